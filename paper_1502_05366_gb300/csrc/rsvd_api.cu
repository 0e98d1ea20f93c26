// C ABI of the library (include/rsvd.h) and the host-side launch sequences.
//
// Every entry point validates its arguments, carves the caller's workspace
// with a bump allocator (the same code computes the *_workspace_size values
// by running without launching), and enqueues kernels on the caller's stream.
// No device memory is allocated and the host never waits for the device.  The
// combined SVD + ID/CUR call forks one kernel (the Jacobi SVD: an 8-CTA
// cluster for FP32 cores of 32 <= l <= 256, one CTA otherwise) onto an
// auxiliary stream and joins it back with events; that stream and its two
// events are created once per device on first use and kept until the process
// exits (a cudaDeviceReset invalidates them: do not call the library on that
// device afterwards).
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace rsvd {

// ------------------------------------------------------------------------
// options, workspace arena, launch context
// ------------------------------------------------------------------------
struct Opts {
  int s = 1, max_sweeps = 30, precision = RSVD_PREC_TC;
};

static bool read_opts(const rsvd_opts* o, Opts* out) {
  Opts d;
  if (o) {
    if (o->s < 1 || o->max_sweeps < 1 || o->max_sweeps > 1000) return false;
    if (o->precision != RSVD_PREC_TC && o->precision != RSVD_PREC_SIMT &&
        o->precision != RSVD_PREC_MIXED)
      return false;
    for (int i = 0; i < 13; ++i)
      if (o->reserved[i] != 0) return false;
    d.s = o->s;
    d.max_sweeps = o->max_sweeps;
    d.precision = o->precision;
  }
  *out = d;
  return true;
}

struct Ctx {
  bool dry = true;
  char* base = nullptr;
  size_t cap = 0;
  size_t off = 0;
  cudaStream_t stream = nullptr;
  int* d_info = nullptr;
  cudaError_t err = cudaSuccess;
  // A holds bf16 values (RSVD_BF16, tensor-core path): the passes over A read
  // it as bf16 and the CUR gathers convert; everything else is fp32
  int abf = 0;
  // host-input call: A arrives in row chunks, chunk ci complete at chunk_ev[ci]
  int nchunks = 0;
  int64_t chunk_rows = 0;
  cudaEvent_t* chunk_ev = nullptr;

  template <typename T>
  T* take(size_t count) {
    off = (size_t)round_up((int64_t)off, 256);
    T* p = dry ? nullptr : reinterpret_cast<T*>(base + off);
    off += count * sizeof(T) + 16;
    return p;
  }
  bool run(cudaError_t e) {
    if (e != cudaSuccess && err == cudaSuccess) err = e;
    return e == cudaSuccess;
  }
};

#define LK(...)                                      \
  do {                                               \
    if (!c.dry) {                                    \
      if (!c.run(__VA_ARGS__)) return RSVD_ERR_CUDA; \
    }                                                \
  } while (0)

static inline int padL(int l) { return (int)round_up(l, 16); }
static inline int64_t pad8(int64_t r) { return round_up(r, 8); }

// ------------------------------------------------------------------------
// Engine: the path for one element type.  T = float uses the tensor-core GEMMs
// (unless the SIMT option is chosen or A is not TMA-addressable); T = double
// runs the SIMT FP64 kernels.
// ------------------------------------------------------------------------
template <typename T>
struct Engine {
  Ctx& c;
  Opts o;
  bool tc;
  int sms;
  explicit Engine(Ctx& ctx, const Opts& op, bool use_tc) : c(ctx), o(op), tc(use_tc) {
    sms = device_sm_count();
  }

  // Split-transposed bf16 operand buffers (L x ld rows).
  struct Split {
    void* hi = nullptr;
    void* lo = nullptr;
    int64_t ld = 0;
    void* lo2 = nullptr;   // third term (R^-1 operands only)
  };
  Split take_split(int L, int64_t rows) {
    Split s;
    s.ld = pad8(rows);
    s.hi = c.template take<uint16_t>((size_t)L * s.ld);
    s.lo = c.template take<uint16_t>((size_t)L * s.ld);
    return s;
  }

  // ---------------- GEMM building blocks ----------------
  // Y (rows x L) = A (rows x K) * W.  omega: W = Omega(seed) with lvalid columns.
  rsvd_status gemm_n(int64_t rows, int64_t K, int L, const T* A, int64_t lda, int64_t a_rows,
                     int64_t a_cols, bool omega, uint64_t seed, int lvalid, const Split* w,
                     const T* Wsimt, int64_t ldws, T* out, int64_t ldo, int ncols, Split* out_split,
                     float* part, const int* skip, bool a_bf16 = false) {
    if (tc) {
      TcGemm g{};
      g.form = 0;
      g.a_bf16 = a_bf16 ? 1 : 0;
      g.omega = omega ? 1 : 0;
      g.seed = seed;
      g.rows = rows;
      g.K = K;
      g.L = L;
      g.lvalid = lvalid;
      g.A = (const float*)A;
      g.lda = lda;
      g.a_rows_total = a_rows;
      g.a_cols_total = a_cols;
      g.Whi = w ? w->hi : nullptr;
      g.Wlo = w ? w->lo : nullptr;
      g.Wlo2 = w ? w->lo2 : nullptr;
      g.wterms = (w && !w->lo) ? 1 : ((w && w->lo2) ? 3 : 2);
      g.ldw = w ? w->ld : 0;
      g.part = part;
      g.out = (float*)out;
      g.ldo = ldo;
      g.ncols = ncols;
      g.out_hi = out_split ? out_split->hi : nullptr;
      g.out_lo = out_split ? out_split->lo : nullptr;
      g.ldt = out_split ? out_split->ld : 0;
      g.skip = skip;
      g.d_info = c.d_info;
      LK(launch_tc_gemm(g, c.stream));
    } else {
      LK(launch_gemm_nn<T>(rows, ncols, K, A, lda, omega ? nullptr : Wsimt, ldws, out, ldo,
                           seed, lvalid, c.stream));
    }
    return RSVD_OK;
  }

  // Z (rows x L) = A^T W with A (K x rows).
  rsvd_status gemm_t(int64_t rows, int64_t K, int L, const T* A, int64_t lda, const Split* w,
                     const T* Wsimt, int64_t ldws, T* out, int64_t ldo, int ncols,
                     Split* out_split, float* part, T* slabs, const int* skip, bool gram = false,
                     bool a_bf16 = false) {
    if (tc) {
      TcGemm g{};
      g.form = 1;
      g.a_bf16 = a_bf16 ? 1 : 0;
      g.rows = rows;
      g.K = K;
      g.L = L;
      g.lvalid = L;
      g.A = (const float*)A;
      g.lda = lda;
      g.a_rows_total = K;
      g.a_cols_total = rows;
      g.Whi = w->hi;
      g.Wlo = w->lo;
      g.Wlo2 = nullptr;
      g.wterms = w->lo ? 2 : 1;
      g.gram = gram ? 1 : 0;
      g.ldw = w->ld;
      g.part = part;
      g.out = (float*)out;
      g.ldo = ldo;
      g.ncols = ncols;
      g.out_hi = out_split ? out_split->hi : nullptr;
      g.out_lo = out_split ? out_split->lo : nullptr;
      g.ldt = out_split ? out_split->ld : 0;
      g.skip = skip;
      g.d_info = c.d_info;
      LK(launch_tc_gemm(g, c.stream));
    } else {
      int ns;
      int64_t kc;
      tn_split(rows, ncols, K, sms, &ns, &kc);
      LK(launch_gemm_tn_partial<T>(rows, ncols, K, A, lda, Wsimt, ldws, slabs, ncols, ns, kc,
                                   c.stream));
      LK(launch_reduce_slabs<T>(rows, ncols, ns, slabs, ncols, out, ldo, c.stream));
    }
    return RSVD_OK;
  }

  // Scratch sizes for GEMMs of the given shapes.
  size_t part_bytes_n(int64_t rows, int64_t K, int L) {
    return tc ? tc_part_bytes(rows, K, L) : 0;
  }
  size_t slab_elems_t(int64_t rows, int64_t K, int ncols) {
    if (tc) return 0;
    int ns;
    int64_t kc;
    tn_split(rows, ncols, K, sms, &ns, &kc);
    return (size_t)ns * rows * ncols;
  }

  // ---------------- orth: CholeskyQR with two or three passes ----------------
  struct OrthBufs {
    T* G;        // L x L
    T* R;        // L x L
    T* Rinv;     // L x L
    T* Racc;     // L x L
    T* tmpLL;    // L x L
    void* Whi;   // L x L bf16, three terms of (R^-1)^T
    void* Wlo;
    void* Wlo2;
    int* flags;  // 4 ints
    T* chol_scratch;
  };
  OrthBufs take_orth_bufs(int L) {
    OrthBufs b;
    b.G = c.template take<T>((size_t)L * L);
    b.R = c.template take<T>((size_t)L * L);
    b.Rinv = c.template take<T>((size_t)L * L);
    b.Racc = c.template take<T>((size_t)L * L);
    b.tmpLL = c.template take<T>((size_t)L * L);
    b.Whi = c.template take<uint16_t>((size_t)L * L);
    b.Wlo = c.template take<uint16_t>((size_t)L * L);
    b.Wlo2 = c.template take<uint16_t>((size_t)L * L);
    b.flags = c.template take<int>(4);
    const size_t cs = chol_scratch_bytes(L, sizeof(T));
    b.chol_scratch = cs ? c.template take<T>(cs / sizeof(T)) : nullptr;
    return b;
  }

  // X (rows x L, l valid columns, zero padding) -> Q in Y (rows x L).  For the
  // tensor-core path `split` holds the hi/lo of X^T on entry and of Q^T on exit.
  // When want_R, ob.Racc ends as R with X = Q R.
  // full = true: CholeskyQR2 plus the conditional third pass (orthonormal Q).
  // full = false (inside the power scheme, where any well-conditioned basis of
  // range(X) gives the same subspace): one pass, and the second and third
  // passes only when the first one needed a shift (numerically rank-deficient
  // X), decided on the device.
  rsvd_status orth(int64_t rows, int l, int L, T* X, T* Y, Split* split, OrthBufs& ob,
                   float* part, T* slabs, bool want_R, bool full = true) {
    LK(cudaMemsetAsync(ob.flags, 0, 4 * sizeof(int), c.stream));
    T* src = X;
    T* dst = Y;
    for (int pass = 1; pass <= 3; ++pass) {
      const int skip_idx = (pass == 3) ? 2 : ((pass == 2 && !full) ? 3 : -1);
      const int* skip = skip_idx >= 0 ? ob.flags + skip_idx : nullptr;
      // Gram G = src^T src
      rsvd_status st = gemm_t(L, rows, L, src, L, split, src, L, ob.G, L, L, nullptr, part, slabs,
                              skip, true);
      if (st != RSVD_OK) return st;
      CholArgs a{};
      a.l = l;
      a.L = L;
      a.G = ob.G;
      a.ldg = L;
      a.R = want_R ? ob.R : nullptr;
      a.Rinv = tc ? nullptr : ob.Rinv;   // the tensor-core apply takes the bf16 terms
      a.Whi = tc ? ob.Whi : nullptr;
      a.Wlo = tc ? ob.Wlo : nullptr;
      a.Wlo2 = tc ? ob.Wlo2 : nullptr;
      a.scratch = ob.chol_scratch;
      a.flags = ob.flags;
      a.pass = pass;
      a.skip_idx = skip_idx;
      a.d_info = c.d_info;
      LK(launch_chol<T>(a, c.stream));
      if (want_R) {
        if (pass == 1)
          LK(cudaMemcpyAsync(ob.Racc, ob.R, sizeof(T) * L * L, cudaMemcpyDeviceToDevice,
                             c.stream));
        else
          LK(launch_trmm_upper<T>(L, ob.R, ob.Racc, ob.tmpLL, c.stream));
      }
      // apply: dst = src R^{-1}
      Split w{ob.Whi, ob.Wlo, L, ob.Wlo2};
      st = gemm_n(rows, L, L, src, L, rows, L, false, 0, L, &w, ob.Rinv, L, dst, L, L, split,
                  part, skip);
      if (st != RSVD_OK) return st;
      if (skip && tc) {  // pass skipped: the previous Q carried over unchanged
        if (!c.dry) {
          if (!c.run(launch_cond_copy<float>(skip, rows * (int64_t)L, (const float*)src,
                                             (float*)dst, c.stream)))
            return RSVD_ERR_CUDA;
        }
      }
      T* t = src;
      src = dst;
      dst = t;
    }
    // three passes (run or carried over) leave the result in Y (X -> Y -> X -> Y)
    return RSVD_OK;
  }

  // ---------------- QB: range finder + power scheme + Bt ----------------
  struct QBBufs {
    T* Y;        // m x L
    T* Ytmp;     // m x L
    T* Z;        // n x L
    T* Ztmp;     // n x L
    Split ys, zs;
    float* part;
    T* slabs;
    OrthBufs ob;
  };

  QBBufs take_qb(int64_t m, int64_t n, int L) {
    QBBufs b;
    b.Y = c.template take<T>((size_t)m * L);
    b.Ytmp = c.template take<T>((size_t)m * L);
    b.Z = c.template take<T>((size_t)n * L);
    b.Ztmp = c.template take<T>((size_t)n * L);
    if (tc) {
      b.ys = take_split(L, m);
      b.zs = take_split(L, n);
    }
    size_t pb = 0;
    if (tc) {
      pb = std::max(pb, tc_part_bytes(m, n, L));   // Y = A Omega, Y = A Z
      pb = std::max(pb, tc_part_bytes(n, m, L));   // Z = A^T Y, Bt
      pb = std::max(pb, tc_part_bytes(L, m, L));   // Gram of m-row X
      pb = std::max(pb, tc_part_bytes(L, n, L));   // Gram of n-row X
      pb = std::max(pb, tc_part_bytes(m, L, L));   // apply on m rows
      pb = std::max(pb, tc_part_bytes(n, L, L));   // apply on n rows
    }
    b.part = pb ? c.template take<float>(pb / sizeof(float)) : nullptr;
    size_t se = 0;
    if (!tc) {
      se = std::max(se, slab_elems_t(n, m, L));
      se = std::max(se, slab_elems_t(L, m, L));
      se = std::max(se, slab_elems_t(L, n, L));
    }
    b.slabs = se ? c.template take<T>(se) : nullptr;
    b.ob = take_orth_bufs(L);
    return b;
  }

  // Range finder up to its last product (Alg. 5 first part): on exit b.Y holds
  // Y = A Z (or A Omega when q = 0), not yet orthonormalised, with its split in
  // b.ys on the tensor-core path.
  rsvd_status power(QBBufs& b, int64_t m, int64_t n, int l, int q, uint64_t seed, const T* A,
                    int64_t lda) {
    const int L = padL(l);
    rsvd_status st;
    if (!tc) LK(launch_fill<T>(m, L, b.Y, L, T(0), c.stream));
    // Y = A Omega (Fig. 1 step 2); for a host-input call, row chunk by row
    // chunk as the chunks of A land (the rows of Y are independent)
    if (c.nchunks > 0 && tc) {
      for (int ci = 0; ci < c.nchunks; ++ci) {
        const int64_t r0 = ci * c.chunk_rows, r1 = std::min(m, r0 + c.chunk_rows);
        if (r1 <= r0) break;
        LK(cudaStreamWaitEvent(c.stream, c.chunk_ev[ci], 0));
        Split ysc = b.ys;
        ysc.hi = (uint16_t*)b.ys.hi + r0;
        ysc.lo = (uint16_t*)b.ys.lo + r0;
        const T* Ac = reinterpret_cast<const T*>(reinterpret_cast<const char*>(A) +
                                                 r0 * lda * (c.abf ? 2 : (int64_t)sizeof(T)));
        st = gemm_n(r1 - r0, n, L, Ac, lda, r1 - r0, n, true, seed, l, nullptr, nullptr, 0,
                    b.Y + r0 * L, L, L, &ysc, b.part, nullptr, c.abf != 0);
        if (st != RSVD_OK) return st;
      }
    } else {
      st = gemm_n(m, n, L, A, lda, m, n, true, seed, l, nullptr, nullptr, 0, b.Y, L, L, &b.ys,
                  b.part, nullptr, c.abf != 0);
      if (st != RSVD_OK) return st;
    }
    // RSVD_PREC_MIXED: the passes of the power scheme take one bf16 term of the
    // stored operand (one product per K-step); the sketch, the orthonormalisations
    // and Bt = A^T Q keep the split arithmetic
    const bool mixed = tc && o.precision == RSVD_PREC_MIXED;
    Split ys1 = b.ys, zs1 = b.zs;
    if (mixed) ys1.lo = zs1.lo = nullptr;
    int prod = 0;  // index of the next product with A or A^T (Alg. 5 orth test)
    for (int j = 1; j <= q; ++j) {
      if (prod % o.s == 0) {
        st = orth(m, l, L, b.Y, b.Ytmp, &b.ys, b.ob, b.part, b.slabs, false, false);
        if (st != RSVD_OK) return st;
        std::swap(b.Y, b.Ytmp);
      }
      ++prod;
      // Z = A^* Y (Sec. 3.2)
      st = gemm_t(n, m, L, A, lda, mixed ? &ys1 : &b.ys, b.Y, L, b.Z, L, L, &b.zs, b.part, b.slabs,
                  nullptr, false, c.abf != 0);
      if (st != RSVD_OK) return st;
      if (prod % o.s == 0) {
        st = orth(n, l, L, b.Z, b.Ztmp, &b.zs, b.ob, b.part, b.slabs, false, false);
        if (st != RSVD_OK) return st;
        std::swap(b.Z, b.Ztmp);
      }
      ++prod;
      // Y = A Z
      st = gemm_n(m, n, L, A, lda, m, n, false, 0, L, mixed ? &zs1 : &b.zs, b.Z, L, b.Y, L, L,
                  &b.ys, b.part, nullptr, c.abf != 0);
      if (st != RSVD_OK) return st;
    }
    return RSVD_OK;
  }

  // On exit: b.Y holds Q (m x L, padded), b.Z holds Bt (n x L, padded); for
  // the tensor-core path b.zs holds the split of Bt^T.
  rsvd_status qb(QBBufs& b, int64_t m, int64_t n, int l, int q, uint64_t seed, const T* A,
                 int64_t lda) {
    const int L = padL(l);
    rsvd_status st = power(b, m, n, l, q, seed, A, lda);
    if (st != RSVD_OK) return st;
    // Q = orth(Y)
    st = orth(m, l, L, b.Y, b.Ytmp, &b.ys, b.ob, b.part, b.slabs, false);
    if (st != RSVD_OK) return st;
    std::swap(b.Y, b.Ytmp);
    // Bt = A^* Q (Alg. 5)
    st = gemm_t(n, m, L, A, lda, &b.ys, b.Y, L, b.Z, L, L, &b.zs, b.part, b.slabs, nullptr, false,
                c.abf != 0);
    return st;
  }

  // ---------------- one block of the adaptive QB (Alg. 7) ----------------
  // Q_t from the range finder on the current residual A (seed of this block),
  // re-projected against the done = b t columns already in Qo and
  // re-orthonormalised; Bt_t = A^* Q_t; both appended to the outputs at column
  // `done`; then A <- A - Q_t Bt_t^T with the squared norms of the updated tiles
  // in sq.  Ct (b x done) and cslabs are the re-projection's scratch.
  rsvd_status qb2_block(QBBufs& b, int64_t m, int64_t n, int bs, int q, uint64_t seed, T* A,
                        int64_t lda, T* Qo, int64_t ldq, T* Bto, int64_t ldbt, int64_t done,
                        T* Ct, T* cslabs, double* sq) {
    const int L = padL(bs);
    rsvd_status st = power(b, m, n, bs, q, seed, A, lda);
    if (st != RSVD_OK) return st;
    st = orth(m, bs, L, b.Y, b.Ytmp, &b.ys, b.ob, b.part, b.slabs, false);
    if (st != RSVD_OK) return st;
    std::swap(b.Y, b.Ytmp);
    if (done > 0) {
      // Ct = Q_t^* Qbar (b x done): split-K partial products summed in a fixed order
      int ns;
      int64_t kc;
      tn_split(bs, done, m, sms, &ns, &kc);
      LK(launch_gemm_tn_partial<T>(bs, done, m, b.Y, L, Qo, ldq, cslabs, done, ns, kc,
                                   c.stream));
      LK(launch_reduce_slabs<T>(bs, done, ns, cslabs, done, Ct, done, c.stream));
      // Q_t <- Q_t - Qbar Ct^T, then orth again
      LK(launch_rank_update<T>(m, bs, b.Y, L, Qo, ldq, Ct, done, (int)done, nullptr, c.stream));
      if (tc)
        LK(launch_split_transpose(m, bs, L, (const float*)b.Y, L, b.ys.hi, b.ys.lo, b.ys.ld,
                                  c.stream));
      st = orth(m, bs, L, b.Y, b.Ytmp, &b.ys, b.ob, b.part, b.slabs, false);
      if (st != RSVD_OK) return st;
      std::swap(b.Y, b.Ytmp);
    }
    // Bt_t = A^* Q_t (B_t = Q_t^* A)
    st = gemm_t(n, m, L, A, lda, &b.ys, b.Y, L, b.Z, L, L, &b.zs, b.part, b.slabs, nullptr,
                false);
    if (st != RSVD_OK) return st;
    LK(launch_copy2d<T, T>(m, bs, b.Y, L, Qo + done, ldq, c.stream));
    LK(launch_copy2d<T, T>(n, bs, b.Z, L, Bto + done, ldbt, c.stream));
    // A <- A - Q_t B_t
    LK(launch_rank_update<T>(m, n, A, lda, b.Y, L, b.Z, L, bs, sq, c.stream));
    return RSVD_OK;
  }

  // ---------------- small SVD of R-hat and lift (Alg. 5 tail) ----------------
  struct SvdBufs {
    T* Uh;       // L x L
    T* Vh;       // L x L
    double* Sh;  // L
    T* Uj;       // l x l: Jacobi's left vectors before the final sort
    T* P;        // l x l: M^T Uj
    double* Sj;  // l
    T* jac_scratch;
    T* vslabs;
    int* signs;
  };
  SvdBufs take_svd(int l, int L, int k) {
    SvdBufs s;
    s.Uh = c.template take<T>((size_t)L * L);
    s.Vh = c.template take<T>((size_t)L * L);
    s.Sh = c.template take<double>((size_t)L);
    s.Uj = c.template take<T>((size_t)l * l);
    s.P = c.template take<T>((size_t)l * l);
    s.Sj = c.template take<double>((size_t)l);
    const size_t js = jacobi_scratch_bytes(l, sizeof(T));
    s.jac_scratch = js ? c.template take<T>(js / sizeof(T)) : nullptr;
    int ns;
    int64_t kc;
    tn_split(l, l, l, sms, &ns, &kc);
    s.vslabs = c.template take<T>((size_t)ns * l * l);
    s.signs = c.template take<int>((size_t)k + 1);
    return s;
  }

  // M (l x l, ldm) = Uh diag(Sh) Vh^T: Jacobi for the left vectors, then
  // P = M^T Uh, sigma_j = ||P(:, j)||, Vh = P diag(1/sigma), sorted.
  rsvd_status small_svd(int l, const T* M, int64_t ldm, SvdBufs& s, T* Uh, int64_t lduh,
                        double* Sh, T* Vh, int64_t ldvh) {
    rsvd_status st = small_svd_jacobi(l, M, ldm, s, c.stream);
    if (st != RSVD_OK) return st;
    return small_svd_finish(l, M, ldm, s, Uh, lduh, Sh, Vh, ldvh);
  }
  // The Jacobi sweeps alone (one CTA), on stream js.
  rsvd_status small_svd_jacobi(int l, const T* M, int64_t ldm, SvdBufs& s, cudaStream_t js) {
    LK(launch_jacobi<T>(l, M, ldm, s.Uj, l, s.Sj, nullptr, 0, s.jac_scratch, o.max_sweeps,
                        c.d_info, js));
    return RSVD_OK;
  }
  rsvd_status small_svd_finish(int l, const T* M, int64_t ldm, SvdBufs& s, T* Uh, int64_t lduh,
                               double* Sh, T* Vh, int64_t ldvh) {
    int ns;
    int64_t kc;
    tn_split(l, l, l, sms, &ns, &kc);
    LK(launch_gemm_tn_partial<T>(l, l, l, M, ldm, s.Uj, l, s.vslabs, l, ns, kc, c.stream));
    LK(launch_reduce_slabs<T>(l, l, ns, s.vslabs, l, s.P, l, c.stream));
    LK(launch_svd_finalize<T>(l, s.P, l, s.Uj, l, Uh, lduh, Sh, Vh, ldvh, c.d_info, c.stream));
    return RSVD_OK;
  }

  // From QB: U = Q Vh(:, :k), V = Qh Uh(:, :k), S = Sh(:k), signs fixed.
  rsvd_status svd_from_qb(QBBufs& b, SvdBufs& s, int64_t m, int64_t n, int k, int l, T* U,
                          int64_t ldu, double* S, T* V, int64_t ldv) {
    rsvd_status st = svd_prep(b, s, n, l);
    if (st != RSVD_OK) return st;
    st = small_svd_jacobi(l, b.ob.Racc, padL(l), s, c.stream);
    if (st != RSVD_OK) return st;
    return svd_finish(b, s, m, n, k, l, U, ldu, S, V, ldv);
  }
  // [Qh, Rh] = qr(Bt): Qh into Ztmp, Rh = Racc (overwrites Bt).
  rsvd_status svd_prep(QBBufs& b, SvdBufs& s, int64_t n, int l) {
    (void)s;
    return orth(n, l, padL(l), b.Z, b.Ztmp, &b.zs, b.ob, b.part, b.slabs, true);
  }
  // After the Jacobi sweeps on Rh: its right vectors and sigma, then the lifts.
  rsvd_status svd_finish(QBBufs& b, SvdBufs& s, int64_t m, int64_t n, int k, int l, T* U,
                         int64_t ldu, double* S, T* V, int64_t ldv) {
    const int L = padL(l);
    T* Qh = b.Ztmp;
    rsvd_status st = small_svd_finish(l, b.ob.Racc, L, s, s.Uh, L, s.Sh, s.Vh, L);
    if (st != RSVD_OK) return st;
    LK(launch_gemm_nn<T>(m, k, l, b.Y, L, s.Vh, L, U, ldu, 0, k, c.stream));   // U = Q Vh
    LK(launch_gemm_nn<T>(n, k, l, Qh, L, s.Uh, L, V, ldv, 0, k, c.stream));    // V = Qh Uh
    LK(launch_sign_fix<T>(m, n, k, U, ldu, V, ldv, s.signs, c.stream));
    LK(cudaMemcpyAsync(S, s.Sh, sizeof(double) * k, cudaMemcpyDeviceToDevice, c.stream));
    return RSVD_OK;
  }

  // ---------------- ID (Sec. 3.5) and CUR (Sec. 3.6) ----------------
  struct IdBufs {
    double* W;       // r x n row-major
    int64_t* where;  // n
    double* pval;
    int64_t* pidx;
    double* nrm;     // n
    double* diagR;   // k
    unsigned* bar;
    double* S11;     // k x k
    double* S12;     // k x (n-k) row-major
    int32_t* J;      // n (internal copy)
    T* Tt;           // (n-k) x k
  };
  IdBufs take_id(int r, int64_t n, int k, bool with_T = true) {
    IdBufs d;
    d.W = c.template take<double>((size_t)n * r);
    d.where = c.template take<int64_t>((size_t)n);
    d.pval = c.template take<double>(2 * 1024 * 2);
    d.pidx = c.template take<int64_t>(2 * 1024);
    d.nrm = c.template take<double>((size_t)2 * n);
    d.diagR = c.template take<double>((size_t)k);
    d.bar = c.template take<unsigned>(4);
    d.J = c.template take<int32_t>((size_t)n);
    if (with_T) {
      d.S11 = c.template take<double>((size_t)k * k + k);   // + diagonal reciprocals (df path)
      d.S12 = c.template take<double>((size_t)(n - k) * k + 1);
      d.Tt = c.template take<T>((size_t)(n - k) * k + 1);
    } else {
      d.S11 = nullptr;
      d.S12 = nullptr;
      d.Tt = nullptr;
    }
    return d;
  }

  // CPQR of the r x n row-major matrix in d.W (already filled), k steps; J
  // into d.J; Tt ((n-k) x k) = (S11^{-1} S12)^T.
  rsvd_status id_core(IdBufs& d, int r, int64_t n, int k, double* gaps) {
    CpqrArgs a{};
    a.r = r;
    a.n = n;
    a.k = k;
    a.W = d.W;
    a.J = d.J;
    a.where = d.where;
    a.gaps = gaps;
    a.pval = d.pval;
    a.pidx = d.pidx;
    a.nrm = d.nrm;
    a.diagR = d.diagR;
    a.bar = d.bar;
    a.d_info = c.d_info;
    int grid = 0;
    // FP32 data: double-float arithmetic on the working area as two float planes
    constexpr bool DF = sizeof(T) == 4;
    if (DF)
      LK(launch_cpqr_df(a, &grid, c.stream));
    else
      LK(launch_cpqr(a, &grid, c.stream));
    if (!d.Tt) return RSVD_OK;   // pivots only (row ID of the CUR)
    if (DF)
      LK(launch_id_extract_df(r, n, k, d.W, d.J, d.diagR, d.S11, d.S12, c.stream));
    else
      LK(launch_id_extract(r, n, k, d.W, d.J, d.diagR, d.S11, d.S12, c.stream));
    // S11 column-major: U(i, t) = S11[t*k + i]; rhs(i, c) = S12[i*(n-k) + c];
    // out Tt(c, i) = Tt[c*k + i]
    if (DF)
      LK(launch_upper_solve_df<float2, float>(k, n - k, d.S11, (const float2*)d.S12, n - k, 1,
                                              (float*)d.Tt, 1, k, c.d_info, c.stream));
    else
      LK(launch_upper_solve<double, T>(k, n - k, d.S11, 1, k, d.S12, n - k, 1, d.Tt, 1, k,
                                       c.d_info, c.stream));
    return RSVD_OK;
  }

  struct CurBufs {
    IdBufs rid;       // row ID of C^T: r = k, n = m
    T* R;             // k x n
    T* RT;            // n x Kp
    T* RTtmp;         // n x Kp
    Split rts;
    OrthBufs ob;
    float* part;
    T* slabs;
    T* QRg;           // (n-k) x Kp
    T* M1;            // k x Kp
    T* M1b;           // k x Kp
    T* mslabs;
    double* RR64;     // Kp x Kp
  };
  CurBufs take_cur(int64_t m, int64_t n, int k) {
    CurBufs u;
    const int Kp = padL(k);
    u.rid = take_id(k, m, k, false);
    u.R = c.template take<T>((size_t)k * n);
    u.RT = c.template take<T>((size_t)n * Kp);
    u.RTtmp = c.template take<T>((size_t)n * Kp);
    if (tc) u.rts = take_split(Kp, n);
    u.ob = take_orth_bufs(Kp);
    size_t pb = 0;
    if (tc) {
      pb = std::max(pb, tc_part_bytes(Kp, n, Kp));
      pb = std::max(pb, tc_part_bytes(n, Kp, Kp));
    }
    u.part = pb ? c.template take<float>(pb / sizeof(float)) : nullptr;
    const size_t se = tc ? 0 : slab_elems_t(Kp, n, Kp);
    u.slabs = se ? c.template take<T>(se) : nullptr;
    u.QRg = c.template take<T>((size_t)(n - k) * Kp + 1);
    u.M1 = c.template take<T>((size_t)k * Kp);
    u.M1b = c.template take<T>((size_t)k * Kp);
    int ns;
    int64_t kc;
    tn_split(k, Kp, n - k, sms, &ns, &kc);
    u.mslabs = c.template take<T>((size_t)ns * k * Kp);
    u.RR64 = c.template take<double>((size_t)Kp * Kp + Kp);
    return u;
  }

  // CUR from the column ID (J in idb.J, Tt): Jc, Ir, Ucur.
  rsvd_status cur_from_id(CurBufs& u, IdBufs& idb, int64_t m, int64_t n, int k, const T* A,
                          int64_t lda, int32_t* Jc, int32_t* Ir, T* Ucur, int64_t ldu,
                          double* rgaps) {
    const int Kp = padL(k);
    // C^T columns (rows of C = A(:, J[:k])) in the CPQR layout
    if (sizeof(T) == 4)
      LK(launch_gather_ct_df(m, k, A, lda, c.abf, idb.J, u.rid.W, c.stream));
    else
      LK(launch_gather_ct<T>(m, k, A, lda, idb.J, u.rid.W, c.stream));
    rsvd_status st = id_core(u.rid, k, m, k, rgaps);
    if (st != RSVD_OK) return st;
    if (Jc) LK(launch_copy_i32(k, idb.J, Jc, c.stream));
    if (Ir) LK(launch_copy_i32(k, u.rid.J, Ir, c.stream));
    // R = A(I, :), R^T (n x Kp, zero padded)
    if (c.abf)
      LK(launch_gather_rows_bf16(k, n, A, lda, u.rid.J, (float*)u.R, n, c.stream));
    else
      LK(launch_gather_rows<T>(k, n, A, lda, u.rid.J, u.R, n, c.stream));
    LK(cudaMemsetAsync(u.RT, 0, sizeof(T) * n * Kp, c.stream));
    LK(launch_transpose<T, T>(k, n, u.R, n, u.RT, Kp, c.stream));
    if (tc)
      LK(launch_split_transpose(n, Kp, Kp, (const float*)u.RT, Kp, u.rts.hi, u.rts.lo, u.rts.ld,
                                c.stream));
    // R^* = Q_R R_R
    st = orth(n, k, Kp, u.RT, u.RTtmp, &u.rts, u.ob, u.part, u.slabs, true);
    if (st != RSVD_OK) return st;
    const T* QR = u.RTtmp;
    // M1 = V^* Q_R = Q_R(J[:k], :) + T Q_R(J[k:], :)
    LK(launch_gather_rows_by_perm<T>(n - k, Kp, QR, Kp, idb.J + k, u.QRg, Kp, c.stream));
    int ns;
    int64_t kc;
    tn_split(k, Kp, n - k, sms, &ns, &kc);
    LK(launch_gemm_tn_partial<T>(k, Kp, n - k, idb.Tt, k, u.QRg, Kp, u.mslabs, Kp, ns, kc,
                                 c.stream));
    LK(launch_reduce_slabs<T>(k, Kp, ns, u.mslabs, Kp, u.M1, Kp, c.stream));
    LK(launch_gather_rows_by_perm<T>(k, Kp, QR, Kp, idb.J, u.M1b, Kp, c.stream));
    LK(launch_add_inplace<T>(k, Kp, u.M1b, Kp, u.M1, Kp, c.stream));
    // U R_R^T = M1  ->  R_R U(c, :)^T = M1(c, :)^T
    if (sizeof(T) == 4 && k <= 1024) {
      LK(launch_upper_to_df<float>(k, (const float*)u.ob.Racc, Kp, u.RR64, c.stream));
      LK(launch_upper_solve_df<float, float>(k, k, u.RR64, (const float*)u.M1, 1, Kp,
                                             (float*)Ucur, 1, ldu, c.d_info, c.stream));
    } else {
      LK(launch_copy2d<T, double>(Kp, Kp, u.ob.Racc, Kp, u.RR64, Kp, c.stream));
      LK(launch_upper_solve<T, T>(k, k, u.RR64, Kp, 1, u.M1, 1, Kp, Ucur, 1, ldu, c.d_info,
                                  c.stream));
    }
    return RSVD_OK;
  }
};

// ------------------------------------------------------------------------
// argument checks
// ------------------------------------------------------------------------
static bool base_args_ok(int64_t m, int64_t n, int k, int p, int q, int dtype) {
  if (dtype != RSVD_F32 && dtype != RSVD_F64 && dtype != RSVD_BF16) return false;
  if (m < 1 || n < 1 || k < 1 || p < 0 || q < 0 || q > 64) return false;
  const int64_t l = (int64_t)k + p;
  if (l > m || l > n || l > 1024) return false;
  if (m > 0x7fffffffLL || n > 0x7fffffffLL) return false;
  return true;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Tensor-core path usable: FP32 or BF16 A, requested, width fits, A
// TMA-addressable (16-byte aligned base and rows).
static bool want_tc(int dtype, const Opts& o, int l, const void* A, int64_t lda) {
  if (dtype != RSVD_F32 && dtype != RSVD_BF16) return false;
  if (o.precision != RSVD_PREC_TC && o.precision != RSVD_PREC_MIXED) return false;
  if (padL(l) > 1024) return false;   // widths above 256 run in column chunks
  if (A && !aligned16(A)) return false;
  if (lda % (dtype == RSVD_BF16 ? 8 : 4) != 0) return false;
  return true;
}

static void reset_info(Ctx& c) {
  if (c.d_info && !c.dry) c.run(cudaMemsetAsync(c.d_info, 0, sizeof(int), c.stream));
}

enum Want { W_Q = 1, W_SVD = 2, W_ID = 4, W_CUR = 8 };

// Auxiliary stream and fork/join events of one device (created on first use,
// kept for the life of the process).  The host-side enqueue of a forked call
// holds the device's mutex so that concurrent callers do not interleave their
// records of the shared events.
constexpr int MAX_CHUNKS = 16;
struct SideStream {
  std::mutex mu;
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t chunk[MAX_CHUNKS] = {};
};
static SideStream* side_stream() {
  static SideStream g_side[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  SideStream* ss = &g_side[dev];
  std::lock_guard<std::mutex> lk(ss->mu);
  if (!ss->s) {
    cudaStream_t st = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    if (cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess) {
      if (a) cudaEventDestroy(a);
      cudaStreamDestroy(st);
      return nullptr;
    }
    for (int i = 0; i < MAX_CHUNKS; ++i) {
      if (cudaEventCreateWithFlags(&ss->chunk[i], cudaEventDisableTiming) != cudaSuccess) {
        for (int q = 0; q < i; ++q) cudaEventDestroy(ss->chunk[q]);
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        cudaStreamDestroy(st);
        return nullptr;
      }
    }
    ss->fork = a;
    ss->join = b;
    ss->s = st;
  }
  return ss;
}

template <typename T>
static rsvd_status run_all(Ctx& c, const Opts& o, bool tc, int64_t m, int64_t n, int k, int p,
                           int q, uint64_t seed, const T* A, int64_t lda, int want, T* Qo,
                           int64_t ldq, T* Bto, int64_t ldbt, T* U, int64_t ldu, double* S, T* V,
                           int64_t ldv, int32_t* J, T* Tout, int64_t ldt, int32_t* Jc,
                           int32_t* Ir, T* Ucur, int64_t lducur, const T* A_host = nullptr) {
  Engine<T> e(c, o, tc);
  const int l = k + p, L = padL(l);
  auto qbb = e.take_qb(m, n, L);
  typename Engine<T>::SvdBufs sb{};
  if (want & W_SVD) sb = e.take_svd(l, L, k);
  typename Engine<T>::IdBufs idb{};
  if (want & (W_ID | W_CUR)) idb = e.take_id(l, n, k);
  typename Engine<T>::CurBufs cb{};
  if (want & W_CUR) cb = e.take_cur(m, n, k);
  if (c.dry) return RSVD_OK;
  if (c.off > c.cap) return RSVD_ERR_WORKSPACE;

  reset_info(c);
  // host input: A is copied into the caller's device buffer (same leading
  // dimension); on the tensor-core path in row chunks on the auxiliary stream,
  // so that the sketch Y = A Omega runs behind the copy
  std::unique_lock<std::mutex> host_lock;
  if (A_host) {
    if (tc) {
      SideStream* hs = side_stream();
      if (!hs) return RSVD_ERR_CUDA;
      host_lock = std::unique_lock<std::mutex>(hs->mu);
      int nch = (int)std::min<int64_t>(8, ceil_div(m, 256));
      const int64_t rows = round_up(ceil_div(m, nch), 256);
      nch = (int)ceil_div(m, rows);
      LK(cudaEventRecord(hs->fork, c.stream));
      LK(cudaStreamWaitEvent(hs->s, hs->fork, 0));
      for (int ci = 0; ci < nch; ++ci) {
        const int64_t r0 = ci * rows, r1 = std::min(m, r0 + rows);
        const size_t es = c.abf ? 2 : sizeof(T);
        LK(cudaMemcpyAsync((char*)A + r0 * lda * es, (const char*)A_host + r0 * lda * es,
                           es * (size_t)(r1 - r0) * lda, cudaMemcpyHostToDevice, hs->s));
        LK(cudaEventRecord(hs->chunk[ci], hs->s));
      }
      c.nchunks = nch;
      c.chunk_rows = rows;
      c.chunk_ev = hs->chunk;
    } else {
      LK(cudaMemcpyAsync((T*)A, A_host, (c.abf ? 2 : sizeof(T)) * (size_t)m * lda,
                         cudaMemcpyHostToDevice, c.stream));
    }
  }
  rsvd_status st = e.qb(qbb, m, n, l, q, seed, A, lda);
  c.nchunks = 0;
  if (host_lock.owns_lock()) host_lock.unlock();
  if (st != RSVD_OK) return st;
  if (want & W_Q) {
    if (Qo) LK(launch_copy2d<T, T>(m, l, qbb.Y, L, Qo, ldq, c.stream));
    if (Bto) LK(launch_copy2d<T, T>(n, l, qbb.Z, L, Bto, ldbt, c.stream));
  }
  const bool idcur = (want & (W_ID | W_CUR)) != 0;
  if (idcur) {
    // B = Bt^T (l x n), taken before the SVD reuses Bt's buffer: row-major
    // FP64, or column-major double-float planes (hi = B, lo = 0) for FP32 data
    if (sizeof(T) == 4) {
      // column-major planes: column c of B is row c of Bt
      float* Wh = reinterpret_cast<float*>(idb.W);
      LK(launch_copy2d<float, float>(n, l, (const float*)qbb.Z, L, Wh, l, c.stream));
      LK(cudaMemsetAsync(Wh + (int64_t)l * n, 0, sizeof(float) * (size_t)l * n, c.stream));
    } else {
      LK(launch_transpose<T, double>(n, l, qbb.Z, L, idb.W, n, c.stream));
    }
  }
  // With the ID/CUR requested too, the Jacobi sweeps of the SVD run on the
  // auxiliary stream, beside the CPQR and solves; the SVD is finished on the
  // caller's stream after the join.  The double-float CPQR grid leaves eight
  // SMs free and the FP64 one one SM, room for the 8-CTA cluster or the
  // one-CTA Jacobi; whether the cluster is placed beside the running
  // cooperative grid is the hardware scheduler's choice (it needs eight free
  // SMs of one GPC), so the overlap is partial and the results do not depend
  // on it.  The two branches share no buffer: the Jacobi reads Rh and writes
  // the SVD buffers only.
  SideStream* ss = nullptr;
  std::unique_lock<std::mutex> side_lock;
  if (want & W_SVD) {
    st = e.svd_prep(qbb, sb, n, l);
    if (st != RSVD_OK) return st;
    if (idcur) {
      ss = side_stream();
      if (!ss) return RSVD_ERR_CUDA;
      side_lock = std::unique_lock<std::mutex>(ss->mu);
      LK(cudaEventRecord(ss->fork, c.stream));
      LK(cudaStreamWaitEvent(ss->s, ss->fork, 0));
      st = e.small_svd_jacobi(l, qbb.ob.Racc, L, sb, ss->s);
      if (st != RSVD_OK) return st;
      LK(cudaEventRecord(ss->join, ss->s));
    } else {
      st = e.small_svd_jacobi(l, qbb.ob.Racc, L, sb, c.stream);
      if (st != RSVD_OK) return st;
    }
  }
  if (idcur) {
    st = e.id_core(idb, l, n, k, nullptr);
    if (st != RSVD_OK) return st;
    if (J) LK(launch_copy_i32(n, idb.J, J, c.stream));
    if (Tout) LK(launch_transpose<T, T>(n - k, k, idb.Tt, k, Tout, ldt, c.stream));
  }
  if (want & W_CUR) {
    st = e.cur_from_id(cb, idb, m, n, k, A, lda, Jc, Ir, Ucur, lducur, nullptr);
    if (st != RSVD_OK) return st;
  }
  if (want & W_SVD) {
    if (ss) LK(cudaStreamWaitEvent(c.stream, ss->join, 0));
    st = e.svd_finish(qbb, sb, m, n, k, l, U, ldu, S, V, ldv);
    if (st != RSVD_OK) return st;
  }
  return RSVD_OK;
}

template <typename T>
static size_t size_all(const Opts& o, bool tc, int64_t m, int64_t n, int k, int p, int want) {
  Ctx c;
  c.dry = true;
  run_all<T>(c, o, tc, m, n, k, p, 0, 0, nullptr, 0, want, nullptr, 0, nullptr, 0, nullptr, 0,
             nullptr, nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, nullptr, 0);
  return c.off + 256;
}

static size_t ws_query(int64_t m, int64_t n, int k, int p, int q, int dtype,
                       const rsvd_opts* opts, int want) {
  Opts o;
  if (!read_opts(opts, &o) || !base_args_ok(m, n, k, p, q, dtype)) return 0;
  const bool tc = want_tc(dtype, o, k + p, nullptr, 0);
  if (dtype == RSVD_F64) return size_all<double>(o, false, m, n, k, p, want);
  if (dtype == RSVD_BF16) return tc ? size_all<float>(o, true, m, n, k, p, want) : 0;
  // Both variants may be chosen at call time (alignment of A): report the max.
  size_t s1 = size_all<float>(o, false, m, n, k, p, want);
  size_t s2 = tc ? size_all<float>(o, true, m, n, k, p, want) : 0;
  return s1 > s2 ? s1 : s2;
}

static int d_abf(int dtype) { return dtype == RSVD_BF16 ? 1 : 0; }

static rsvd_status dispatch(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                            const void* A, int64_t lda, int want, void* Qo, int64_t ldq,
                            void* Bto, int64_t ldbt, void* U, int64_t ldu, double* S, void* V,
                            int64_t ldv, int32_t* J, void* Tout, int64_t ldt, int32_t* Jc,
                            int32_t* Ir, void* Ucur, int64_t lducur, void* work,
                            size_t work_bytes, int* d_info, void* stream,
                            const rsvd_opts* opts, const void* A_host = nullptr) {
  Opts o;
  if (!read_opts(opts, &o)) return RSVD_ERR_INVALID_ARG;
  if (!base_args_ok(m, n, k, p, q, dtype)) return RSVD_ERR_INVALID_ARG;
  if (!A || lda < n) return RSVD_ERR_INVALID_ARG;
  const int l = k + p;
  if ((want & W_Q) && ((Qo && ldq < l) || (Bto && ldbt < l) || (!Qo && !Bto)))
    return RSVD_ERR_INVALID_ARG;
  if ((want & W_SVD) && (!U || !S || !V || ldu < k || ldv < k)) return RSVD_ERR_INVALID_ARG;
  if ((want & W_ID) && (k >= n) ) return RSVD_ERR_INVALID_ARG;
  if (want & W_ID) {
    if (!J && !Tout) return RSVD_ERR_INVALID_ARG;
    if (Tout && ldt < n - k) return RSVD_ERR_INVALID_ARG;
  }
  if ((want & W_CUR) && (!Jc || !Ir || !Ucur || lducur < k || k >= n || k >= m))
    return RSVD_ERR_INVALID_ARG;
  if ((want & (W_ID | W_CUR)) && k > UPPER_SOLVE_MAX_K) return RSVD_ERR_UNSUPPORTED;
  if (!work && work_bytes) return RSVD_ERR_INVALID_ARG;
  if (work && !aligned16(work)) return RSVD_ERR_INVALID_ARG;
  Ctx c;
  c.dry = false;
  c.base = (char*)work;
  c.cap = work_bytes;
  c.stream = (cudaStream_t)stream;
  c.d_info = d_info;
  rsvd_status st;
  if (dtype == RSVD_F64) {
    // workspace check first (dry pass with the same carving)
    Ctx d;
    run_all<double>(d, o, false, m, n, k, p, q, seed, nullptr, lda, want, nullptr, 0, nullptr, 0,
                    nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr,
                    nullptr, 0);
    if (d.off > work_bytes) return RSVD_ERR_WORKSPACE;
    st = run_all<double>(c, o, false, m, n, k, p, q, seed, (const double*)A, lda, want,
                         (double*)Qo, ldq, (double*)Bto, ldbt, (double*)U, ldu, S, (double*)V,
                         ldv, J, (double*)Tout, ldt, Jc, Ir, (double*)Ucur, lducur,
                         (const double*)A_host);
  } else {
    const bool tc = want_tc(dtype, o, l, A, lda);
    // bf16 A runs on the tensor-core path only (its SIMT kernels read fp32)
    if (dtype == RSVD_BF16 && !tc) return RSVD_ERR_UNSUPPORTED;
    c.abf = d_abf(dtype);
    Ctx d;
    d.abf = c.abf;
    run_all<float>(d, o, tc, m, n, k, p, q, seed, nullptr, lda, want, nullptr, 0, nullptr, 0,
                   nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr,
                   nullptr, 0);
    if (d.off > work_bytes) return RSVD_ERR_WORKSPACE;
    st = run_all<float>(c, o, tc, m, n, k, p, q, seed, (const float*)A, lda, want, (float*)Qo,
                        ldq, (float*)Bto, ldbt, (float*)U, ldu, S, (float*)V, ldv, J,
                        (float*)Tout, ldt, Jc, Ir, (float*)Ucur, lducur, (const float*)A_host);
  }
  if (st == RSVD_OK && c.err != cudaSuccess) st = RSVD_ERR_CUDA;
  return st;
}

// ------------------------------------------------------------------------
// blocked adaptive QB to a tolerance (Alg. 7)
// ------------------------------------------------------------------------
// Reads a device value into host memory; the stream is synchronised.
static bool read_back(Ctx& c, const void* src, void* dst, size_t bytes) {
  if (!c.run(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c.stream))) return false;
  return c.run(cudaStreamSynchronize(c.stream));
}

template <typename T>
static rsvd_status run_qb_adaptive(Ctx& c, const Opts& o, bool tc, int64_t m, int64_t n, int bs,
                                   int M, int q, double eps, int relative, uint64_t seed, T* A,
                                   int64_t lda, T* Qo, int64_t ldq, T* Bto, int64_t ldbt,
                                   double* resid, int* rank) {
  Engine<T> e(c, o, tc);
  const int L = padL(bs);
  auto qbb = e.take_qb(m, n, L);
  // re-projection scratch: Ct (b x b(M-1)) and the split-K slabs of its product
  const int64_t cmax = (int64_t)bs * (M - 1);
  size_t se = 0;
  for (int t = 1; t < M; ++t) {
    int ns;
    int64_t kc;
    tn_split(bs, (int64_t)bs * t, m, e.sms, &ns, &kc);
    se = std::max(se, (size_t)ns * bs * bs * t);
  }
  T* Ct = cmax > 0 ? c.template take<T>((size_t)bs * cmax) : nullptr;
  T* cslabs = se ? c.template take<T>(se) : nullptr;
  const int64_t ntiles = rank_update_tiles(m, n);
  double* sq = c.template take<double>((size_t)ntiles);
  if (c.dry) return RSVD_OK;
  if (c.off > c.cap) return RSVD_ERR_WORKSPACE;

  reset_info(c);
  *rank = 0;
  // resid[0] = ||A_in||_F (a read-only pass: K = 0)
  LK(launch_rank_update<T>(m, n, A, lda, nullptr, 0, nullptr, 0, 0, sq, c.stream));
  LK(launch_sumsq_finish(ntiles, sq, resid, c.d_info, c.stream));
  double tol = eps;
  if (relative) {
    double a0 = 0.0;
    if (!read_back(c, resid, &a0, sizeof(double))) return RSVD_ERR_CUDA;
    tol = eps * a0;
  }
  for (int t = 0; t < M; ++t) {
    const int64_t done = (int64_t)bs * t;
    rsvd_status st = e.qb2_block(qbb, m, n, bs, q, seed + (uint64_t)t, A, lda, Qo, ldq, Bto,
                                 ldbt, done, Ct, cslabs, sq);
    if (st != RSVD_OK) return st;
    LK(launch_sumsq_finish(ntiles, sq, resid + t + 1, c.d_info, c.stream));
    *rank = (int)(done + bs);
    // the stopping test of Alg. 7 needs the residual norm on the host
    double r = 0.0;
    int info = 0;
    if (!read_back(c, resid + t + 1, &r, sizeof(double))) return RSVD_ERR_CUDA;
    if (c.d_info && !read_back(c, c.d_info, &info, sizeof(int))) return RSVD_ERR_CUDA;
    if (info != 0 || r < tol) break;
  }
  return RSVD_OK;
}

static bool qb_adaptive_args_ok(int64_t m, int64_t n, int bs, int M, int q, int dtype) {
  if (dtype != RSVD_F32 && dtype != RSVD_F64) return false;
  if (m < 1 || n < 1 || m > 0x7fffffffLL || n > 0x7fffffffLL) return false;
  if (bs < 1 || bs > 1024 || M < 1 || q < 0 || q > 64) return false;
  const int64_t cols = (int64_t)bs * M;
  return cols <= m && cols <= n;
}

template <typename T>
static size_t size_qb_adaptive(const Opts& o, bool tc, int64_t m, int64_t n, int bs, int M) {
  Ctx c;
  c.dry = true;
  int rank = 0;
  run_qb_adaptive<T>(c, o, tc, m, n, bs, M, 0, 0.0, 0, 0, nullptr, 0, nullptr, 0, nullptr, 0,
                     nullptr, &rank);
  return c.off + 256;
}

}  // namespace rsvd

using namespace rsvd;

extern "C" {

void rsvd_opts_default(rsvd_opts* opts) {
  if (!opts) return;
  std::memset(opts, 0, sizeof(*opts));
  opts->s = 1;
  opts->max_sweeps = 30;
  opts->precision = RSVD_PREC_TC;
}

const char* rsvd_status_string(int status) {
  switch (status) {
    case RSVD_OK: return "RSVD_OK";
    case RSVD_ERR_INVALID_ARG: return "RSVD_ERR_INVALID_ARG";
    case RSVD_ERR_WORKSPACE: return "RSVD_ERR_WORKSPACE";
    case RSVD_ERR_CUDA: return "RSVD_ERR_CUDA";
    case RSVD_ERR_UNSUPPORTED: return "RSVD_ERR_UNSUPPORTED";
    case RSVD_ERR_NOT_SPD: return "RSVD_ERR_NOT_SPD";
    case RSVD_ERR_NO_CONVERGENCE: return "RSVD_ERR_NO_CONVERGENCE";
    case RSVD_ERR_NUMERIC: return "RSVD_ERR_NUMERIC";
    case RSVD_ERR_TIMEOUT: return "RSVD_ERR_TIMEOUT";
    default: return "RSVD_ERR_UNKNOWN";
  }
}

int rsvd_version(void) { return 100; }

size_t rsvd_qb_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                              const rsvd_opts* opts) {
  return ws_query(m, n, k, p, q, dtype, opts, W_Q);
}
size_t rsvd_svd_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                               const rsvd_opts* opts) {
  return ws_query(m, n, k, p, q, dtype, opts, W_SVD);
}
size_t rsvd_id_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                              const rsvd_opts* opts) {
  if (k >= n) return 0;
  return ws_query(m, n, k, p, q, dtype, opts, W_ID);
}
size_t rsvd_cur_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                               const rsvd_opts* opts) {
  if (k >= n || k >= m) return 0;
  return ws_query(m, n, k, p, q, dtype, opts, W_ID | W_CUR);
}
size_t rsvd_svd_id_cur_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                                      const rsvd_opts* opts) {
  if (k >= n || k >= m) return 0;
  return ws_query(m, n, k, p, q, dtype, opts, W_SVD | W_ID | W_CUR);
}

rsvd_status rsvd_qb(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                    const void* A, int64_t lda, void* Q, int64_t ldq, void* Bt, int64_t ldbt,
                    void* work, size_t work_bytes, int* d_info, void* stream,
                    const rsvd_opts* opts) {
  return dispatch(m, n, k, p, q, seed, dtype, A, lda, W_Q, Q, ldq, Bt, ldbt, nullptr, 0, nullptr,
                  nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, nullptr, 0, work,
                  work_bytes, d_info, stream, opts);
}

rsvd_status rsvd_svd(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                     const void* A, int64_t lda, void* U, int64_t ldu, double* S, void* V,
                     int64_t ldv, void* work, size_t work_bytes, int* d_info, void* stream,
                     const rsvd_opts* opts) {
  return dispatch(m, n, k, p, q, seed, dtype, A, lda, W_SVD, nullptr, 0, nullptr, 0, U, ldu, S, V,
                  ldv, nullptr, nullptr, 0, nullptr, nullptr, nullptr, 0, work, work_bytes,
                  d_info, stream, opts);
}

rsvd_status rsvd_id(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                    const void* A, int64_t lda, int32_t* J, void* T, int64_t ldt, void* work,
                    size_t work_bytes, int* d_info, void* stream, const rsvd_opts* opts) {
  return dispatch(m, n, k, p, q, seed, dtype, A, lda, W_ID, nullptr, 0, nullptr, 0, nullptr, 0,
                  nullptr, nullptr, 0, J, T, ldt, nullptr, nullptr, nullptr, 0, work, work_bytes,
                  d_info, stream, opts);
}

rsvd_status rsvd_cur(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                     const void* A, int64_t lda, int32_t* Jc, int32_t* Ir, void* U, int64_t ldu,
                     void* work, size_t work_bytes, int* d_info, void* stream,
                     const rsvd_opts* opts) {
  return dispatch(m, n, k, p, q, seed, dtype, A, lda, W_ID | W_CUR, nullptr, 0, nullptr, 0,
                  nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, 0, Jc, Ir, U, ldu, work,
                  work_bytes, d_info, stream, opts);
}

rsvd_status rsvd_svd_id_cur(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                            const void* A, int64_t lda, void* U, int64_t ldu, double* S, void* V,
                            int64_t ldv, int32_t* J, void* T, int64_t ldt, int32_t* Jc,
                            int32_t* Ir, void* Ucur, int64_t lducur, void* work,
                            size_t work_bytes, int* d_info, void* stream,
                            const rsvd_opts* opts) {
  int want = 0;
  if (U || S || V) want |= W_SVD;
  if (J || T) want |= W_ID;
  if (Jc || Ir || Ucur) want |= W_ID | W_CUR;
  if (!want) return RSVD_ERR_INVALID_ARG;
  return dispatch(m, n, k, p, q, seed, dtype, A, lda, want, nullptr, 0, nullptr, 0, U, ldu, S, V,
                  ldv, J, T, ldt, Jc, Ir, Ucur, lducur, work, work_bytes, d_info, stream, opts);
}

rsvd_status rsvd_svd_id_cur_host(int64_t m, int64_t n, int k, int p, int q, uint64_t seed,
                                 int dtype, const void* A_host, void* A, int64_t lda, void* U,
                                 int64_t ldu, double* S, void* V, int64_t ldv, int32_t* J,
                                 void* T, int64_t ldt, int32_t* Jc, int32_t* Ir, void* Ucur,
                                 int64_t lducur, void* work, size_t work_bytes, int* d_info,
                                 void* stream, const rsvd_opts* opts) {
  if (!A_host) return RSVD_ERR_INVALID_ARG;
  int want = 0;
  if (U || S || V) want |= W_SVD;
  if (J || T) want |= W_ID;
  if (Jc || Ir || Ucur) want |= W_ID | W_CUR;
  if (!want) return RSVD_ERR_INVALID_ARG;
  return dispatch(m, n, k, p, q, seed, dtype, A, lda, want, nullptr, 0, nullptr, 0, U, ldu, S, V,
                  ldv, J, T, ldt, Jc, Ir, Ucur, lducur, work, work_bytes, d_info, stream, opts,
                  A_host);
}

size_t rsvd_qb_adaptive_workspace_size(int64_t m, int64_t n, int b, int M, int q, int dtype,
                                       const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !qb_adaptive_args_ok(m, n, b, M, q, dtype)) return 0;
  if (dtype == RSVD_F64) return size_qb_adaptive<double>(o, false, m, n, b, M);
  const bool tc = want_tc(dtype, o, b, nullptr, 0);
  size_t s1 = size_qb_adaptive<float>(o, false, m, n, b, M);
  size_t s2 = tc ? size_qb_adaptive<float>(o, true, m, n, b, M) : 0;
  return s1 > s2 ? s1 : s2;
}

rsvd_status rsvd_qb_adaptive(int64_t m, int64_t n, int b, int M, int q, double eps, int relative,
                             uint64_t seed, int dtype, void* A, int64_t lda, void* Q, int64_t ldq,
                             void* Bt, int64_t ldbt, double* resid, int* rank, void* work,
                             size_t work_bytes, int* d_info, void* stream,
                             const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o)) return RSVD_ERR_INVALID_ARG;
  if (dtype == RSVD_BF16) return RSVD_ERR_UNSUPPORTED;
  if (!qb_adaptive_args_ok(m, n, b, M, q, dtype)) return RSVD_ERR_INVALID_ARG;
  if (!(eps >= 0.0) || eps > 1e300) return RSVD_ERR_INVALID_ARG;   // also rejects NaN
  const int64_t cols = (int64_t)b * M;
  if (!A || !Q || !Bt || !resid || !rank) return RSVD_ERR_INVALID_ARG;
  if (lda < n || ldq < cols || ldbt < cols) return RSVD_ERR_INVALID_ARG;
  if (!work && work_bytes) return RSVD_ERR_INVALID_ARG;
  if (work && !aligned16(work)) return RSVD_ERR_INVALID_ARG;
  Ctx c;
  c.dry = false;
  c.base = (char*)work;
  c.cap = work_bytes;
  c.stream = (cudaStream_t)stream;
  c.d_info = d_info;
  rsvd_status st;
  if (dtype == RSVD_F64) {
    if (size_qb_adaptive<double>(o, false, m, n, b, M) - 256 > work_bytes)
      return RSVD_ERR_WORKSPACE;
    st = run_qb_adaptive<double>(c, o, false, m, n, b, M, q, eps, relative, seed, (double*)A, lda,
                                 (double*)Q, ldq, (double*)Bt, ldbt, resid, rank);
  } else {
    const bool tc = want_tc(dtype, o, b, A, lda);
    if (size_qb_adaptive<float>(o, tc, m, n, b, M) - 256 > work_bytes) return RSVD_ERR_WORKSPACE;
    st = run_qb_adaptive<float>(c, o, tc, m, n, b, M, q, eps, relative, seed, (float*)A, lda,
                                (float*)Q, ldq, (float*)Bt, ldbt, resid, rank);
  }
  if (st == RSVD_OK && c.err != cudaSuccess) st = RSVD_ERR_CUDA;
  return st;
}

}  // extern "C"

// ==========================================================================
// Step-level entry points
// ==========================================================================
namespace rsvd {

static bool dtype_ok(int dtype) { return dtype == RSVD_F32 || dtype == RSVD_F64; }
// The passes over A (sample, apply) also take bf16 A, on the tensor-core path.
static bool a_dtype_ok(int dtype) { return dtype_ok(dtype) || dtype == RSVD_BF16; }

template <typename T>
static rsvd_status sample_impl(Ctx& c, const Opts& o, bool tc, int64_t m, int64_t n, int l,
                               uint64_t seed, const T* A, int64_t lda, T* Y, int64_t ldy) {
  Engine<T> e(c, o, tc);
  const int L = padL(l);
  float* part = tc ? c.template take<float>(tc_part_bytes(m, n, L) / sizeof(float)) : nullptr;
  if (c.dry) return RSVD_OK;
  if (c.off > c.cap) return RSVD_ERR_WORKSPACE;
  return e.gemm_n(m, n, L, A, lda, m, n, true, seed, l, nullptr, nullptr, 0, Y, ldy, l, nullptr,
                  part, nullptr, c.abf != 0);
}

template <typename T>
static rsvd_status apply_impl(Ctx& c, const Opts& o, bool tc, int64_t m, int64_t n, int l,
                              int trans, const T* A, int64_t lda, const T* X, int64_t ldx, T* Y,
                              int64_t ldy) {
  Engine<T> e(c, o, tc);
  const int L = padL(l);
  const int64_t K = trans ? m : n;
  const int64_t rows = trans ? n : m;
  typename Engine<T>::Split w{};
  float* part = nullptr;
  T* slabs = nullptr;
  if (tc) {
    w = e.take_split(L, K);
    part = c.template take<float>(tc_part_bytes(rows, K, L) / sizeof(float));
  } else if (trans) {
    slabs = c.template take<T>(e.slab_elems_t(rows, K, l));
  }
  if (c.dry) return RSVD_OK;
  if (c.off > c.cap) return RSVD_ERR_WORKSPACE;
  if (tc) LK(launch_split_transpose(K, l, L, (const float*)X, ldx, w.hi, w.lo, w.ld, c.stream));
  if (!trans)
    return e.gemm_n(rows, K, L, A, lda, m, n, false, 0, L, &w, X, ldx, Y, ldy, l, nullptr, part,
                    nullptr, c.abf != 0);
  return e.gemm_t(rows, K, L, A, lda, &w, X, ldx, Y, ldy, l, nullptr, part, slabs, nullptr, false,
                  c.abf != 0);
}

template <typename T>
static rsvd_status orth_impl(Ctx& c, const Opts& o, bool tc, int64_t rows, int l, const T* X,
                             int64_t ldx, T* Q, int64_t ldq, T* R, int64_t ldr) {
  Engine<T> e(c, o, tc);
  const int L = padL(l);
  T* Xb = c.template take<T>((size_t)rows * L);
  T* Yb = c.template take<T>((size_t)rows * L);
  typename Engine<T>::Split sp{};
  float* part = nullptr;
  T* slabs = nullptr;
  if (tc) {
    sp = e.take_split(L, rows);
    size_t pb = std::max(tc_part_bytes(L, rows, L), tc_part_bytes(rows, L, L));
    part = c.template take<float>(pb / sizeof(float));
  } else {
    slabs = c.template take<T>(e.slab_elems_t(L, rows, L));
  }
  auto ob = e.take_orth_bufs(L);
  if (c.dry) return RSVD_OK;
  if (c.off > c.cap) return RSVD_ERR_WORKSPACE;
  LK(cudaMemsetAsync(Xb, 0, sizeof(T) * rows * L, c.stream));
  LK(launch_copy2d<T, T>(rows, l, X, ldx, Xb, L, c.stream));
  if (tc) LK(launch_split_transpose(rows, L, L, (const float*)Xb, L, sp.hi, sp.lo, sp.ld, c.stream));
  rsvd_status st = e.orth(rows, l, L, Xb, Yb, &sp, ob, part, slabs, R != nullptr);
  if (st != RSVD_OK) return st;
  LK(launch_copy2d<T, T>(rows, l, Yb, L, Q, ldq, c.stream));
  if (R) LK(launch_copy2d<T, T>(l, l, ob.Racc, L, R, ldr, c.stream));
  return RSVD_OK;
}

template <typename T>
static rsvd_status small_svd_impl(Ctx& c, const Opts& o, int l, const T* M, int64_t ldm, T* Uh,
                                  int64_t lduh, double* Sh, T* Vh, int64_t ldvh) {
  Engine<T> e(c, o, false);
  auto sb = e.take_svd(l, padL(l), 1);
  if (c.dry) return RSVD_OK;
  if (c.off > c.cap) return RSVD_ERR_WORKSPACE;
  return e.small_svd(l, M, ldm, sb, Uh, lduh, Sh, Vh, ldvh);
}

// Column ID of an explicit r x n matrix: FP64 arithmetic for double M, the
// double-float kernel (as on the FP32 path) for float M.
template <typename T>
static rsvd_status cpqr_impl(Ctx& c, int r, int64_t n, int k, const T* M, int64_t ldm,
                             int32_t* J, T* Tout, int64_t ldt, double* gaps) {
  Opts o;
  Engine<T> e(c, o, false);
  auto idb = e.take_id(r, n, k, true);
  if (c.dry) return RSVD_OK;
  if (c.off > c.cap) return RSVD_ERR_WORKSPACE;
  if (sizeof(T) == 4) {
    float* Wh = reinterpret_cast<float*>(idb.W);
    LK(launch_transpose<float, float>(r, n, (const float*)M, ldm, Wh, r, c.stream));
    LK(cudaMemsetAsync(Wh + (int64_t)r * n, 0, sizeof(float) * (size_t)r * n, c.stream));
  } else {
    LK(launch_copy2d<double, double>(r, n, (const double*)M, ldm, idb.W, n, c.stream));
  }
  rsvd_status st = e.id_core(idb, r, n, k, gaps);
  if (st != RSVD_OK) return st;
  LK(launch_copy_i32(n, idb.J, J, c.stream));
  if (Tout && n > k) LK(launch_transpose<T, T>(n - k, k, idb.Tt, k, Tout, ldt, c.stream));
  return RSVD_OK;
}

static Ctx make_ctx(void* work, size_t bytes, int* d_info, void* stream) {
  Ctx c;
  c.dry = false;
  c.base = (char*)work;
  c.cap = bytes;
  c.d_info = d_info;
  c.stream = (cudaStream_t)stream;
  return c;
}

static rsvd_status finish(Ctx& c, rsvd_status st) {
  if (st == RSVD_OK && c.err != cudaSuccess) return RSVD_ERR_CUDA;
  return st;
}

}  // namespace rsvd

extern "C" {

rsvd_status rsvd_omega(int64_t n, int l, uint64_t seed, int dtype, void* Omega, int64_t ldo,
                       void* stream) {
  if (!dtype_ok(dtype) || n < 1 || l < 1 || !Omega || ldo < l) return RSVD_ERR_INVALID_ARG;
  if (n > 0xffffffffLL) return RSVD_ERR_INVALID_ARG;
  cudaError_t e = (dtype == RSVD_F64)
                      ? launch_omega<double>(n, l, seed, (double*)Omega, ldo, (cudaStream_t)stream)
                      : launch_omega<float>(n, l, seed, (float*)Omega, ldo, (cudaStream_t)stream);
  return e == cudaSuccess ? RSVD_OK : RSVD_ERR_CUDA;
}

rsvd_status rsvd_omega_words(int64_t n, int l, uint64_t seed, uint32_t* out, void* stream) {
  if (n < 1 || l < 1 || !out || ((uintptr_t)out & 15u)) return RSVD_ERR_INVALID_ARG;
  if (n > 0xffffffffLL) return RSVD_ERR_INVALID_ARG;
  return launch_omega_words(n, l, seed, out, (cudaStream_t)stream) == cudaSuccess ? RSVD_OK
                                                                                 : RSVD_ERR_CUDA;
}

static bool sizes_ok(int64_t m, int64_t n, int l) {
  return m >= 1 && n >= 1 && l >= 1 && l <= 1024 && m <= 0x7fffffffLL && n <= 0x7fffffffLL;
}

size_t rsvd_sample_workspace_size(int64_t m, int64_t n, int l, int dtype, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !a_dtype_ok(dtype) || !sizes_ok(m, n, l)) return 0;
  Ctx c;
  const bool tc = want_tc(dtype, o, l, nullptr, 0);
  if (dtype == RSVD_BF16 && !tc) return 0;
  if (dtype == RSVD_F64)
    sample_impl<double>(c, o, false, m, n, l, 0, nullptr, n, nullptr, l);
  else
    sample_impl<float>(c, o, tc, m, n, l, 0, nullptr, n, nullptr, l);
  return c.off + 256;
}

rsvd_status rsvd_sample(int64_t m, int64_t n, int l, uint64_t seed, int dtype, const void* A,
                        int64_t lda, void* Y, int64_t ldy, void* work, size_t work_bytes,
                        void* stream, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !a_dtype_ok(dtype) || !sizes_ok(m, n, l))
    return RSVD_ERR_INVALID_ARG;
  if (!A || !Y || lda < n || ldy < l) return RSVD_ERR_INVALID_ARG;
  if (work && ((uintptr_t)work & 15u)) return RSVD_ERR_INVALID_ARG;
  Ctx c = make_ctx(work, work_bytes, nullptr, stream);
  rsvd_status st;
  if (dtype == RSVD_F64) {
    st = sample_impl<double>(c, o, false, m, n, l, seed, (const double*)A, lda, (double*)Y, ldy);
  } else {
    const bool tc = want_tc(dtype, o, l, A, lda);
    if (dtype == RSVD_BF16 && !tc) return RSVD_ERR_UNSUPPORTED;
    c.abf = dtype == RSVD_BF16 ? 1 : 0;
    st = sample_impl<float>(c, o, tc, m, n, l, seed, (const float*)A, lda, (float*)Y, ldy);
  }
  return finish(c, st);
}

size_t rsvd_apply_workspace_size(int64_t m, int64_t n, int l, int dtype, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !a_dtype_ok(dtype) || !sizes_ok(m, n, l)) return 0;
  if (dtype == RSVD_BF16 && !want_tc(dtype, o, l, nullptr, 0)) return 0;
  size_t best = 0;
  for (int trans = 0; trans < 2; ++trans) {
    Ctx c;
    const bool tc = want_tc(dtype, o, l, nullptr, 0);
    if (dtype == RSVD_F64)
      apply_impl<double>(c, o, false, m, n, l, trans, nullptr, n, nullptr, l, nullptr, l);
    else {
      apply_impl<float>(c, o, tc, m, n, l, trans, nullptr, n, nullptr, l, nullptr, l);
      Ctx c2;
      apply_impl<float>(c2, o, false, m, n, l, trans, nullptr, n, nullptr, l, nullptr, l);
      best = std::max(best, c2.off);
    }
    best = std::max(best, c.off);
  }
  return best + 256;
}

rsvd_status rsvd_apply(int64_t m, int64_t n, int l, int trans, int dtype, const void* A,
                       int64_t lda, const void* X, int64_t ldx, void* Y, int64_t ldy, void* work,
                       size_t work_bytes, void* stream, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !a_dtype_ok(dtype) || !sizes_ok(m, n, l))
    return RSVD_ERR_INVALID_ARG;
  if (trans != 0 && trans != 1) return RSVD_ERR_INVALID_ARG;
  if (!A || !X || !Y || lda < n || ldx < l || ldy < l) return RSVD_ERR_INVALID_ARG;
  if (work && ((uintptr_t)work & 15u)) return RSVD_ERR_INVALID_ARG;
  Ctx c = make_ctx(work, work_bytes, nullptr, stream);
  rsvd_status st;
  if (dtype == RSVD_F64) {
    st = apply_impl<double>(c, o, false, m, n, l, trans, (const double*)A, lda, (const double*)X,
                            ldx, (double*)Y, ldy);
  } else {
    const bool tc = want_tc(dtype, o, l, A, lda);
    if (dtype == RSVD_BF16 && !tc) return RSVD_ERR_UNSUPPORTED;
    c.abf = dtype == RSVD_BF16 ? 1 : 0;
    st = apply_impl<float>(c, o, tc, m, n, l, trans, (const float*)A, lda, (const float*)X, ldx,
                           (float*)Y, ldy);
  }
  return finish(c, st);
}

size_t rsvd_orth_workspace_size(int64_t rows, int l, int dtype, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !dtype_ok(dtype) || !sizes_ok(rows, l, l) || rows < l) return 0;
  Ctx c, c2;
  if (dtype == RSVD_F64) {
    orth_impl<double>(c, o, false, rows, l, nullptr, l, nullptr, l, nullptr, l);
  } else {
    const bool tc = want_tc(dtype, o, l, nullptr, 0);
    orth_impl<float>(c, o, tc, rows, l, nullptr, l, nullptr, l, nullptr, l);
    orth_impl<float>(c2, o, false, rows, l, nullptr, l, nullptr, l, nullptr, l);
  }
  return std::max(c.off, c2.off) + 256;
}

rsvd_status rsvd_orth(int64_t rows, int l, int dtype, const void* X, int64_t ldx, void* Q,
                      int64_t ldq, void* R, int64_t ldr, void* work, size_t work_bytes,
                      int* d_info, void* stream, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !dtype_ok(dtype) || !sizes_ok(rows, l, l) || rows < l)
    return RSVD_ERR_INVALID_ARG;
  if (!X || !Q || ldx < l || ldq < l || (R && ldr < l)) return RSVD_ERR_INVALID_ARG;
  if (work && ((uintptr_t)work & 15u)) return RSVD_ERR_INVALID_ARG;
  Ctx c = make_ctx(work, work_bytes, d_info, stream);
  reset_info(c);
  rsvd_status st;
  if (dtype == RSVD_F64) {
    st = orth_impl<double>(c, o, false, rows, l, (const double*)X, ldx, (double*)Q, ldq,
                           (double*)R, ldr);
  } else {
    const bool tc = want_tc(dtype, o, l, nullptr, 0);
    st = orth_impl<float>(c, o, tc, rows, l, (const float*)X, ldx, (float*)Q, ldq, (float*)R,
                          ldr);
  }
  return finish(c, st);
}

size_t rsvd_small_svd_workspace_size(int l, int dtype, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !dtype_ok(dtype) || l < 1 || l > 1024) return 0;
  Ctx c;
  if (dtype == RSVD_F64)
    small_svd_impl<double>(c, o, l, nullptr, l, nullptr, l, nullptr, nullptr, l);
  else
    small_svd_impl<float>(c, o, l, nullptr, l, nullptr, l, nullptr, nullptr, l);
  return c.off + 256;
}

rsvd_status rsvd_small_svd(int l, int dtype, const void* M, int64_t ldm, void* Uh, int64_t lduh,
                           double* Sh, void* Vh, int64_t ldvh, void* work, size_t work_bytes,
                           int* d_info, void* stream, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !dtype_ok(dtype) || l < 1 || l > 1024) return RSVD_ERR_INVALID_ARG;
  if (!M || !Uh || !Sh || !Vh || ldm < l || lduh < l || ldvh < l) return RSVD_ERR_INVALID_ARG;
  if (work && ((uintptr_t)work & 15u)) return RSVD_ERR_INVALID_ARG;
  Ctx c = make_ctx(work, work_bytes, d_info, stream);
  reset_info(c);
  rsvd_status st;
  if (dtype == RSVD_F64)
    st = small_svd_impl<double>(c, o, l, (const double*)M, ldm, (double*)Uh, lduh, Sh,
                                (double*)Vh, ldvh);
  else
    st = small_svd_impl<float>(c, o, l, (const float*)M, ldm, (float*)Uh, lduh, Sh, (float*)Vh,
                               ldvh);
  return finish(c, st);
}

size_t rsvd_cpqr_workspace_size(int r, int64_t n, int k) {
  if (r < 1 || n < 1 || k < 1 || k > r || k > n || r > 8192 || k > UPPER_SOLVE_MAX_K ||
      n > 0x7fffffffLL)
    return 0;
  Ctx c;
  cpqr_impl<double>(c, r, n, k, nullptr, n, nullptr, nullptr, 0, nullptr);
  return c.off + 256;
}

rsvd_status rsvd_cpqr_id(int r, int64_t n, int k, const double* M, int64_t ldm, int32_t* J,
                         double* T, int64_t ldt, double* gaps, void* work, size_t work_bytes,
                         int* d_info, void* stream) {
  if (r < 1 || n < 1 || k < 1 || k > r || k > n || r > 8192 || n > 0x7fffffffLL)
    return RSVD_ERR_INVALID_ARG;
  if (k > UPPER_SOLVE_MAX_K) return RSVD_ERR_UNSUPPORTED;
  if (!M || !J || ldm < n || (T && n > k && ldt < n - k)) return RSVD_ERR_INVALID_ARG;
  if (work && ((uintptr_t)work & 15u)) return RSVD_ERR_INVALID_ARG;
  Ctx c = make_ctx(work, work_bytes, d_info, stream);
  reset_info(c);
  return finish(c, cpqr_impl<double>(c, r, n, k, M, ldm, J, T, ldt, gaps));
}

size_t rsvd_cpqr_f32_workspace_size(int r, int64_t n, int k) {
  if (r < 1 || n < 1 || k < 1 || k > r || k > n || r > 8192 || k > UPPER_SOLVE_MAX_K ||
      n > 0x7fffffffLL)
    return 0;
  Ctx c;
  cpqr_impl<float>(c, r, n, k, nullptr, n, nullptr, nullptr, 0, nullptr);
  return c.off + 256;
}

rsvd_status rsvd_cpqr_id_f32(int r, int64_t n, int k, const float* M, int64_t ldm, int32_t* J,
                             float* T, int64_t ldt, double* gaps, void* work, size_t work_bytes,
                             int* d_info, void* stream) {
  if (r < 1 || n < 1 || k < 1 || k > r || k > n || r > 8192 || n > 0x7fffffffLL)
    return RSVD_ERR_INVALID_ARG;
  if (k > UPPER_SOLVE_MAX_K) return RSVD_ERR_UNSUPPORTED;
  if (!M || !J || ldm < n || (T && n > k && ldt < n - k)) return RSVD_ERR_INVALID_ARG;
  if (work && ((uintptr_t)work & 15u)) return RSVD_ERR_INVALID_ARG;
  Ctx c = make_ctx(work, work_bytes, d_info, stream);
  reset_info(c);
  return finish(c, cpqr_impl<float>(c, r, n, k, M, ldm, J, T, ldt, gaps));
}

}  // extern "C"
