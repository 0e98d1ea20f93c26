// The launch engine shared by the host-side entry points: options, the
// workspace arena (a bump allocator that also computes the workspace sizes by
// running without launching), the per-element-type sequences of the path
// (GEMM building blocks, CholeskyQR, the QB step with its power scheme, the
// left sketch, the small SVD, ID and CUR), and the argument checks.
#pragma once

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

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
        o->precision != RSVD_PREC_MIXED && o->precision != RSVD_PREC_FP8)
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
// K-chunks (of 32) per tensor-core accumulation run in the products whose scale
// matters (Bt = A^* Q): 2048 terms keep the accumulation's drift near 3e-6.
constexpr int kDrainQB = 64;
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

  // FP8 sketch (RSVD_PREC_FP8): the quantised Omega^T (L x omq_ld bf16),
  // generated once per call by the first sketch product.
  uint16_t* omq = nullptr;
  int64_t omq_ld = 0;
  bool omq_done = false;
  void take_omq(int64_t n, int L) {
    if (tc && o.precision == RSVD_PREC_FP8) {
      omq_ld = pad8(n);
      omq = c.template take<uint16_t>((size_t)L * omq_ld);
    }
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
    // the FP8 sketch exists on the tensor-core path only
    if (omega && o.precision == RSVD_PREC_FP8 && !tc) return RSVD_ERR_UNSUPPORTED;
    if (tc) {
      TcGemm g{};
      g.form = 0;
      g.a_bf16 = a_bf16 ? 1 : 0;
      g.omega = omega ? 1 : 0;
      if (omega && o.precision == RSVD_PREC_FP8) {
        // Y = q(A) q(Omega): A quantised by the GEMM's converters, Omega^T
        // quantised once into the workspace
        if (!omq && !c.dry) return RSVD_ERR_INVALID_ARG;
        if (!omq_done) {
          LK(launch_omega_fp8_t(K, lvalid, L, seed, omq, omq_ld, c.stream));
          omq_done = true;
        }
        g.omega = 0;
        g.q8 = 1;
        w = nullptr;
      }
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
      if (g.q8) {
        g.Whi = omq;
        g.Wlo = g.Wlo2 = nullptr;
        g.wterms = 1;
        g.ldw = omq_ld;
      }
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
  // drain > 0: the tensor-core accumulation runs hold at most `drain` K-chunks
  // of 32 (see tc_unit_kernel); used where the result's scale matters, not
  // only its span (the QB projection Bt = A^* Q).
  rsvd_status gemm_t(int64_t rows, int64_t K, int L, const T* A, int64_t lda, const Split* w,
                     const T* Wsimt, int64_t ldws, T* out, int64_t ldo, int ncols,
                     Split* out_split, float* part, T* slabs, const int* skip, bool gram = false,
                     bool a_bf16 = false, int drain = 0) {
    if (tc) {
      TcGemm g{};
      g.form = 1;
      g.drain = drain;
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
      // pass skipped: the previous Q carried over unchanged.  Inside the power
      // scheme a skipped second pass implies a skipped third one (only a
      // second pass that runs can ask for the third), and the two carries
      // Y -> X -> Y would cancel: the second pass copies nothing, and the third
      // copies only when the second one ran (flags[3] != 1).
      if (skip && tc && !(pass == 2 && !full)) {
        if (!c.dry) {
          const int* veto = (pass == 3 && !full) ? ob.flags + 3 : nullptr;
          if (!c.run(launch_cond_copy<float>(skip, veto, rows * (int64_t)L, (const float*)src,
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
    take_omq(n, L);
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
    // Bt = A^* Q (Alg. 5); its scale sets the singular values: bounded
    // accumulation runs
    st = gemm_t(n, m, L, A, lda, &b.ys, b.Y, L, b.Z, L, L, &b.zs, b.part, b.slabs, nullptr, false,
                c.abf != 0, kDrainQB);
    return st;
  }

  // ---------------- left sketch of the ID (Sec. 3.5, Alg. 6) ----------------
  // Y = Omega~ A (A^* A)^q with Omega~ l x m Gaussian (Philox tag 1, stored
  // transposed as the m x l right-hand operand), orthonormalising before every
  // product: Z = A^* Omega~^*; for j = 1..q: Y = A orth(Z), Z = A^* orth(Y).
  // On exit b.Z holds Y^* (n x L, padded).  The last orth before the last
  // product is a full CholeskyQR (orthonormal, like the oracle's Householder
  // Q); the earlier ones keep only the span, which is all the next product
  // needs.  Any orthonormal basis there changes Y by a left orthogonal factor,
  // which leaves the pivoted QR of Y (pivots, T) unchanged.
  rsvd_status power_left(QBBufs& b, int64_t m, int64_t n, int l, int q, uint64_t seed,
                         const T* A, int64_t lda) {
    const int L = padL(l);
    rsvd_status st;
    LK(launch_fill<T>(m, L, b.Ytmp, L, T(0), c.stream));
    LK(launch_omega<T>(m, l, seed, b.Ytmp, L, c.stream, 1u));
    Split om = b.ys;
    if (tc) {
      // the bf16-exact Gaussians: one term (lo is zero)
      LK(launch_split_transpose(m, l, L, (const float*)b.Ytmp, L, b.ys.hi, b.ys.lo, b.ys.ld,
                                c.stream));
      om.lo = nullptr;
    }
    if (!tc) LK(launch_fill<T>(n, L, b.Z, L, T(0), c.stream));
    st = gemm_t(n, m, L, A, lda, &om, b.Ytmp, L, b.Z, L, L, &b.zs, b.part, b.slabs, nullptr,
                false, c.abf != 0);
    if (st != RSVD_OK) return st;
    for (int j = 1; j <= q; ++j) {
      st = orth(n, l, L, b.Z, b.Ztmp, &b.zs, b.ob, b.part, b.slabs, false, false);
      if (st != RSVD_OK) return st;
      std::swap(b.Z, b.Ztmp);
      st = gemm_n(m, n, L, A, lda, m, n, false, 0, L, &b.zs, b.Z, L, b.Y, L, L, &b.ys, b.part,
                  nullptr, c.abf != 0);
      if (st != RSVD_OK) return st;
      st = orth(m, l, L, b.Y, b.Ytmp, &b.ys, b.ob, b.part, b.slabs, false, j == q);
      if (st != RSVD_OK) return st;
      std::swap(b.Y, b.Ytmp);
      st = gemm_t(n, m, L, A, lda, &b.ys, b.Y, L, b.Z, L, L, &b.zs, b.part, b.slabs, nullptr,
                  false, c.abf != 0);
      if (st != RSVD_OK) return st;
    }
    return RSVD_OK;
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
                false, false, kDrainQB);
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
    double* psum;    // 2 x 1024 per-CTA residual sums (tolerance mode)
    int* k_out;      // steps taken (tolerance mode)
  };
  // kmin < k: the T buffers also fit every rank in [kmin, k] (tolerance mode,
  // where the rank is known only after the pivoted QR)
  IdBufs take_id(int r, int64_t n, int k, bool with_T = true, int kmin = -1) {
    IdBufs d;
    d.psum = c.template take<double>(2 * 1024);
    d.k_out = c.template take<int>(1);
    d.W = c.template take<double>((size_t)n * r);
    d.where = c.template take<int64_t>((size_t)n);
    d.pval = c.template take<double>(2 * 1024 * 2);
    d.pidx = c.template take<int64_t>(2 * 1024);
    d.nrm = c.template take<double>((size_t)2 * n);
    d.diagR = c.template take<double>((size_t)k);
    d.bar = c.template take<unsigned>(4);
    d.J = c.template take<int32_t>((size_t)n);
    if (with_T) {
      size_t t12 = (size_t)(n - k) * k;
      for (int kk = kmin > 0 ? kmin : k; kk < k; ++kk)
        t12 = std::max(t12, (size_t)(n - kk) * kk);
      d.S11 = c.template take<double>((size_t)k * k + k);   // + diagonal reciprocals (df path)
      d.S12 = c.template take<double>(t12 + 1);
      d.Tt = c.template take<T>(t12 + 1);
    } else {
      d.S11 = nullptr;
      d.S12 = nullptr;
      d.Tt = nullptr;
    }
    return d;
  }

  // CPQR of the r x n row-major matrix in d.W (already filled), k steps; J
  // into d.J; Tt ((n-k) x k) = (S11^{-1} S12)^T.
  // Tolerance mode (tol > 0; Sec. 2.6): the factorisation stops at the first
  // j >= 1 with ||S22(j)||_F < tol, at the latest after k steps; the host
  // then reads the rank (one synchronisation) into *k_taken, which is 0 when a
  // device failure cut the factorisation short (the code is in d_info).
  rsvd_status id_core(IdBufs& d, int r, int64_t n, int k, double* gaps, double tol = 0.0,
                      int* k_taken = nullptr) {
    CpqrArgs a{};
    if (tol > 0.0) {
      a.tol2 = tol * tol;
      a.k_out = d.k_out;
      a.psum = d.psum;
      LK(cudaMemsetAsync(d.k_out, 0, sizeof(int), c.stream));
    }
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
    if (tol > 0.0 && !c.dry) {
      int kk = 0;
      if (!c.run(cudaMemcpyAsync(&kk, d.k_out, sizeof(int), cudaMemcpyDeviceToHost, c.stream)) ||
          !c.run(cudaStreamSynchronize(c.stream)))
        return RSVD_ERR_CUDA;
      *k_taken = (kk >= 1 && kk <= k) ? kk : 0;
      if (*k_taken == 0) return RSVD_OK;
      k = kk;
    }
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
  if (o.precision == RSVD_PREC_SIMT) return false;
  if (padL(l) > 1024) return false;   // widths above 256 run in column chunks
  if (A && !aligned16(A)) return false;
  if (lda % (dtype == RSVD_BF16 ? 8 : 4) != 0) return false;
  return true;
}

static void reset_info(Ctx& c) {
  if (c.d_info && !c.dry) c.run(cudaMemsetAsync(c.d_info, 0, sizeof(int), c.stream));
}

}  // namespace rsvd
