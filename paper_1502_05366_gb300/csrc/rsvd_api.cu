// C ABI of the library (include/rsvd.h) and the host-side launch sequences.
//
// Every entry point validates its arguments, carves the caller's workspace
// with a bump allocator (the same code computes the *_workspace_size values
// by running without launching), and enqueues kernels on the caller's stream.
// No device memory is allocated, and the host waits for the device only in the
// calls whose rank depends on the result (the tolerance modes and the adaptive
// QB), which read that rank back.  The
// combined SVD + ID/CUR call forks one kernel (the Jacobi SVD: an 8-CTA
// cluster for FP32 cores of 32 <= l <= 256, one CTA otherwise) onto an
// auxiliary stream and joins it back with events; that stream and its two
// events are created once per device on first use and kept until the process
// exits (a cudaDeviceReset invalidates them: do not call the library on that
// device afterwards).
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "engine.cuh"
#include "kernels.h"

namespace rsvd {


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

// ID and CUR to a tolerance (Sec. 2.6; Sec. 4 TOL mode) and the left-sketch ID
// (Sec. 3.5, Alg. 6).  The sketch is the QB step's B = Q^* A (l = kmax + p) or,
// with `left`, Y = Omega~ A (A^* A)^q; its pivoted QR runs k = kmax steps or,
// with tol > 0, stops at the first j >= 1 with ||S22(j)||_F < tol, and the host
// reads that rank back (one synchronisation).  The CUR buffers are carved once
// the rank is known; the dry run (workspace size) covers every rank <= kmax.
template <typename T>
static rsvd_status run_id_ext(Ctx& c, const Opts& o, bool tc, int64_t m, int64_t n, int kmax,
                              int p, int q, uint64_t seed, const T* A, int64_t lda, bool left,
                              double tol, int32_t* J, T* Tout, int64_t ldt, int32_t* Jc,
                              int32_t* Ir, T* Ucur, int64_t lducur, int* rank) {
  Engine<T> e(c, o, tc);
  const int l = kmax + p, L = padL(l);
  const bool want_cur = Jc != nullptr;
  auto qbb = e.take_qb(m, n, L);
  auto idb = e.take_id(l, n, kmax, true, tol > 0.0 ? 1 : kmax);
  if (c.dry) {
    if (want_cur) {
      const size_t base = c.off;
      size_t most = 0;
      for (int k = (tol > 0.0 ? 1 : kmax); k <= kmax; ++k) {
        c.off = base;
        e.take_cur(m, n, k);
        most = std::max(most, c.off);
      }
      c.off = most;
    }
    return RSVD_OK;
  }
  reset_info(c);
  rsvd_status st = left ? e.power_left(qbb, m, n, l, q, seed, A, lda)
                        : e.qb(qbb, m, n, l, q, seed, A, lda);
  if (st != RSVD_OK) return st;
  // the sketch (l x n) into the pivoted-QR layout: column c is row c of qbb.Z
  if (sizeof(T) == 4) {
    float* Wh = reinterpret_cast<float*>(idb.W);
    LK(launch_copy2d<float, float>(n, l, (const float*)qbb.Z, L, Wh, l, c.stream));
    LK(cudaMemsetAsync(Wh + (int64_t)l * n, 0, sizeof(float) * (size_t)l * n, c.stream));
  } else {
    LK(launch_transpose<T, double>(n, l, qbb.Z, L, idb.W, n, c.stream));
  }
  int k = kmax;
  st = e.id_core(idb, l, n, kmax, nullptr, tol, &k);
  if (st != RSVD_OK) return st;
  if (rank) *rank = k;
  if (k == 0) return RSVD_OK;            // a device failure, recorded in d_info
  if (J) LK(launch_copy_i32(n, idb.J, J, c.stream));
  if (Tout) LK(launch_transpose<T, T>(n - k, k, idb.Tt, k, Tout, ldt, c.stream));
  if (want_cur) {
    auto cb = e.take_cur(m, n, k);
    if (c.off > c.cap) return RSVD_ERR_WORKSPACE;
    st = e.cur_from_id(cb, idb, m, n, k, A, lda, Jc, Ir, Ucur, lducur, nullptr);
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
  if (o.precision == RSVD_PREC_FP8 && !tc) return 0;   // FP8 sketch: tensor cores only
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

// ID / CUR to a tolerance and the left-sketch ID: argument checks, workspace
// check by a dry run, then the launch sequence of run_id_ext.
static size_t ws_query_ext(int64_t m, int64_t n, int kmax, int p, int q, int dtype,
                           const rsvd_opts* opts, bool tolmode, bool cur, bool left) {
  Opts o;
  if (!read_opts(opts, &o) || !base_args_ok(m, n, kmax, p, q, dtype)) return 0;
  if (kmax >= n || (cur && kmax >= m) || kmax > UPPER_SOLVE_MAX_K) return 0;
  const double tol = tolmode ? 1.0 : 0.0;
  int32_t* jc = cur ? reinterpret_cast<int32_t*>(16) : nullptr;   // only tested for null
  auto one = [&](bool tc, auto tag) -> size_t {
    using T = decltype(tag);
    Ctx c;
    c.dry = true;
    c.abf = dtype == RSVD_BF16 ? 1 : 0;
    run_id_ext<T>(c, o, tc, m, n, kmax, p, q, 0, nullptr, n, left, tol, nullptr, nullptr, 0,
                  jc, nullptr, nullptr, 0, nullptr);
    return c.off + 256;
  };
  const bool tc = want_tc(dtype, o, kmax + p, nullptr, 0);
  if (o.precision == RSVD_PREC_FP8 && !tc) return 0;   // FP8 sketch: tensor cores only
  if (dtype == RSVD_F64) return one(false, double{});
  if (dtype == RSVD_BF16) return tc ? one(true, float{}) : 0;
  const size_t s1 = one(false, float{});
  const size_t s2 = tc ? one(true, float{}) : 0;
  return s1 > s2 ? s1 : s2;
}

static rsvd_status dispatch_ext(int64_t m, int64_t n, int kmax, int p, int q, double tol,
                                uint64_t seed, int dtype, const void* A, int64_t lda, bool left,
                                int32_t* J, void* Tout, int64_t ldt, int32_t* Jc, int32_t* Ir,
                                void* Ucur, int64_t lducur, int* rank, void* work,
                                size_t work_bytes, int* d_info, void* stream,
                                const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o)) return RSVD_ERR_INVALID_ARG;
  if (!base_args_ok(m, n, kmax, p, q, dtype)) return RSVD_ERR_INVALID_ARG;
  if (!A || lda < n || kmax >= n) return RSVD_ERR_INVALID_ARG;
  const bool tolmode = tol > 0.0;
  if (tol < 0.0 || !(tol < 1e300) || (tolmode && !rank)) return RSVD_ERR_INVALID_ARG;
  const bool cur = Jc != nullptr;
  if (cur && (!Ir || !Ucur || lducur < kmax || kmax >= m)) return RSVD_ERR_INVALID_ARG;
  if (!cur && !J && !Tout) return RSVD_ERR_INVALID_ARG;
  if (Tout && ldt < (tolmode ? n - 1 : n - kmax)) return RSVD_ERR_INVALID_ARG;
  if (kmax > UPPER_SOLVE_MAX_K) return RSVD_ERR_UNSUPPORTED;
  if (!work && work_bytes) return RSVD_ERR_INVALID_ARG;
  if (work && !aligned16(work)) return RSVD_ERR_INVALID_ARG;
  const size_t need = ws_query_ext(m, n, kmax, p, q, dtype, opts, tolmode, cur, left);
  if (need == 0) return RSVD_ERR_INVALID_ARG;
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  Ctx c;
  c.dry = false;
  c.base = (char*)work;
  c.cap = work_bytes;
  c.stream = (cudaStream_t)stream;
  c.d_info = d_info;
  rsvd_status st;
  if (dtype == RSVD_F64) {
    st = run_id_ext<double>(c, o, false, m, n, kmax, p, q, seed, (const double*)A, lda, left, tol,
                            J, (double*)Tout, ldt, Jc, Ir, (double*)Ucur, lducur, rank);
  } else {
    const bool tc = want_tc(dtype, o, kmax + p, A, lda);
    if (dtype == RSVD_BF16 && !tc) return RSVD_ERR_UNSUPPORTED;
    c.abf = d_abf(dtype);
    st = run_id_ext<float>(c, o, tc, m, n, kmax, p, q, seed, (const float*)A, lda, left, tol, J,
                           (float*)Tout, ldt, Jc, Ir, (float*)Ucur, lducur, rank);
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
  if (k >= n || k > UPPER_SOLVE_MAX_K) return 0;
  return ws_query(m, n, k, p, q, dtype, opts, W_ID);
}
size_t rsvd_cur_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                               const rsvd_opts* opts) {
  if (k >= n || k >= m || k > UPPER_SOLVE_MAX_K) return 0;
  return ws_query(m, n, k, p, q, dtype, opts, W_ID | W_CUR);
}
size_t rsvd_svd_id_cur_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                                      const rsvd_opts* opts) {
  if (k >= n || k >= m || k > UPPER_SOLVE_MAX_K) return 0;
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

size_t rsvd_id_tol_workspace_size(int64_t m, int64_t n, int kmax, int p, int q, int dtype,
                                  const rsvd_opts* opts) {
  return ws_query_ext(m, n, kmax, p, q, dtype, opts, true, false, false);
}
size_t rsvd_cur_tol_workspace_size(int64_t m, int64_t n, int kmax, int p, int q, int dtype,
                                   const rsvd_opts* opts) {
  return ws_query_ext(m, n, kmax, p, q, dtype, opts, true, true, false);
}
size_t rsvd_id_left_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                                   const rsvd_opts* opts) {
  return ws_query_ext(m, n, k, p, q, dtype, opts, false, false, true);
}

rsvd_status rsvd_id_tol(int64_t m, int64_t n, int kmax, int p, int q, double tol, uint64_t seed,
                        int dtype, const void* A, int64_t lda, int32_t* J, void* T, int64_t ldt,
                        int* rank, void* work, size_t work_bytes, int* d_info, void* stream,
                        const rsvd_opts* opts) {
  if (!(tol > 0.0)) return RSVD_ERR_INVALID_ARG;
  return dispatch_ext(m, n, kmax, p, q, tol, seed, dtype, A, lda, false, J, T, ldt, nullptr,
                      nullptr, nullptr, 0, rank, work, work_bytes, d_info, stream, opts);
}

rsvd_status rsvd_cur_tol(int64_t m, int64_t n, int kmax, int p, int q, double tol, uint64_t seed,
                         int dtype, const void* A, int64_t lda, int32_t* Jc, int32_t* Ir, void* U,
                         int64_t ldu, int* rank, void* work, size_t work_bytes, int* d_info,
                         void* stream, const rsvd_opts* opts) {
  if (!(tol > 0.0) || !Jc) return RSVD_ERR_INVALID_ARG;
  return dispatch_ext(m, n, kmax, p, q, tol, seed, dtype, A, lda, false, nullptr, nullptr, 0, Jc,
                      Ir, U, ldu, rank, work, work_bytes, d_info, stream, opts);
}

rsvd_status rsvd_id_left(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                         const void* A, int64_t lda, int32_t* J, void* T, int64_t ldt, void* work,
                         size_t work_bytes, int* d_info, void* stream, const rsvd_opts* opts) {
  return dispatch_ext(m, n, k, p, q, 0.0, seed, dtype, A, lda, true, J, T, ldt, nullptr, nullptr,
                      nullptr, 0, nullptr, work, work_bytes, d_info, stream, opts);
}

rsvd_status rsvd_svd_tol(int64_t m, int64_t n, int kmax, int p, int q, double tol, uint64_t seed,
                         int dtype, const void* A, int64_t lda, void* U, int64_t ldu, double* S,
                         void* V, int64_t ldv, int* rank, void* work, size_t work_bytes,
                         int* d_info, void* stream, const rsvd_opts* opts) {
  if (!(tol > 0.0) || !(tol < 1e300) || !rank) return RSVD_ERR_INVALID_ARG;
  rsvd_status st = dispatch(m, n, kmax, p, q, seed, dtype, A, lda, W_SVD, nullptr, 0, nullptr, 0,
                            U, ldu, S, V, ldv, nullptr, nullptr, 0, nullptr, nullptr, nullptr, 0,
                            work, work_bytes, d_info, stream, opts);
  if (st != RSVD_OK) return st;
  // the rank: the number of singular values above tol, at least one
  std::vector<double> h((size_t)kmax);
  cudaStream_t cs = (cudaStream_t)stream;
  if (cudaMemcpyAsync(h.data(), S, sizeof(double) * kmax, cudaMemcpyDeviceToHost, cs) !=
          cudaSuccess ||
      cudaStreamSynchronize(cs) != cudaSuccess)
    return RSVD_ERR_CUDA;
  int r = 0;
  for (int i = 0; i < kmax; ++i)
    if (h[i] > tol) ++r;
  *rank = r > 0 ? r : 1;
  return RSVD_OK;
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
  if (o.precision == RSVD_PREC_FP8 && !tc) return 0;   // FP8 sketch: tensor cores only
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
  e.take_omq(n, L);
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
  // bounded accumulation runs: the result is returned to the caller as is
  return e.gemm_t(rows, K, L, A, lda, &w, X, ldx, Y, ldy, l, nullptr, part, slabs, nullptr, false,
                  c.abf != 0, kDrainQB);
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

rsvd_status rsvd_omega_fp8(int64_t n, int l, uint64_t seed, float* Omega, int64_t ldo,
                           void* stream) {
  if (n < 1 || l < 1 || l > 4096 || !Omega || ldo < l || n > 0xffffffffLL)
    return RSVD_ERR_INVALID_ARG;
  return launch_omega_fp8(n, l, seed, Omega, ldo, (cudaStream_t)stream) == cudaSuccess
             ? RSVD_OK
             : RSVD_ERR_CUDA;
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
  if (o.precision == RSVD_PREC_FP8 && !tc) return 0;   // FP8 sketch: tensor cores only
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
