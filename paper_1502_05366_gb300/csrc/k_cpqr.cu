// k-step column-pivoted Householder QR (Sec. 2.3) of an r x n sketch in FP64,
// the ID coefficients T = S11^{-1} S12 (Sec. 2.4; Alg. 1), and a generic
// many-right-hand-side upper-triangular solve.
//
// One persistent cooperative grid; CTA b owns a contiguous slab of columns.
// Step j: every CTA proposes the best active column of its slab (largest
// residual norm, ties to the lowest column index) -> grid barrier -> every CTA
// reduces the proposals, rebuilds the Householder vector of the pivot column
// (rows j..r-1) and applies it to its own active columns, recomputing their
// residual norms exactly.  Columns never move; the LAPACK-style exchange
// (positions j <-> where(p)) is kept in the permutation J.  The grid barrier
// waits are bounded: after ~2 s of spinning the kernel reports RSVD_ERR_TIMEOUT
// and every CTA returns.
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int PT = 1024;
constexpr long long SPIN_LIMIT_CYCLES = 4000000000LL;
}

// Proposal slots: 2 x 1024 CTAs x (2 doubles) and 2 x 1024 x int64.
size_t cpqr_scratch_bytes(int64_t n) {
  (void)n;
  return 2 * 1024 * (2 * sizeof(double) + sizeof(int64_t));
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Returns false when the wait ran out.
__device__ bool grid_barrier(unsigned* bar, unsigned target, int* d_info) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const long long t0 = clock64();
    int ok = 1;
    unsigned it = 0;
    while (ld_acquire_u32(bar) < target) {
      __nanosleep(100);
      if (((++it) & 255u) == 0 && clock64() - t0 > SPIN_LIMIT_CYCLES) {
        set_info(d_info, RSVD_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct Top2 {
  double b1;
  int64_t i1;
  double b2;
};

__device__ __forceinline__ Top2 merge_top2(Top2 x, Top2 y) {
  Top2 r;
  const bool xfirst = (x.b1 > y.b1) || (x.b1 == y.b1 && x.i1 < y.i1);
  if (xfirst) {
    r.b1 = x.b1;
    r.i1 = x.i1;
    r.b2 = max(x.b2, y.b1);
  } else {
    r.b1 = y.b1;
    r.i1 = y.i1;
    r.b2 = max(y.b2, x.b1);
  }
  return r;
}

__device__ Top2 block_top2(Top2 v) {
  __shared__ double sb1[PT / 32], sb2[PT / 32];
  __shared__ int64_t si1[PT / 32];
  __shared__ Top2 s_res;
  for (int o = 16; o > 0; o >>= 1) {
    Top2 w;
    w.b1 = __shfl_xor_sync(0xffffffffu, v.b1, o);
    w.i1 = __shfl_xor_sync(0xffffffffu, v.i1, o);
    w.b2 = __shfl_xor_sync(0xffffffffu, v.b2, o);
    v = merge_top2(v, w);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sb1[warp] = v.b1;
    si1[warp] = v.i1;
    sb2[warp] = v.b2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Top2 r{sb1[0], si1[0], sb2[0]};
    for (int w = 1; w < PT / 32; ++w) r = merge_top2(r, Top2{sb1[w], si1[w], sb2[w]});
    s_res = r;
  }
  __syncthreads();
  Top2 r = s_res;
  __syncthreads();
  return r;
}

// W is the r x n sketch in FP64, ROW-major (element (i, c) at W[i*n + c]), so a
// warp's 32 threads, one column each, touch 32 consecutive doubles of a row.
// Residual norms are downdated, nu_c^2 <- nu_c^2 - W(j, c)^2 after step j (the
// reflector keeps ||W(j:, c)||), and recomputed exactly from the column when
// the downdated value falls below sqrt(eps) of its last exact value (the
// LAPACK dgeqp3 safeguard); the pivot relative error stays below ~1e-8.
__global__ void __launch_bounds__(PT) cpqr_kernel(CpqrArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  double* v = (double*)dsm;  // Householder vector, r entries
  __shared__ double s_tau, s_beta;
  __shared__ double s_part[PT];
  const int r = a.r;
  const int64_t n = a.n;
  const int G = gridDim.x;
  const int64_t per = ceil_div(n, G);
  const int64_t c0 = (int64_t)blockIdx.x * per;
  const int64_t c1 = min(n, c0 + per);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = PT / 32;
  double* W = a.W;
  double* __restrict__ nrm = a.nrm;
  double* __restrict__ nref = a.nrm + n;     // norm^2 at the last exact computation
  double* __restrict__ diagR = a.diagR;
  const double tol3z = 1.4901161193847656e-08;   // sqrt(eps_fp64)

  // exact initial norms of the own columns
  for (int64_t c = c0 + tid; c < c1; c += PT) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) {
      const double x = W[(int64_t)i * n + c];
      s = fma(x, x, s);
    }
    nrm[c] = s;
    nref[c] = s;
  }
  if (blockIdx.x == 0)
    for (int64_t c = tid; c < n; c += PT) {
      a.J[c] = (int32_t)c;
      a.where[c] = c;
    }
  __syncthreads();

  for (int j = 0; j < a.k; ++j) {
    Top2 loc{-1.0, 0x7fffffffffffffffLL, -1.0};
    for (int64_t c = c0 + tid; c < c1; c += PT) {
      const double x = nrm[c];
      if (x >= 0.0) loc = merge_top2(loc, Top2{x, c, -1.0});
    }
    loc = block_top2(loc);
    const int slot = j & 1;
    if (tid == 0) {
      a.pval[(size_t)slot * 2 * G + 2 * blockIdx.x] = loc.b1;
      a.pval[(size_t)slot * 2 * G + 2 * blockIdx.x + 1] = loc.b2;
      a.pidx[(size_t)slot * G + blockIdx.x] = loc.i1;
    }
    if (!grid_barrier(a.bar, (unsigned)(j + 1) * (unsigned)G, a.d_info)) return;
    Top2 g{-1.0, 0x7fffffffffffffffLL, -1.0};
    for (int b = tid; b < G; b += PT)
      g = merge_top2(g, Top2{__ldcg(a.pval + (size_t)slot * 2 * G + 2 * b),
                             __ldcg(reinterpret_cast<const long long*>(a.pidx) +
                                    (size_t)slot * G + b),
                             __ldcg(a.pval + (size_t)slot * 2 * G + 2 * b + 1)});
    g = block_top2(g);
    const int64_t p = g.i1;
    if (p < 0 || p >= n) {  // no active column left (cannot happen for k <= min(r, n))
      set_info(a.d_info, RSVD_ERR_NUMERIC);
      return;
    }
    // Householder vector of the pivot column, rows j..r-1 (read-only this step)
    const int len = r - j;
    double part = 0.0;
    for (int i = tid; i < len; i += PT) {
      const double x = __ldcg(W + (int64_t)(j + i) * n + p);
      v[i] = x;
      part = fma(x, x, part);
    }
    __shared__ double s_red[PT / 32];
    part = warp_sum(part);
    if (lane == 0) s_red[warp] = part;
    __syncthreads();
    if (tid == 0) {
      double nx2 = 0.0;
      for (int w = 0; w < nwarp; ++w) nx2 += s_red[w];
      const double nx = sqrt(nx2);
      const double x0 = v[0];
      const double beta = (x0 >= 0.0) ? -nx : nx;
      s_beta = beta;
      if (nx > 0.0) {
        v[0] = x0 - beta;
        const double vv = nx2 - x0 * x0 + v[0] * v[0];
        s_tau = 2.0 / vv;
      } else {
        s_tau = 0.0;
      }
    }
    __syncthreads();
    const double tau = s_tau;
    // TPC threads per column, each on a chunk of the len active rows; the
    // partial dot products meet in shared memory.
    const int cw = PT / a.tpc;                 // columns per pass
    const int h = tid / cw, cc = tid - h * cw;
    const int clen = (len + a.tpc - 1) / a.tpc;
    const int i0 = h * clen, i1 = min(len, i0 + clen);
    for (int64_t cb = c0; cb < c1; cb += cw) {
      const int64_t c = cb + cc;
      const bool act = c < c1 && c != p && nrm[c] >= 0.0;
      double* col = W + (int64_t)j * n + c;
      if (act) {
        double w0 = 0.0, w1 = 0.0, w2 = 0.0, w3 = 0.0;
        int i = i0;
        for (; i + 4 <= i1; i += 4) {
          w0 = fma(v[i], col[(int64_t)i * n], w0);
          w1 = fma(v[i + 1], col[(int64_t)(i + 1) * n], w1);
          w2 = fma(v[i + 2], col[(int64_t)(i + 2) * n], w2);
          w3 = fma(v[i + 3], col[(int64_t)(i + 3) * n], w3);
        }
        for (; i < i1; ++i) w0 = fma(v[i], col[(int64_t)i * n], w0);
        s_part[h * cw + cc] = (w0 + w1) + (w2 + w3);
      }
      __syncthreads();
      if (act) {
        double w = 0.0;
        for (int t = 0; t < a.tpc; ++t) w += s_part[t * cw + cc];
        w *= tau;
#pragma unroll 4
        for (int i = i0; i < i1; ++i) col[(int64_t)i * n] -= w * v[i];
      }
      __syncthreads();
      if (act && h == 0) {
        const double top = col[0];
        const double nc = nrm[c];
        double nn = nc - top * top;
        if (!(nn > tol3z * nref[c]) && j + 1 < r) {   // cancellation: recompute exactly
          nn = 0.0;
          for (int i = 1; i < len; ++i) {
            const double x = col[(int64_t)i * n];
            nn = fma(x, x, nn);
          }
          nref[c] = nn;
        }
        nrm[c] = nn > 0.0 ? nn : 0.0;
      }
    }
    if (p >= c0 && p < c1 && tid == 0) nrm[p] = -1.0;
    if (blockIdx.x == 0 && tid == 0) {
      diagR[j] = s_beta;
      const int64_t P = a.where[p];
      const int32_t cj = a.J[j];
      a.J[P] = cj;
      a.where[cj] = P;
      a.J[j] = (int32_t)p;
      a.where[p] = j;
      if (a.gaps) {
        const double n1 = sqrt(g.b1);
        a.gaps[j] = (g.b2 < 0.0) ? __longlong_as_double(0x7ff0000000000000LL)
                                 : (n1 > 0.0 ? (n1 - sqrt(g.b2)) / n1 : 0.0);
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_cpqr(const CpqrArgs& a, int* grid_out, cudaStream_t s) {
  if (a.r > 8192) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const size_t dyn = (size_t)a.r * sizeof(double);
  e = cudaFuncSetAttribute(cpqr_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cpqr_kernel, PT, dyn);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // one SM is left to a single-CTA kernel running beside the CPQR on another
  // stream (the Jacobi SVD of the combined SVD + ID/CUR call)
  int64_t G = sms > 1 ? sms - 1 : 1;
  const int64_t byn = ceil_div(a.n, 32);
  if (G > byn) G = byn;
  if (G > 1024) G = 1024;
  if (G < 1) G = 1;
  *grid_out = (int)G;
  // threads per column: the largest power of two that keeps one pass per step
  const int64_t per = ceil_div(a.n, G);
  int tpc = 1;
  while (tpc < 8 && (int64_t)(PT / (tpc * 2)) >= per) tpc *= 2;
  e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  CpqrArgs b = a;
  b.tpc = tpc;
  void* args[] = {(void*)&b};
  count_launch();
  const int tr = trace_begin(RSVD_TRACE_CPQR, s);
  e = cudaLaunchCooperativeKernel((const void*)cpqr_kernel, dim3((unsigned)G), dim3(PT), args,
                                  dyn, s);
  trace_end(tr, s);
  return e;
}

// S11 (k x k, column-major, upper triangular incl. beta on the diagonal) and
// S12 (k x (n-k), row-major; column c' = position k + c') in pivot order, from
// the row-major working array W (r x n).
__global__ void id_extract_kernel(int r, int64_t n, int k, const double* __restrict__ W,
                                  const int32_t* __restrict__ J, const double* __restrict__ diagR,
                                  double* __restrict__ S11, double* __restrict__ S12) {
  const int64_t total = n * (int64_t)k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = t / k;
    const int i = (int)(t - pos * k);
    const int64_t c = J[pos];
    if (pos < k) {
      double v;
      if (i < pos) v = W[(int64_t)i * n + c];
      else if (i == pos) v = diagR[pos];
      else v = 0.0;
      S11[pos * k + i] = v;
    } else {
      S12[(int64_t)i * (n - k) + (pos - k)] = W[(int64_t)i * n + c];
    }
  }
}

cudaError_t launch_id_extract(int r, int64_t n, int k, const double* W, const int32_t* J,
                                const double* diagR, double* S11, double* S12, cudaStream_t s) {
  const int64_t total = n * (int64_t)k;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 16384) blocks = 16384;
  id_extract_kernel<<<(unsigned)blocks, 256, 0, s>>>(r, n, k, W, J, diagR, S11, S12);
  count_launch();
  return cudaGetLastError();
}

// One thread per right-hand side; the running right-hand side sits in shared
// memory (sv[i * blockDim + thread]).  Column-oriented back substitution:
//   for i = kk-1 .. 0: x_i = s_i / U(i,i); s(0:i) -= x_i U(0:i, i),
// with U read by all threads at the same address (broadcast).
template <typename TR, typename TO>
__global__ void upper_solve_kernel(int kk, int64_t ncols, const double* __restrict__ Ug,
                                   int64_t us_i, int64_t us_t, const TR* __restrict__ rhs,
                                   int64_t rs_i, int64_t rs_c, TO* __restrict__ out,
                                   int64_t os_i, int64_t os_c, int* d_info) {
  extern __shared__ __align__(16) unsigned char dsm[];
  double* sv = (double*)dsm;
  const int t = threadIdx.x, bd = blockDim.x;
  for (int64_t cb = (int64_t)blockIdx.x * bd; cb < ncols; cb += (int64_t)gridDim.x * bd) {
    const int64_t c = cb + t;
    const bool act = c < ncols;
    if (act)
      for (int i = 0; i < kk; ++i) sv[i * bd + t] = (double)rhs[i * rs_i + c * rs_c];
    for (int i = kk - 1; i >= 0; --i) {
      const double d = Ug[i * us_i + i * us_t];
      if (!(d != 0.0)) {
        if (act) sv[i * bd + t] = 0.0;
        if (t == 0) set_info(d_info, RSVD_ERR_NUMERIC);
        continue;
      }
      if (act) {
        const double xi = sv[i * bd + t] / d;
        sv[i * bd + t] = xi;
        const double* ucol = Ug + i * us_t;
        for (int q = 0; q < i; ++q) sv[q * bd + t] = fma(-xi, ucol[q * us_i], sv[q * bd + t]);
      }
    }
    if (act)
      for (int i = 0; i < kk; ++i) out[i * os_i + c * os_c] = (TO)sv[i * bd + t];
  }
}

template <typename TR, typename TO>
cudaError_t launch_upper_solve(int kk, int64_t ncols, const double* Ug, int64_t us_i,
                               int64_t us_t, const TR* rhs, int64_t rs_i, int64_t rs_c, TO* out,
                               int64_t os_i, int64_t os_c, int* d_info, cudaStream_t s) {
  if (kk <= 0 || ncols <= 0) return cudaSuccess;
  if (kk > UPPER_SOLVE_MAX_K) return cudaErrorInvalidValue;
  // threads per block: as many as fit 8*kk bytes each in 220 KB of shared
  // memory (multiples of 32, at most 128), and no more blocks than columns need
  int bd = (int)((220 * 1024) / ((size_t)kk * sizeof(double)));
  bd = bd > 128 ? 128 : (bd / 32) * 32;
  if (bd < 32) return cudaErrorInvalidValue;
  const int sms = device_sm_count();
  while (bd > 32 && ceil_div(ncols, bd) < sms) bd -= 32;
  const size_t dyn = (size_t)bd * kk * sizeof(double);
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(upper_solve_kernel<TR, TO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  int64_t blocks = ceil_div(ncols, bd);
  if (blocks > 65535) blocks = 65535;
  const int tr_ = trace_begin(RSVD_TRACE_SOLVE, s);
  upper_solve_kernel<TR, TO><<<(unsigned)blocks, bd, dyn, s>>>(
      kk, ncols, Ug, us_i, us_t, rhs, rs_i, rs_c, out, os_i, os_c, d_info);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

template cudaError_t launch_upper_solve<double, double>(int, int64_t, const double*, int64_t,
                                                        int64_t, const double*, int64_t,
                                                        int64_t, double*, int64_t, int64_t,
                                                        int*, cudaStream_t);
template cudaError_t launch_upper_solve<double, float>(int, int64_t, const double*, int64_t,
                                                       int64_t, const double*, int64_t, int64_t,
                                                       float*, int64_t, int64_t, int*,
                                                       cudaStream_t);
template cudaError_t launch_upper_solve<float, float>(int, int64_t, const double*, int64_t,
                                                      int64_t, const float*, int64_t, int64_t,
                                                      float*, int64_t, int64_t, int*,
                                                      cudaStream_t);

}  // namespace rsvd
