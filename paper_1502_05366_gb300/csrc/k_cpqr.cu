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
#include "df.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int PT = 1024;
constexpr long long SPIN_LIMIT_CYCLES = 4000000000LL;
// Test aid (rsvd_test_set_barrier_wait): a shorter bound on the grid-barrier
// waits and, optionally, CTA 0 withholding its arrival at the first barrier so
// that every wait runs out.  0 / 0 = the defaults.
long long g_test_spin_limit = 0;
int g_test_withhold = 0;
}

extern "C" rsvd_status rsvd_test_set_barrier_wait(long long cycles, int withhold) {
  if (cycles < 0) return RSVD_ERR_INVALID_ARG;
  if (cycles == 0) withhold = 0;
  g_test_spin_limit = cycles;
  g_test_withhold = withhold ? 1 : 0;
  return RSVD_OK;
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

// Returns false when the wait ran out.  `limit` bounds the wait in SM clock
// cycles; `arrive` false withholds this CTA's arrival (test aid only).
__device__ bool grid_barrier(unsigned* bar, unsigned target, int* d_info, long long limit,
                             bool arrive) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (arrive) atomicAdd(bar, 1u);
    const long long t0 = clock64();
    int ok = 1;
    unsigned it = 0;
    while (ld_acquire_u32(bar) < target) {
      __nanosleep(100);
      if (((++it) & 255u) == 0 && clock64() - t0 > limit) {
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

template <int NT>
__device__ Top2 block_top2_n(Top2 v) {
  __shared__ double sb1[NT / 32], sb2[NT / 32];
  __shared__ int64_t si1[NT / 32];
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
    for (int w = 1; w < NT / 32; ++w) r = merge_top2(r, Top2{sb1[w], si1[w], sb2[w]});
    s_res = r;
  }
  __syncthreads();
  Top2 r = s_res;
  __syncthreads();
  return r;
}


__device__ __forceinline__ Top2 block_top2(Top2 v) { return block_top2_n<PT>(v); }

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

  const bool tolmode = a.tol2 > 0.0;
  __shared__ double s_wsum[PT / 32];
  __shared__ double s_tot;
  int steps = a.k;
  for (int j = 0; j < a.k; ++j) {
    Top2 loc{-1.0, 0x7fffffffffffffffLL, -1.0};
    double cs = 0.0;
    for (int64_t c = c0 + tid; c < c1; c += PT) {
      const double x = nrm[c];
      if (x >= 0.0) {
        loc = merge_top2(loc, Top2{x, c, -1.0});
        cs += x;
      }
    }
    loc = block_top2(loc);
    const int slot = j & 1;
    if (tolmode) {   // the CTA's sum of residual norms^2, in a fixed order
      cs = warp_sum(cs);
      if (lane == 0) s_wsum[warp] = cs;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < nwarp; ++w) t += s_wsum[w];
        a.psum[(size_t)slot * G + blockIdx.x] = t;
      }
    }
    if (tid == 0) {
      a.pval[(size_t)slot * 2 * G + 2 * blockIdx.x] = loc.b1;
      a.pval[(size_t)slot * 2 * G + 2 * blockIdx.x + 1] = loc.b2;
      a.pidx[(size_t)slot * G + blockIdx.x] = loc.i1;
    }
    if (!grid_barrier(a.bar, (unsigned)(j + 1) * (unsigned)G, a.d_info, a.spin_limit,
                      !(a.withhold && j == 0 && blockIdx.x == 0)))
      return;
    Top2 g{-1.0, 0x7fffffffffffffffLL, -1.0};
    for (int b = tid; b < G; b += PT)
      g = merge_top2(g, Top2{__ldcg(a.pval + (size_t)slot * 2 * G + 2 * b),
                             __ldcg(reinterpret_cast<const long long*>(a.pidx) +
                                    (size_t)slot * G + b),
                             __ldcg(a.pval + (size_t)slot * 2 * G + 2 * b + 1)});
    g = block_top2(g);
    if (tolmode && j >= 1) {
      // ||S22(j)||_F^2: every CTA adds the G partials in the same order
      if (warp == 0) {
        double t = 0.0;
        for (int b = lane; b < G; b += 32) t += __ldcg(a.psum + (size_t)slot * G + b);
        t = warp_sum(t);
        if (lane == 0) s_tot = t;
      }
      __syncthreads();
      if (s_tot < a.tol2) {
        steps = j;
        break;
      }
    }
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
  if (a.k_out && blockIdx.x == 0 && tid == 0) *a.k_out = steps;
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
  // one SM is left to the one-CTA FP64 Jacobi SVD that runs beside the CPQR
  // on another stream in the combined SVD + ID/CUR call
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
  b.spin_limit = g_test_spin_limit > 0 ? g_test_spin_limit : SPIN_LIMIT_CYCLES;
  b.withhold = g_test_withhold;
  void* args[] = {(void*)&b};
  count_launch();
  const int tr = trace_begin(RSVD_TRACE_CPQR, s);
  e = cudaLaunchCooperativeKernel((const void*)cpqr_kernel, dim3((unsigned)G), dim3(PT), args,
                                  dyn, s);
  trace_end(tr, s);
  return e;
}

// ---------------------------------------------------------------------------
// Double-float variant (sketches of FP32 data).
//
// GB300 issues FP64 fused multiply-adds at 2 per clock per SM, 1/64 of the
// FP32 rate, so the bulk arithmetic of the pivoted QR (dot product and rank-1
// update on every active entry, 4 flops per entry per step) runs in
// double-float: every entry of W is the unevaluated sum hi + lo of two floats
// (about 48 significant bits), held in two planes Wh, Wl.  The dot products
// use the compensated scheme Dot2 (Ogita, Rump & Oishi 2005: TwoProduct by
// fma, TwoSum, errors summed in a second float), the updates TwoProduct /
// TwoSum with a final renormalisation (Dekker 1971).  Per-column and per-step
// scalars (residual norms, tau, beta, pivots, gaps) stay FP64.  With a
// relative error near 2^-47 per operation the pivot choices are those of an
// FP64 computation unless two residual norms agree to about 1e-13.
// The rounding primitives use the _rn intrinsics so that no product is fused
// into a neighbouring sum.
// ---------------------------------------------------------------------------
template <int NT>
__device__ Top2F block_top2f(Top2F v) {
  __shared__ float sb[NT / 32][4];
  __shared__ int64_t si1[NT / 32];
  __shared__ Top2F s_res;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Top2F w;
    w.b1.h = __shfl_xor_sync(0xffffffffu, v.b1.h, o);
    w.b1.l = __shfl_xor_sync(0xffffffffu, v.b1.l, o);
    w.i1 = __shfl_xor_sync(0xffffffffu, v.i1, o);
    w.b2.h = __shfl_xor_sync(0xffffffffu, v.b2.h, o);
    w.b2.l = __shfl_xor_sync(0xffffffffu, v.b2.l, o);
    v = merge_top2f(v, w);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sb[warp][0] = v.b1.h;
    sb[warp][1] = v.b1.l;
    sb[warp][2] = v.b2.h;
    sb[warp][3] = v.b2.l;
    si1[warp] = v.i1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Top2F r{{sb[0][0], sb[0][1]}, si1[0], {sb[0][2], sb[0][3]}};
    for (int w = 1; w < NT / 32; ++w)
      r = merge_top2f(r, Top2F{{sb[w][0], sb[w][1]}, si1[w], {sb[w][2], sb[w][3]}});
    s_res = r;
  }
  __syncthreads();
  Top2F r = s_res;
  __syncthreads();
  return r;
}
// Row-slot granularity of the specialised column passes: single slots for
// r <= 256, groups of 4 for r <= 1024 (8 instantiations either way).
template <int RPL>
__host__ __device__ constexpr int SLOT_STEP() { return RPL <= 8 ? 1 : RPL / 8; }

// One step's dot products, rank-1 updates and norm downdates over the CTA's
// columns (one warp per column), with S row slots per lane.
// The 8-slot form (r <= 256): each warp loads its next column into registers
// while it processes the current one (CPQR_PIPE), at 16 warps per CTA so
// that the second set of registers fits (CPQR_NT8).  Measured against no
// pipelining at 24 warps: 2.78 / 4.46 ms against 2.84 / 4.62 ms per launch on
// 220 x 20000 / 200 x 50000; 20 or 14 warps with it, or 16 without it, were
// slower.
#ifndef CPQR_PIPE
#define CPQR_PIPE 1
#endif
#ifndef CPQR_NT8
#define CPQR_NT8 512
#endif
__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Warp-wide best two of (value, index) proposals; every lane ends with it.
__device__ __forceinline__ Top2F warp_top2f(Top2F v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Top2F w;
    w.b1.h = __shfl_xor_sync(0xffffffffu, v.b1.h, o);
    w.b1.l = __shfl_xor_sync(0xffffffffu, v.b1.l, o);
    w.i1 = __shfl_xor_sync(0xffffffffu, v.i1, o);
    w.b2.h = __shfl_xor_sync(0xffffffffu, v.b2.h, o);
    w.b2.l = __shfl_xor_sync(0xffffffffu, v.b2.l, o);
    v = merge_top2f(v, w);
  }
  return v;
}

struct CpqrDfCol {
  float* Wh;
  float* Wl;
  float2* nrm2;       // residual norms of columns cbase.. (shared or global memory)
  float* nref;
  int64_t cbase;
  const float* svh;
  const float* svl;
  int r, j, len;
  int64_t p, c0, c1;
  float tauh, taul;
  bool zero;
  int lane, warp;
  bool tol;           // tolerance mode: sum the residual norms^2 (lane 0)

  // Returns (on lane 0) the warp's best two residual norms after the step and
  // adds them all, as doubles, to `acc` (lane 0; read in tolerance mode only).
  // VS: the Householder vector is read from shared memory at each use instead
  // of being held in registers (the 32-slot form, whose registers would
  // otherwise limit it to 8 warps per SM).
  template <int S, int NWARP, bool VS>
  __device__ __forceinline__ Top2F run(double& acc) const {
    const DF none{-1.f, 0.f};
    Top2F best{none, 0x7fffffffffffffffLL, none};
    const float tol3z = 1.4901161193847656e-08f;   // sqrt(eps_fp64), as in the FP64 kernel
    constexpr int SV = VS ? 1 : S;
    float vh[SV], vl[SV];
    if (!VS) {
#pragma unroll
      for (int t = 0; t < SV; ++t) {
        const int i = lane + 32 * t;
        vh[t] = i < len ? svh[i] : 0.f;
        vl[t] = i < len ? svl[i] : 0.f;
      }
    }
    // slot t of v (zero beyond the active rows)
    auto vslot = [&](int t, float& h, float& l) {
      if (VS) {
        const int i = lane + 32 * t;
        h = i < len ? svh[i] : 0.f;
        l = i < len ? svl[i] : 0.f;
      } else {
        h = vh[VS ? 0 : t];
        l = vl[VS ? 0 : t];
      }
    };
    // Norm bookkeeping of the pass, batched over up to 32 columns (lane q
    // holds the q-th column of the batch) instead of run by lane 0 column by
    // column: the downdate nu^2 - W(j, c)^2 in double-float, the exact
    // recompute on cancellation (LAPACK safeguard; from the stored column,
    // the values the lane itself wrote), the new norms and the warp's best
    // two.  Every column's arithmetic is the one lane 0 ran, the best two do
    // not depend on the order of merging, and the tolerance sum is taken in
    // column order, so the results are those of the column-by-column form.
    float st_nx = 0.f, st_ny = 0.f, st_wh = 0.f, st_wl = 0.f;
    int64_t st_c = 0;
    int nst = 0;
    auto flush = [&]() {
      if (nst == 0) return;
      float nh = 0.f, nl = 0.f;
      int rec = 0;
      if (lane < nst) {
        float ph, pe, sh, se;
        df_sqr(st_wh, st_wl, ph, pe);
        df_two_sum(st_nx, -ph, sh, se);
        se = __fadd_rn(se, __fsub_rn(st_ny, pe));
        df_fast_two_sum(sh, se, nh, nl);
        rec = (!(nh > tol3z * nref[st_c - cbase]) && j + 1 < r) ? 1 : 0;
      }
      unsigned rm = __ballot_sync(0xffffffffu, rec);
      while (rm) {
        const int q = __ffs(rm) - 1;
        rm &= rm - 1;
        const int64_t cq = __shfl_sync(0xffffffffu, st_c, q);
        const float* ch = Wh + cq * r + j;
        const float* cl = Wl + cq * r + j;
        float qs = 0.f, qe = 0.f;
#pragma unroll
        for (int t = 0; t < S; ++t) {
          const int i = lane + 32 * t;
          if (i >= 1 && i < len) df_acc_sqr(ch[i], cl[i], qs, qe);
        }
        df_warp_sum(qs, qe);
        float h, l;
        df_fast_two_sum(qs, qe, h, l);
        if (lane == q) {
          nh = h;
          nl = l;
          nref[st_c - cbase] = h;
        }
      }
      float2 nv = make_float2(0.f, 0.f);
      Top2F cand{none, 0x7fffffffffffffffLL, none};
      if (lane < nst) {
        nv = nh > 0.f ? make_float2(nh, nl) : make_float2(0.f, 0.f);
        nrm2[st_c - cbase] = nv;
        cand = Top2F{DF{nv.x, nv.y}, st_c, none};
      }
      best = merge_top2f(best, warp_top2f(cand));
      if (tol) {
        for (int q = 0; q < nst; ++q) {
          const float a = __shfl_sync(0xffffffffu, nv.x, q);
          const float b = __shfl_sync(0xffffffffu, nv.y, q);
          if (lane == 0) acc += (double)a + (double)b;
        }
      }
      nst = 0;
    };
    // The 32-slot form (VS) prefetches the warp's next column into L1 while
    // this one is processed; the 8-slot form does not: its pass is
    // issue-bound, and two prefetches per row slot cost more than the latency
    // they hid (C2: 9.42 -> 8.77 ms per step without them; the 32-slot form at
    // r = 550: 100 -> 106 ms without them).
    // PIPE (8-slot form): the warp's next column is loaded into registers
    // while this one is processed
    constexpr bool PIPE = CPQR_PIPE && !VS;
    constexpr int SP = PIPE ? S : 1;
    float xh[SP], xl[SP];
    if (PIPE) {
      const int64_t cf = c0 + warp;
#pragma unroll
      for (int t = 0; t < SP; ++t) {
        const int i = lane + 32 * t;
        xh[t] = (cf < c1 && i < len) ? Wh[cf * r + j + i] : 0.f;
        xl[t] = (cf < c1 && i < len) ? Wl[cf * r + j + i] : 0.f;
      }
    }
    for (int64_t c = c0 + warp; c < c1; c += NWARP) {
      if (VS && c + NWARP < c1) {
#pragma unroll
        for (int t = 0; t < S; ++t) {
          const int i = lane + 32 * t;
          if (i < len) {
            prefetch_l1(Wh + (c + NWARP) * r + j + i);
            prefetch_l1(Wl + (c + NWARP) * r + j + i);
          }
        }
      }
      float wh[S], wl[S];
      if (PIPE) {
        const int64_t cn = c + NWARP;
#pragma unroll
        for (int t = 0; t < S; ++t) {
          const int i = lane + 32 * t;
          wh[t] = xh[PIPE ? t : 0];
          wl[t] = xl[PIPE ? t : 0];
          xh[PIPE ? t : 0] = (cn < c1 && i < len) ? Wh[cn * r + j + i] : 0.f;
          xl[PIPE ? t : 0] = (cn < c1 && i < len) ? Wl[cn * r + j + i] : 0.f;
        }
      }
      if (c == p) continue;                                  // warp-uniform
      const float2 nc = nrm2[c - cbase];
      if (nc.x < 0.f) continue;                              // already pivoted
      float* colh = Wh + c * r + j;
      float* coll = Wl + c * r + j;
      if (!PIPE) {
#pragma unroll
        for (int t = 0; t < S; ++t) {
          const int i = lane + 32 * t;
          wh[t] = i < len ? colh[i] : 0.f;
          wl[t] = i < len ? coll[i] : 0.f;
        }
      }
      if (!zero) {
        // Dot2 in two independent chains (even / odd slots), then joined
        float sd = 0.f, ed = 0.f, sd2 = 0.f, ed2 = 0.f;
#pragma unroll
        for (int t = 0; t < S; ++t) {
          float vht, vlt;
          vslot(t, vht, vlt);
          const float ph = __fmul_rn(vht, wh[t]);
          float pe = __fmaf_rn(vht, wh[t], -ph);
          pe = __fmaf_rn(vht, wl[t], pe);
          pe = __fmaf_rn(vlt, wh[t], pe);
          float e;
          if (t & 1) {
            df_two_sum(sd2, ph, sd2, e);
            ed2 = __fadd_rn(ed2, __fadd_rn(e, pe));
          } else {
            df_two_sum(sd, ph, sd, e);
            ed = __fadd_rn(ed, __fadd_rn(e, pe));
          }
        }
        {
          float e;
          df_two_sum(sd, sd2, sd, e);
          ed = __fadd_rn(ed, __fadd_rn(ed2, e));
        }
        df_warp_sum(sd, ed);
        float dh, dl;
        df_fast_two_sum(sd, ed, dh, dl);
        // t = tau * (v . w) as a double-float pair
        const float qh = __fmul_rn(tauh, dh);
        float qe = __fmaf_rn(tauh, dh, -qh);
        qe = __fmaf_rn(tauh, dl, qe);
        qe = __fmaf_rn(taul, dh, qe);
        float th, tl;
        df_fast_two_sum(qh, qe, th, tl);
#pragma unroll
        for (int t = 0; t < S; ++t) {
          float vht, vlt;
          vslot(t, vht, vlt);
          const float ph = __fmul_rn(th, vht);
          float pe = __fmaf_rn(th, vht, -ph);
          pe = __fmaf_rn(th, vlt, pe);
          pe = __fmaf_rn(tl, vht, pe);
          float sh, se;
          df_two_sum(wh[t], -ph, sh, se);
          se = __fadd_rn(se, __fsub_rn(wl[t], pe));
          df_fast_two_sum(sh, se, wh[t], wl[t]);
          const int i = lane + 32 * t;
          if (i < len) {
            colh[i] = wh[t];
            coll[i] = wl[t];
          }
        }
      }
      // the column's norm bookkeeping goes to lane nst of the batch: its old
      // residual norm and the updated W(j, c) (held by lane 0)
      const float w0h = __shfl_sync(0xffffffffu, wh[0], 0);
      const float w0l = __shfl_sync(0xffffffffu, wl[0], 0);
      if (lane == nst) {
        st_nx = nc.x;
        st_ny = nc.y;
        st_wh = w0h;
        st_wl = w0l;
        st_c = c;
      }
      if (++nst == 32) flush();
    }
    flush();
    if (VS) {   // the warp's first column of the next step (stored rows j + 1 ..)
      const int64_t c = c0 + warp;
      if (c < c1) {
#pragma unroll
        for (int t = 0; t < S; ++t) {
          const int i = lane + 32 * t + 1;
          if (i < len) {
            prefetch_l1(Wh + c * r + j + i);
            prefetch_l1(Wl + c * r + j + i);
          }
        }
      }
    }
    return best;
  }
};

// Grid barrier entered by one warp of each CTA (lane 0 arrives and polls);
// false on every lane when the wait ran out.
// Arrival is a release-ordered reduction (no returned value to wait for; the
// CTA's proposal, written by the same thread before it, is visible to whoever
// acquires the count); the poll is an acquire load, which orders the reads of
// other CTAs' proposals.
__device__ __forceinline__ bool grid_barrier_warp(unsigned* bar, unsigned target, int* d_info,
                                                  long long limit, bool arrive) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    if (arrive) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    const long long t0 = clock64();
    unsigned it = 0;
    while (ld_acquire_u32(bar) < target) {
      if (((++it) & 1023u) == 0 && clock64() - t0 > limit) {
        set_info(d_info, RSVD_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
  }
  // lanes other than 0 read the proposals after this; order them after lane
  // 0's acquire
  __syncwarp();
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// Threads of the 32-slot form (256 < r <= 1024); above 256 the Householder
// vector is read from shared memory (registers for 16 warps).
#ifndef CPQR_DF_NT32
#define CPQR_DF_NT32 512
#endif

// W is COLUMN-major here (element (i, c) in Wh[c*r + i], Wl[c*r + i]), so one
// warp owns a column per iteration: lane l holds rows j + l + 32 t
// (t < RPL) of it in registers from the load through the dot product, the
// warp-shuffle reduction and the update to the store, with no block-wide
// synchronisation inside the column loop.  Warp 0 builds the Householder
// vector of the pivot column once per CTA and step (shared memory); its
// scalars (norm, beta, tau) are the only FP64 arithmetic of a step.
// The residual norms live in a.nrm as double-float pairs: float2 nrm2[c] =
// (hi, lo) of nu_c^2 (hi = -1 once pivoted), float nref[c] (the value at the
// last exact computation) at nrm2 + n.
template <int RPL, int NT, bool VS>
__global__ void __launch_bounds__(NT) cpqr_df_kernel(CpqrArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  float* svh = (float*)dsm;        // Householder vector, hi parts (r entries)
  float* svl = svh + a.r;          // lo parts
  __shared__ double s_beta;
  __shared__ float s_th, s_tl;     // tau as a double-float pair
  __shared__ int s_zero;           // zero pivot column: nothing to reflect
  const int r = a.r;
  const int64_t n = a.n;
  const int G = gridDim.x;
  const int64_t per = ceil_div(n, G);
  const int64_t c0 = (int64_t)blockIdx.x * per;
  const int64_t c1 = min(n, c0 + per);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWARP = NT / 32;
  float* Wh = reinterpret_cast<float*>(a.W);
  float* Wl = Wh + (int64_t)r * n;
  // residual norms of this CTA's columns: in shared memory after the
  // Householder vector when they fit (a.nrm_local), else in global memory
  const int64_t cbase = a.nrm_local ? c0 : 0;
  float2* nrm2;
  float* nref;
  if (a.nrm_local) {
    nrm2 = reinterpret_cast<float2*>(svh + 2 * a.r);
    nref = reinterpret_cast<float*>(nrm2 + per);
  } else {
    nrm2 = reinterpret_cast<float2*>(a.nrm);
    nref = reinterpret_cast<float*>(nrm2 + n);
  }
  float4* __restrict__ pv = reinterpret_cast<float4*>(a.pval);   // (b1h, b1l, b2h, b2l)
  double* __restrict__ diagR = a.diagR;

  __shared__ float s_wt[NWARP][4];          // per-warp best two norms (hi, lo, hi, lo)
  __shared__ int64_t s_wi[NWARP];           // per-warp best column
  __shared__ int64_t s_p;                   // this step's pivot column
  __shared__ float s_g[4];                  // the step's best two norms (for the gaps)
  __shared__ int s_abort;
  __shared__ int s_stop;                    // tolerance mode: ||S22(j)||_F below tol
  __shared__ double s_wsum[NWARP];          // per-warp sums of residual norms^2
  const bool tolmode = a.tol2 > 0.0;
  const DF none{-1.f, 0.f};

  // exact initial squared norms, one warp per column; each warp keeps its best two
  {
    Top2F best{none, 0x7fffffffffffffffLL, none};
    double acc = 0.0;
    for (int64_t c = c0 + warp; c < c1; c += NWARP) {
      float sh = 0.f, se = 0.f;
      for (int i = lane; i < r; i += 32) df_acc_sqr(Wh[c * r + i], Wl[c * r + i], sh, se);
      df_warp_sum(sh, se);
      if (lane == 0) {
        float h, l;
        df_fast_two_sum(sh, se, h, l);
        nrm2[c - cbase] = make_float2(h, l);
        nref[c - cbase] = h;
        best = merge_top2f(best, Top2F{DF{h, l}, c, none});
        if (tolmode) acc += (double)h + (double)l;
      }
    }
    if (lane == 0) {
      s_wsum[warp] = acc;
      s_wt[warp][0] = best.b1.h;
      s_wt[warp][1] = best.b1.l;
      s_wt[warp][2] = best.b2.h;
      s_wt[warp][3] = best.b2.l;
      s_wi[warp] = best.i1;
    }
  }
  if (blockIdx.x == 0)
    for (int64_t c = tid; c < n; c += NT) {
      a.J[c] = (int32_t)c;
      a.where[c] = c;
    }
  if (tid == 0) {
    s_abort = 0;
    s_stop = 0;
  }
  __syncthreads();

  int steps = a.k;
  for (int j = 0; j < a.k; ++j) {
    const int len = r - j;
    // ---- warp 0: CTA proposal, grid barrier, global pivot, Householder vector ----
    if (warp == 0) {
      Top2F v{none, 0x7fffffffffffffffLL, none};
      if (lane < NWARP)
        v = Top2F{DF{s_wt[lane][0], s_wt[lane][1]}, s_wi[lane], DF{s_wt[lane][2], s_wt[lane][3]}};
      v = warp_top2f(v);
      const int slot = j & 1;
      if (tolmode) {
        // the CTA's sum of residual norms^2 (warps in a fixed order)
        double ws = lane < NWARP ? s_wsum[lane] : 0.0;
        ws = warp_sum(ws);
        if (lane == 0) a.psum[(size_t)slot * G + blockIdx.x] = ws;
      }
      if (lane == 0) {
        pv[(size_t)slot * G + blockIdx.x] = make_float4(v.b1.h, v.b1.l, v.b2.h, v.b2.l);
        a.pidx[(size_t)slot * G + blockIdx.x] = v.i1;
      }
      if (!grid_barrier_warp(a.bar, (unsigned)(j + 1) * (unsigned)G, a.d_info, a.spin_limit,
                             !(a.withhold && j == 0 && blockIdx.x == 0))) {
        if (lane == 0) s_abort = 1;
      } else {
        Top2F g{none, 0x7fffffffffffffffLL, none};
        for (int b0 = 0; b0 < G; b0 += 4 * 32) {     // 4 loads in flight per lane
          float4 q[4];
          long long qi[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int b = b0 + u * 32 + lane;
            if (b < G) {
              q[u] = __ldcg(pv + (size_t)slot * G + b);
              qi[u] = __ldcg(reinterpret_cast<const long long*>(a.pidx) + (size_t)slot * G + b);
            }
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (b0 + u * 32 + lane < G)
              g = merge_top2f(g, Top2F{DF{q[u].x, q[u].y}, qi[u], DF{q[u].z, q[u].w}});
        }
        g = warp_top2f(g);
        const int64_t p = g.i1;
        bool stop = false;
        if (tolmode && j >= 1) {
          // ||S22(j)||_F^2 = the sum of all residual norms^2: every CTA adds
          // the G partials in the same order, so all take the same decision
          double t = 0.0;
          for (int b = lane; b < G; b += 32) t += __ldcg(a.psum + (size_t)slot * G + b);
          t = __shfl_sync(0xffffffffu, warp_sum(t), 0);
          stop = t < a.tol2;
        }
        if (stop) {
          if (lane == 0) s_stop = 1;
        } else if (p < 0 || p >= n) {
          if (lane == 0) {
            set_info(a.d_info, RSVD_ERR_NUMERIC);
            s_abort = 1;
          }
        } else {
          // the pivot column into shared memory (all loads independent), then
          // its squared norm
#pragma unroll 8
          for (int i = lane; i < len; i += 32) {
            svh[i] = __ldcg(Wh + p * r + j + i);
            svl[i] = __ldcg(Wl + p * r + j + i);
          }
          __syncwarp();
          float ss = 0.f, se = 0.f;
          for (int i = lane; i < len; i += 32) df_acc_sqr(svh[i], svl[i], ss, se);
          df_warp_sum(ss, se);
          __syncwarp();
          if (lane == 0) {
            s_p = p;
            // reflector scalars in double-float: nx = sqrt(nx2), beta = -sign(x0) nx,
            // v0 = x0 - beta, tau = 2 / (nx2 - x0^2 + v0^2) = 1 / (nx (nx + |x0|))
            float n2h, n2l;
            df_fast_two_sum(ss, se, n2h, n2l);
            const float x0h = svh[0], x0l = svl[0];
            if (n2h > 0.f) {
              float nxh, nxl;
              df_sqrt(n2h, n2l, nxh, nxl);
              const bool pos = (x0h > 0.f) || (x0h == 0.f && x0l >= 0.f);
              // v0 = x0 + sign(x0) nx (no cancellation)
              float vh, vl;
              df_add(x0h, x0l, pos ? nxh : -nxh, pos ? nxl : -nxl, vh, vl);
              svh[0] = vh;
              svl[0] = vl;
              // tau = 1 / (nx (nx + |x0|))
              float ah, al;
              df_add(nxh, nxl, pos ? x0h : -x0h, pos ? x0l : -x0l, ah, al);
              float dh, dl;
              df_mul(nxh, nxl, ah, al, dh, dl);
              float th, tl;
              df_recip(dh, dl, th, tl);
              s_th = th;
              s_tl = tl;
              s_beta = pos ? -((double)nxh + (double)nxl) : ((double)nxh + (double)nxl);
              s_zero = 0;
            } else {
              s_beta = 0.0;
              s_th = 0.f;
              s_tl = 0.f;
              s_zero = 1;
            }
            s_g[0] = g.b1.h;
            s_g[1] = g.b1.l;
            s_g[2] = g.b2.h;
            s_g[3] = g.b2.l;
          }
        }
      }
    }
    __syncthreads();
    if (s_abort) return;
    if (s_stop) {
      steps = j;
      break;
    }
    const int64_t p = s_p;
    const float tauh = s_th, taul = s_tl;
    const bool zero = s_zero != 0;
    // pivot bookkeeping (block 0, warp 1), off the path to the next barrier
    if (blockIdx.x == 0 && warp == 1 && lane == 0) {
      diagR[j] = s_beta;
      const int64_t P = a.where[p];
      const int32_t cj = a.J[j];
      a.J[P] = cj;
      a.where[cj] = P;
      a.J[j] = (int32_t)p;
      a.where[p] = j;
      if (a.gaps) {
        const double n1 = sqrt((double)s_g[0] + (double)s_g[1]);
        a.gaps[j] = (s_g[2] < 0.f) ? __longlong_as_double(0x7ff0000000000000LL)
                                   : (n1 > 0.0 ? (n1 - sqrt((double)s_g[2] + (double)s_g[3])) / n1
                                               : 0.0);
      }
    }
    // the column pass specialised on the row slots in use, so that no
    // instruction is spent on slots beyond the active rows
    const int nt = (len + 31) >> 5;
    CpqrDfCol cp{Wh, Wl, nrm2, nref, cbase, svh, svl, r, j, len, p, c0, c1, tauh, taul, zero,
                 lane, warp, tolmode};
    Top2F best;
    double acc = 0.0;
    switch ((nt + SLOT_STEP<RPL>() - 1) / SLOT_STEP<RPL>()) {
      case 1: best = cp.template run<1 * SLOT_STEP<RPL>(), NWARP, VS>(acc); break;
      case 2: best = cp.template run<2 * SLOT_STEP<RPL>(), NWARP, VS>(acc); break;
      case 3: best = cp.template run<3 * SLOT_STEP<RPL>(), NWARP, VS>(acc); break;
      case 4: best = cp.template run<4 * SLOT_STEP<RPL>(), NWARP, VS>(acc); break;
      case 5: best = cp.template run<5 * SLOT_STEP<RPL>(), NWARP, VS>(acc); break;
      case 6: best = cp.template run<6 * SLOT_STEP<RPL>(), NWARP, VS>(acc); break;
      case 7: best = cp.template run<7 * SLOT_STEP<RPL>(), NWARP, VS>(acc); break;
      default: best = cp.template run<8 * SLOT_STEP<RPL>(), NWARP, VS>(acc); break;
    }
    if (lane == 0) {
      s_wsum[warp] = acc;
      s_wt[warp][0] = best.b1.h;
      s_wt[warp][1] = best.b1.l;
      s_wt[warp][2] = best.b2.h;
      s_wt[warp][3] = best.b2.l;
      s_wi[warp] = best.i1;
    }
    if (p >= c0 && p < c1 && tid == 0) nrm2[p - cbase] = make_float2(-1.f, 0.f);
    __syncthreads();
  }
  if (a.k_out && blockIdx.x == 0 && tid == 0) *a.k_out = steps;
}

template <int RPL, int NT, bool VS>
static cudaError_t launch_cpqr_df_t(const CpqrArgs& a, int sms, cudaStream_t s) {
  auto kern = cpqr_df_kernel<RPL, NT, VS>;
  // eight SMs are left to the Jacobi SVD (one 8-CTA cluster) that runs beside
  // the CPQR on another stream in the combined SVD + ID/CUR call
  int64_t G = sms > 16 ? sms - 8 : (sms > 1 ? sms - 1 : 1);
  const int64_t byn = ceil_div(a.n, 8);
  if (G > byn) G = byn;
  if (G > 1024) G = 1024;
  if (G < 1) G = 1;
  // the CTA's residual norms (12 bytes a column) go to shared memory when they
  // fit beside the Householder vector
  const int64_t per = ceil_div(a.n, G);
  size_t dyn = (size_t)a.r * 2 * sizeof(float);
  const size_t local = (size_t)per * (sizeof(float2) + sizeof(float));
  const bool nrm_local = dyn + local <= (size_t)160 * 1024;
  if (nrm_local) dyn += local;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  if (e != cudaSuccess) return e;
  if (dyn > 48 * 1024) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, dyn);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  CpqrArgs b = a;
  b.nrm_local = nrm_local ? 1 : 0;
  b.spin_limit = g_test_spin_limit > 0 ? g_test_spin_limit : SPIN_LIMIT_CYCLES;
  b.withhold = g_test_withhold;
  void* args[] = {(void*)&b};
  count_launch();
  const int tr = trace_begin(RSVD_TRACE_CPQR, s);
  e = cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)G), dim3(NT), args, dyn, s);
  trace_end(tr, s);
  return e;
}

cudaError_t launch_cpqr_df(const CpqrArgs& a, int* grid_out, cudaStream_t s) {
  (void)grid_out;
  if (a.r > 1024) return cudaErrorInvalidValue;
  const int sms = device_sm_count();
  if (a.r <= 256) return launch_cpqr_df_t<8, CPQR_NT8, false>(a, sms, s);
  return launch_cpqr_df_t<32, CPQR_DF_NT32, (CPQR_DF_NT32 > 256)>(a, sms, s);
}

// S11 (k x k, column-major, upper triangular with beta on the diagonal), the
// reciprocals of its diagonal and S12 (k x (n-k), row-major) as double-float
// pairs (float2 hi, lo), in pivot order, from the column-major planes.
__global__ void id_extract_df_kernel(int r, int64_t n, int k, const float* __restrict__ Wh,
                                     const float* __restrict__ Wl,
                                     const int32_t* __restrict__ J,
                                     const double* __restrict__ diagR, float2* __restrict__ S11,
                                     float2* __restrict__ dinv, float2* __restrict__ S12) {
  const int64_t total = n * (int64_t)k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t pos = t / k;
    const int i = (int)(t - pos * k);
    const int64_t c = J[pos];
    const int64_t o = c * r + i;            // column-major planes
    if (pos < k) {
      float2 v = make_float2(0.f, 0.f);
      if (i < pos) {
        v = make_float2(Wh[o], Wl[o]);
      } else if (i == pos) {
        float h, l;
        d_to_df(diagR[pos], h, l);
        v = make_float2(h, l);
        const double d = diagR[pos];
        float ih = 0.f, il = 0.f;
        if (d != 0.0) d_to_df(1.0 / d, ih, il);
        dinv[pos] = make_float2(ih, il);
      }
      S11[pos * k + i] = v;
    } else {
      S12[(int64_t)i * (n - k) + (pos - k)] = make_float2(Wh[o], Wl[o]);
    }
  }
}

cudaError_t launch_id_extract_df(int r, int64_t n, int k, const double* W, const int32_t* J,
                                 const double* diagR, double* S11, double* S12, cudaStream_t s) {
  const int64_t total = n * (int64_t)k;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 16384) blocks = 16384;
  const float* Wh = reinterpret_cast<const float*>(W);
  float2* s11 = reinterpret_cast<float2*>(S11);
  id_extract_df_kernel<<<(unsigned)blocks, 256, 0, s>>>(r, n, k, Wh, Wh + (int64_t)r * n, J,
                                                        diagR, s11, s11 + (int64_t)k * k,
                                                        reinterpret_cast<float2*>(S12));
  count_launch();
  return cudaGetLastError();
}

// Double-float back substitution for many right-hand sides,
// x_i = s_i (1 / U_ii); s_q -= x_i U_qi, with U (column-major k x k, float2)
// and the reciprocals of its diagonal as written by launch_id_extract_df.
__device__ __forceinline__ float2 df_mul2(float2 a, float2 b) {
  const float ph = __fmul_rn(a.x, b.x);
  float pe = __fmaf_rn(a.x, b.x, -ph);
  pe = __fmaf_rn(a.x, b.y, pe);
  pe = __fmaf_rn(a.y, b.x, pe);
  float h, l;
  df_fast_two_sum(ph, pe, h, l);
  return make_float2(h, l);
}
// s - x u
__device__ __forceinline__ float2 df_fms2(float2 s, float2 x, float2 u) {
  const float ph = __fmul_rn(x.x, u.x);
  float pe = __fmaf_rn(x.x, u.x, -ph);
  pe = __fmaf_rn(x.x, u.y, pe);
  pe = __fmaf_rn(x.y, u.x, pe);
  float a, b;
  df_two_sum(s.x, -ph, a, b);
  b = __fadd_rn(b, __fsub_rn(s.y, pe));
  float h, l;
  df_fast_two_sum(a, b, h, l);
  return make_float2(h, l);
}

// One warp solves NC right-hand sides at once (kk <= 32 RPL); lane l holds rows l + 32 t (t < RPL) of each.  Step i: the lane owning
// row i forms x_i = s_i / U_ii and broadcasts it; every lane updates its rows
// q < i with U(q, i), read coalesced from the column-major U.
__device__ __forceinline__ float2 load_df(const float2* p) { return *p; }
__device__ __forceinline__ float2 load_df(const float* p) { return make_float2(*p, 0.f); }

#ifndef SOLVE_NC8
#define SOLVE_NC8 2        // right-hand sides per warp of the 8-slot form
#endif
#ifndef SOLVE_MINB
#define SOLVE_MINB 3       // resident blocks per SM the 8-slot form's registers are set for
#endif
template <typename TR, typename TO, int NC, int RPL>
__global__ void __launch_bounds__(256, RPL <= 8 ? SOLVE_MINB : 2) upper_solve_df_warp_kernel(
    int kk, int64_t ncols, const float2* __restrict__ U, const float2* __restrict__ dinv,
    const TR* __restrict__ rhs, int64_t rs_i, int64_t rs_c, TO* __restrict__ out,
    int64_t os_i, int64_t os_c, int* d_info) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int nt = (kk + 31) >> 5;
  for (int64_t grp = gw; grp * NC < ncols; grp += nw) {
    const int64_t cbase = grp * NC;
    float sh[NC][RPL], sl[NC][RPL];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int i = lane + 32 * t;
        float2 v = make_float2(0.f, 0.f);
        if (t < nt && i < kk && cbase + c < ncols) v = load_df(rhs + i * rs_i + (cbase + c) * rs_c);
        sh[c][t] = v.x;
        sl[c][t] = v.y;
      }
    // steps i = kk - 1 .. 0 by row slot TI = i / 32, top slot first: inside a
    // slot its index is a compile-time constant, so x_i is read straight from
    // the owner's register and the slots below TI update without a test
    // (their rows q < 32 TI <= i)
#pragma unroll
    for (int TI = RPL - 1; TI >= 0; --TI) {
      if (TI >= nt) continue;                                  // uniform
      const int itop = min(kk - 1, 32 * TI + 31);
      for (int i = itop; i >= 32 * TI; --i) {
        const int owner = i & 31;
        const float2 di = __ldg(dinv + i);
        if (di.x == 0.f && grp == 0 && lane == 0) set_info(d_info, RSVD_ERR_NUMERIC);
        float xh[NC], xl[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const float2 x = df_mul2(make_float2(sh[c][TI], sl[c][TI]), di);
          xh[c] = __shfl_sync(0xffffffffu, x.x, owner);
          xl[c] = __shfl_sync(0xffffffffu, x.y, owner);
        }
        const float2* ucol = U + (int64_t)i * kk;
#pragma unroll
        for (int t = 0; t < TI; ++t) {
          const float2 u = __ldg(ucol + lane + 32 * t);
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            const float2 r = df_fms2(make_float2(sh[c][t], sl[c][t]), make_float2(xh[c], xl[c]), u);
            sh[c][t] = r.x;
            sl[c][t] = r.y;
          }
        }
        {
          const int q = lane + 32 * TI;
          if (q < i) {
            const float2 u = __ldg(ucol + q);
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              const float2 r =
                  df_fms2(make_float2(sh[c][TI], sl[c][TI]), make_float2(xh[c], xl[c]), u);
              sh[c][TI] = r.x;
              sl[c][TI] = r.y;
            }
          } else if (q == i) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              sh[c][TI] = xh[c];
              sl[c][TI] = xl[c];
            }
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int t = 0; t < RPL; ++t) {
        const int i = lane + 32 * t;
        if (t < nt && i < kk && cbase + c < ncols)
          out[i * os_i + (cbase + c) * os_c] = (TO)((double)sh[c][t] + (double)sl[c][t]);
      }
  }
}

template <typename TR, typename TO, int NC, int RPL>
static cudaError_t launch_solve_warp(int kk, int64_t ncols, const double* S11, const TR* rhs,
                                     int64_t rs_i, int64_t rs_c, TO* out, int64_t os_i,
                                     int64_t os_c, int* d_info, cudaStream_t s) {
  const float2* U = reinterpret_cast<const float2*>(S11);
  // one wave of resident blocks; warps stride over the column groups
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &per_sm, upper_solve_df_warp_kernel<TR, TO, NC, RPL>, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int64_t warps = ceil_div(ncols, NC);
  int64_t blocks = ceil_div(warps, 8);
  const int64_t cap = (int64_t)device_sm_count() * per_sm;
  if (blocks > cap) blocks = cap;
  const int tr_ = trace_begin(RSVD_TRACE_SOLVE, s);
  upper_solve_df_warp_kernel<TR, TO, NC, RPL><<<(unsigned)blocks, 256, 0, s>>>(
      kk, ncols, U, U + (int64_t)kk * kk, rhs, rs_i, rs_c, out, os_i, os_c, d_info);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

template <typename TR, typename TO>
cudaError_t launch_upper_solve_df(int kk, int64_t ncols, const double* S11, const TR* rhs,
                                  int64_t rs_i, int64_t rs_c, TO* out, int64_t os_i,
                                  int64_t os_c, int* d_info, cudaStream_t s) {
  if (kk <= 0 || ncols <= 0) return cudaSuccess;
  if (kk <= 256)
    return launch_solve_warp<TR, TO, SOLVE_NC8, 8>(kk, ncols, S11, rhs, rs_i, rs_c, out, os_i, os_c,
                                           d_info, s);
  if (kk <= 1024)
    return launch_solve_warp<TR, TO, 1, 32>(kk, ncols, S11, rhs, rs_i, rs_c, out, os_i, os_c,
                                            d_info, s);
  return cudaErrorInvalidValue;
}

// Upper-triangular R (kk x kk, R(i, t) = R[i*ldr + t], fp32 values) as the
// column-major float2 matrix and diagonal reciprocals of the solve above.
template <typename T>
__global__ void upper_to_df_kernel(int kk, const T* __restrict__ R, int64_t ldr,
                                   float2* __restrict__ U, float2* __restrict__ dinv) {
  const int64_t total = (int64_t)kk * kk;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(e / kk), i = (int)(e - (int64_t)t * kk);
    float2 v = make_float2(0.f, 0.f);
    if (i <= t) {
      float h, l;
      d_to_df((double)R[(int64_t)i * ldr + t], h, l);
      v = make_float2(h, l);
    }
    U[e] = v;
    if (i == t) {
      const double d = (double)R[(int64_t)i * ldr + i];
      float ih = 0.f, il = 0.f;
      if (d != 0.0) d_to_df(1.0 / d, ih, il);
      dinv[i] = make_float2(ih, il);
    }
  }
}

template <typename T>
cudaError_t launch_upper_to_df(int kk, const T* R, int64_t ldr, double* S11, cudaStream_t s) {
  if (kk <= 0) return cudaSuccess;
  float2* U = reinterpret_cast<float2*>(S11);
  const int64_t total = (int64_t)kk * kk;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 4096) blocks = 4096;
  upper_to_df_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(kk, R, ldr, U, U + total);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_upper_to_df<float>(int, const float*, int64_t, double*, cudaStream_t);

template cudaError_t launch_upper_solve_df<float2, float>(int, int64_t, const double*,
                                                          const float2*, int64_t, int64_t, float*,
                                                          int64_t, int64_t, int*, cudaStream_t);
template cudaError_t launch_upper_solve_df<float, float>(int, int64_t, const double*,
                                                         const float*, int64_t, int64_t, float*,
                                                         int64_t, int64_t, int*, cudaStream_t);

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
