// Cholesky factor and inverse of the l x l Gram matrix for CholeskyQR.
//
// orth(X) (Sec. 2.1: an unpivoted QR whose Q is unique by diag(R) > 0) is
// computed as Q = X R^{-1} with G = X^T X = R^T R, repeated two or three times
// (CholeskyQR2/3).  A pass whose Gram has a pivot below tau * max(diag G),
// tau = 4 l eps, is redone with a diagonal shift (shifted CholeskyQR, Fukaya et
// al. 2020), the shift growing tenfold per retry; any shifted pass, or a second
// pass whose Gram is far from I, requests the third pass.  One CTA of 1024
// threads holds the matrix in shared memory (global memory beyond the limit).
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int CT = 512;
constexpr size_t SMEM_LIMIT = 212 * 1024;   // dynamic part; static arrays take <= 9 KB
template <typename T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ float eps_of<float>() { return 5.9604645e-8f; }
template <> __device__ __forceinline__ double eps_of<double>() { return 1.1102230246251565e-16; }
}  // namespace

// Global fallback when l x l does not fit in shared memory: the matrix plus a
// 32 x l block-row buffer for the blocked inverse.
size_t chol_scratch_bytes(int l, int elem) {
  const size_t b = (size_t)l * l * elem;
  return b <= SMEM_LIMIT ? 0 : b + (size_t)32 * l * elem;
}

template <typename T>
__device__ void block_max(T v, T* red, T* out) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nw = (blockDim.x * blockDim.y) / 32;
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    T w = tid < nw ? red[tid] : T(0);
    for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    if (tid == 0) *out = w;
  }
  __syncthreads();
}

template <typename T>
__device__ void write_identity_outputs(const CholArgs& a) {
  const int L = a.L;
  for (int i = threadIdx.y; i < L; i += blockDim.y)
  for (int c = threadIdx.x; c < L; c += blockDim.x) {
    const int t = i * L + c;
    const T v = (i == c) ? T(1) : T(0);
    if (a.R) ((T*)a.R)[t] = v;
    if (a.Rinv) ((T*)a.Rinv)[t] = v;
    if (a.Whi) {
      ((__nv_bfloat16*)a.Whi)[t] = __float2bfloat16_rn((float)v);
      ((__nv_bfloat16*)a.Wlo)[t] = __float2bfloat16_rn(0.0f);
      ((__nv_bfloat16*)a.Wlo2)[t] = __float2bfloat16_rn(0.0f);
    }
  }
}

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky G = R^T R on the l x l row-major matrix S
// (upper triangle used, R left there), panels of NB = 32 columns:
//   (a) the diagonal block is factored by warp 0 in registers (lane c holds
//       column c of the block; row j of R is shared by shuffles);
//   (b) the panel row block becomes R_pp^{-T} S_panel (one thread per column);
//   (c) the trailing upper triangle is updated with 4 x 4 register tiles.
// A pivot not above thr stops the factorization and records its column.
// ---------------------------------------------------------------------------
constexpr int NB = 32;

template <typename T>
__device__ void chol_blocked(T* S, int l, T thr, int* s_fail) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nthr = blockDim.x * blockDim.y;
  for (int p0 = 0; p0 < l; p0 += NB) {
    const int pb = min(NB, l - p0);
    if (warp == 0) {
      T d[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i)
        d[i] = (lane < pb && i <= lane) ? S[(p0 + i) * l + p0 + lane] : T(0);
      int failed = -1;
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) {
        if (jj < pb && failed < 0) {
          const T piv = __shfl_sync(0xffffffffu, d[jj], jj);
          if (!(piv > thr)) {
            failed = jj;
          } else {
            const T r = sqrt(piv);
            T rj = d[jj];
            if (lane == jj) rj = r;
            else if (lane > jj) rj = rj / r;
            d[jj] = rj;
#pragma unroll
            for (int i = jj + 1; i < NB; ++i) {
              const T ri = __shfl_sync(0xffffffffu, rj, i);
              if (lane >= i) d[i] -= ri * rj;
            }
          }
        }
      }
      if (failed < 0) {
#pragma unroll
        for (int i = 0; i < NB; ++i)
          if (lane < pb && i <= lane) S[(p0 + i) * l + p0 + lane] = d[i];
      } else if (lane == 0) {
        *s_fail = p0 + failed;
      }
    }
    __syncthreads();
    if (*s_fail >= 0) return;
    const int c0 = p0 + pb, nt = l - c0;
    if (nt <= 0) return;
    // (b) X = R_pp^{-T} S(p0:p0+pb, c0:l), forward substitution per column
    for (int c = c0 + tid; c < l; c += nthr) {
      T x[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i < pb) {
          T acc = S[(p0 + i) * l + c];
#pragma unroll
          for (int t = 0; t < i; ++t) acc -= S[(p0 + t) * l + p0 + i] * x[t];
          x[i] = acc / S[(p0 + i) * l + p0 + i];
        } else {
          x[i] = T(0);
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < pb) S[(p0 + i) * l + c] = x[i];
    }
    __syncthreads();
    // (c) trailing update of the upper triangle: S(i, c) -= sum_t X(t, i) X(t, c)
    const int nT = (nt + 3) / 4;
    for (int tt = tid; tt < nT * nT; tt += nthr) {
      const int ti = tt / nT, tc = tt - ti * nT;
      if (tc < ti) continue;
      const int i0 = c0 + 4 * ti, k0 = c0 + 4 * tc;
      T acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = T(0);
      for (int t = 0; t < pb; ++t) {
        const T* row = S + (p0 + t) * l;
        T xi[4], xc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xi[q] = (i0 + q < l) ? row[i0 + q] : T(0);
          xc[q] = (k0 + q < l) ? row[k0 + q] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] = fma(xi[q], xc[w], acc[q][w]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int i = i0 + q, c = k0 + w;
          if (i < l && c < l && c >= i) S[i * l + c] -= acc[q][w];
        }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// In-place inverse of the upper-triangular R held in the upper triangle of S
// (l x l row-major), by block rows from the bottom:
//   T = E_I - R(I, I+1:) X(I+1:, :)   (E_I: rows of the identity)
//   X(I, :) = R_II^{-1} T             (back substitution, one thread per column)
// R_II is copied aside first since X(I, :) overwrites row block I.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void inv_upper_blocked(T* S, int l, T* ttmp) {
  __shared__ T Rd[NB][NB + 1];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
  const int nb = (l + NB - 1) / NB;
  constexpr int MAXE = 16;
  for (int Ib = nb - 1; Ib >= 0; --Ib) {
    const int r0 = Ib * NB, rb = min(NB, l - r0);
    const int ncol = l - r0;
    const int ne = rb * ncol;
    for (int t = tid; t < NB * NB; t += nthr) {
      const int i = t / NB, c = t - i * NB;
      Rd[i][c] = (i < rb && c < rb && c >= i) ? S[(r0 + i) * l + r0 + c] : T(0);
    }
    if (ttmp) {   // large l: T through the global buffer
      for (int e = tid; e < ne; e += nthr) {
        const int i = r0 + e / ncol, c = r0 + e % ncol;
        T acc = (i == c) ? T(1) : T(0);
        for (int t = r0 + rb; t <= c; ++t) acc -= S[i * l + t] * S[t * l + c];
        ttmp[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < ne; e += nthr) S[(r0 + e / ncol) * l + r0 + e % ncol] = ttmp[e];
    } else {      // T into registers (at most MAXE elements per thread)
      T tv[MAXE];
#pragma unroll
      for (int u = 0; u < MAXE; ++u) {
        const int e = tid + u * nthr;
        tv[u] = T(0);
        if (e < ne) {
          const int i = r0 + e / ncol, c = r0 + e % ncol;
          T acc = (i == c) ? T(1) : T(0);
          for (int t = r0 + rb; t <= c; ++t) acc -= S[i * l + t] * S[t * l + c];
          tv[u] = acc;
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < MAXE; ++u) {
        const int e = tid + u * nthr;
        if (e < ne) S[(r0 + e / ncol) * l + r0 + e % ncol] = tv[u];
      }
    }
    __syncthreads();
    // X(I, c) = R_II^{-1} T(:, c)
    for (int c = r0 + tid; c < l; c += nthr) {
      T x[NB];
#pragma unroll
      for (int i = NB - 1; i >= 0; --i) {
        if (i < rb) {
          T acc = S[(r0 + i) * l + c];
#pragma unroll
          for (int t = i + 1; t < NB; ++t)
            if (t < rb) acc -= Rd[i][t] * x[t];
          x[i] = acc / Rd[i][i];
        } else {
          x[i] = T(0);
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < rb) S[(r0 + i) * l + c] = x[i];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(CT) chol_kernel(CholArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ T red[32];
  __shared__ T s_maxdiag, s_dev;
  __shared__ int s_fail;
  const int l = a.l, L = a.L;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int tx = threadIdx.x, ty = threadIdx.y, nty = blockDim.y;
  T* S = a.scratch ? (T*)a.scratch : (T*)dsm;
  const T* G = (const T*)a.G;
  const int64_t ldg = a.ldg;

  if (a.skip_idx >= 0 && a.flags && a.flags[a.skip_idx] == 1) {  // pass not needed: R = I
    write_identity_outputs<T>(a);
    return;
  }

  // scale of G and, on the second pass, its distance to I
  T md = T(0), dev = T(0);
  bool bad = false;
  for (int i = ty; i < l; i += nty)
    for (int c = tx; c < l; c += 32) {
      const T g = G[(int64_t)i * ldg + c];
      if (!isfinite(g)) bad = true;
      if (i == c) md = max(md, g);
      dev = max(dev, abs(g - (i == c ? T(1) : T(0))));
    }
  if (bad) set_info(a.d_info, RSVD_ERR_NUMERIC);
  block_max<T>(md, red, &s_maxdiag);
  block_max<T>(dev, red, &s_dev);
  const T maxdiag = s_maxdiag;
  if (!(maxdiag > T(0))) {                       // X = 0 or non-finite: no basis
    set_info(a.d_info, RSVD_ERR_NOT_SPD);
    write_identity_outputs<T>(a);
    return;
  }
  const T tau = T(4) * T(l) * eps_of<T>();
  T shift = T(0);
  int used_shift = 0;
  int fail = -1;
  for (int attempt = 0; attempt < 12; ++attempt) {
    for (int i = ty; i < l; i += nty)
      for (int c = tx; c < l; c += 32) S[i * l + c] = G[(int64_t)i * ldg + c] + ((i == c) ? shift : T(0));
    if (tid == 0) s_fail = -1;
    __syncthreads();
    chol_blocked<T>(S, l, tau * maxdiag, &s_fail);
    fail = s_fail;
    __syncthreads();
    if (fail < 0) break;
    shift = (shift == T(0)) ? tau * maxdiag : shift * T(10);
    used_shift = 1;
  }
  if (fail >= 0) {
    set_info(a.d_info, RSVD_ERR_NOT_SPD);
    write_identity_outputs<T>(a);
    return;
  }
  if (tid == 0 && a.flags) {
    if (a.pass == 1) {
      a.flags[1] = used_shift;
      // conditional second pass (inside the power scheme): only after a shift;
      // the third pass is skipped unless the second one asks for it
      a.flags[3] = used_shift ? 0 : 1;
      a.flags[2] = 1;
    } else if (a.pass == 2) {
      a.flags[1] |= used_shift;
      a.flags[0] = (a.flags[1] || T(l) * s_dev > T(0.5)) ? 1 : 0;
      a.flags[2] = 1 - a.flags[0];   // skip flag of the third pass
    }
  }
  // R out (identity on the padding)
  if (a.R) {
    T* R = (T*)a.R;
    for (int i = ty; i < L; i += nty)
      for (int c = tx; c < L; c += 32) {
        T v;
        if (i < l && c < l) v = (c >= i) ? S[i * l + c] : T(0);
        else v = (i == c) ? T(1) : T(0);
        R[i * L + c] = v;
      }
  }
  inv_upper_blocked<T>(S, l, a.scratch ? (T*)a.scratch + (size_t)l * l : nullptr);
  if (a.Rinv) {
    T* Ri = (T*)a.Rinv;
    for (int i = ty; i < L; i += nty)
      for (int c = tx; c < L; c += 32) {
        T v;
        if (i < l && c < l) v = (c >= i) ? S[i * l + c] : T(0);
        else v = (i == c) ? T(1) : T(0);
        Ri[i * L + c] = v;
      }
  }
  if (a.Whi) {  // W^T with W = R^{-1}: Wt[j][kk] = Rinv[kk][j], three bf16 terms (24 bits)
    __nv_bfloat16* hi = (__nv_bfloat16*)a.Whi;
    __nv_bfloat16* lo = (__nv_bfloat16*)a.Wlo;
    __nv_bfloat16* lo2 = (__nv_bfloat16*)a.Wlo2;
    for (int j = ty; j < L; j += nty)
    for (int kk = tx; kk < L; kk += 32) {
      const int t = j * L + kk;
      float v;
      if (j < l && kk < l) v = (j >= kk) ? (float)S[kk * l + j] : 0.0f;
      else v = (j == kk) ? 1.0f : 0.0f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(h);
      const __nv_bfloat16 mdl = __float2bfloat16_rn(r1);
      hi[t] = h;
      lo[t] = mdl;
      lo2[t] = __float2bfloat16_rn(r1 - __bfloat162float(mdl));
    }
  }
}

// Racc <- R * Racc for upper-triangular L x L matrices (through tmp).
template <typename T>
__global__ void trmm_upper_kernel(int L, const T* __restrict__ R, const T* __restrict__ Racc,
                                  T* __restrict__ tmp) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L * L; t += gridDim.x * blockDim.x) {
    const int i = t / L, c = t - i * L;
    T s = T(0);
    if (c >= i)
      for (int q = i; q <= c; ++q) s += R[i * L + q] * Racc[q * L + c];
    tmp[t] = s;
  }
}

template <typename T>
cudaError_t launch_chol(const CholArgs& a, cudaStream_t s) {
  const size_t bytes = (size_t)a.l * a.l * sizeof(T);
  CholArgs b = a;
  size_t dyn = 0;
  if (bytes <= SMEM_LIMIT) {
    b.scratch = nullptr;
    dyn = bytes;
  } else if (a.scratch == nullptr) {
    return cudaErrorInvalidValue;
  }
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(chol_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  const int tr_ = trace_begin(RSVD_TRACE_CHOL, s);
  chol_kernel<T><<<1, dim3(32, CT / 32), dyn, s>>>(b);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trmm_upper(int L, const T* R, T* Racc, T* tmp, cudaStream_t s) {
  const int blocks = (L * L + 255) / 256;
  trmm_upper_kernel<T><<<blocks, 256, 0, s>>>(L, R, Racc, tmp);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(Racc, tmp, sizeof(T) * L * L, cudaMemcpyDeviceToDevice, s);
}

template cudaError_t launch_chol<float>(const CholArgs&, cudaStream_t);
template cudaError_t launch_chol<double>(const CholArgs&, cudaStream_t);
template cudaError_t launch_trmm_upper<float>(int, const float*, float*, float*, cudaStream_t);
template cudaError_t launch_trmm_upper<double>(int, const double*, double*, double*,
                                               cudaStream_t);

}  // namespace rsvd
