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
constexpr int CT = 1024;
constexpr size_t SMEM_LIMIT = 212 * 1024;   // dynamic part; static arrays take <= 9 KB
template <typename T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ float eps_of<float>() { return 5.9604645e-8f; }
template <> __device__ __forceinline__ double eps_of<double>() { return 1.1102230246251565e-16; }
}  // namespace

size_t chol_scratch_bytes(int l, int elem) {
  const size_t b = (size_t)l * l * elem;
  return b <= SMEM_LIMIT ? 0 : b;
}

template <typename T>
__device__ void block_max(T v, T* red, T* out) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    T w = red[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    if (threadIdx.x == 0) *out = w;
  }
  __syncthreads();
}

template <typename T>
__device__ void write_identity_outputs(const CholArgs& a) {
  const int L = a.L;
  for (int t = threadIdx.x; t < L * L; t += blockDim.x) {
    const int i = t / L, c = t - i * L;
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

template <typename T>
__global__ void __launch_bounds__(CT) chol_kernel(CholArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ T dg[1024];
  __shared__ T red[32];
  __shared__ T s_maxdiag, s_dev;
  __shared__ int s_fail;
  const int l = a.l, L = a.L;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = CT / 32;
  T* S = a.scratch ? (T*)a.scratch : (T*)dsm;
  const T* G = (const T*)a.G;
  const int64_t ldg = a.ldg;

  if (a.pass == 3 && a.flags && a.flags[0] == 0) {  // third pass not needed: R = I
    write_identity_outputs<T>(a);
    return;
  }

  // scale of G and, on the second pass, its distance to I
  T md = T(0), dev = T(0);
  bool bad = false;
  for (int t = tid; t < l * l; t += CT) {
    const int i = t / l, c = t - i * l;
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
    for (int t = tid; t < l * l; t += CT) {
      const int i = t / l, c = t - i * l;
      S[t] = G[(int64_t)i * ldg + c] + ((i == c) ? shift : T(0));
    }
    if (tid == 0) s_fail = -1;
    __syncthreads();
    // right-looking Cholesky G = R^T R, R in the upper triangle of S
    for (int j = 0; j < l; ++j) {
      if (tid == 0) {
        const T d = S[j * l + j];
        if (!(d > tau * maxdiag)) s_fail = j;
        else dg[j] = sqrt(d);
      }
      __syncthreads();
      if (s_fail >= 0) break;
      const T r = dg[j];
      for (int c = j + 1 + tid; c < l; c += CT) S[j * l + c] /= r;
      if (tid == 0) S[j * l + j] = r;
      __syncthreads();
      for (int i = j + 1 + warp; i < l; i += nwarp) {
        const T sji = S[j * l + i];
        for (int c = i + lane; c < l; c += 32) S[i * l + c] -= sji * S[j * l + c];
      }
      __syncthreads();
    }
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
    } else if (a.pass == 2) {
      a.flags[1] |= used_shift;
      a.flags[0] = (a.flags[1] || T(l) * s_dev > T(0.5)) ? 1 : 0;
      a.flags[2] = 1 - a.flags[0];   // skip flag of the third pass
    }
  }
  // R out (identity on the padding)
  if (a.R) {
    T* R = (T*)a.R;
    for (int t = tid; t < L * L; t += CT) {
      const int i = t / L, c = t - i * L;
      T v;
      if (i < l && c < l) v = (c >= i) ? S[i * l + c] : T(0);
      else v = (i == c) ? T(1) : T(0);
      R[t] = v;
    }
  }
  // R^T into the strict lower triangle, diagonal kept in dg
  for (int t = tid; t < l * l; t += CT) {
    const int i = t / l, c = t - i * l;
    if (c < i) S[i * l + c] = S[c * l + i];
  }
  __syncthreads();
  for (int t = tid; t < l * l; t += CT) {
    const int i = t / l, c = t - i * l;
    if (c >= i) S[t] = (i == c) ? T(1) : T(0);   // B = I in the upper triangle
  }
  __syncthreads();
  // back substitution R X = I, row i from the bottom; X overwrites B (upper)
  for (int i = l - 1; i >= 0; --i) {
    const T inv = T(1) / dg[i];
    for (int c = i + tid; c < l; c += CT) S[i * l + c] *= inv;
    __syncthreads();
    for (int r = warp; r < i; r += nwarp) {
      const T rri = S[i * l + r];                 // R[r][i]
      for (int c = i + lane; c < l; c += 32) S[r * l + c] -= rri * S[i * l + c];
    }
    __syncthreads();
  }
  if (a.Rinv) {
    T* Ri = (T*)a.Rinv;
    for (int t = tid; t < L * L; t += CT) {
      const int i = t / L, c = t - i * L;
      T v;
      if (i < l && c < l) v = (c >= i) ? S[i * l + c] : T(0);
      else v = (i == c) ? T(1) : T(0);
      Ri[t] = v;
    }
  }
  if (a.Whi) {  // W^T with W = R^{-1}: Wt[j][kk] = Rinv[kk][j], three bf16 terms (24 bits)
    __nv_bfloat16* hi = (__nv_bfloat16*)a.Whi;
    __nv_bfloat16* lo = (__nv_bfloat16*)a.Wlo;
    __nv_bfloat16* lo2 = (__nv_bfloat16*)a.Wlo2;
    for (int t = tid; t < L * L; t += CT) {
      const int j = t / L, kk = t - j * L;
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
  chol_kernel<T><<<1, CT, dyn, s>>>(b);
  count_launch();
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
