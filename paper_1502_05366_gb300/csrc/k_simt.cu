// Plain SIMT GEMMs (fp32 / fp64 FMA): the arithmetic of the FP64 path, the
// RSVD_PREC_SIMT cross-check path and the small (k x k, l x l) products.
//
// gemm_nn:  C = A B      (sketch Y = A Omega with Omega generated per tile,
//                         power step Y = A Z, lift U = Q Vh)
// gemm_tn:  C = A^T B    (power step Z = A^* Y, QB step Bt = A^* Q, Gram X^T X)
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, NT = 256;
}

template <typename T, bool OMEGA>
__global__ void __launch_bounds__(NT) gemm_nn_kernel(int64_t M, int64_t N, int64_t K,
                                                     const T* __restrict__ A, int64_t lda,
                                                     const T* __restrict__ B, int64_t ldb,
                                                     T* __restrict__ C, int64_t ldc,
                                                     uint64_t seed, int64_t nvalid) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int64_t k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int t = 0; t < (BM * BK) / NT; ++t) {
      const int e = tid + NT * t;
      const int r = e / BK, kk = e % BK;
      const int64_t gr = m0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < K) ? A[gr * lda + gk] : T(0);
    }
    if (OMEGA) {
      const int kk = tid / 16, q = tid % 16;
      const int64_t gk = k0 + kk;
      T z[4];
      OmegaGen<T>::quad(seed, (uint32_t)gk, (uint32_t)(n0 / 4 + q), z);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t gc = n0 + 4 * q + c;
        Bs[kk][4 * q + c] = (gk < K && gc < nvalid) ? z[c] : T(0);
      }
    } else {
#pragma unroll
      for (int t = 0; t < (BN * BK) / NT; ++t) {
        const int e = tid + NT * t;
        const int kk = e / BN, c = e % BN;
        const int64_t gk = k0 + kk, gc = n0 + c;
        Bs[kk][c] = (gk < K && gc < N) ? B[gk * ldb + gc] : T(0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = m0 + ty + 16 * i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gc = n0 + tx + 16 * j;
      if (gc < N) C[gr * ldc + gc] = acc[i][j];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) gemm_tn_kernel(int64_t M, int64_t N, int64_t K,
                                                     const T* __restrict__ A, int64_t lda,
                                                     const T* __restrict__ B, int64_t ldb,
                                                     T* __restrict__ P, int64_t ldp,
                                                     int64_t kchunk) {
  __shared__ T As[BK][BM];
  __shared__ T Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t m0 = (int64_t)blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * BN;
  const int64_t kb = (int64_t)blockIdx.z * kchunk;
  const int64_t ke = min(K, kb + kchunk);
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

  for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int t = 0; t < (BM * BK) / NT; ++t) {
      const int e = tid + NT * t;
      const int kk = e / BM, r = e % BM;
      const int64_t gk = k0 + kk, gr = m0 + r;
      As[kk][r] = (gk < ke && gr < M) ? A[gk * lda + gr] : T(0);
    }
#pragma unroll
    for (int t = 0; t < (BN * BK) / NT; ++t) {
      const int e = tid + NT * t;
      const int kk = e / BN, c = e % BN;
      const int64_t gk = k0 + kk, gc = n0 + c;
      Bs[kk][c] = (gk < ke && gc < N) ? B[gk * ldb + gc] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  T* Pz = P + (int64_t)blockIdx.z * M * ldp;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = m0 + ty + 16 * i;
    if (gr >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gc = n0 + tx + 16 * j;
      if (gc < N) Pz[gr * ldp + gc] = acc[i][j];
    }
  }
}

template <typename T>
__global__ void reduce_slabs_kernel(int64_t M, int64_t ncols, int nsplit,
                                    const T* __restrict__ P, int64_t ldp, T* __restrict__ out,
                                    int64_t ldo) {
  const int64_t total = M * ncols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / ncols, j = t - i * ncols;
    T s = T(0);
    for (int z = 0; z < nsplit; ++z) s += P[(int64_t)z * M * ldp + i * ldp + j];
    out[i * ldo + j] = s;
  }
}

template <typename T>
cudaError_t launch_gemm_nn(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda,
                           const T* B, int64_t ldb, T* C, int64_t ldc, uint64_t seed,
                           int64_t nvalid, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(N, BN), (unsigned)ceil_div(M, BM));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  const int tr_ = trace_begin(RSVD_TRACE_SIMT, s);
  if (B == nullptr)
    gemm_nn_kernel<T, true><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, seed, nvalid);
  else
    gemm_nn_kernel<T, false><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, seed, nvalid);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

void tn_split(int64_t M, int64_t N, int64_t K, int num_sms, int* nsplit, int64_t* kchunk) {
  const int64_t base = ceil_div(M, BM) * ceil_div(N, BN);
  const int64_t target = 4LL * (num_sms > 0 ? num_sms : 148);
  int64_t ns = ceil_div(target, base);
  const int64_t maxs = ceil_div(K, 256);
  if (ns > maxs) ns = maxs;
  if (ns < 1) ns = 1;
  int64_t kc = round_up(ceil_div(K, ns), BK);
  if (kc < BK) kc = BK;
  *kchunk = kc;
  *nsplit = (int)ceil_div(K, kc);
  if (*nsplit < 1) *nsplit = 1;
}

template <typename T>
cudaError_t launch_gemm_tn_partial(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda,
                                   const T* B, int64_t ldb, T* P, int64_t ldp, int nsplit,
                                   int64_t kchunk, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(N, BN), (unsigned)ceil_div(M, BM), (unsigned)nsplit);
  if (grid.y > 65535u || grid.z > 65535u) return cudaErrorInvalidConfiguration;
  const int tr_ = trace_begin(RSVD_TRACE_SIMT, s);
  gemm_tn_kernel<T><<<grid, NT, 0, s>>>(M, N, K, A, lda, B, ldb, P, ldp, kchunk);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_reduce_slabs(int64_t M, int64_t ncols, int nsplit, const T* P, int64_t ldp,
                                T* out, int64_t ldo, cudaStream_t s) {
  const int64_t total = M * ncols;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = ceil_div(total, 256);
  if (blocks > 8192) blocks = 8192;
  reduce_slabs_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(M, ncols, nsplit, P, ldp, out, ldo);
  count_launch();
  return cudaGetLastError();
}

#define INST(T)                                                                             \
  template cudaError_t launch_gemm_nn<T>(int64_t, int64_t, int64_t, const T*, int64_t,       \
                                         const T*, int64_t, T*, int64_t, uint64_t, int64_t,  \
                                         cudaStream_t);                                      \
  template cudaError_t launch_gemm_tn_partial<T>(int64_t, int64_t, int64_t, const T*,        \
                                                 int64_t, const T*, int64_t, T*, int64_t,    \
                                                 int, int64_t, cudaStream_t);                \
  template cudaError_t launch_reduce_slabs<T>(int64_t, int64_t, int, const T*, int64_t, T*,  \
                                              int64_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace rsvd
