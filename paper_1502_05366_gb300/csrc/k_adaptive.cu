// Kernels of the blocked adaptive QB (Alg. 7): the update of a matrix by a
// rank-K product, X <- X - Q Bt^T, with the squared Frobenius norm of the
// updated X reduced per CTA, and the fixed-order finish of that norm.
//
// The same kernel serves the two updates of Alg. 7: A <- A - Q_t B_t (K = b,
// X = A, m x n: one read and one write of A, HBM-bound) and the re-projection
// Q_t <- Q_t - Qbar (Qbar^* Q_t) (K = b t, X = Q_t, m x b).  With K = 0 it only
// reads X and reduces its norm (||A_in||_F for a relative tolerance).
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int RU_T = 256;   // 16 x 16 threads, each 4 x 4 outputs
constexpr int RU_M = 64;    // tile rows
constexpr int RU_N = 64;    // tile columns
constexpr int RU_K = 16;    // contraction chunk staged in shared memory
}  // namespace

int64_t rank_update_tiles(int64_t rows, int64_t cols) {
  return ceil_div(rows, RU_M) * ceil_div(cols, RU_N);
}

// Tile (r0, c0) of X (rows x cols, ld ldx): X(r, c) -= sum_k Q(r, k) Bt(c, k).
// Thread (ty, tx) owns rows r0 + ty + 16 i and columns c0 + tx + 16 j.  When
// sumsq is set, sumsq[tile] = sum of X(r, c)^2 over the updated tile, in a
// fixed order (per thread, then a shared-memory tree).
template <typename T>
__global__ void __launch_bounds__(RU_T) rank_update_kernel(int64_t rows, int64_t cols,
                                                           T* __restrict__ X, int64_t ldx,
                                                           const T* __restrict__ Q, int64_t ldq,
                                                           const T* __restrict__ Bt, int64_t ldb,
                                                           int K, int64_t ntc,
                                                           double* __restrict__ sumsq) {
  __shared__ T Qs[RU_K][RU_M + 4];   // Qs[kk][r] = Q(r0 + r, k0 + kk)
  __shared__ T Bs[RU_K][RU_N + 4];   // Bs[kk][c] = Bt(c0 + c, k0 + kk)
  __shared__ double red[RU_T];
  const int64_t tile = blockIdx.x;
  const int64_t r0 = (tile / ntc) * RU_M, c0 = (tile % ntc) * RU_N;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < K; k0 += RU_K) {
    for (int e = tid; e < RU_M * RU_K; e += RU_T) {
      const int r = e / RU_K, kk = e - (e / RU_K) * RU_K;
      const int k = k0 + kk;
      const int64_t gr = r0 + r, gc = c0 + r;
      Qs[kk][r] = (gr < rows && k < K) ? Q[gr * ldq + k] : T(0);
      Bs[kk][r] = (gc < cols && k < K) ? Bt[gc * ldb + k] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < RU_K; ++kk) {
      T a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Qs[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  double ss = 0.0;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t gr = r0 + ty + 16 * i;
    if (gr >= rows) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gc = c0 + tx + 16 * j;
      if (gc >= cols) continue;
      T v = X[gr * ldx + gc];
      if (K > 0) {
        v -= acc[i][j];
        X[gr * ldx + gc] = v;
      }
      ss += (double)v * (double)v;
    }
  }
  if (!sumsq) return;   // uniform over the CTA
  red[tid] = ss;
  __syncthreads();
  for (int o = RU_T / 2; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  if (tid == 0) sumsq[tile] = red[0];
}

template <typename T>
cudaError_t launch_rank_update(int64_t rows, int64_t cols, T* X, int64_t ldx, const T* Q,
                               int64_t ldq, const T* Bt, int64_t ldb, int K, double* sumsq,
                               cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  if (K < 0 || (K > 0 && (!Q || !Bt))) return cudaErrorInvalidValue;
  const int64_t tiles = rank_update_tiles(rows, cols);
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  rank_update_kernel<T><<<(unsigned)tiles, RU_T, 0, s>>>(rows, cols, X, ldx, Q, ldq, Bt, ldb, K,
                                                         ceil_div(cols, RU_N), sumsq);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_rank_update<float>(int64_t, int64_t, float*, int64_t, const float*,
                                               int64_t, const float*, int64_t, int, double*,
                                               cudaStream_t);
template cudaError_t launch_rank_update<double>(int64_t, int64_t, double*, int64_t,
                                                const double*, int64_t, const double*, int64_t,
                                                int, double*, cudaStream_t);

// *out = sqrt(sum of the nparts partial sums), summed in a fixed order (strided
// per thread, then a tree); a non-finite result sets RSVD_ERR_NUMERIC.
__global__ void __launch_bounds__(1024) sumsq_finish_kernel(int64_t nparts,
                                                            const double* __restrict__ parts,
                                                            double* __restrict__ out,
                                                            int* d_info) {
  __shared__ double red[1024];
  const int tid = threadIdx.x;
  double s = 0.0;
  for (int64_t t = tid; t < nparts; t += 1024) s += parts[t];
  red[tid] = s;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  if (tid == 0) {
    const double v = sqrt(red[0]);
    *out = v;
    if (!isfinite(v)) set_info(d_info, RSVD_ERR_NUMERIC);
  }
}

cudaError_t launch_sumsq_finish(int64_t nparts, const double* parts, double* out, int* d_info,
                                cudaStream_t s) {
  if (nparts <= 0) return cudaErrorInvalidValue;
  sumsq_finish_kernel<<<1, 1024, 0, s>>>(nparts, parts, out, d_info);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rsvd
