// One-sided (Hestenes) Jacobi SVD of the small l x l core of Alg. 5.
//
// The columns x_j of M are rotated in pairs until every pair is orthogonal to
// |x_a . x_b| <= tol ||x_a|| ||x_b|| (tol = sqrt(l) eps), so M V = X with
// orthogonal columns; then sigma_j = ||x_j||, Uh(:, rank(j)) = x_j / sigma_j
// with the ranks sorting sigma in descending order (ties: lower column first).
// Rounded fp32 rotations are not exactly orthogonal, so the column norms of X
// drift by O(eps) per rotation; the singular values are therefore taken
// afterwards from the original matrix, sigma_j = ||M^T u_j|| (M^T u_j = sigma_j
// v_j), which also gives v_j (svd_finalize_kernel, after P = M^T Uh).
// Pairs are visited in the round-robin (circle) order, l/2 disjoint pairs per
// round, one warp per pair; one CTA of 1024 threads holds X in shared memory
// (global memory beyond the limit).
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int JT = 1024;
constexpr size_t JSMEM_LIMIT = 212 * 1024;
template <typename T> __device__ __forceinline__ T jeps();
template <> __device__ __forceinline__ float jeps<float>() { return 5.9604645e-8f; }
template <> __device__ __forceinline__ double jeps<double>() { return 1.1102230246251565e-16; }
}  // namespace

size_t jacobi_scratch_bytes(int l, int elem) {
  const size_t b = (size_t)l * l * elem;
  return b <= JSMEM_LIMIT ? 0 : b;
}

__device__ __forceinline__ void rr_pair(int r, int p, int N, int* a, int* b) {
  if (p == 0) {
    *a = N - 1;
    *b = r;
  } else {
    *a = (r + p) % (N - 1);
    *b = (r - p + N - 1) % (N - 1);
  }
}

template <typename T>
__global__ void __launch_bounds__(JT) jacobi_kernel(int l, const T* __restrict__ M, int64_t ldm,
                                                    T* __restrict__ Uh, int64_t lduh,
                                                    double* __restrict__ Sh, T* scratch,
                                                    int max_sweeps, int* d_info) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double s_sig[1024];
  __shared__ int s_rot;
  T* X = scratch ? scratch : (T*)dsm;  // column-major: X[j*l + i]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = JT / 32;
  for (int t = tid; t < l * l; t += JT) {
    const int j = t / l, i = t - j * l;
    X[t] = M[(int64_t)i * ldm + j];
  }
  __syncthreads();
  const int N = l + (l & 1);
  const T tol = sqrt((T)l) * jeps<T>();
  bool converged = (l == 1);
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    if (tid == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      for (int p = warp; p < N / 2; p += nwarp) {
        int a, b;
        rr_pair(r, p, N, &a, &b);
        if (a >= l || b >= l) continue;
        T* xa = X + (int64_t)a * l;
        T* xb = X + (int64_t)b * l;
        T al = T(0), be = T(0), ga = T(0);
        for (int i = lane; i < l; i += 32) {
          const T u = xa[i], v = xb[i];
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
        al = warp_sum(al);
        be = warp_sum(be);
        ga = warp_sum(ga);
        if (!(al > T(0)) || !(be > T(0))) continue;
        if (!(abs(ga) > tol * sqrt(al) * sqrt(be))) continue;
        const T zeta = (be - al) / (T(2) * ga);
        const T t = (zeta >= T(0) ? T(1) : T(-1)) / (abs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t);
        const T s = c * t;
        for (int i = lane; i < l; i += 32) {
          const T u = xa[i], v = xb[i];
          xa[i] = c * u - s * v;
          xb[i] = s * u + c * v;
        }
        if (lane == 0) atomicAdd(&s_rot, 1);
      }
      __syncthreads();
    }
    converged = (s_rot == 0);
    __syncthreads();
  }
  if (!converged) set_info(d_info, RSVD_ERR_NO_CONVERGENCE);
  for (int j = warp; j < l; j += nwarp) {
    const T* xj = X + (int64_t)j * l;
    double acc = 0.0;
    T s = T(0);
    for (int i = lane; i < l; i += 32) s = fma(xj[i], xj[i], s);
    s = warp_sum(s);
    acc = (double)sqrt(s);
    if (lane == 0) {
      s_sig[j] = acc;
      if (!isfinite(acc)) set_info(d_info, RSVD_ERR_NUMERIC);
    }
  }
  __syncthreads();
  for (int j = warp; j < l; j += nwarp) {
    const double sj = s_sig[j];
    int rank = 0;
    for (int i = lane; i < l; i += 32) {
      const double si = s_sig[i];
      rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const T inv = sj > 0.0 ? (T)(1.0 / sj) : T(0);
    const T* xj = X + (int64_t)j * l;
    for (int i = lane; i < l; i += 32) Uh[(int64_t)i * lduh + rank] = xj[i] * inv;
    if (lane == 0) Sh[rank] = sj;
  }
}

// P = M^T Uh (l x l): sigma_j = ||P(:, j)|| (FP64 accumulation), sorted in
// descending order (ties: lower column first); Sh, Vh(:, r) = P(:, j) / sigma_j
// and Uh(:, r) = Uin(:, j) with r the rank of column j.
template <typename T>
__global__ void __launch_bounds__(1024) svd_finalize_kernel(int l, const T* __restrict__ P,
                                                            int64_t ldp, const T* __restrict__ Uin,
                                                            int64_t ldin, T* __restrict__ Uh,
                                                            int64_t lduh, double* __restrict__ Sh,
                                                            T* __restrict__ Vh, int64_t ldvh,
                                                            int* d_info) {
  __shared__ double s_sig[1024];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x / 32;
  for (int j = warp; j < l; j += nwarp) {
    double s = 0.0;
    for (int i = lane; i < l; i += 32) {
      const double v = (double)P[(int64_t)i * ldp + j];
      s = fma(v, v, s);
    }
    s = warp_sum(s);
    if (lane == 0) {
      s_sig[j] = sqrt(s);
      if (!isfinite(s)) set_info(d_info, RSVD_ERR_NUMERIC);
    }
  }
  __syncthreads();
  for (int j = warp; j < l; j += nwarp) {
    const double sj = s_sig[j];
    int rank = 0;
    for (int i = lane; i < l; i += 32) {
      const double si = s_sig[i];
      rank += (si > sj || (si == sj && i < j)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const double inv = sj > 0.0 ? 1.0 / sj : 0.0;
    for (int i = lane; i < l; i += 32) {
      Vh[(int64_t)i * ldvh + rank] = (T)((double)P[(int64_t)i * ldp + j] * inv);
      Uh[(int64_t)i * lduh + rank] = Uin[(int64_t)i * ldin + j];
    }
    if (lane == 0) Sh[rank] = sj;
  }
}

template <typename T>
cudaError_t launch_svd_finalize(int l, const T* P, int64_t ldp, const T* Uin, int64_t ldin, T* Uh,
                                int64_t lduh, double* Sh, T* Vh, int64_t ldvh, int* d_info,
                                cudaStream_t s) {
  if (l > 1024) return cudaErrorInvalidValue;
  svd_finalize_kernel<T><<<1, 1024, 0, s>>>(l, P, ldp, Uin, ldin, Uh, lduh, Sh, Vh, ldvh, d_info);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_svd_finalize<float>(int, const float*, int64_t, const float*, int64_t,
                                                float*, int64_t, double*, float*, int64_t, int*,
                                                cudaStream_t);
template cudaError_t launch_svd_finalize<double>(int, const double*, int64_t, const double*,
                                                 int64_t, double*, int64_t, double*, double*,
                                                 int64_t, int*, cudaStream_t);

template <typename T>
cudaError_t launch_jacobi(int l, const T* M, int64_t ldm, T* Uh, int64_t lduh, double* Sh,
                          T* Vh, int64_t ldvh, T* scratch, int max_sweeps, int* d_info,
                          cudaStream_t s) {
  (void)Vh;
  (void)ldvh;
  if (l > 1024) return cudaErrorInvalidValue;
  const size_t bytes = (size_t)l * l * sizeof(T);
  size_t dyn = 0;
  T* scr = nullptr;
  if (bytes <= JSMEM_LIMIT) {
    dyn = bytes;
  } else {
    if (!scratch) return cudaErrorInvalidValue;
    scr = scratch;
  }
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(jacobi_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  jacobi_kernel<T><<<1, JT, dyn, s>>>(l, M, ldm, Uh, lduh, Sh, scr, max_sweeps, d_info);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_jacobi<float>(int, const float*, int64_t, float*, int64_t, double*,
                                          float*, int64_t, float*, int, int*, cudaStream_t);
template cudaError_t launch_jacobi<double>(int, const double*, int64_t, double*, int64_t,
                                           double*, double*, int64_t, double*, int, int*,
                                           cudaStream_t);

}  // namespace rsvd
