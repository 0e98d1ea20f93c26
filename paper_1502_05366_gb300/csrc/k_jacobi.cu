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

// Error-free transformations (Knuth TwoSum; TwoProduct through fma) for the
// compensated dot product Dot2 of Ogita, Rump & Oishi (SIAM J. Sci. Comput.
// 2005): the result is as accurate as if computed in twice the working
// precision, so pairs are judged orthogonal on their stored values and not on
// rounding noise of the dot product.
template <typename T>
__device__ __forceinline__ void two_sum(T a, T b, T& s, T& e) {
  s = a + b;
  const T z = s - a;
  e = (a - (s - z)) + (b - z);
}

// Warp-level reduction of one (p, s) compensated pair (TwoSum on the leading
// parts, errors accumulated).
template <typename T>
__device__ __forceinline__ void warp_sum2(T& p, T& s) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const T op = __shfl_xor_sync(0xffffffffu, p, o);
    const T os = __shfl_xor_sync(0xffffffffu, s, o);
    T q;
    two_sum(p, op, p, q);
    s += os + q;
  }
}

// 1024 threads for fp32; 512 for fp64.
template <typename T>
__host__ __device__ constexpr int jthreads() { return sizeof(T) == 8 ? 512 : 1024; }

// One group of 8 lanes per column pair, so a round's l/2 pairs run at once;
// each lane strides over the rows with step 8.  The dot products are plain;
// when a pair's cosine is within a factor 64 of the threshold, gamma is
// recomputed with Dot2 so convergence is judged on accurate values.
template <typename T>
__global__ void __launch_bounds__(jthreads<T>()) jacobi_kernel(int l, const T* __restrict__ M,
                                                              int64_t ldm, T* __restrict__ Uh,
                                                              int64_t lduh,
                                                              double* __restrict__ Sh, T* scratch,
                                                              int max_sweeps, int* d_info) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double s_sig[1024];
  __shared__ int s_rot;
  T* X = scratch ? scratch : (T*)dsm;  // column-major: X[j*l + i]
  constexpr int NT = jthreads<T>();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = NT / 32;
  const int g = tid >> 3, gl = tid & 7, ngroups = NT / 8;
  const unsigned gmask = 0xffu << (lane & ~7);
  for (int t = tid; t < l * l; t += NT) {
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
      for (int p = g; p < N / 2; p += ngroups) {
        int a, b;
        rr_pair(r, p, N, &a, &b);
        if (a >= l || b >= l) continue;          // uniform within the group
        T* xa = X + (int64_t)a * l;
        T* xb = X + (int64_t)b * l;
        T al = T(0), be = T(0), ga = T(0);
        for (int i = gl; i < l; i += 8) {
          const T u = xa[i], v = xb[i];
          al = fma(u, u, al);
          be = fma(v, v, be);
          ga = fma(u, v, ga);
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
          al += __shfl_xor_sync(gmask, al, o, 8);
          be += __shfl_xor_sync(gmask, be, o, 8);
          ga += __shfl_xor_sync(gmask, ga, o, 8);
        }
        if (!(al > T(0)) || !(be > T(0))) continue;
        const T scale = sqrt(al) * sqrt(be);
        if (abs(ga) < T(64) * tol * scale) {     // near the threshold: Dot2
          T gp = T(0), gs = T(0);
          for (int i = gl; i < l; i += 8) {
            const T u = xa[i], v = xb[i];
            const T h = u * v;
            const T hr = fma(u, v, -h);
            T e;
            two_sum(gp, h, gp, e);
            gs += e + hr;
          }
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) {
            const T op = __shfl_xor_sync(gmask, gp, o, 8);
            const T os = __shfl_xor_sync(gmask, gs, o, 8);
            T e;
            two_sum(gp, op, gp, e);
            gs += os + e;
          }
          ga = gp + gs;
        }
        if (!(abs(ga) > tol * scale)) continue;
        const T zeta = (be - al) / (T(2) * ga);
        const T t = (zeta >= T(0) ? T(1) : T(-1)) / (abs(zeta) + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + t * t);
        const T sn = c * t;
        for (int i = gl; i < l; i += 8) {
          const T u = xa[i], v = xb[i];
          xa[i] = c * u - sn * v;
          xb[i] = sn * u + c * v;
        }
        if (gl == 0) atomicAdd(&s_rot, 1);
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
  const int tr_ = trace_begin(RSVD_TRACE_JACOBI, s);
  svd_finalize_kernel<T><<<1, 1024, 0, s>>>(l, P, ldp, Uin, ldin, Uh, lduh, Sh, Vh, ldvh, d_info);
  count_launch();
  trace_end(tr_, s);
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
  const int tr_ = trace_begin(RSVD_TRACE_JACOBI, s);
  jacobi_kernel<T><<<1, jthreads<T>(), dyn, s>>>(l, M, ldm, Uh, lduh, Sh, scr, max_sweeps,
                                                  d_info);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

template cudaError_t launch_jacobi<float>(int, const float*, int64_t, float*, int64_t, double*,
                                          float*, int64_t, float*, int, int*, cudaStream_t);
template cudaError_t launch_jacobi<double>(int, const double*, int64_t, double*, int64_t,
                                           double*, double*, int64_t, double*, int, int*,
                                           cudaStream_t);

}  // namespace rsvd
