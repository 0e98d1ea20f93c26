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
#include <cooperative_groups.h>

#include <algorithm>

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

// Cluster variant (fp32): a thread-block cluster of JC CTAs, each holding two
// blocks of w = ceil(l / 2 JC) columns and two inbox blocks in shared memory
// (4 w l floats).  8 CTAs of 512 threads for 32 <= l <= 256; 16 CTAs (the
// opt-in cluster size) of 1024 threads for 256 < l <= 672, where 4 w l floats
// still fit a CTA's shared memory.  One warp per pair of a sub-round (w <= 21).
constexpr int JC_MAX = 16;
constexpr int JC_LMAX = 672;
static inline int jacobi_cluster_size(int l, int elem) {
  if (elem != 4 || l < 32 || l > JC_LMAX) return 0;
  return l <= 256 ? 8 : 16;
}
static inline bool jacobi_use_cluster(int l, int elem) { return jacobi_cluster_size(l, elem) > 0; }
__host__ __device__ inline int jc_width(int l, int jc) { return (l + 2 * jc - 1) / (2 * jc); }

size_t jacobi_scratch_bytes(int l, int elem) {
  const int jc = jacobi_cluster_size(l, elem);
  // the cluster kernel's sigma exchange, and the one-CTA kernel's fallback
  // storage when the cluster cannot be placed
  const size_t b = (size_t)l * l * elem;
  const size_t one = b <= JSMEM_LIMIT ? 0 : b;
  if (jc) return std::max((size_t)2 * jc * jc_width(l, jc) * sizeof(double), one);
  return one;
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
// The sweeps and the sorted output of one matrix by one CTA of NT threads; X
// (l*l, column-major: X[j*l + i]) and s_sig (l doubles) are the CTA's working
// storage.
template <typename T, int NT>
__device__ void jacobi_body(int l, const T* __restrict__ M, int64_t ldm, T* __restrict__ Uh,
                            int64_t lduh, double* __restrict__ Sh, T* X, double* s_sig,
                            int& s_rot, int max_sweeps, int* d_info) {
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

template <typename T>
__global__ void __launch_bounds__(jthreads<T>()) jacobi_kernel(int l, const T* __restrict__ M,
                                                              int64_t ldm, T* __restrict__ Uh,
                                                              int64_t lduh,
                                                              double* __restrict__ Sh, T* scratch,
                                                              int max_sweeps, int* d_info) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double s_sig[1024];
  __shared__ int s_rot;
  T* X = scratch ? scratch : (T*)dsm;
  jacobi_body<T, jthreads<T>()>(l, M, ldm, Uh, lduh, Sh, X, s_sig, s_rot, max_sweeps, d_info);
}

// ---------------------------------------------------------------------------
// Block one-sided Jacobi on a thread-block cluster (fp32).
//
// The l columns (padded with zero columns to 16 w) form 16 blocks of w
// columns.  CTA c of the 8-CTA cluster holds two blocks ("top" and "bottom")
// in its shared memory.  A sweep is: the pairs inside every block (first
// block-round), then 15 block-rounds in the circle order of the 16 blocks
// (top block of CTA 0 fixed), in which each CTA orthogonalises all w^2 cross
// pairs between its two blocks, w disjoint pairs per sub-round, one warp per
// pair.  Between block-rounds the blocks move to the neighbouring CTAs through
// distributed shared memory (two cluster barriers).  Every pair of columns
// meets once per sweep, as in the cyclic one-sided method; the rotation of a
// pair is the same formula as in jacobi_kernel.  The sweep loop ends for all
// CTAs together (rotation counts exchanged in distributed shared memory), so
// every CTA passes the same sequence of cluster barriers.
// ---------------------------------------------------------------------------
namespace cg = cooperative_groups;

// Rotate columns xa, xb (l floats each, shared memory) of one warp's pair;
// true when a rotation was applied.
__device__ __forceinline__ bool jc_rotate(float* xa, float* xb, int l, float tol, int lane) {
  float al = 0.f, be = 0.f, ga = 0.f;
  for (int i = lane; i < l; i += 32) {
    const float u = xa[i], v = xb[i];
    al = fmaf(u, u, al);
    be = fmaf(v, v, be);
    ga = fmaf(u, v, ga);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    al += __shfl_xor_sync(0xffffffffu, al, o);
    be += __shfl_xor_sync(0xffffffffu, be, o);
    ga += __shfl_xor_sync(0xffffffffu, ga, o);
  }
  if (!(al > 0.f) || !(be > 0.f)) return false;
  const float scale = sqrtf(al) * sqrtf(be);
  if (fabsf(ga) < 64.f * tol * scale) {   // near the threshold: Dot2
    float gp = 0.f, gs = 0.f;
    for (int i = lane; i < l; i += 32) {
      const float u = xa[i], v = xb[i];
      const float h = u * v;
      const float hr = fmaf(u, v, -h);
      float e;
      two_sum(gp, h, gp, e);
      gs += e + hr;
    }
    warp_sum2(gp, gs);
    ga = gp + gs;
  }
  if (!(fabsf(ga) > tol * scale)) return false;
  const float zeta = (be - al) / (2.f * ga);
  const float t = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
  const float c = 1.f / sqrtf(1.f + t * t);
  const float sn = c * t;
  for (int i = lane; i < l; i += 32) {
    const float u = xa[i], v = xb[i];
    xa[i] = c * u - sn * v;
    xb[i] = sn * u + c * v;
  }
  return true;
}

template <int JC, int JCT>
__global__ void __launch_bounds__(JCT)
    jacobi_cluster_kernel(int l, const float* __restrict__ M, int64_t ldm, float* __restrict__ Uh,
                          int64_t lduh, double* __restrict__ Sh, double* __restrict__ sig,
                          int max_sweeps, int* d_info) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  extern __shared__ __align__(16) float jsm[];
  __shared__ int s_rot;
  __shared__ int s_cnt[JC];
  __shared__ int s_in[2];                    // this CTA's current inbox buffers (top, bottom)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NWARP = JCT / 32;
  const int w = jc_width(l, JC);
  const int bsz = w * l;                     // floats per block, column-major X[a*l + i]
  // buffer roles (indices into the four block buffers)
  int iT = 0, iB = 1, inT = 2, inB = 3;
  // initial blocks: top = block c, bottom = block 2 JC - 1 - c; block q holds
  // columns q w .. q w + w - 1 of M (zero beyond l)
  {
    const int qT = rank, qB = 2 * JC - 1 - rank;
    for (int e = tid; e < 2 * bsz; e += JCT) {
      const int which = e / bsz, rem = e - which * bsz;
      const int a = rem / l, i = rem - a * l;
      const int col = (which == 0 ? qT : qB) * w + a;
      jsm[(which == 0 ? iT : iB) * bsz + rem] = col < l ? M[(int64_t)i * ldm + col] : 0.f;
    }
  }
  if (tid == 0) {
    s_rot = 0;
    s_in[0] = inT;
    s_in[1] = inB;
  }
  __syncthreads();
  const float tol = sqrtf((float)l) * 5.9604645e-8f;
  const int wp = w + (w & 1);                // players of the in-block round robin
  bool converged = false;
  int sweep = 0;
  for (; sweep < max_sweeps && !converged; ++sweep) {
    // ---- pairs inside the two blocks held now (covers all blocks) ----
    for (int rr = 0; rr < wp - 1; ++rr) {
      const int half = wp / 2;
      if (warp < 2 * half) {
        const int blk = warp / half, pi = warp - blk * half;
        int a, b;
        if (pi == 0) {
          a = wp - 1;
          b = rr;
        } else {
          a = (rr + pi) % (wp - 1);
          b = (rr - pi + wp - 1) % (wp - 1);
        }
        if (a < w && b < w) {
          float* base = jsm + (blk == 0 ? iT : iB) * bsz;
          if (jc_rotate(base + a * l, base + b * l, l, tol, lane) && lane == 0)
            atomicAdd(&s_rot, 1);
        }
      }
      __syncthreads();
    }
    // ---- 2 JC - 1 block-rounds of cross pairs, blocks rotating between CTAs ----
    for (int br = 0; br < 2 * JC - 1; ++br) {
      for (int sr = 0; sr < w; ++sr) {
        if (warp < w) {
          const int a = warp, b = (warp + sr) % w;
          if (jc_rotate(jsm + iT * bsz + a * l, jsm + iB * bsz + b * l, l, tol, lane) &&
              lane == 0)
            atomicAdd(&s_rot, 1);
        }
        __syncthreads();
      }
      const bool last = (br == 2 * JC - 2);
      cluster.sync();                         // (A) every CTA done with its blocks
      // send: CTA 0 its bottom to CTA 1's top inbox; CTA c in 1..JC-2 its top
      // to CTA c+1's top inbox; CTA c >= 1 its bottom to CTA c-1's bottom inbox
      {
        // the receivers' inbox buffers (their roles differ from this CTA's)
        float* dstT = nullptr;
        const float* srcT = nullptr;
        if (rank <= JC - 2) {
          const int q = rank + 1;
          dstT = cluster.map_shared_rank(jsm, q) + *cluster.map_shared_rank(&s_in[0], q) * bsz;
          srcT = jsm + (rank == 0 ? iB : iT) * bsz;
        }
        float* dstB = nullptr;
        if (rank >= 1) {
          const int q = rank - 1;
          dstB = cluster.map_shared_rank(jsm, q) + *cluster.map_shared_rank(&s_in[1], q) * bsz;
        }
        const float* srcB = jsm + iB * bsz;
        for (int e = tid; e < bsz; e += JCT) {
          if (dstT) dstT[e] = srcT[e];
          if (dstB) dstB[e] = srcB[e];
        }
      }
      if (last && tid == 0) {
        // this sweep's rotation count to every CTA of the cluster
        for (int q = 0; q < JC; ++q) cluster.map_shared_rank(s_cnt, q)[rank] = s_rot;
      }
      cluster.sync();                         // (B) inboxes filled
      if (rank == 0) {
        const int t = iB;
        iB = inB;
        inB = t;
      } else if (rank <= JC - 2) {
        int t = iT;
        iT = inT;
        inT = t;
        t = iB;
        iB = inB;
        inB = t;
      } else {
        const int oT = iT, oB = iB;
        iT = inT;
        iB = oT;                              // own top becomes the bottom
        inT = oB;
      }
      if (last) {
        int tot = 0;
        for (int q = 0; q < JC; ++q) tot += s_cnt[q];
        converged = (tot == 0);
      }
      // publish the new inbox roles: peers read them only after the next (A)
      __syncthreads();
      if (tid == 0) {
        s_in[0] = inT;
        s_in[1] = inB;
        if (last) s_rot = 0;
      }
      __syncthreads();
    }
  }
  if (!converged && rank == 0 && tid == 0) set_info(d_info, RSVD_ERR_NO_CONVERGENCE);
  // ---- sigma of the 2 w columns held, their global ranks, Uh columns ----
  __shared__ double s_sig[64];
  for (int a = warp; a < 2 * w; a += NWARP) {
    const float* x = jsm + (a < w ? iT : iB) * bsz + (a % w) * l;
    float sq = 0.f;
    for (int i = lane; i < l; i += 32) sq = fmaf(x[i], x[i], sq);
    sq = warp_sum(sq);
    if (lane == 0) {
      const double sg = (double)sqrtf(sq);
      s_sig[a] = sg;
      sig[rank * 2 * w + a] = sg;
      if (!isfinite(sg)) set_info(d_info, RSVD_ERR_NUMERIC);
    }
  }
  cluster.sync();                             // every sigma written (cluster scope)
  const int N = 2 * JC * w;
  for (int a = warp; a < 2 * w; a += NWARP) {
    const int slot = rank * 2 * w + a;
    const double sj = s_sig[a];
    int rk = 0;
    for (int q = lane; q < N; q += 32) {
      const double sq = __ldcg(sig + q);
      rk += (sq > sj || (sq == sj && q < slot)) ? 1 : 0;
    }
    for (int o = 16; o > 0; o >>= 1) rk += __shfl_xor_sync(0xffffffffu, rk, o);
    if (rk < l) {
      const float inv = sj > 0.0 ? (float)(1.0 / sj) : 0.f;
      const float* x = jsm + (a < w ? iT : iB) * bsz + (a % w) * l;
      for (int i = lane; i < l; i += 32) Uh[(int64_t)i * lduh + rk] = x[i] * inv;
      if (lane == 0) Sh[rk] = sj;
    }
  }
  cluster.sync();                             // keep every CTA's shared memory alive to the end
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

// One CTA per problem: Jacobi sweeps on M (l x l <= 128, row-major ld l),
// P = M^T Uj, sigma_j = ||P(:, j)||, Vh(:, rank) = P(:, j) / sigma_j,
// Uh(:, rank) = Uj(:, j) (the steps of jacobi_kernel and svd_finalize_kernel).
constexpr int SB_T = 256;
__global__ void __launch_bounds__(SB_T) small_svd_batched_kernel(const BSvd* __restrict__ tasks,
                                                                  int max_sweeps, int* d_info) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ double s_sig[BATCH_LMAX];
  __shared__ int s_rot;
  const BSvd tk = tasks[blockIdx.x];
  const int l = tk.l;
  float* X = reinterpret_cast<float*>(dsm);          // l*l
  float* Ms = X + l * l;                              // l*l
  float* Pm = Ms + l * l;                             // l*l
  jacobi_body<float, SB_T>(l, tk.M, l, tk.Uj, l, tk.Sh, X, s_sig, s_rot, max_sweeps, d_info);
  __syncthreads();
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarp = SB_T / 32;
  for (int t = tid; t < l * l; t += SB_T) {
    Ms[t] = tk.M[t];
    X[t] = tk.Uj[t];
  }
  __syncthreads();
  for (int t = tid; t < l * l; t += SB_T) {   // P[i][j] = sum_r M[r][i] Uj[r][j]
    const int i = t / l, j = t - (t / l) * l;
    float acc = 0.f;
    for (int r = 0; r < l; ++r) acc = fmaf(Ms[r * l + i], X[r * l + j], acc);
    Pm[t] = acc;
  }
  __syncthreads();
  for (int j = warp; j < l; j += nwarp) {
    double sq = 0.0;
    for (int i = lane; i < l; i += 32) {
      const double v = (double)Pm[i * l + j];
      sq = fma(v, v, sq);
    }
    sq = warp_sum(sq);
    if (lane == 0) {
      s_sig[j] = sqrt(sq);
      if (!isfinite(sq)) set_info(d_info, RSVD_ERR_NUMERIC);
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
      tk.Vh[i * l + rank] = (float)((double)Pm[i * l + j] * inv);
      tk.Uh[i * l + rank] = X[i * l + j];
    }
    if (lane == 0) tk.Sh[rank] = sj;
  }
}

cudaError_t launch_small_svd_batched(const BSvd* tasks, int batch, int lmax, int max_sweeps,
                                     int* d_info, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  if (lmax > BATCH_LMAX) return cudaErrorInvalidValue;
  const size_t dyn = (size_t)3 * lmax * lmax * sizeof(float);
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(small_svd_batched_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  const int tr_ = trace_begin(RSVD_TRACE_JACOBI, s);
  small_svd_batched_kernel<<<batch, SB_T, dyn, s>>>(tasks, max_sweeps, d_info);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

// The cluster kernel through cudaLaunchKernelEx (cluster size set at launch;
// 16 needs the non-portable size opt-in).  *placed = false, and nothing is
// launched, when the device cannot hold one such cluster.
static cudaError_t launch_jacobi_cluster(int jc, int l, const float* M, int64_t ldm, float* Uh,
                                         int64_t lduh, double* Sh, double* sig, int max_sweeps,
                                         int* d_info, cudaStream_t s, bool* placed) {
  *placed = false;
  const size_t dyn = (size_t)4 * jc_width(l, jc) * l * sizeof(float);
  const void* kern = jc == 8 ? (const void*)jacobi_cluster_kernel<8, 512>
                             : (const void*)jacobi_cluster_kernel<16, 1024>;
  const int threads = jc == 8 ? 512 : 1024;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
  if (e != cudaSuccess) return e;
  if (jc > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)jc);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)jc;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  e = cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg);
  if (e != cudaSuccess) return e;
  if (nclusters < 1) return cudaSuccess;
  *placed = true;
  const int tr_ = trace_begin(RSVD_TRACE_JACOBI, s);
  if (jc == 8)
    e = cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<8, 512>, l, M, ldm, Uh, lduh, Sh, sig,
                           max_sweeps, d_info);
  else
    e = cudaLaunchKernelEx(&cfg, jacobi_cluster_kernel<16, 1024>, l, M, ldm, Uh, lduh, Sh, sig,
                           max_sweeps, d_info);
  count_launch();
  trace_end(tr_, s);
  return e;
}

template <typename T>
cudaError_t launch_jacobi(int l, const T* M, int64_t ldm, T* Uh, int64_t lduh, double* Sh,
                          T* Vh, int64_t ldvh, T* scratch, int max_sweeps, int* d_info,
                          cudaStream_t s) {
  (void)Vh;
  (void)ldvh;
  if (l > 1024) return cudaErrorInvalidValue;
  const int jc = jacobi_cluster_size(l, (int)sizeof(T));
  if (jc) {
    if (!scratch) return cudaErrorInvalidValue;
    bool placed = false;
    const cudaError_t e = launch_jacobi_cluster(jc, l, (const float*)M, ldm, (float*)Uh, lduh, Sh,
                                                (double*)scratch, max_sweeps, d_info, s, &placed);
    // a cluster that cannot be placed falls through to the one-CTA kernel
    if (e != cudaSuccess || placed) return e;
  }
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
