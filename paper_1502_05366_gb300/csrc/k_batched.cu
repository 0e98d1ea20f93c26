// Kernels of the batched path: many small, unevenly sized RSVD problems, each
// step of Alg. 5 one launch over every problem of the batch.
//
// bgemm_kernel is a grouped fp32 GEMM: a task is (problem GEMM, 64-row block of
// its output); the CTA computes the block's full width (N <= 128) over the
// whole contraction, in 32-deep chunks staged in shared memory.  The sketch's
// Omega is generated in the chunk instead of read (Sec. 3.1: Gaussian test
// matrix; the problem index is the counter's batch word).  Products are plain
// fp32 FMAs: the problems are small, so the work is spread over many CTAs and
// bound by the bytes of A.
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int BG_T = 256;             // threads: 16 row groups of 4 rows x 16 column lanes
constexpr int BG_TK = 32;             // contraction chunk
constexpr int BG_AP = BGEMM_TM + 4;   // padded row of the staged A chunk (float4-aligned)
constexpr int BG_WP = BATCH_LMAX + 4;
}  // namespace

__global__ void __launch_bounds__(BG_T) bgemm_kernel(const BGemm* __restrict__ gemms,
                                                     const int2* __restrict__ tasks,
                                                     uint64_t seed) {
  __shared__ __align__(16) float As[BG_TK][BG_AP];   // As[kk][r] = op(A)(row0 + r, k0 + kk)
  __shared__ __align__(16) float Ws[BG_TK][BG_WP];   // Ws[kk][c] = W(k0 + kk, c)
  const int2 tk = tasks[blockIdx.x];
  const BGemm g = gemms[tk.x];
  const int row0 = tk.y;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int M = g.M, N = g.N, K = g.K;
  const int nc = (N + 15) >> 4;             // column lanes per thread (<= 8)
  float acc[4][8];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[q][c] = 0.f;
  for (int k0 = 0; k0 < K; k0 += BG_TK) {
    if (!g.transA) {   // A is M x K: rows of 32 contiguous values
      for (int e = tid; e < BGEMM_TM * BG_TK; e += BG_T) {
        const int r = e >> 5, kk = e & 31;
        const int gr = row0 + r, gk = k0 + kk;
        As[kk][r] = (gr < M && gk < K) ? g.A[(int64_t)gr * g.lda + gk] : 0.f;
      }
    } else {           // A is stored K x M: op(A)(r, kk) = A(kk, r), rows of 64 values
      for (int e = tid; e < BGEMM_TM * BG_TK; e += BG_T) {
        const int kk = e >> 6, r = e & 63;
        const int gr = row0 + r, gk = k0 + kk;
        As[kk][r] = (gr < M && gk < K) ? g.A[(int64_t)gk * g.lda + gr] : 0.f;
      }
    }
    if (g.W) {
      for (int e = tid; e < BG_TK * N; e += BG_T) {
        const int kk = e / N, c = e - (e / N) * N;
        const int gk = k0 + kk;
        Ws[kk][c] = gk < K ? g.W[(int64_t)gk * g.ldw + c] : 0.f;
      }
    } else {
      const int nq = (N + 3) >> 2;
      for (int e = tid; e < BG_TK * nq; e += BG_T) {
        const int kk = e / nq, qd = e - (e / nq) * nq;
        const int gk = k0 + kk;
        float z[4] = {0.f, 0.f, 0.f, 0.f};
        if (gk < K) {
          gauss4_f(omega_words(seed, (uint32_t)gk, (uint32_t)qd, 0u, (uint32_t)g.batch), z);
#pragma unroll
          for (int t = 0; t < 4; ++t) z[t] = round_bf16(z[t]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
          if (4 * qd + t < N) Ws[kk][4 * qd + t] = z[t];
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < BG_TK; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      float wv[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) wv[c] = (c < nc) ? Ws[kk][tx + 16 * c] : 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[q][c] = fmaf(av[q], wv[c], acc[q][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gr = row0 + 4 * ty + q;
    if (gr >= M) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int col = tx + 16 * c;
      if (c < nc && col < g.ncol) g.C[(int64_t)gr * g.ldc + col] = acc[q][c];
    }
  }
}

cudaError_t launch_bgemm(const BGemm* gemms, const int2* tasks, int ntasks, uint64_t seed,
                         cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  bgemm_kernel<<<ntasks, BG_T, 0, s>>>(gemms, tasks, seed);
  count_launch();
  return cudaGetLastError();
}

// One CTA per problem: for each column j < k, the row of the largest |V(i, j)|
// (lowest index on ties) decides the sign; U(:, j) and V(:, j) take it, and
// S[j] = Sh[j].
__global__ void __launch_bounds__(256) sign_batched_kernel(const BSign* __restrict__ tasks) {
  __shared__ float s_best[256];
  __shared__ int64_t s_idx[256];
  __shared__ float s_val[256];
  __shared__ float s_sign;
  const BSign tk = tasks[blockIdx.x];
  const int tid = threadIdx.x;
  for (int j = 0; j < tk.k; ++j) {
    float best = -1.f, bv = 0.f;
    int64_t bi = INT64_MAX;
    for (int64_t i = tid; i < tk.n; i += 256) {
      const float v = tk.V[i * tk.k + j];
      const float a = fabsf(v);
      if (a > best || (a == best && i < bi)) {
        best = a;
        bi = i;
        bv = v;
      }
    }
    s_best[tid] = best;
    s_idx[tid] = bi;
    s_val[tid] = bv;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (tid < o) {
        const float b2 = s_best[tid + o];
        const int64_t i2 = s_idx[tid + o];
        if (b2 > s_best[tid] || (b2 == s_best[tid] && i2 < s_idx[tid])) {
          s_best[tid] = b2;
          s_idx[tid] = i2;
          s_val[tid] = s_val[tid + o];
        }
      }
      __syncthreads();
    }
    if (tid == 0) {
      s_sign = s_val[0] < 0.f ? -1.f : 1.f;
      tk.S[j] = tk.Sh[j];
    }
    __syncthreads();
    const float sg = s_sign;
    if (sg < 0.f) {
      for (int64_t i = tid; i < tk.m; i += 256) tk.U[i * tk.k + j] = -tk.U[i * tk.k + j];
      for (int64_t i = tid; i < tk.n; i += 256) tk.V[i * tk.k + j] = -tk.V[i * tk.k + j];
    }
    __syncthreads();
  }
}

cudaError_t launch_sign_batched(const BSign* tasks, int batch, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  sign_batched_kernel<<<batch, 256, 0, s>>>(tasks);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rsvd
