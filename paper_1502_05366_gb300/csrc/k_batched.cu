// Kernels of the batched path: many small, unevenly sized RSVD problems, each
// step of Alg. 5 one launch over every problem of the batch.
//
// bgemm_kernel is a grouped fp32 GEMM: a task is (problem GEMM, block of 64, 128
// or 256 output rows, by the width); the CTA computes the block's full width
// (N <= 128) over the whole contraction, in 32-deep chunks staged in shared
// memory.  The sketch's
// Omega is generated in the chunk instead of read (Sec. 3.1: Gaussian test
// matrix; the problem index is the counter's batch word).  Products are plain
// fp32 FMAs: the problems are small, so the work is spread over many CTAs and
// bound by the bytes of A.
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int BG_T = 256;             // threads: 16 row groups x 16 column lanes
constexpr int BG_TK = 32;             // contraction chunk
}  // namespace

// RPT rows per thread: the tile is TM = 16 RPT rows by NC * 16 columns, NC = 32 / RPT
// (64 x 128, 128 x 64 or 256 x 32), so that every thread holds 32 accumulators
// whatever the width.  The next chunk's A and W values are prefetched into
// registers while the current chunk is multiplied from shared memory.
template <int RPT>
__global__ void __launch_bounds__(BG_T, 2) bgemm_kernel(const BGemm* __restrict__ gemms,
                                                     const int2* __restrict__ tasks,
                                                     uint64_t seed) {
  constexpr int TM = 16 * RPT;
  constexpr int NC = 32 / RPT;
  constexpr int NW = NC * 16;               // widest W handled
  constexpr int PA = TM * BG_TK / BG_T;     // A values per thread and chunk
  constexpr int PW = BG_TK * NW / BG_T;     // W values per thread and chunk (at most)
  __shared__ __align__(16) float As[BG_TK][TM + 4];   // As[kk][r] = op(A)(row0 + r, k0 + kk)
  __shared__ __align__(16) float Ws[BG_TK][NW + 4];   // Ws[kk][c] = W(k0 + kk, c)
  const int2 tk = tasks[blockIdx.x];
  const BGemm g = gemms[tk.x];
  const int row0 = tk.y;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int M = g.M, N = g.N, K = g.K;
  const int nc = (N + 15) >> 4;
  float ra[PA], rw[PW];
  auto load_chunk = [&](int k0) {
#pragma unroll
    for (int j = 0; j < PA; ++j) {
      const int e = tid + j * BG_T;
      int r, kk;
      if (!g.transA) {
        r = e >> 5;
        kk = e & 31;
      } else {
        kk = e / TM;
        r = e - kk * TM;
      }
      const int gr = row0 + r, gk = k0 + kk;
      float v = 0.f;
      if (gr < M && gk < K)
        v = g.transA ? g.A[(int64_t)gk * g.lda + gr] : g.A[(int64_t)gr * g.lda + gk];
      ra[j] = v;
    }
    if (g.W) {
#pragma unroll
      for (int j = 0; j < PW; ++j) {
        const int e = tid + j * BG_T;
        const int kk = e / NW, c = e - (e / NW) * NW;
        const int gk = k0 + kk;
        rw[j] = (c < N && gk < K) ? g.W[(int64_t)gk * g.ldw + c] : 0.f;
      }
    }
  };
  auto store_chunk = [&](int k0) {
#pragma unroll
    for (int j = 0; j < PA; ++j) {
      const int e = tid + j * BG_T;
      int r, kk;
      if (!g.transA) {
        r = e >> 5;
        kk = e & 31;
      } else {
        kk = e / TM;
        r = e - kk * TM;
      }
      As[kk][r] = ra[j];
    }
    if (g.W) {
#pragma unroll
      for (int j = 0; j < PW; ++j) {
        const int e = tid + j * BG_T;
        Ws[e / NW][e - (e / NW) * NW] = rw[j];
      }
    } else {   // Omega rows k0 .. k0 + 31, generated
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
          if (4 * qd + t < NW) Ws[kk][4 * qd + t] = (4 * qd + t < N) ? z[t] : 0.f;
      }
    }
  };
  float acc[RPT][NC];
#pragma unroll
  for (int q = 0; q < RPT; ++q)
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[q][c] = 0.f;
  load_chunk(0);
  for (int k0 = 0; k0 < K; k0 += BG_TK) {
    store_chunk(k0);
    __syncthreads();
    if (k0 + BG_TK < K) load_chunk(k0 + BG_TK);
#pragma unroll 4
    for (int kk = 0; kk < BG_TK; ++kk) {
      float av[RPT];
#pragma unroll
      for (int q4 = 0; q4 < RPT / 4; ++q4) {
        const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][RPT * ty + 4 * q4]);
        av[4 * q4] = a4.x;
        av[4 * q4 + 1] = a4.y;
        av[4 * q4 + 2] = a4.z;
        av[4 * q4 + 3] = a4.w;
      }
      float wv[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) wv[c] = Ws[kk][tx + 16 * c];
#pragma unroll
      for (int q = 0; q < RPT; ++q)
#pragma unroll
        for (int c = 0; c < NC; ++c) acc[q][c] = fmaf(av[q], wv[c], acc[q][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int gr = row0 + RPT * ty + q;
    if (gr >= M) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int col = tx + 16 * c;
      if (c < nc && col < g.ncol) g.C[(int64_t)gr * g.ldc + col] = acc[q][c];
    }
  }
}

int bgemm_rows(int N) { return N > 64 ? 64 : (N > 32 ? 128 : 256); }

cudaError_t launch_bgemm(const BGemm* gemms, const int2* tasks, int ntasks, int rows,
                         uint64_t seed, cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  if (rows == 64)
    bgemm_kernel<4><<<ntasks, BG_T, 0, s>>>(gemms, tasks, seed);
  else if (rows == 128)
    bgemm_kernel<8><<<ntasks, BG_T, 0, s>>>(gemms, tasks, seed);
  else if (rows == 256)
    bgemm_kernel<16><<<ntasks, BG_T, 0, s>>>(gemms, tasks, seed);
  else
    return cudaErrorInvalidValue;
  count_launch();
  return cudaGetLastError();
}

// Split-K partials of one problem summed in slice order (the Grams of tall
// samples run as one GEMM task per 512-row slice).
__global__ void __launch_bounds__(256) sum_batched_kernel(const BSum* __restrict__ tasks) {
  const BSum tk = tasks[blockIdx.x];
  for (int e = threadIdx.x; e < tk.count; e += blockDim.x) {
    float acc = 0.f;
    for (int sl = 0; sl < tk.nslice; ++sl) acc += tk.part[(int64_t)sl * tk.count + e];
    tk.out[e] = acc;
  }
}

cudaError_t launch_sum_batched(const BSum* tasks, int batch, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  sum_batched_kernel<<<batch, 256, 0, s>>>(tasks);
  count_launch();
  return cudaGetLastError();
}

// Negates the entries of the row-major X (cnt entries, k columns) whose column
// sign is negative, four loads in flight per thread.  Entry e is in column
// e % k; the column advances by 256 % k per 256-entry sweep.
__device__ __forceinline__ void flip_columns(float* __restrict__ X, int64_t cnt, int k,
                                             const float* s_sign) {
  const int adv = 256 % k;
  int c = threadIdx.x % k;
  for (int64_t e0 = threadIdx.x; e0 < cnt; e0 += 4 * 256) {
    float v[4];
    bool f[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t e = e0 + 256 * u;
      f[u] = e < cnt && s_sign[c] < 0.f;
      v[u] = f[u] ? X[e] : 0.f;
      c += adv;
      if (c >= k) c -= k;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (f[u]) X[e0 + 256 * u] = -v[u];
  }
}

// One CTA per problem: for each column j < k, the row of the largest |V(i, j)|
// (lowest index on ties) decides the sign; U(:, j) and V(:, j) take it, and
// S[j] = Sh[j].  All k columns at once (k <= BATCH_LMAX <= 256): thread t
// scans column t % k over the rows t / k, t / k + R, ... (R = 256 / k rows per
// sweep, so that a warp reads consecutive entries of a row), the R candidates
// of a column are merged by its thread t < k, and the flips run over U and V
// in storage order.  The order (|v| descending, row ascending) is total on
// the non-NaN entries, so the chosen row does not depend on the merge order.
static_assert(BATCH_LMAX <= 256, "sign_batched_kernel holds one column per thread");
__global__ void __launch_bounds__(256) sign_batched_kernel(const BSign* __restrict__ tasks) {
  __shared__ float s_best[256];
  __shared__ int64_t s_idx[256];
  __shared__ float s_val[256];
  __shared__ float s_sign[256];
  const BSign tk = tasks[blockIdx.x];
  const int tid = threadIdx.x;
  const int k = tk.k;
  if (k < 1 || k > 256) return;
  const int R = 256 / k;
  const int j = tid % k, rr = tid / k;
  float best = -1.f, bv = 0.f;
  int64_t bi = INT64_MAX;
  if (rr < R) {
    // four rows in flight, compared in increasing row order
    for (int64_t i0 = rr; i0 < tk.n; i0 += 4 * (int64_t)R) {
      float vv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + (int64_t)u * R;
        vv[u] = i < tk.n ? tk.V[i * k + j] : 0.f;
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t i = i0 + (int64_t)u * R;
        const float a = fabsf(vv[u]);
        if (i < tk.n && (a > best || (a == best && i < bi))) {
          best = a;
          bi = i;
          bv = vv[u];
        }
      }
    }
  }
  s_best[tid] = best;
  s_idx[tid] = bi;
  s_val[tid] = bv;
  __syncthreads();
  if (tid < k) {
    for (int u = tid + k; u < R * k; u += k) {
      const float b2 = s_best[u];
      const int64_t i2 = s_idx[u];
      if (b2 > best || (b2 == best && i2 < bi)) {
        best = b2;
        bi = i2;
        bv = s_val[u];
      }
    }
    s_sign[tid] = bv < 0.f ? -1.f : 1.f;
    tk.S[tid] = tk.Sh[tid];
  }
  __syncthreads();
  flip_columns(tk.U, tk.m * k, k, s_sign);
  flip_columns(tk.V, tk.n * k, k, s_sign);
}

cudaError_t launch_sign_batched(const BSign* tasks, int batch, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  sign_batched_kernel<<<batch, 256, 0, s>>>(tasks);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rsvd
