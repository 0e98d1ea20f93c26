// Grouped tcgen05 GEMM of the batched path: the passes over A of many small
// problems of uneven sizes (Alg. 5 per problem) in one persistent launch.
//
//   form 0:  C_i (M_i x l_i) = A_i W_i         Y = A Omega, Y = A Z
//   form 1:  C_i (M_i x l_i) = A_i^T W_i       Z = A^* Y, Bt = A^* Q
//
// A task is one 128-row output tile of one problem over its whole
// contraction (no split K, so no partial tiles and no reduce); CTA b takes
// tasks b, b + G, ... of a table ordered by decreasing cost.  Per problem the
// launch gets three tensor maps: A (fp32, rows padded to a 16-byte pitch by
// launch_pad_rows_batched; tiles beyond the matrix read as zeros) and the
// bf16 terms of W^T (launch_split_t_batched, launch_omega_t_batched).  The
// arithmetic is that of k_tc.cu: a = a0 + a1 (bf16 hi, lo), products a0 w0 +
// a1 w0 (+ a0 w1 for a stored W), fp32 accumulation in tensor memory.
//
// The CholeskyQR steps of the power scheme run here too: the Gram X^T X
// (form 1, W = X) and the apply X R^-1 (form 0, W = R^-1 in three bf16
// terms); X has an l-float pitch, so these take TMA maps of X itself when
// every l is a multiple of 4.  The final orthonormalisations and the lifts
// U = Q Vh, V = Qh Uh stay on the fp32 SIMT GEMM (the split products hold Q
// to 16 bits, short of the orthogonality the returned U and V need).
//
// Roles (256 threads): warp 0 TMA producer, warp 1 MMA issuer and TMEM owner,
// warps 4-7 converters (fp32 A rows -> bf16 hi/lo in TMEM) and the epilogue of
// each task (TMEM -> C_i rows).  The MMA width N_i = round_up(l_i, 16) is the
// task's own (instruction descriptor built per task).  Every mbarrier wait is
// bounded (~1 s); on expiry the kernel records RSVD_ERR_TIMEOUT and every role
// leaves its loop.
#include <cuda.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace rsvd {

using namespace tc;

namespace {
constexpr int GB_BM = 128;                     // output rows per task (MMA M)
constexpr int GB_BK = 32;                      // K per stage
constexpr int GB_ST = 4;                       // stages
constexpr int GB_ASTAGE = GB_BM * GB_BK * 4;   // 16 KB: the fp32 A tile
constexpr int GB_WTILE = TG_NMAX * GB_BK * 2;  // 8 KB: one bf16 term of W^T (N <= 128 rows)
// W terms and products per K-step (the rules of k_tc.cu):
//   NWT 1         a0 w0 + a1 w0                 (Omega: bf16-exact)
//   NWT 2         a0 w0 + a1 w0 + a0 w1         (a stored operand)
//   NWT 2, GRAM   a0 w0 + a1 w0 + a0 w1 + a1 w1 (Gram X^T X: W is X itself)
//   NWT 3         a0 w0 + a1 w0 + a0 w1 + a0 w2 (the fixed factor R^-1)
constexpr int GB_NCONV = 4;                    // warps 4..7
constexpr uint32_t GB_TMEM_COLS = 256;         // accumulator at 0 (<= 128 columns), A stages after
constexpr uint32_t GB_TMEM_A0 = 128;
// K-chunks per accumulation run: the tensor cores' fp32 accumulation in TMEM
// is not rounded to nearest and drifts one way over a long contraction
// (~1.2e-5 relative over 4096 terms); each run of at most 1024 terms is
// added into C in fp32 with round to nearest.
constexpr int GB_DRAIN = 32;

__host__ __device__ constexpr int gb_stage_bytes(int nwt) { return GB_ASTAGE + nwt * GB_WTILE; }
size_t gb_smem(int nwt) { return 1024 + (size_t)GB_ST * gb_stage_bytes(nwt) + (3 * GB_ST + 2) * 8 + 16; }
}  // namespace

template <int FORM, int NWT, bool GRAM>
__global__ void __launch_bounds__(256, 1)
    tc_group_kernel(const TgProb* __restrict__ probs, const TgTask* __restrict__ tasks, int ntasks,
                    const CUtensorMap* __restrict__ maps, int* d_info) {
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  unsigned char* dsm = (unsigned char*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  constexpr int SB = gb_stage_bytes(NWT);
  uint64_t* bars = (uint64_t*)(dsm + GB_ST * SB);
  uint64_t* full = bars;                  // TMA landed (A and the W terms)
  uint64_t* conv = bars + GB_ST;          // A stage written to TMEM
  uint64_t* done = bars + 2 * GB_ST;      // MMAs of the stage finished
  uint64_t* acc_full = bars + 3 * GB_ST;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_holder = (uint32_t*)(acc_empty + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x;

  if (threadIdx.x == 0) {
    for (int s = 0; s < GB_ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], GB_NCONV);
      mbar_init(&done[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, GB_NCONV);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(GB_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int64_t issued = 0;
      bool ok = true;
      const uint64_t pol_a = l2_policy_evict_first(), pol_w = l2_policy_evict_last();
      for (int t = blockIdx.x; t < ntasks && ok; t += G) {
        const TgTask tk = tasks[t];
        const TgProb pr = probs[tk.prob];
        const CUtensorMap* mA = maps + 4 * (int64_t)tk.prob;
        prefetch_map(mA);
        prefetch_map(mA + 1);
        if (NWT >= 2) prefetch_map(mA + 2);
        if (NWT == 3) prefetch_map(mA + 3);
        const int kiters = (pr.K + GB_BK - 1) / GB_BK;
        const uint32_t bytes = (uint32_t)GB_ASTAGE + (uint32_t)NWT * (uint32_t)pr.N * GB_BK * 2u;
        for (int kc = 0; kc < kiters; ++kc) {
          if (!mbar_wait(&done[s], ph ^ 1u, abort_flag, d_info)) {
            ok = false;
            break;
          }
          unsigned char* st = dsm + s * SB;
          mbar_arrive_expect_tx(&full[s], bytes);
          if (FORM == 0)
            tma_load_2d_hint(st, mA, &full[s], kc * GB_BK, tk.r0, pol_a);
          else
            tma_load_2d_hint(st, mA, &full[s], tk.r0, kc * GB_BK, pol_a);
          tma_load_2d_hint(st + GB_ASTAGE, mA + 1, &full[s], kc * GB_BK, 0, pol_w);
          if (NWT >= 2) tma_load_2d_hint(st + GB_ASTAGE + GB_WTILE, mA + 2, &full[s], kc * GB_BK, 0, pol_w);
          if (NWT == 3) tma_load_2d_hint(st + GB_ASTAGE + 2 * GB_WTILE, mA + 3, &full[s], kc * GB_BK, 0, pol_w);
          ++issued;
          if (++s == GB_ST) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
      if (*abort_flag && issued > 0) {
        // drain: wait (bounded) for the copies this thread issued
        const int64_t first = issued - GB_ST > 0 ? issued - GB_ST : 0;
        for (int64_t li = first; li < issued; ++li) {
          const int sd = (int)(li % GB_ST);
          const uint32_t pd = (uint32_t)((li / GB_ST) & 1);
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[sd], pd) && clock64() - t0 < WAIT_LIMIT) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------- MMA issuer -------------------------------
    if (lane == 0) {
      int s = 0;
      uint32_t ph = 0;
      int run = 0;              // accumulation runs of this CTA so far
      bool ok = true;
      for (int t = blockIdx.x; t < ntasks && ok; t += G) {
        const TgProb pr = probs[tasks[t].prob];
        const uint32_t idesc = make_idesc(GB_BM, pr.N);
        const int kiters = (pr.K + GB_BK - 1) / GB_BK;
        for (int kc = 0; kc < kiters; ++kc) {
          const bool first = kc % GB_DRAIN == 0;
          const bool last = kc % GB_DRAIN == GB_DRAIN - 1 || kc + 1 == kiters;
          if (first && run > 0 &&
              !mbar_wait(acc_empty, (uint32_t)((run - 1) & 1), abort_flag, d_info)) {
            ok = false;
            break;
          }
          if (!mbar_wait(&conv[s], ph, abort_flag, d_info) ||
              !mbar_wait(&full[s], ph, abort_flag, d_info)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t wbase = smem_u32(dsm + s * SB + GB_ASTAGE);
          const uint32_t a_col = tmem + GB_TMEM_A0 + 32u * (uint32_t)s;
#pragma unroll
          for (int kk = 0; kk < GB_BK / 16; ++kk) {
            const uint64_t bhi = sw64_desc(wbase + 32u * kk);
            const uint32_t ahi = a_col + 8u * kk;
            const uint32_t alo = a_col + 16u + 8u * kk;
            mma_ts(tmem, ahi, bhi, idesc, (first && kk == 0) ? 0u : 1u);
            mma_ts(tmem, alo, bhi, idesc, 1u);
            if (NWT >= 2) {
              const uint64_t b1 = sw64_desc(wbase + GB_WTILE + 32u * kk);
              mma_ts(tmem, ahi, b1, idesc, 1u);
              if (GRAM) mma_ts(tmem, alo, b1, idesc, 1u);
            }
            if (NWT == 3) mma_ts(tmem, ahi, sw64_desc(wbase + 2 * GB_WTILE + 32u * kk), idesc, 1u);
          }
          mma_commit(&done[s]);
          if (last) {
            mma_commit(acc_full);
            ++run;
          }
          if (++s == GB_ST) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp >= 4) {
    // ------------------------ converters and epilogue -------------------------
    const int q = warp - 4;                 // TMEM lane quadrant (= warp % 4)
    const int r = 32 * q + lane;            // tile row handled by this thread
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    int s = 0;
    uint32_t ph = 0;
    int run = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < ntasks && ok; t += G) {
      const TgTask tk = tasks[t];
      const TgProb pr = probs[tk.prob];
      const int kiters = (pr.K + GB_BK - 1) / GB_BK;
      for (int kc = 0; kc < kiters; ++kc) {
        if (!mbar_wait(&full[s], ph, abort_flag, d_info)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const unsigned char* st = dsm + s * SB;
        const uint32_t a_col = tmem + GB_TMEM_A0 + 32u * (uint32_t)s;
        float x[32];
        if (FORM == 0) {
          // 128B-swizzled rows of 32 fp32: 16-byte chunk c of row r sits at c ^ (r & 7)
          const unsigned char* row = st + r * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(row + ((c ^ (r & 7)) << 4));
            x[4 * c] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
          }
        } else {
          // plain 32 x 128 fp32 tile, row = k; this thread reads column r
          const float* tl = reinterpret_cast<const float*>(st);
#pragma unroll
          for (int k = 0; k < 32; ++k) x[k] = tl[k * GB_BM + r];
        }
        uint32_t hi[16], lo[16];
        split_row(x, hi, lo);
        tmem_st16(lane_base + a_col, hi);
        tmem_st16(lane_base + a_col + 16u, lo);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[s]);
        if (kc % GB_DRAIN == GB_DRAIN - 1 || kc + 1 == kiters) {
          // end of an accumulation run: the first run of the task stores its
          // rows of C, later ones add into them (fp32, round to nearest)
          if (!mbar_wait(acc_full, (uint32_t)(run & 1), abort_flag, d_info)) {
            ok = false;
            break;
          }
          ++run;
          tc_fence_after();
          const bool add = kc >= GB_DRAIN;
          const int64_t gr = (int64_t)tk.r0 + r;
          for (int c0 = 0; c0 < pr.N; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + tmem + (uint32_t)c0, v);
            tmem_wait_ld();
            if (gr < pr.M) {
              float* orow = pr.C + gr * pr.ldc + c0;
#pragma unroll
              for (int c = 0; c < 16; ++c)
                if (c0 + c < pr.ncol)
                  orow[c] = add ? __fadd_rn(orow[c], __uint_as_float(v[c])) : __uint_as_float(v[c]);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acc_empty);
        }
        if (++s == GB_ST) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(GB_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Operand preparation of the grouped passes.
// ---------------------------------------------------------------------------

// Rows of every problem's A copied to a 16-byte pitch (TMA); one block per
// (problem, 32-row chunk).
__global__ void __launch_bounds__(256) pad_rows_batched_kernel(const TgPad* __restrict__ jobs,
                                                                const int2* __restrict__ chunks) {
  const int2 ch = chunks[blockIdx.x];
  const TgPad jb = jobs[ch.x];
  const int64_t r1 = min((int64_t)ch.y + 32, jb.rows);
  for (int64_t r = ch.y + threadIdx.y; r < r1; r += blockDim.y)
    for (int64_t c = threadIdx.x; c < jb.cols; c += blockDim.x)
      jb.dst[r * jb.ldd + c] = __ldg(jb.src + r * jb.lds + c);
}

// W^T split into bf16 hi / lo (K-major rows of the MMA's B operand): row j < l
// of the output is column j of W (rows x l, ld l); rows l .. N - 1 are zero.
// One block per (problem, 32-row chunk of W).
__global__ void __launch_bounds__(256) split_t_batched_kernel(const TgSplit* __restrict__ jobs,
                                                               const int2* __restrict__ chunks) {
  __shared__ float tile[32][TG_NMAX + 1];
  const int2 ch = chunks[blockIdx.x];
  const TgSplit jb = jobs[ch.x];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int64_t k0 = ch.y;
  const int kr = (int)min((int64_t)32, jb.rows - k0);
  for (int e = tid; e < 32 * jb.l; e += 256) {
    const int kk = e / jb.l, j = e - kk * jb.l;
    tile[kk][j] = kk < kr ? jb.W[(k0 + kk) * jb.ldw + j] : 0.f;
  }
  __syncthreads();
  for (int e = tid; e < jb.N * 32; e += 256) {
    const int j = e >> 5, kk = e & 31;
    if (kk >= kr) continue;
    const float v = j < jb.l ? tile[kk][j] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r1);
    const int64_t o = (int64_t)j * jb.ldt + k0 + kk;
    reinterpret_cast<__nv_bfloat16*>(jb.hi)[o] = h;
    reinterpret_cast<__nv_bfloat16*>(jb.lo)[o] = lo;
    if (jb.lo2)   // third term: the rest of the 24 bits
      reinterpret_cast<__nv_bfloat16*>(jb.lo2)[o] = __float2bfloat16_rn(r1 - __bfloat162float(lo));
  }
}

// Omega^T of every problem as bf16 (exact: the Gaussians are rounded to bf16,
// the same values the SIMT path draws): row j < l, column k is Omega(k, j)
// of the problem's stream (batch word = the problem index); rows l .. N - 1
// zero.  One block per (problem, 32-row chunk of Omega).
__global__ void __launch_bounds__(256) omega_t_batched_kernel(const TgSplit* __restrict__ jobs,
                                                               const int2* __restrict__ chunks,
                                                               uint64_t seed) {
  const int2 ch = chunks[blockIdx.x];
  const TgSplit jb = jobs[ch.x];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int64_t k0 = ch.y;
  const int kr = (int)min((int64_t)32, jb.rows - k0);
  const int nq = jb.N / 4;
  for (int e = tid; e < 32 * nq; e += 256) {
    const int kk = e / nq, qd = e - kk * nq;
    if (kk >= kr) continue;
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (4 * qd < jb.l) {
      gauss4_f(omega_words(seed, (uint32_t)(k0 + kk), (uint32_t)qd, 0u, (uint32_t)jb.batch), z);
#pragma unroll
      for (int t = 0; t < 4; ++t) z[t] = round_bf16(z[t]);
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int j = 4 * qd + t;
      reinterpret_cast<__nv_bfloat16*>(jb.hi)[(int64_t)j * jb.ldt + k0 + kk] =
          __float2bfloat16_rn(j < jb.l ? z[t] : 0.f);
    }
  }
}

// ------------------------------- host side ---------------------------------

bool tg_encode_maps(int form, int nwt, const float* Ap, int64_t m, int64_t n, int64_t ldap,
                    const void* whi, const void* wlo, const void* wlo2, int64_t K, int N,
                    int64_t ldt, CUtensorMap out[4]) {
  memset(out, 0, 4 * sizeof(CUtensorMap));
  bool ok;
  if (form == 0)   // rows of 32 fp32 (128 bytes), swizzled
    ok = encode_2d(&out[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Ap, (uint64_t)n, (uint64_t)m,
                   (uint64_t)ldap, GB_BK, GB_BM, CU_TENSOR_MAP_SWIZZLE_128B);
  else             // 32 rows of 128 columns
    ok = encode_2d(&out[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, Ap, (uint64_t)n, (uint64_t)m,
                   (uint64_t)ldap, GB_BM, GB_BK, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!ok) return false;
  const void* wp[3] = {whi, wlo, wlo2};
  for (int t = 0; t < nwt; ++t) {
    if (!wp[t]) return false;
    ok = encode_2d(&out[1 + t], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, wp[t], (uint64_t)K,
                   (uint64_t)N, (uint64_t)ldt, GB_BK, (uint32_t)N, CU_TENSOR_MAP_SWIZZLE_64B);
    if (!ok) return false;
  }
  for (int t = nwt; t < 3; ++t) out[1 + t] = out[1];
  return true;
}

cudaError_t launch_tc_group(int form, int nwt, bool gram, const TgProb* probs,
                            const TgTask* tasks, int ntasks, const CUtensorMap* maps, int* d_info,
                            cudaStream_t s) {
  if (ntasks <= 0) return cudaSuccess;
  const int G = std::min(ntasks, device_sm_count());
  const size_t smem = gb_smem(nwt);
  void (*kern)(const TgProb*, const TgTask*, int, const CUtensorMap*, int*) = nullptr;
  if (form == 0 && nwt == 1 && !gram) kern = tc_group_kernel<0, 1, false>;
  else if (form == 0 && nwt == 2 && !gram) kern = tc_group_kernel<0, 2, false>;
  else if (form == 0 && nwt == 3 && !gram) kern = tc_group_kernel<0, 3, false>;
  else if (form == 1 && nwt == 2 && !gram) kern = tc_group_kernel<1, 2, false>;
  else if (form == 1 && nwt == 2 && gram) kern = tc_group_kernel<1, 2, true>;
  else return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  const int cls = gram ? RSVD_TRACE_GRAM
                      : (nwt == 3 ? RSVD_TRACE_APPLY
                                  : (form == 1 ? RSVD_TRACE_AT_W
                                               : (nwt == 1 ? RSVD_TRACE_A_OMEGA : RSVD_TRACE_A_W)));
  const int tr = trace_begin(cls, s);
  kern<<<G, 256, smem, s>>>(probs, tasks, ntasks, maps, d_info);
  count_launch();
  trace_end(tr, s);
  return cudaGetLastError();
}

cudaError_t launch_pad_rows_batched(const TgPad* jobs, const int2* chunks, int nchunks,
                                    cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  pad_rows_batched_kernel<<<nchunks, dim3(64, 4), 0, s>>>(jobs, chunks);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_split_t_batched(const TgSplit* jobs, const int2* chunks, int nchunks,
                                   cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  split_t_batched_kernel<<<nchunks, dim3(32, 8), 0, s>>>(jobs, chunks);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_omega_t_batched(const TgSplit* jobs, const int2* chunks, int nchunks,
                                   uint64_t seed, cudaStream_t s) {
  if (nchunks <= 0) return cudaSuccess;
  omega_t_batched_kernel<<<nchunks, dim3(32, 8), 0, s>>>(jobs, chunks, seed);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rsvd
