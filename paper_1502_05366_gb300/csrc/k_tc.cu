// tcgen05 (5th-generation tensor core) GEMMs for the passes over A.
//
//   form 0:  Y (rows x L) = A (rows x K) W       power step Y = A Z, orth apply X R^-1
//                                                (the sketch Y = A Omega: k_omega.cu)
//   form 1:  Z (rows x L) = A^T W, A is K x rows  power step Z = A^* Y (Sec. 3.2),
//                                                QB step Bt = A^* Q (Alg. 5), Gram X^T X
//
// Arithmetic: every fp32 entry x of A is split as x ~ a0 + a1 with a0 = bf16(x),
// a1 = bf16(x - a0) (16 significant bits).  W comes in NW bf16 terms:
//   NW = 1  one term (the mixed-precision power scheme): a0 w0 only
//           (Omega, bf16-exact, takes a0 w0 + a1 w0 in k_omega.cu)
//   NW = 2  stored matrix of generic data (Q, Z, X): a0 w0 + a1 w0 + a0 w1
//   NW = 3  the l x l factor R^-1 of CholeskyQR:     a0 w0 + a1 w0 + a0 w1 + a0 w2
//   NW = 4  Gram X^T X (W = split of X itself):      a0 w0 + a1 w0 + a0 w1 + a1 w1
// A stored in bf16 (a_bf16) is exact as a0 (a1 = 0): its passes issue one
// product per W term and stream half the bytes.
// For two different matrices the dropped term a1 w1 and the rounding residuals
// are independent from entry to entry and only add noise of relative size
// 2^-17.  R^-1 is one fixed matrix applied to every row, so its rounding would
// bias the result: it keeps 24 bits.  In a Gram both factors carry the same
// residual a1 and sum_i a1_i^2 is a positive bias on the diagonal: kept.  The products run as
// tcgen05.mma kind::f16 with fp32 accumulation in tensor memory (TMEM).
//
// Data flow per CTA (one CTA per SM, persistent, stream-K over the flattened
// (tile, k-chunk) iteration space so that every SM gets the same share):
//   warp 0      TMA producer: fp32 A tile (128 x 32) and the W hi/lo tiles
//   warp 1      MMA issuer (one thread) and TMEM owner
//   warps 4-7   converters: fp32 A tile (shared) -> bf16 hi/lo rows -> TMEM
//               (tcgen05.st), then the epilogue (tcgen05.ld -> partial tile)
// Partial tiles are summed in a fixed order by tc_reduce_kernel, which writes
// the fp32 result and, on request, the transposed bf16 hi/lo split that the
// next GEMM consumes.
//
// Every mbarrier wait is bounded (~1 s of clock): on expiry the kernel records
// RSVD_ERR_TIMEOUT, every role leaves its loop, the producer waits (bounded)
// for its own copies in flight, TMEM is freed and the CTA returns.
#include <cuda.h>
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "fp8.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace rsvd {

using namespace tc;

namespace {
constexpr int BM = 128;             // output rows per tile (MMA M)
constexpr int BK = 32;              // K per stage
constexpr int MAXST = 4;            // stages (3 when W has three bf16 terms)
constexpr int A_STAGE_BYTES = BM * BK * 4;   // 16 KB fp32 (a bf16 A tile uses the first half)
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t TMEM_A0 = 256;   // first TMEM column of the A stages
constexpr int NCONV = 4;            // converter / epilogue warps (4..7)

__host__ __device__ constexpr int w_tile_bytes(int L) { return L * BK * 2; }
__host__ __device__ constexpr int stages_for(int nw) { return nw == 3 ? 3 : 4; }
// W tiles per stage: stored 2, R^-1 3, Gram 2.
__host__ __device__ constexpr int w_tiles(int nw) { return nw == 4 ? 2 : nw; }
__host__ __device__ constexpr int stage_bytes(int L, int nw) {
  return A_STAGE_BYTES + w_tiles(nw) * w_tile_bytes(L);
}
}  // namespace


// Stream-K bounds of CTA b.
__device__ __forceinline__ int64_t sk_start(int64_t b, int64_t total, int64_t G) {
  return (b * total) / G;
}

template <int FORM, int NW, bool ABF, bool Q8 = false>
__global__ void __launch_bounds__(256, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                   const __grid_constant__ CUtensorMap mapW0,
                   const __grid_constant__ CUtensorMap mapW1,
                   const __grid_constant__ CUtensorMap mapW2, TcParams P) {
  constexpr bool GRAM = (NW == 4);
  constexpr int NWT = w_tiles(NW);   // W tiles loaded per stage
  constexpr int STAGES = stages_for(NW);
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  if (P.skip && *P.skip) return;
  unsigned char* dsm = (unsigned char*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int L = P.L;
  const int SB = stage_bytes(L, NW);
  uint64_t* bars = (uint64_t*)(dsm + STAGES * SB);
  uint64_t* full = bars;                  // TMA landed (A [+ W])
  uint64_t* conv = bars + STAGES;         // A stage written to TMEM
  uint64_t* done = bars + 2 * STAGES;     // MMAs of the stage finished
  uint64_t* acc_full = bars + 3 * STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_holder = (uint32_t*)(acc_empty + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t it0 = sk_start(blockIdx.x, P.total, G);
  const int64_t it1 = sk_start(blockIdx.x + 1, P.total, G);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], NCONV);
      mbar_init(&done[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NCONV);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane == 0) {
    prefetch_map(&mapA);
    prefetch_map(&mapW0);
    if (NWT >= 2) prefetch_map(&mapW1);
    if (NWT == 3) prefetch_map(&mapW2);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(TMEM_COLS)
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
      const uint32_t bytes =
          (ABF ? A_STAGE_BYTES / 2 : A_STAGE_BYTES) + (uint32_t)NWT * (uint32_t)w_tile_bytes(L);
      int64_t last_issued = -1;
      int64_t tile = it0 / P.kiters, kc = it0 - tile * P.kiters;
      int s = 0;
      uint32_t ph = 0;
      // A streams through once: evict first; the W tiles are re-read by every
      // output tile: evict last
      const uint64_t pol_a = l2_policy_evict_first(), pol_w = l2_policy_evict_last();
      for (int64_t it = it0; it < it1; ++it) {
        const int64_t li = it - it0;
        if (!mbar_wait(&done[s], ph ^ 1u, abort_flag, P.d_info)) break;
        unsigned char* st = dsm + s * SB;
        mbar_arrive_expect_tx(&full[s], bytes);
        if (FORM == 0)
          tma_load_2d_hint(st, &mapA, &full[s], (int)(kc * BK), (int)(tile * BM), pol_a);
        else
          tma_load_2d_hint(st, &mapA, &full[s], (int)(tile * BM), (int)(kc * BK), pol_a);
        tma_load_2d_hint(st + A_STAGE_BYTES, &mapW0, &full[s], (int)(kc * BK), 0, pol_w);
        if (NWT >= 2)
          tma_load_2d_hint(st + A_STAGE_BYTES + w_tile_bytes(L), &mapW1, &full[s], (int)(kc * BK),
                           0, pol_w);
        if (NWT == 3)
          tma_load_2d_hint(st + A_STAGE_BYTES + 2 * w_tile_bytes(L), &mapW2, &full[s],
                           (int)(kc * BK), 0, pol_w);
        last_issued = li;
        if (++kc == P.kiters) {
          kc = 0;
          ++tile;
        }
        if (++s == STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
      if (*abort_flag && last_issued >= 0) {
        // drain: wait (bounded) for the copies this thread issued
        const int64_t first = last_issued - STAGES + 1 > 0 ? last_issued - STAGES + 1 : 0;
        for (int64_t li = first; li <= last_issued; ++li) {
          const int sd = (int)(li % STAGES);
          const uint32_t pd = (uint32_t)((li / STAGES) & 1);
          const long long t0 = clock64();
          while (!mbar_try_wait(&full[sd], pd) && clock64() - t0 < WAIT_LIMIT) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------- MMA issuer -------------------------------
    if (lane == 0) {
      const uint32_t idesc = make_idesc(BM, L);
      int64_t seg = -1;
      int64_t kc = it0 % P.kiters;
      int s = 0;
      uint32_t ph = 0;
      for (int64_t it = it0; it < it1; ++it) {
        const bool seg_start = (it == it0) || (kc == 0);
        if (seg_start) {
          ++seg;
          if (seg > 0 && !mbar_wait(acc_empty, (uint32_t)((seg - 1) & 1), abort_flag, P.d_info))
            break;
        }
        if (!mbar_wait(&conv[s], ph, abort_flag, P.d_info)) break;
        if (!mbar_wait(&full[s], ph, abort_flag, P.d_info)) break;
        tc_fence_after();
        const uint32_t wbase = smem_u32(dsm + s * SB + A_STAGE_BYTES);
        const uint32_t a_col = tmem + TMEM_A0 + 32u * (uint32_t)s;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint64_t bhi = sw64_desc(wbase + 32u * kk);
          const uint32_t ahi = a_col + 8u * kk;
          const uint32_t alo = a_col + 16u + 8u * kk;
          const uint32_t acc0 = (seg_start && kk == 0) ? 0u : 1u;
          mma_ts(tmem, ahi, bhi, idesc, acc0);
          if (!ABF && NW != 1) mma_ts(tmem, alo, bhi, idesc, 1u);
#pragma unroll
          for (int t = 1; t < NWT; ++t) {
            const uint64_t bt = sw64_desc(wbase + (uint32_t)(t * w_tile_bytes(L)) + 32u * kk);
            mma_ts(tmem, ahi, bt, idesc, 1u);
            if (GRAM) mma_ts(tmem, alo, bt, idesc, 1u);
          }
        }
        mma_commit(&done[s]);
        const bool seg_end = (it + 1 == it1) || (kc + 1 == P.kiters);
        if (seg_end) mma_commit(acc_full);
        if (++kc == P.kiters) kc = 0;
        if (++s == STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
  } else if (warp >= 4 && warp < 4 + NCONV) {
    // ------------------------ converters and epilogue -------------------------
    const int q = warp - 4;                 // TMEM lane quadrant (= warp % 4)
    const int r = 32 * q + lane;            // tile row handled by this thread
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    int64_t seg = -1;
    int64_t tile = it0 / P.kiters, kc = it0 - tile * P.kiters;
    const int64_t tile0 = tile;
    bool whole = false;                     // current segment started at k-chunk 0
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    for (int64_t it = it0; it < it1 && ok; ++it) {
      if (it == it0 || kc == 0) {
        ++seg;
        whole = (kc == 0);
      }
      if (!mbar_wait(&full[s], ph, abort_flag, P.d_info)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const unsigned char* st = dsm + s * SB;
      const uint32_t a_col = tmem + TMEM_A0 + 32u * (uint32_t)s;
      if (Q8) {
        // FP8 sketch (form 0): the row's 32 values of this K-chunk are one
        // block; quantised to E4M3 with its scale, exact in bf16 (one term)
        float x[32];
        if (ABF) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint4 v = *reinterpret_cast<const uint4*>(st + sw64_off((uint32_t)r, (uint32_t)c));
            const uint32_t wv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              x[8 * c + 2 * e] = __uint_as_float(wv[e] << 16);
              x[8 * c + 2 * e + 1] = __uint_as_float(wv[e] & 0xffff0000u);
            }
          }
        } else {
          const unsigned char* row = st + r * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(row + ((c ^ (r & 7)) << 4));
            x[4 * c] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
          }
        }
        uint32_t hi[16];
        e4m3_block_bf16(x, hi);
        tmem_st16(lane_base + a_col, hi);
      } else if (ABF) {
        // bf16 A: the tile row (form 0, 64-byte swizzled rows of 32 values) or
        // column (form 1, plain 32 x 128 tile) goes to TMEM as it is
        uint32_t hi[16];
        if (FORM == 0) {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint4 v = *reinterpret_cast<const uint4*>(st + sw64_off((uint32_t)r, (uint32_t)c));
            hi[4 * c] = v.x;
            hi[4 * c + 1] = v.y;
            hi[4 * c + 2] = v.z;
            hi[4 * c + 3] = v.w;
          }
        } else {
          const unsigned short* t = reinterpret_cast<const unsigned short*>(st);
#pragma unroll
          for (int k = 0; k < 16; ++k)
            hi[k] = (uint32_t)t[(2 * k) * BM + r] | ((uint32_t)t[(2 * k + 1) * BM + r] << 16);
        }
        tmem_st16(lane_base + a_col, hi);
      } else {
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
        const float* t = reinterpret_cast<const float*>(st);
#pragma unroll
        for (int k = 0; k < 32; ++k) x[k] = t[k * BM + r];
      }
      uint32_t hi[16], lo[16];
      split_row(x, hi, lo);
      tmem_st16(lane_base + a_col, hi);
      tmem_st16(lane_base + a_col + 16u, lo);
      }
      tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&conv[s]);
      const bool seg_end = (it + 1 == it1) || (kc + 1 == P.kiters);
      if (seg_end) {
        if (!mbar_wait(acc_full, (uint32_t)(seg & 1), abort_flag, P.d_info)) {
          ok = false;
          break;
        }
        tc_fence_after();
        if (whole && kc + 1 == P.kiters) {
          // this CTA holds the whole tile: final rows (+ transposed bf16 split)
          const int64_t gr = tile * BM + r;
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + tmem + (uint32_t)c0, v);
            tmem_wait_ld();
            if (gr < P.rows) {
              float* orow = P.out + gr * P.ldo + c0;
              const bool vec = (c0 + 16 <= P.ncols) && ((reinterpret_cast<uintptr_t>(orow) & 15u) == 0);
              if (vec) {
#pragma unroll
                for (int c = 0; c < 16; c += 4)
                  *reinterpret_cast<float4*>(orow + c) =
                      make_float4(__uint_as_float(v[c]), __uint_as_float(v[c + 1]),
                                  __uint_as_float(v[c + 2]), __uint_as_float(v[c + 3]));
              }
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const int col = c0 + c;
                const float val = __uint_as_float(v[c]);
                if (!vec && col < P.ncols) orow[c] = val;
                if (P.out_hi) {
                  const float w = col < P.ncols ? val : 0.0f;
                  const __nv_bfloat16 h = __float2bfloat16_rn(w);
                  P.out_hi[(int64_t)col * P.ldt + gr] = h;
                  P.out_lo[(int64_t)col * P.ldt + gr] = __float2bfloat16_rn(w - __bfloat162float(h));
                }
              }
            }
          }
        } else {
          float* dst = P.part + ((int64_t)blockIdx.x * P.maxseg + (tile - tile0)) * (int64_t)BM * L;
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + tmem + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; ++c) dst[(int64_t)(c0 + c) * BM + r] = __uint_as_float(v[c]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
      }
      if (++kc == P.kiters) {
        kc = 0;
        ++tile;
      }
      if (++s == STAGES) {
        s = 0;
        ph ^= 1u;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// Fixed-order sum of the stream-K partials of the tiles split between CTAs.
// Block (sub, z): boundary b = z + 1 (start of CTA b); the tile containing it
// is handled by the first boundary inside it; the block sums one 32 x 32
// sub-tile over the contributing CTAs in increasing order and writes the fp32
// output and, when requested, the transposed bf16 split (padding zero).
// The boundaries that start a split tile (the only ones with work), found on
// the host; n = 0: every boundary b = blockIdx.y + 1 (more than 256 CTAs).
struct RedList {
  int n;
  int b[256];
};

__global__ void tc_reduce_kernel(TcParams P, int G, const __grid_constant__ RedList R) {
  if (P.skip && *P.skip) return;
  __shared__ float tile_s[32][33];
  __shared__ int64_t s_base[1024];
  const int64_t b = R.n > 0 ? (int64_t)R.b[blockIdx.y] : (int64_t)blockIdx.y + 1;
  const int64_t sb = (b * P.total) / G;
  const int64_t t = sb / P.kiters;
  if (sb == t * P.kiters) return;                           // boundary at a tile start
  const int64_t sprev = ((b - 1) * P.total) / G;
  if (b - 1 >= 1 && sprev > t * P.kiters) return;          // not the first boundary in t
  const int64_t last = (t + 1) * P.kiters - 1;
  const int64_t blo = b - 1;
  const int L = P.L;
  const int tid = threadIdx.x + threadIdx.y * 32;
  // contributors blo .. bhi: CTA c contributes iff start(c) <= last
  int nctr;
  __shared__ int s_n;
  if (tid == 0) {
    int64_t c = b;
    while (c < G && (c * P.total) / G <= last) ++c;
    s_n = (int)(c - blo);
  }
  __syncthreads();
  nctr = s_n;
  if (nctr > 1024) nctr = 1024;
  for (int i = tid; i < nctr; i += 256) {
    const int64_t c = blo + i;
    const int64_t tile0 = ((c * P.total) / G) / P.kiters;
    s_base[i] = ((c * P.wmul + P.wadd) * P.maxseg + (t - tile0)) * (int64_t)P.bm * L;
  }
  __syncthreads();
  const int rg = blockIdx.x % (P.bm / 32), jg = blockIdx.x / (P.bm / 32);
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  // contributors are added in increasing order; each thread's four rows and 8
  // contributors are loaded together so that a load's latency is not paid per
  // contributor
  {
    float sum[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i0 = 0; i0 < nctr; i0 += 8) {
      float v[4][8];
#pragma unroll
      for (int a4 = 0; a4 < 4; ++a4) {
        const int j = jg * 32 + ty + 8 * a4;
        const int64_t off = (int64_t)j * P.bm + rg * 32 + tx;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          v[a4][u] = (j < L && i0 + u < nctr) ? P.part[s_base[min(i0 + u, nctr - 1)] + off] : 0.f;
      }
#pragma unroll
      for (int a4 = 0; a4 < 4; ++a4)
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (i0 + u < nctr) sum[a4] += v[a4][u];
    }
#pragma unroll
    for (int a4 = 0; a4 < 4; ++a4) tile_s[ty + 8 * a4][tx] = sum[a4];
  }
  __syncthreads();
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t i = t * P.ustride + P.uoff + rg * 32 + rr;
    const int j = jg * 32 + tx;
    if (i < P.rows && j < P.ncols) P.out[i * P.ldo + j] = tile_s[tx][rr];
  }
  if (P.out_hi) {
    for (int jj = ty; jj < 32; jj += 8) {
      const int j = jg * 32 + jj;
      const int64_t i = t * P.ustride + P.uoff + rg * 32 + tx;
      if (j < L && i < P.rows) {
        const float v = (j < P.ncols) ? tile_s[jj][tx] : 0.0f;
        const __nv_bfloat16 h = __float2bfloat16_rn(v);
        P.out_hi[(int64_t)j * P.ldt + i] = h;
        P.out_lo[(int64_t)j * P.ldt + i] = __float2bfloat16_rn(v - __bfloat162float(h));
      }
    }
  }
}

// ------------------------------- host side ---------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn get_encode() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

bool encode_2d(CUtensorMap* map, CUtensorMapDataType dt, int elem, const void* base,
                      uint64_t inner, uint64_t outer, uint64_t pitch_elems, uint32_t box_inner,
                      uint32_t box_outer, CUtensorMapSwizzle sw) {
  EncodeTiledFn fn = get_encode();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {pitch_elems * (uint64_t)elem};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  return fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 148;
  return sms;
}

bool tc_supported(int L) { return L >= 16 && L <= 256 && L % 16 == 0; }

void sk_plan(int64_t rows, int64_t K, int bm, int bk, int G_hint, int64_t* tiles, int64_t* kiters,
             int64_t* total, int64_t* G, int* maxseg) {
  *tiles = ceil_div(rows, bm);
  *kiters = ceil_div(K, bk);
  *total = (*tiles) * (*kiters);
  int64_t g = G_hint;
  if (g > *total) g = *total;
  if (g < 1) g = 1;
  *G = g;
  int ms = 1;
  for (int64_t b = 0; b < g; ++b) {
    const int64_t s = (b * (*total)) / g, e = ((b + 1) * (*total)) / g;
    if (e <= s) continue;
    const int segs = (int)((e - 1) / (*kiters) - s / (*kiters) + 1);
    if (segs > ms) ms = segs;
  }
  *maxseg = ms;
}

// Partial-tile buffer of one GEMM: the larger of the one-tile (128-row) plan
// and the two-tile (256-row) plan of the Omega kernel.
size_t tc_part_bytes(int64_t rows, int64_t K, int L) {
  size_t best = 0;
  for (int bm = 128; bm <= 256; bm *= 2) {
    int64_t tiles, kiters, total, G;
    int maxseg;
    sk_plan(rows, K, bm, BK, device_sm_count(), &tiles, &kiters, &total, &G, &maxseg);
    const size_t b = (size_t)G * maxseg * bm * L * sizeof(float);
    if (b > best) best = b;
  }
  {  // two-CTA Omega kernel: 512-row units over SMs / 2 pairs, 256-row partials per CTA
    int64_t tiles, kiters, total, G;
    int maxseg;
    sk_plan(rows, K, 512, BK, device_sm_count() / 2, &tiles, &kiters, &total, &G, &maxseg);
    const size_t b = (size_t)2 * G * maxseg * 256 * L * sizeof(float);
    if (b > best) best = b;
  }
  return best;
}

cudaError_t launch_tc_reduce(const TcParams& P, int G, cudaStream_t s) {
  if (G <= 1) return cudaSuccess;
  // the kernel's own test, on the host: boundary b = start of CTA b works iff
  // it falls inside a tile and is the first boundary inside that tile
  RedList R;
  R.n = 0;
  int ny = G - 1;
  if (G - 1 <= 256) {
    for (int64_t b = 1; b < G; ++b) {
      const int64_t sb = (b * P.total) / G;
      const int64_t t = sb / P.kiters;
      if (sb == t * P.kiters) continue;
      const int64_t sprev = ((b - 1) * P.total) / G;
      if (b - 1 >= 1 && sprev > t * P.kiters) continue;
      R.b[R.n++] = (int)b;
    }
    if (R.n == 0) return cudaSuccess;   // no tile is split between CTAs
    ny = R.n;
  }
  dim3 rgrid((unsigned)((P.bm / 32) * ceil_div(P.L, 32)), (unsigned)ny);
  const int tr = trace_begin(RSVD_TRACE_REDUCE, s);
  tc_reduce_kernel<<<rgrid, dim3(32, 8), 0, s>>>(P, G, R);
  count_launch();
  trace_end(tr, s);
  return cudaGetLastError();
}

template <int FORM, int NW, bool ABF = false, bool Q8 = false>
static cudaError_t launch_form(const CUtensorMap& ma, const CUtensorMap* mw, const TcParams& P,
                               int G, size_t smem, cudaStream_t s) {
  auto kern = tc_gemm_kernel<FORM, NW, ABF, Q8>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  // trace classes (include/rsvd.h): 0 A Omega, 1 A W, 2 A^T W, 3 Gram, 4 orth apply
  const int cls = Q8 ? RSVD_TRACE_A_OMEGA
                     : (FORM == 1 ? (NW == 4 ? RSVD_TRACE_GRAM : RSVD_TRACE_AT_W)
                                  : (NW == 3 ? RSVD_TRACE_APPLY : RSVD_TRACE_A_W));
  const int tr = trace_begin(cls, s);
  kern<<<G, 256, smem, s>>>(ma, mw[0], mw[1], mw[2], P);
  count_launch();
  trace_end(tr, s);
  return cudaGetLastError();
}

cudaError_t launch_tc_gemm(const TcGemm& g, cudaStream_t s) {
  if (g.L > 256 && g.L % 16 == 0 && g.L <= 1024) {
    // wider outputs (the sketch width l > 256): column chunks of at most 256,
    // one launch each over the whole of A.  Chunk c0 takes rows c0.. of the
    // transposed bf16 operand and of the transposed output split, output
    // columns c0.., and for Omega the columns c0.. of the Gaussian stream.
    for (int c0 = 0; c0 < g.L; c0 += 256) {
      const int Lc = std::min(256, g.L - c0);
      TcGemm gc = g;
      gc.L = Lc;
      gc.col0 = g.col0 + c0;
      gc.lvalid = std::max(0, std::min(g.lvalid - c0, Lc));
      gc.ncols = std::max(0, std::min(g.ncols - c0, Lc));
      gc.out = g.out + c0;
      auto off16 = [&](const void* p, int64_t ld) -> const void* {
        return p ? (const void*)((const __nv_bfloat16*)p + (int64_t)c0 * ld) : nullptr;
      };
      gc.Whi = off16(g.Whi, g.ldw);
      gc.Wlo = off16(g.Wlo, g.ldw);
      gc.Wlo2 = off16(g.Wlo2, g.ldw);
      gc.out_hi = g.out_hi ? (void*)((__nv_bfloat16*)g.out_hi + (int64_t)c0 * g.ldt) : nullptr;
      gc.out_lo = g.out_lo ? (void*)((__nv_bfloat16*)g.out_lo + (int64_t)c0 * g.ldt) : nullptr;
      cudaError_t e = launch_tc_gemm(gc, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (!tc_supported(g.L)) return cudaErrorInvalidValue;
  if (g.form == 1 && g.omega) return cudaErrorInvalidValue;
  if (g.form == 0 && g.omega) return launch_tc_omega(g, s);
  if (g.q8 && (g.form != 0 || g.wterms != 1 || g.gram)) return cudaErrorInvalidValue;
  // the passes over A with a stored operand: two M-tiles per CTA (k_tc2.cu)
  if (!g.q8 && tc_unit_supported(g)) return launch_tc_unit(g, s);
  int64_t tiles, kiters, total, G;
  int maxseg;
  const int sms = device_sm_count();
  sk_plan(g.rows, g.K, BM, BK, sms, &tiles, &kiters, &total, &G, &maxseg);
  // Short contractions (the R^-1 apply of CholeskyQR, K = L): one CTA per
  // output tile instead of stream-K, so that no tile is split and the reduce
  // launch disappears (a few waves of short CTAs cost less than the split
  // tiles' partial writes and the extra launch)
  bool whole_tiles = false;
  if (kiters <= 8 && tiles > sms && tiles <= 4 * (int64_t)sms) {
    G = tiles;
    maxseg = 1;
    whole_tiles = true;
  }
  TcParams P;
  P.rows = g.rows;
  P.K = g.K;
  P.bm = BM;
  P.ustride = BM;
  P.uoff = 0;
  P.wmul = 1;
  P.wadd = 0;
  P.L = g.L;
  P.lvalid = g.lvalid;
  P.seed = g.seed;
  P.tiles = tiles;
  P.kiters = kiters;
  P.total = total;
  P.maxseg = maxseg;
  P.part = g.part;
  P.out = g.out;
  P.ldo = g.ldo;
  P.ncols = g.ncols;
  P.out_hi = (__nv_bfloat16*)g.out_hi;
  P.out_lo = (__nv_bfloat16*)g.out_lo;
  P.ldt = g.ldt;
  P.skip = g.skip;
  P.d_info = g.d_info;

  CUtensorMap ma, mw[3];
  memset(&ma, 0, sizeof(ma));
  memset(mw, 0, sizeof(mw));
  bool ok;
  const bool abf = g.a_bf16 != 0;
  const CUtensorMapDataType adt = abf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const int aes = abf ? 2 : 4;
  if (g.form == 0)   // rows of BK values: 128 bytes (fp32) or 64 bytes (bf16), swizzled
    ok = encode_2d(&ma, adt, aes, g.A, (uint64_t)g.a_cols_total, (uint64_t)g.a_rows_total,
                   (uint64_t)g.lda, BK, BM,
                   abf ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
  else
    ok = encode_2d(&ma, adt, aes, g.A, (uint64_t)g.a_cols_total, (uint64_t)g.a_rows_total,
                   (uint64_t)g.lda, BM, BK, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!ok) return cudaErrorInvalidValue;
  const int nw = g.gram ? 4 : g.wterms;
  if (nw < 1 || nw > 4 || (g.gram && g.wterms != 2))
    return cudaErrorInvalidValue;
  if (abf && nw > 2) return cudaErrorInvalidValue;   // bf16 A: stored-W passes only
  const int nwt = w_tiles(nw);
  const void* wp[3] = {g.Whi, g.Wlo, g.Wlo2};
  for (int t = 0; t < nwt; ++t) {
    if (!wp[t]) return cudaErrorInvalidValue;
    ok = encode_2d(&mw[t], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, wp[t], (uint64_t)g.K,
                   (uint64_t)g.L, (uint64_t)g.ldw, BK, (uint32_t)g.L, CU_TENSOR_MAP_SWIZZLE_64B);
    if (!ok) return cudaErrorInvalidValue;
  }
  for (int t = nwt; t < 3; ++t) mw[t] = mw[0];
  const size_t smem = (size_t)stages_for(nw) * stage_bytes(g.L, nw) + 1024 /*align*/ +
                      (4 * MAXST + 2) * 8 + 16;
  cudaError_t e;
  if (g.q8)
    e = abf ? launch_form<0, 1, true, true>(ma, mw, P, (int)G, smem, s)
            : launch_form<0, 1, false, true>(ma, mw, P, (int)G, smem, s);
  else if (nw == 1)
    e = g.form == 0 ? (abf ? launch_form<0, 1, true>(ma, mw, P, (int)G, smem, s)
                           : launch_form<0, 1, false>(ma, mw, P, (int)G, smem, s))
                    : (abf ? launch_form<1, 1, true>(ma, mw, P, (int)G, smem, s)
                           : launch_form<1, 1, false>(ma, mw, P, (int)G, smem, s));
  else if (abf && g.form == 0)
    e = launch_form<0, 2, true>(ma, mw, P, (int)G, smem, s);
  else if (abf)
    e = launch_form<1, 2, true>(ma, mw, P, (int)G, smem, s);
  else if (g.form == 0 && nw == 2)
    e = launch_form<0, 2>(ma, mw, P, (int)G, smem, s);
  else if (g.form == 0 && nw == 3)
    e = launch_form<0, 3>(ma, mw, P, (int)G, smem, s);
  else if (g.form == 1 && nw == 2)
    e = launch_form<1, 2>(ma, mw, P, (int)G, smem, s);
  else if (g.form == 1 && nw == 4)
    e = launch_form<1, 4>(ma, mw, P, (int)G, smem, s);
  else
    return cudaErrorInvalidValue;
  if (e != cudaSuccess) return e;
  // fixed-order reduction of the tiles split between CTAs
  if (!whole_tiles) {
    e = launch_tc_reduce(P, (int)G, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace rsvd
