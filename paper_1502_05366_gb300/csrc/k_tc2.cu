// Passes over A with a stored right-hand operand, on 256-row units:
//
//   form 0:  Y (rows x L) = A (rows x K) W        power step Y = A Z (Sec. 3.2)
//   form 1:  Z (rows x L) = A^T W, A is K x rows  power step Z = A^* Y, QB step
//                                                  Bt = A^* Q (Alg. 5)
//
// Each CTA (one per SM, persistent, stream-K over (unit, k-chunk)) computes
// two 128-row M-tiles of a 256-row unit, and both tiles share every stage of
// W.  Against one tile per CTA this halves the W traffic (W is re-read from L2
// for every unit and K-chunk) and spreads each stage's synchronisation over
// 256 rows.  A is fp32 (split a0 + a1 as in k_tc.cu) or bf16 (exact a0).
// Products per K-step and tile: a0 w0, plus a1 w0 for fp32 A when W has two
// terms, plus a0 w1 when W has two terms (NW = 2); NW = 1 (the mixed-precision
// power scheme) is a0 w0 alone.  bf16 in, fp32 accumulation in TMEM.
//
// Roles:
//   warp 0      TMA of the A stage: 256 rows (form 0) or 256 columns (form 1)
//               of 32 K-values, fp32 or bf16
//   warp 1      MMA issuer and TMEM owner (accumulators at columns 0 and 256)
//   warp 2      TMA of the W stage (NW bf16 terms, L rows of 32 K-values)
//   warps 4-11  converters: one A row per thread -> bf16 hi (and lo) rows of
//               K-major 64-byte-swizzled tiles in shared memory; then the
//               epilogue of their tile (t = (warp - 4) / 4, TMEM lane quadrant
//               warp % 4) into the output or a stream-K partial
// Bounded accumulation runs (P.drain > 0): the tensor cores' fp32 accumulation
// into TMEM is not rounded to nearest, and over a long contraction its error
// drifts one way (over the 50000-row contraction of Bt = A^* Q a TMEM
// accumulator holding ~800 K-chunks came out ~6.5e-5 small in relative
// terms).  With drain = D the accumulator holds at most D K-chunks; the
// epilogue then adds it into the CTA's partial tile in fp32 with round to
// nearest, and the MMAs restart on a fresh accumulator.
//
// Every mbarrier wait is bounded: on expiry the kernel records
// RSVD_ERR_TIMEOUT, the roles leave their loops, the producers wait (bounded)
// for their copies in flight, TMEM is freed and the CTA returns.
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace rsvd {

using namespace tc;

namespace {
constexpr int U_BM = 128;                     // rows of an M-tile (MMA M)
constexpr int U_ROWS = 2 * U_BM;              // rows of a unit
constexpr int U_BK = 32;                      // K per stage
constexpr int U_FST = 3;                      // A stages as loaded
constexpr int U_BST = 2;                      // operand stages (bf16 A tiles + W)
constexpr int U_FBYTES = U_ROWS * U_BK * 4;   // 32 KB: an fp32 stage (bf16 uses half)
constexpr int U_AT = U_BM * U_BK * 2;         // 8 KB: one bf16 tile
constexpr int U_NCONV = 8;                    // warps 4..11
constexpr int U_THREADS = 32 * (4 + U_NCONV); // 384
constexpr uint32_t U_TMEM_COLS = 512;
constexpr uint32_t U_ACC2 = 256;              // TMEM column of the second accumulator

__host__ __device__ constexpr int u_wtile(int L) { return L * U_BK * 2; }
__host__ __device__ constexpr int u_bstage(int L, int nw) { return 4 * U_AT + nw * u_wtile(L); }
size_t u_smem(int L, int nw) {
  return 1024 + (size_t)U_FST * U_FBYTES + (size_t)U_BST * u_bstage(L, nw) + 256;
}
}  // namespace

template <int FORM, int NW, bool ABF>
__global__ void __launch_bounds__(U_THREADS, 1)
    tc_unit_kernel(const __grid_constant__ CUtensorMap mapA,
                   const __grid_constant__ CUtensorMap mapW0,
                   const __grid_constant__ CUtensorMap mapW1, TcParams P) {
  // the second bf16 term of A exists for fp32 A when W has two terms
  constexpr bool ALO = !ABF && NW == 2;
  // bf16 A in form 0: the TMA lands each stage as two 64-byte-swizzled K-major
  // M-tiles, the layout the MMA reads, so the MMAs take A straight from the
  // A ring (released by their commit) and the converter warps only run the
  // epilogue
  constexpr bool DA = ABF && FORM == 0;
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  if (P.skip && *P.skip) return;
  unsigned char* dsm = (unsigned char*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int L = P.L;
  const int BSB = u_bstage(L, NW);
  const int WT = u_wtile(L);
  unsigned char* fring = dsm;
  unsigned char* bring = dsm + U_FST * U_FBYTES;
  uint64_t* bars = (uint64_t*)(bring + U_BST * BSB);
  uint64_t* ffull = bars;                  // A stage landed
  uint64_t* fempty = bars + U_FST;         // A stage read by the converters
  uint64_t* aready = bars + 2 * U_FST;     // bf16 A tiles written
  uint64_t* wfull = aready + U_BST;        // W stage landed
  uint64_t* bdone = wfull + U_BST;         // MMAs of the operand stage finished
  uint64_t* acc_full = bdone + U_BST;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_holder = (uint32_t*)(acc_empty + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t it0 = ((int64_t)blockIdx.x * P.total) / G;
  const int64_t it1 = ((int64_t)(blockIdx.x + 1) * P.total) / G;

  if (threadIdx.x == 0) {
    for (int s = 0; s < U_FST; ++s) {
      mbar_init(&ffull[s], 1);
      mbar_init(&fempty[s], DA ? 1 : U_NCONV);
    }
    for (int s = 0; s < U_BST; ++s) {
      mbar_init(&aready[s], U_NCONV);
      mbar_init(&wfull[s], 1);
      mbar_init(&bdone[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, U_NCONV);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane == 0) prefetch_map(&mapA);
  if (warp == 2 && lane == 0) {
    prefetch_map(&mapW0);
    if (NW == 2) prefetch_map(&mapW1);
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(U_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ------------------------------ A producer --------------------------------
    if (lane == 0) {
      const uint32_t bytes = ABF ? U_FBYTES / 2 : U_FBYTES;
      int64_t last_issued = -1;
      int64_t unit = it0 / P.kiters, kc = it0 - unit * P.kiters;
      int fs = 0;
      uint32_t fph = 0;
      const uint64_t pol_a = l2_policy_evict_first();   // A streams through once
      for (int64_t it = it0; it < it1; ++it) {
        if (!mbar_wait(&fempty[fs], fph ^ 1u, abort_flag, P.d_info)) break;
        mbar_arrive_expect_tx(&ffull[fs], bytes);
        if (FORM == 0)
          tma_load_2d_hint(fring + fs * U_FBYTES, &mapA, &ffull[fs], (int)(kc * U_BK),
                           (int)(unit * U_ROWS), pol_a);
        else
          tma_load_2d_hint(fring + fs * U_FBYTES, &mapA, &ffull[fs], (int)(unit * U_ROWS),
                           (int)(kc * U_BK), pol_a);
        last_issued = it - it0;
        if (++kc == P.kiters) {
          kc = 0;
          ++unit;
        }
        if (++fs == U_FST) {
          fs = 0;
          fph ^= 1u;
        }
      }
      if (*abort_flag && last_issued >= 0) {
        const int64_t first = last_issued - U_FST + 1 > 0 ? last_issued - U_FST + 1 : 0;
        for (int64_t li = first; li <= last_issued; ++li) {
          const int sd = (int)(li % U_FST);
          const uint32_t pd = (uint32_t)((li / U_FST) & 1);
          const long long t0 = clock64();
          while (!mbar_try_wait(&ffull[sd], pd) && clock64() - t0 < WAIT_LIMIT) {
          }
        }
      }
    }
  } else if (warp == 2) {
    // ------------------------------ W producer --------------------------------
    if (lane == 0) {
      int64_t last_issued = -1;
      int64_t kc = it0 % P.kiters;
      int bs = 0;
      uint32_t bph = 0;
      const uint64_t pol_w = l2_policy_evict_last();    // W is re-read by every unit
      for (int64_t it = it0; it < it1; ++it) {
        if (!mbar_wait(&bdone[bs], bph ^ 1u, abort_flag, P.d_info)) break;
        unsigned char* wb = bring + bs * BSB + 4 * U_AT;
        mbar_arrive_expect_tx(&wfull[bs], (uint32_t)(NW * WT));
        tma_load_2d_hint(wb, &mapW0, &wfull[bs], (int)(kc * U_BK), 0, pol_w);
        if (NW == 2) tma_load_2d_hint(wb + WT, &mapW1, &wfull[bs], (int)(kc * U_BK), 0, pol_w);
        last_issued = it - it0;
        if (++kc == P.kiters) kc = 0;
        if (++bs == U_BST) {
          bs = 0;
          bph ^= 1u;
        }
      }
      if (*abort_flag && last_issued >= 0) {
        const int64_t first = last_issued - U_BST + 1 > 0 ? last_issued - U_BST + 1 : 0;
        for (int64_t li = first; li <= last_issued; ++li) {
          const int sd = (int)(li % U_BST);
          const uint32_t pd = (uint32_t)((li / U_BST) & 1);
          const long long t0 = clock64();
          while (!mbar_try_wait(&wfull[sd], pd) && clock64() - t0 < WAIT_LIMIT) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------- MMA issuer -------------------------------
    if (lane == 0) {
      const uint32_t idesc = make_idesc(U_BM, L);
      int64_t run = -1;   // accumulation runs: one per segment, or `drain` K-chunks each
      int rc = 0;         // K-chunks in the current run
      int64_t kc = it0 % P.kiters;
      int bs = 0, fs = 0;
      uint32_t bph = 0, fph = 0;
      for (int64_t it = it0; it < it1; ++it) {
        if (it == it0 || kc == 0) rc = 0;
        if (rc == 0) {
          ++run;
          if (run > 0 && !mbar_wait(acc_empty, (uint32_t)((run - 1) & 1), abort_flag, P.d_info))
            break;
        }
        if (DA) {
          if (!mbar_wait(&ffull[fs], fph, abort_flag, P.d_info)) break;
        } else {
          if (!mbar_wait(&aready[bs], bph, abort_flag, P.d_info)) break;
        }
        if (!mbar_wait(&wfull[bs], bph, abort_flag, P.d_info)) break;
        tc_fence_after();
        const uint32_t base = smem_u32(bring + bs * BSB);
        const uint32_t wbase = base + 4u * U_AT;
        // M-tile t of A: tiles 2t (hi), 2t + 1 (lo) of the operand stage, or
        // rows 128 t .. of the landed bf16 stage
        const uint32_t abase = DA ? smem_u32(fring + fs * U_FBYTES) : base;
        const uint32_t astride = DA ? (uint32_t)U_AT : 2u * U_AT;
#pragma unroll
        for (int kk = 0; kk < U_BK / 16; ++kk) {
          const uint64_t bw0 = sw64_desc(wbase + 32u * kk);
          const uint64_t bw1 = sw64_desc(wbase + (uint32_t)WT + 32u * kk);
          const uint32_t acc0 = (rc == 0 && kk == 0) ? 0u : 1u;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const uint32_t d = tmem + U_ACC2 * (uint32_t)t;
            const uint64_t ahi = sw64_desc(abase + (uint32_t)t * astride + 32u * kk);
            mma_ss(d, ahi, bw0, idesc, acc0);
            if (ALO) mma_ss(d, sw64_desc(base + (uint32_t)(2 * t + 1) * U_AT + 32u * kk), bw0,
                            idesc, 1u);
            if (NW == 2) mma_ss(d, ahi, bw1, idesc, 1u);
          }
        }
        mma_commit(&bdone[bs]);
        if (DA) mma_commit(&fempty[fs]);
        ++rc;
        const bool seg_end = (it + 1 == it1) || (kc + 1 == P.kiters);
        if (seg_end || (P.drain > 0 && rc == P.drain)) {
          mma_commit(acc_full);
          rc = 0;
        }
        if (++kc == P.kiters) kc = 0;
        if (++bs == U_BST) {
          bs = 0;
          bph ^= 1u;
        }
        if (DA && ++fs == U_FST) {
          fs = 0;
          fph ^= 1u;
        }
      }
    }
  } else if (warp >= 4 && warp < 4 + U_NCONV) {
    // ------------------------ converters and epilogue -------------------------
    const int t = (warp - 4) >> 2;          // M-tile of the unit
    const int q = warp & 3;                 // TMEM lane quadrant
    const int r = 32 * q + lane;            // row within the tile
    const int rr = t * U_BM + r;            // row within the unit
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t acc = tmem + U_ACC2 * (uint32_t)t;
    int64_t run = -1;     // accumulation runs, counted as the MMA issuer counts them
    int rc = 0, rin = 0;  // K-chunks in the run; runs of this segment already drained
    int64_t unit = it0 / P.kiters, kc = it0 - unit * P.kiters;
    const int64_t unit0 = unit;
    bool whole = false;
    int fs = 0, bs = 0;
    uint32_t fph = 0, bph = 0;
    for (int64_t it = it0; it < it1; ++it) {
      if (it == it0 || kc == 0) {
        whole = (kc == 0);
        rc = 0;
        rin = 0;
      }
      if (rc == 0) ++run;
      if (!DA) {
      if (!mbar_wait(&ffull[fs], fph, abort_flag, P.d_info)) break;
      const unsigned char* st = fring + fs * U_FBYTES;
      uint32_t hi[16], lo[16];
      if (ABF) {
        if (FORM == 0) {      // 64-byte-swizzled rows of 32 bf16
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint4 v =
                *reinterpret_cast<const uint4*>(st + sw64_off((uint32_t)rr, (uint32_t)c));
            hi[4 * c] = v.x;
            hi[4 * c + 1] = v.y;
            hi[4 * c + 2] = v.z;
            hi[4 * c + 3] = v.w;
          }
        } else {              // plain 32 x 256 bf16 tile, row = k: column rr
          const unsigned short* tp = reinterpret_cast<const unsigned short*>(st);
#pragma unroll
          for (int k = 0; k < 16; ++k)
            hi[k] = (uint32_t)tp[(2 * k) * U_ROWS + rr] |
                    ((uint32_t)tp[(2 * k + 1) * U_ROWS + rr] << 16);
        }
      } else {
        float x[32];
        if (FORM == 0) {      // 128-byte-swizzled rows of 32 fp32
          const unsigned char* row = st + rr * 128;
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(row + ((c ^ (rr & 7)) << 4));
            x[4 * c] = v.x;
            x[4 * c + 1] = v.y;
            x[4 * c + 2] = v.z;
            x[4 * c + 3] = v.w;
          }
        } else {              // plain 32 x 256 fp32 tile, row = k: column rr
          const float* tp = reinterpret_cast<const float*>(st);
#pragma unroll
          for (int k = 0; k < 32; ++k) x[k] = tp[k * U_ROWS + rr];
        }
        split_row(x, hi, lo);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&fempty[fs]);
      if (!mbar_wait(&bdone[bs], bph ^ 1u, abort_flag, P.d_info)) break;
      const uint32_t ab = smem_u32(bring + bs * BSB + 2 * t * U_AT);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const uint32_t o = sw64_off((uint32_t)r, (uint32_t)cc);
        st_shared_v4(ab + o, hi[4 * cc], hi[4 * cc + 1], hi[4 * cc + 2], hi[4 * cc + 3]);
        if (ALO)
          st_shared_v4(ab + U_AT + o, lo[4 * cc], lo[4 * cc + 1], lo[4 * cc + 2], lo[4 * cc + 3]);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aready[bs]);
      }
      ++rc;
      const bool seg_end = (it + 1 == it1) || (kc + 1 == P.kiters);
      if (seg_end || (P.drain > 0 && rc == P.drain)) {
        if (!mbar_wait(acc_full, (uint32_t)(run & 1), abort_flag, P.d_info)) break;
        tc_fence_after();
        const int64_t gr = unit * U_ROWS + rr;
        // the CTA's partial tile of this segment (column-major, 256 rows): it
        // receives every run but the last of a whole unit; rows are thread-owned
        float* slot =
            P.part + ((int64_t)blockIdx.x * P.maxseg + (unit - unit0)) * (int64_t)U_ROWS * L;
        if (seg_end && whole && kc + 1 == P.kiters) {
          // this CTA holds the whole unit: final rows (+ transposed bf16 split),
          // the earlier runs' sum added from the partial tile
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + acc + (uint32_t)c0, v);
            tmem_wait_ld();
            if (rin > 0) {
#pragma unroll
              for (int c = 0; c < 16; ++c)
                v[c] = __float_as_uint(slot[(int64_t)(c0 + c) * U_ROWS + rr] +
                                       __uint_as_float(v[c]));
            }
            if (gr < P.rows) {
              float* orow = P.out + gr * P.ldo + c0;
              const bool vec =
                  (c0 + 16 <= P.ncols) && ((reinterpret_cast<uintptr_t>(orow) & 15u) == 0);
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
                  P.out_lo[(int64_t)col * P.ldt + gr] =
                      __float2bfloat16_rn(w - __bfloat162float(h));
                }
              }
            }
          }
        } else {
          // a partial segment's sum for the fixed-order reduce, or a bounded run
          // drained mid-segment: the first run writes, later runs add (fp32,
          // round to nearest, in run order)
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + acc + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              float* d = slot + (int64_t)(c0 + c) * U_ROWS + rr;
              *d = rin > 0 ? *d + __uint_as_float(v[c]) : __uint_as_float(v[c]);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
        ++rin;
        rc = 0;
      }
      if (++kc == P.kiters) {
        kc = 0;
        ++unit;
      }
      if (++fs == U_FST) {
        fs = 0;
        fph ^= 1u;
      }
      if (++bs == U_BST) {
        bs = 0;
        bph ^= 1u;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(U_TMEM_COLS)
                 : "memory");
  }
}

template <int FORM, int NW, bool ABF>
static cudaError_t launch_unit(const CUtensorMap& ma, const CUtensorMap& mw0,
                               const CUtensorMap& mw1, const TcParams& P, int G, size_t smem,
                               cudaStream_t s) {
  auto kern = tc_unit_kernel<FORM, NW, ABF>;
  cudaError_t e =
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tr = trace_begin(FORM == 1 ? RSVD_TRACE_AT_W : RSVD_TRACE_A_W, s);
  kern<<<G, U_THREADS, smem, s>>>(ma, mw0, mw1, P);
  count_launch();
  trace_end(tr, s);
  return cudaGetLastError();
}

bool tc_unit_supported(const TcGemm& g) {
  const int nw = g.wterms;
  if (g.gram || g.omega || (nw != 1 && nw != 2)) return false;
  if (!tc_supported(g.L)) return false;
  return u_smem(g.L, nw) + 64 <= 232448;
}

cudaError_t launch_tc_unit(const TcGemm& g, cudaStream_t s) {
  if (!tc_unit_supported(g)) return cudaErrorInvalidValue;
  const int nw = g.wterms;
  const bool abf = g.a_bf16 != 0;
  int64_t units, kiters, total, G;
  int maxseg;
  sk_plan(g.rows, g.K, U_ROWS, U_BK, device_sm_count(), &units, &kiters, &total, &G, &maxseg);
  TcParams P;
  P.rows = g.rows;
  P.K = g.K;
  P.bm = U_ROWS;
  P.ustride = U_ROWS;
  P.uoff = 0;
  P.wmul = 1;
  P.wadd = 0;
  P.L = g.L;
  P.lvalid = g.lvalid;
  P.seed = g.seed;
  P.tiles = units;
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
  P.drain = g.drain;

  CUtensorMap ma, mw0, mw1;
  memset(&ma, 0, sizeof(ma));
  memset(&mw0, 0, sizeof(mw0));
  memset(&mw1, 0, sizeof(mw1));
  const CUtensorMapDataType adt =
      abf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const int aes = abf ? 2 : 4;
  bool ok;
  if (g.form == 0)   // 256 rows of 32 values: 128-byte (fp32) or 64-byte (bf16) swizzled rows
    ok = encode_2d(&ma, adt, aes, g.A, (uint64_t)g.a_cols_total, (uint64_t)g.a_rows_total,
                   (uint64_t)g.lda, U_BK, U_ROWS,
                   abf ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
  else               // 32 rows (K) of 256 values, unswizzled
    ok = encode_2d(&ma, adt, aes, g.A, (uint64_t)g.a_cols_total, (uint64_t)g.a_rows_total,
                   (uint64_t)g.lda, U_ROWS, U_BK, CU_TENSOR_MAP_SWIZZLE_NONE);
  if (!ok) return cudaErrorInvalidValue;
  if (!g.Whi || (nw == 2 && !g.Wlo)) return cudaErrorInvalidValue;
  ok = encode_2d(&mw0, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.Whi, (uint64_t)g.K, (uint64_t)g.L,
                 (uint64_t)g.ldw, U_BK, (uint32_t)g.L, CU_TENSOR_MAP_SWIZZLE_64B);
  if (ok && nw == 2)
    ok = encode_2d(&mw1, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, g.Wlo, (uint64_t)g.K,
                   (uint64_t)g.L, (uint64_t)g.ldw, U_BK, (uint32_t)g.L,
                   CU_TENSOR_MAP_SWIZZLE_64B);
  if (!ok) return cudaErrorInvalidValue;
  if (nw == 1) mw1 = mw0;
  const size_t smem = u_smem(g.L, nw) + 64;
  cudaError_t e;
  const int Gi = (int)G;
  if (g.form == 0)
    e = nw == 1 ? (abf ? launch_unit<0, 1, true>(ma, mw0, mw1, P, Gi, smem, s)
                       : launch_unit<0, 1, false>(ma, mw0, mw1, P, Gi, smem, s))
                : (abf ? launch_unit<0, 2, true>(ma, mw0, mw1, P, Gi, smem, s)
                       : launch_unit<0, 2, false>(ma, mw0, mw1, P, Gi, smem, s));
  else
    e = nw == 1 ? (abf ? launch_unit<1, 1, true>(ma, mw0, mw1, P, Gi, smem, s)
                       : launch_unit<1, 1, false>(ma, mw0, mw1, P, Gi, smem, s))
                : (abf ? launch_unit<1, 2, true>(ma, mw0, mw1, P, Gi, smem, s)
                       : launch_unit<1, 2, false>(ma, mw0, mw1, P, Gi, smem, s));
  if (e != cudaSuccess) return e;
  return launch_tc_reduce(P, Gi, s);
}

}  // namespace rsvd
