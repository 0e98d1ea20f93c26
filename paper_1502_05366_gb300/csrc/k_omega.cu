// Sketch Y = A Omega (Sec. 3.1, Fig. 1 step 2) on the tcgen05 tensor cores,
// with Omega generated inside the kernel from its Philox counter stream and
// never stored.
//
// Generating Omega is the cost of this GEMM: every 128-row M-tile needs the
// whole n x l Omega, i.e. l/128 Gaussians per entry of A.  Here one stream-K
// unit is a pair of M-tiles (256 rows of A) that share every generated Omega
// stage, which halves the Gaussians per entry of A.  The two fp32 accumulators
// (up to 256 columns each) take all 512 TMEM columns, so the bf16 hi/lo split
// of A is staged in shared memory and both MMA operands come from shared-
// memory descriptors.  Arithmetic as in k_tc.cu: a0 w0 + a1 w0 with
// x ~ a0 + a1 (16 significant bits) and Omega bf16-exact.
//
// Roles (896 threads, one CTA per SM, persistent stream-K over the flattened
// (unit, k-chunk) space):
//   warp 0       TMA producer: fp32 A block (256 rows x 32) into a 3-stage ring
//   warp 1       MMA issuer (one thread) and TMEM owner
//   warps 4-11   converters: fp32 rows -> bf16 hi/lo rows (64-byte swizzled,
//                K-major) in a 2-stage operand ring; then the epilogue of
//                their TMEM lane quadrant of their tile
//   warps 12-27  generators: the bf16 Omega tile (same layout) in the operand
//                ring; one thread makes 4 K-consecutive quads (2 L units per
//                stage, so that every generator thread has work) and stores
//                each of its 4 columns as one 8-byte half chunk
// Every wait is bounded (about 1 s of clock); on expiry the kernel records
// RSVD_ERR_TIMEOUT, all roles leave, the producer drains its copies in flight
// and TMEM is freed.
#include <cuda.h>

#include "common.cuh"
#include "kernels.h"
#include "tc_ptx.cuh"

namespace rsvd {

using namespace tc;

namespace {
constexpr int OBM = 128;                      // rows of one M-tile (MMA M)
constexpr int OUNIT = 2 * OBM;                // rows of one stream-K unit
constexpr int OBK = 32;                       // K per stage
constexpr int F_ST = 2;                       // fp32 A stages
constexpr int B_ST = 3;                       // bf16 operand stages (generation runs ahead)
constexpr int F_BYTES = OUNIT * OBK * 4;      // 32 KB
constexpr int AT_BYTES = OBM * OBK * 2;       // 8 KB: one tile, hi or lo
constexpr int NCONV = 8;                      // warps 4..11
constexpr int NGEN = 16;                      // warps 12..27
constexpr int OTHREADS = 32 * (12 + NGEN);    // 896
constexpr uint32_t TMEM_COLS = 512;
constexpr uint32_t ACC_STRIDE = 256;          // TMEM column of the second accumulator

__host__ __device__ constexpr int w_bytes(int L) { return L * OBK * 2; }
__host__ __device__ constexpr int b_stage_bytes(int L) { return 4 * AT_BYTES + w_bytes(L); }
size_t omega_smem(int L) { return 1024 + (size_t)F_ST * F_BYTES + (size_t)B_ST * b_stage_bytes(L) + 256; }

__device__ __forceinline__ void st_shared_v2(uint32_t addr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}
// Distributed shared memory: this CTA's shared address mapped into the peer
// CTA of the cluster, stores there, and remote mbarrier arrivals.
__device__ __forceinline__ uint32_t mapa_peer(uint32_t addr, uint32_t peer) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(peer));
  return r;
}
__device__ __forceinline__ void st_shared_b32(uint32_t addr, uint32_t a) {
  asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(a) : "memory");
}
__device__ __forceinline__ void st_cluster_b32(uint32_t addr, uint32_t a) {
  asm volatile("st.shared::cluster.b32 [%0], %1;" ::"r"(addr), "r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
               : "memory");
}
// try_wait with cluster-scope acquire (arrivals come from the peer CTA too)
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity,
                                                  volatile int* abort_flag, int* d_info) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait_cluster(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_LIMIT) {
      *abort_flag = 1;
      set_info(d_info, RSVD_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

}  // namespace

__global__ void __launch_bounds__(OTHREADS, 1)
    tc_omega_kernel(const __grid_constant__ CUtensorMap mapA, TcParams P) {
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  if (P.skip && *P.skip) return;
  unsigned char* dsm = (unsigned char*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int L = P.L;
  const int BSB = b_stage_bytes(L);
  unsigned char* fring = dsm;
  unsigned char* bring = dsm + F_ST * F_BYTES;
  uint64_t* bars = (uint64_t*)(bring + B_ST * BSB);
  uint64_t* ffull = bars;                 // fp32 block landed (TMA bytes)
  uint64_t* fempty = bars + F_ST;         // fp32 block read by the converters
  uint64_t* aready = bars + 2 * F_ST;     // bf16 A tiles written
  uint64_t* wready = aready + B_ST;       // Omega tile written
  uint64_t* bdone = wready + B_ST;        // MMAs of the operand stage finished
  uint64_t* acc_full = bdone + B_ST;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_holder = (uint32_t*)(acc_empty + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t G = gridDim.x;
  const int64_t it0 = (blockIdx.x * P.total) / G;
  const int64_t it1 = ((blockIdx.x + 1) * P.total) / G;

  if (threadIdx.x == 0) {
    for (int s = 0; s < F_ST; ++s) {
      mbar_init(&ffull[s], 1);
      mbar_init(&fempty[s], NCONV);
    }
    for (int s = 0; s < B_ST; ++s) {
      mbar_init(&aready[s], NCONV);
      mbar_init(&wready[s], NGEN);
      mbar_init(&bdone[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NCONV);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane == 0) prefetch_map(&mapA);
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
      int64_t last_issued = -1;
      int64_t unit = it0 / P.kiters, kc = it0 - unit * P.kiters;
      int fs = 0;
      uint32_t fph = 0;
      const uint64_t pol_a = l2_policy_evict_first();   // A streams through once
      for (int64_t it = it0; it < it1; ++it) {
        if (!mbar_wait(&fempty[fs], fph ^ 1u, abort_flag, P.d_info)) break;
        mbar_arrive_expect_tx(&ffull[fs], (uint32_t)F_BYTES);
        tma_load_2d_hint(fring + fs * F_BYTES, &mapA, &ffull[fs], (int)(kc * OBK),
                         (int)(unit * OUNIT), pol_a);
        last_issued = it - it0;
        if (++kc == P.kiters) {
          kc = 0;
          ++unit;
        }
        if (++fs == F_ST) {
          fs = 0;
          fph ^= 1u;
        }
      }
      if (*abort_flag && last_issued >= 0) {
        const int64_t first = last_issued - F_ST + 1 > 0 ? last_issued - F_ST + 1 : 0;
        for (int64_t li = first; li <= last_issued; ++li) {
          const int sd = (int)(li % F_ST);
          const uint32_t pd = (uint32_t)((li / F_ST) & 1);
          const long long t0 = clock64();
          while (!mbar_try_wait(&ffull[sd], pd) && clock64() - t0 < WAIT_LIMIT) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------- MMA issuer -------------------------------
    if (lane == 0) {
      const uint32_t idesc = make_idesc(OBM, L);
      int64_t seg = -1;
      int64_t kc = it0 % P.kiters;
      int bs = 0;
      uint32_t bph = 0;
      for (int64_t it = it0; it < it1; ++it) {
        const bool seg_start = (it == it0) || (kc == 0);
        if (seg_start) {
          ++seg;
          if (seg > 0 && !mbar_wait(acc_empty, (uint32_t)((seg - 1) & 1), abort_flag, P.d_info))
            break;
        }
        if (!mbar_wait(&aready[bs], bph, abort_flag, P.d_info)) break;
        if (!mbar_wait(&wready[bs], bph, abort_flag, P.d_info)) break;
        tc_fence_after();
        const uint32_t base = smem_u32(bring + bs * BSB);
#pragma unroll
        for (int kk = 0; kk < OBK / 16; ++kk) {
          const uint64_t bw = sw64_desc(base + 4u * AT_BYTES + 32u * kk);
          const uint32_t acc0 = (seg_start && kk == 0) ? 0u : 1u;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const uint32_t d = tmem + ACC_STRIDE * (uint32_t)t;
            mma_ss(d, sw64_desc(base + (uint32_t)(2 * t) * AT_BYTES + 32u * kk), bw, idesc, acc0);
            mma_ss(d, sw64_desc(base + (uint32_t)(2 * t + 1) * AT_BYTES + 32u * kk), bw, idesc, 1u);
          }
        }
        mma_commit(&bdone[bs]);
        const bool seg_end = (it + 1 == it1) || (kc + 1 == P.kiters);
        if (seg_end) mma_commit(acc_full);
        if (++kc == P.kiters) kc = 0;
        if (++bs == B_ST) {
          bs = 0;
          bph ^= 1u;
        }
      }
    }
  } else if (warp >= 4 && warp < 4 + NCONV) {
    // ------------------------ converters and epilogue -------------------------
    const int t = (warp - 4) >> 2;          // M-tile of the unit
    const int q = warp & 3;                 // TMEM lane quadrant (= warp % 4)
    const int r = 32 * q + lane;            // row within the tile
    const int rr = t * OBM + r;             // row within the fp32 block
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t acc = tmem + ACC_STRIDE * (uint32_t)t;
    int64_t seg = -1;
    int64_t unit = it0 / P.kiters, kc = it0 - unit * P.kiters;
    const int64_t unit0 = unit;
    bool whole = false;
    int fs = 0, bs = 0;
    uint32_t fph = 0, bph = 0;
    for (int64_t it = it0; it < it1; ++it) {
      if (it == it0 || kc == 0) {
        ++seg;
        whole = (kc == 0);
      }
      if (!mbar_wait(&ffull[fs], fph, abort_flag, P.d_info)) break;
      // 128B-swizzled rows of 32 fp32: 16-byte chunk c of row rr sits at c ^ (rr & 7)
      float x[32];
      const unsigned char* row = fring + fs * F_BYTES + rr * 128;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(row + ((c ^ (rr & 7)) << 4));
        x[4 * c] = v.x;
        x[4 * c + 1] = v.y;
        x[4 * c + 2] = v.z;
        x[4 * c + 3] = v.w;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&fempty[fs]);
      uint32_t hi[16], lo[16];
      split_row(x, hi, lo);
      if (!mbar_wait(&bdone[bs], bph ^ 1u, abort_flag, P.d_info)) break;
      const uint32_t ab = smem_u32(bring + bs * BSB + 2 * t * AT_BYTES);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const uint32_t o = sw64_off((uint32_t)r, (uint32_t)cc);
        st_shared_v4(ab + o, hi[4 * cc], hi[4 * cc + 1], hi[4 * cc + 2], hi[4 * cc + 3]);
        st_shared_v4(ab + AT_BYTES + o, lo[4 * cc], lo[4 * cc + 1], lo[4 * cc + 2],
                     lo[4 * cc + 3]);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aready[bs]);
      const bool seg_end = (it + 1 == it1) || (kc + 1 == P.kiters);
      if (seg_end) {
        if (!mbar_wait(acc_full, (uint32_t)(seg & 1), abort_flag, P.d_info)) break;
        tc_fence_after();
        if (whole && kc + 1 == P.kiters) {
          // this CTA holds the whole unit: final rows (+ transposed bf16 split)
          const int64_t gr = unit * OUNIT + rr;
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + acc + (uint32_t)c0, v);
            tmem_wait_ld();
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
          float* dst =
              P.part + ((int64_t)blockIdx.x * P.maxseg + (unit - unit0)) * (int64_t)OUNIT * L;
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + acc + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; ++c)
              dst[(int64_t)(c0 + c) * OUNIT + rr] = __uint_as_float(v[c]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
      }
      if (++kc == P.kiters) {
        kc = 0;
        ++unit;
      }
      if (++fs == F_ST) {
        fs = 0;
        fph ^= 1u;
      }
      if (++bs == B_ST) {
        bs = 0;
        bph ^= 1u;
      }
    }
  } else if (warp >= 12 && warp < 12 + NGEN) {
    // ------------------------- Omega generator warps --------------------------
    const int gt = threadIdx.x - 12 * 32;   // 0 .. 32 NGEN - 1
    const int nunits = 2 * L;               // (L / 4 quads) x (8 groups of 4 K-rows)
    int64_t kc = it0 % P.kiters;
    int bs = 0;
    uint32_t bph = 0;
    for (int64_t it = it0; it < it1; ++it) {
      if (!mbar_wait(&bdone[bs], bph ^ 1u, abort_flag, P.d_info)) break;
      const uint32_t wb = smem_u32(bring + bs * BSB + 4 * AT_BYTES);
      for (int u = gt; u < nunits; u += NGEN * 32) {
        const int kk4 = u & 7, qd = u >> 3;
        uint32_t pk[4][2];
#pragma unroll
        for (int c = 0; c < 4; ++c) pk[c][0] = pk[c][1] = 0u;
        if (4 * qd < P.lvalid) {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int64_t krow = kc * OBK + kk4 * 4 + e;
            float z[4] = {0.f, 0.f, 0.f, 0.f};
            if (krow < P.K) OmegaGen<float>::quad(P.seed, (uint32_t)krow, (uint32_t)(qd + P.qoff), z);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              // z is bf16-exact: its upper 16 bits are the bf16 encoding
              const uint32_t b = (4 * qd + c < P.lvalid) ? (__float_as_uint(z[c]) >> 16) : 0u;
              pk[c][e >> 1] |= b << (16 * (e & 1));
            }
          }
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t o = sw64_off((uint32_t)(4 * qd + c), (uint32_t)(kk4 >> 1)) + 8u * (kk4 & 1);
          st_shared_v2(wb + o, pk[c][0], pk[c][1]);
        }
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&wready[bs]);
      if (++kc == P.kiters) kc = 0;
      if (++bs == B_ST) {
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
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Two-CTA cluster version: a stream-K unit is a super-unit of 512 rows; CTA r
// of the pair takes rows 256 r .. 256 r + 255 of it (two M-tiles) and both run
// the same (super-unit, k-chunk) sequence.  CTA r generates K-rows
// 16 r .. 16 r + 15 of every Omega stage and stores them into its own and the
// peer's operand ring (distributed shared memory), so one generated Omega
// stage feeds four M-tiles.  A peer's ring slot is written only after the
// peer has reported the MMAs of its previous use done (remote arrival on
// pfree); the MMA thread waits for the Omega tile from both CTAs' generators.
// Waits are bounded; a final cluster barrier keeps each CTA's shared memory
// alive until the peer has finished writing into it.
// ---------------------------------------------------------------------------
constexpr int NGEN2 = 16;                       // generator warps 12..27
constexpr int OTHREADS2 = 32 * (12 + NGEN2);    // 896

// ABF: A holds bf16 values; TMA lands each stage as two 64-byte-swizzled
// K-major M-tiles that the MMAs read directly (one product per M-tile and
// K-step); the converter warps only run the epilogue.
template <bool ABF>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(OTHREADS2, 1)
    tc_omega2_kernel(const __grid_constant__ CUtensorMap mapA, TcParams P) {
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  if (P.skip && *P.skip) return;
  unsigned char* dsm = (unsigned char*)(((uintptr_t)dsm_raw + 1023) & ~(uintptr_t)1023);
  const int L = P.L;
  const int BSB = b_stage_bytes(L);
  unsigned char* fring = dsm;
  unsigned char* bring = dsm + F_ST * F_BYTES;
  uint64_t* bars = (uint64_t*)(bring + B_ST * BSB);
  uint64_t* ffull = bars;
  uint64_t* fempty = bars + F_ST;
  uint64_t* aready = bars + 2 * F_ST;
  uint64_t* wready = aready + B_ST;       // Omega tile complete: both CTAs' generators
  uint64_t* bdone = wready + B_ST;
  uint64_t* pfree = bdone + B_ST;         // the peer's ring slot is free (remote arrival)
  uint64_t* acc_full = pfree + B_ST;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_holder = (uint32_t*)(acc_empty + 1);
  volatile int* abort_flag = (volatile int*)(tmem_holder + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_ctarank(), peer = rank ^ 1u;
  const int64_t Gc = gridDim.x >> 1, cid = blockIdx.x >> 1;
  const int64_t it0 = (cid * P.total) / Gc;
  const int64_t it1 = ((cid + 1) * P.total) / Gc;

  if (threadIdx.x == 0) {
    for (int s = 0; s < F_ST; ++s) {
      mbar_init(&ffull[s], 1);
      mbar_init(&fempty[s], ABF ? 1 : NCONV);   // ABF: released by the MMAs' commit
    }
    for (int s = 0; s < B_ST; ++s) {
      mbar_init(&aready[s], NCONV);
      mbar_init(&wready[s], 2 * (NGEN2 / 2));   // one generator group from each CTA
      mbar_init(&bdone[s], 1);
      mbar_init(&pfree[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, NCONV);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0 && lane == 0) prefetch_map(&mapA);
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_holder)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();                     // both CTAs' barriers initialised
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      int64_t last_issued = -1;
      int64_t su = it0 / P.kiters, kc = it0 - su * P.kiters;
      int fs = 0;
      uint32_t fph = 0;
      const uint64_t pol_a = l2_policy_evict_first();
      for (int64_t it = it0; it < it1; ++it) {
        if (!mbar_wait(&fempty[fs], fph ^ 1u, abort_flag, P.d_info)) break;
        mbar_arrive_expect_tx(&ffull[fs], (uint32_t)(ABF ? F_BYTES / 2 : F_BYTES));
        tma_load_2d_hint(fring + fs * F_BYTES, &mapA, &ffull[fs], (int)(kc * OBK),
                         (int)(su * 2 * OUNIT + rank * OUNIT), pol_a);
        last_issued = it - it0;
        if (++kc == P.kiters) {
          kc = 0;
          ++su;
        }
        if (++fs == F_ST) {
          fs = 0;
          fph ^= 1u;
        }
      }
      if (*abort_flag && last_issued >= 0) {
        const int64_t first = last_issued - F_ST + 1 > 0 ? last_issued - F_ST + 1 : 0;
        for (int64_t li = first; li <= last_issued; ++li) {
          const int sd = (int)(li % F_ST);
          const uint32_t pd = (uint32_t)((li / F_ST) & 1);
          const long long t0 = clock64();
          while (!mbar_try_wait(&ffull[sd], pd) && clock64() - t0 < WAIT_LIMIT) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------- MMA issuer -------------------------------
    if (lane == 0) {
      const uint32_t idesc = make_idesc(OBM, L);
      int64_t seg = -1;
      int64_t kc = it0 % P.kiters;
      int bs = 0, fs = 0;
      uint32_t bph = 0, fph = 0;
      for (int64_t it = it0; it < it1; ++it) {
        const bool seg_start = (it == it0) || (kc == 0);
        if (seg_start) {
          ++seg;
          if (seg > 0 && !mbar_wait(acc_empty, (uint32_t)((seg - 1) & 1), abort_flag, P.d_info))
            break;
        }
        if (ABF) {
          if (!mbar_wait(&ffull[fs], fph, abort_flag, P.d_info)) break;
        } else {
          if (!mbar_wait(&aready[bs], bph, abort_flag, P.d_info)) break;
        }
        if (!mbar_wait_cluster(&wready[bs], bph, abort_flag, P.d_info)) break;
        tc_fence_after();
        const uint32_t base = smem_u32(bring + bs * BSB);
        const uint32_t fbase = smem_u32(fring + fs * F_BYTES);
#pragma unroll
        for (int kk = 0; kk < OBK / 16; ++kk) {
          const uint64_t bw = sw64_desc(base + 4u * AT_BYTES + 32u * kk);
          const uint32_t acc0 = (seg_start && kk == 0) ? 0u : 1u;
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            const uint32_t d = tmem + ACC_STRIDE * (uint32_t)t;
            if (ABF) {
              mma_ss(d, sw64_desc(fbase + (uint32_t)t * AT_BYTES + 32u * kk), bw, idesc, acc0);
            } else {
              mma_ss(d, sw64_desc(base + (uint32_t)(2 * t) * AT_BYTES + 32u * kk), bw, idesc,
                     acc0);
              mma_ss(d, sw64_desc(base + (uint32_t)(2 * t + 1) * AT_BYTES + 32u * kk), bw, idesc,
                     1u);
            }
          }
        }
        mma_commit(&bdone[bs]);
        if (ABF) mma_commit(&fempty[fs]);
        if (++fs == F_ST) {
          fs = 0;
          fph ^= 1u;
        }
        const bool seg_end = (it + 1 == it1) || (kc + 1 == P.kiters);
        if (seg_end) mma_commit(acc_full);
        if (++kc == P.kiters) kc = 0;
        if (++bs == B_ST) {
          bs = 0;
          bph ^= 1u;
        }
      }
    }
  } else if (warp == 2) {
    // --------------------------------- forwarder ------------------------------
    // reports every completed use of an operand slot to the peer at once
    if (lane == 0) {
      int bs = 0;
      uint32_t bph = 0;
      for (int64_t it = it0; it < it1; ++it) {
        if (!mbar_wait(&bdone[bs], bph, abort_flag, P.d_info)) break;
        mbar_arrive_remote(mapa_peer(smem_u32(&pfree[bs]), peer));
        if (++bs == B_ST) {
          bs = 0;
          bph ^= 1u;
        }
      }
    }
  } else if (warp >= 4 && warp < 4 + NCONV) {
    // ------------------------ converters and epilogue -------------------------
    const int t = (warp - 4) >> 2;
    const int q = warp & 3;
    const int r = 32 * q + lane;
    const int rr = t * OBM + r;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    const uint32_t acc = tmem + ACC_STRIDE * (uint32_t)t;
    int64_t seg = -1;
    int64_t su = it0 / P.kiters, kc = it0 - su * P.kiters;
    const int64_t su0 = su;
    bool whole = false;
    int fs = 0, bs = 0;
    uint32_t fph = 0, bph = 0;
    for (int64_t it = it0; it < it1; ++it) {
      if (it == it0 || kc == 0) {
        ++seg;
        whole = (kc == 0);
      }
      if (!ABF) {
      if (!mbar_wait(&ffull[fs], fph, abort_flag, P.d_info)) break;
      float x[32];
      const unsigned char* row = fring + fs * F_BYTES + rr * 128;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(row + ((c ^ (rr & 7)) << 4));
        x[4 * c] = v.x;
        x[4 * c + 1] = v.y;
        x[4 * c + 2] = v.z;
        x[4 * c + 3] = v.w;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&fempty[fs]);
      uint32_t hi[16], lo[16];
      split_row(x, hi, lo);
      if (!mbar_wait(&bdone[bs], bph ^ 1u, abort_flag, P.d_info)) break;
      const uint32_t ab = smem_u32(bring + bs * BSB + 2 * t * AT_BYTES);
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) {
        const uint32_t o = sw64_off((uint32_t)r, (uint32_t)cc);
        st_shared_v4(ab + o, hi[4 * cc], hi[4 * cc + 1], hi[4 * cc + 2], hi[4 * cc + 3]);
        st_shared_v4(ab + AT_BYTES + o, lo[4 * cc], lo[4 * cc + 1], lo[4 * cc + 2],
                     lo[4 * cc + 3]);
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) mbar_arrive(&aready[bs]);
      }
      const bool seg_end = (it + 1 == it1) || (kc + 1 == P.kiters);
      if (seg_end) {
        if (!mbar_wait(acc_full, (uint32_t)(seg & 1), abort_flag, P.d_info)) break;
        tc_fence_after();
        const int64_t gr = su * 2 * OUNIT + rank * OUNIT + rr;
        if (whole && kc + 1 == P.kiters) {
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + acc + (uint32_t)c0, v);
            tmem_wait_ld();
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
          float* dst =
              P.part + ((int64_t)blockIdx.x * P.maxseg + (su - su0)) * (int64_t)OUNIT * L;
          for (int c0 = 0; c0 < L; c0 += 16) {
            uint32_t v[16];
            tmem_ld16(lane_base + acc + (uint32_t)c0, v);
            tmem_wait_ld();
#pragma unroll
            for (int c = 0; c < 16; ++c)
              dst[(int64_t)(c0 + c) * OUNIT + rr] = __uint_as_float(v[c]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);
      }
      if (++kc == P.kiters) {
        kc = 0;
        ++su;
      }
      if (++fs == F_ST) {
        fs = 0;
        fph ^= 1u;
      }
      if (++bs == B_ST) {
        bs = 0;
        bph ^= 1u;
      }
    }
  } else if (warp >= 12 && warp < 12 + NGEN2) {
    // -------------------- Omega generators (half the K-rows) ------------------
    // two groups of 8 warps take alternate stages, so that one group's wait for
    // its remote stores (the cluster-scope proxy fence) overlaps the other
    // group's generation; one unit = 2 K-consecutive quads
    const int grp = (warp - 12) >> 3;
    const int gt = threadIdx.x - (12 + 8 * grp) * 32;   // 0 .. 255 within the group
    const int nunits = 2 * L;
    int64_t kc = it0 % P.kiters;
    int bs = 0;
    uint32_t bph = 0;
    for (int64_t it = it0; it < it1; ++it) {
      const bool mine = (((it - it0) & 1) == grp);
      if (mine) {
        if (it - it0 >= B_ST) {
          // this slot's previous MMAs done here and, as reported by the peer's
          // forwarder, in the peer
          if (!mbar_wait(&bdone[bs], bph ^ 1u, abort_flag, P.d_info)) break;
          if (!mbar_wait_cluster(&pfree[bs], bph ^ 1u, abort_flag, P.d_info)) break;
        }
        const uint32_t wb = smem_u32(bring + bs * BSB + 4 * AT_BYTES);
        const uint32_t wb_peer = mapa_peer(wb, peer);
        for (int u = gt; u < nunits; u += 8 * 32) {
          const int kk2 = 8 * (int)rank + (u & 7), qd = u >> 3;   // K-rows 2 kk2, 2 kk2 + 1
          uint32_t pk[4] = {0u, 0u, 0u, 0u};
          if (4 * qd < P.lvalid) {
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const int64_t krow = kc * OBK + kk2 * 2 + e;
              float z[4] = {0.f, 0.f, 0.f, 0.f};
              if (krow < P.K) OmegaGen<float>::quad(P.seed, (uint32_t)krow, (uint32_t)(qd + P.qoff), z);
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                const uint32_t b = (4 * qd + c < P.lvalid) ? (__float_as_uint(z[c]) >> 16) : 0u;
                pk[c] |= b << (16 * e);
              }
            }
          }
          // bf16 elements 2 kk2, 2 kk2 + 1 of each column: one 4-byte word of the
          // column's 16-byte chunk kk2 / 4
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const uint32_t o =
                sw64_off((uint32_t)(4 * qd + c), (uint32_t)(kk2 >> 2)) + 4u * (uint32_t)(kk2 & 3);
            st_shared_b32(wb + o, pk[c]);
            st_cluster_b32(wb_peer + o, pk[c]);
          }
        }
        fence_proxy_async();
        asm volatile("fence.proxy.async.shared::cluster;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&wready[bs]);
          mbar_arrive_remote(mapa_peer(smem_u32(&wready[bs]), peer));
        }
      }
      if (++kc == P.kiters) kc = 0;
      if (++bs == B_ST) {
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
                 "r"(TMEM_COLS)
                 : "memory");
  }
  cluster_sync_all();                     // the peer no longer writes into this CTA
}

template <bool ABF>
static cudaError_t launch_omega2_kernel(const CUtensorMap& ma, const TcParams& P, int64_t Gc,
                                        size_t smem, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(tc_omega2_kernel<ABF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tr = trace_begin(RSVD_TRACE_A_OMEGA, s);
  tc_omega2_kernel<ABF><<<(unsigned)(2 * Gc), OTHREADS2, smem, s>>>(ma, P);
  count_launch();
  trace_end(tr, s);
  return cudaGetLastError();
}

static cudaError_t launch_tc_omega2(const TcGemm& g, cudaStream_t s) {
  int64_t sus, kiters, total, Gc;
  int maxseg;
  sk_plan(g.rows, g.K, 2 * OUNIT, OBK, device_sm_count() / 2, &sus, &kiters, &total, &Gc,
          &maxseg);
  TcParams P;
  P.rows = g.rows;
  P.K = g.K;
  P.bm = OUNIT;
  P.L = g.L;
  P.lvalid = g.lvalid;
  P.qoff = g.col0 / 4;
  P.seed = g.seed;
  P.tiles = sus;
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
  P.ustride = 2 * OUNIT;
  P.uoff = 0;
  P.wmul = 2;
  P.wadd = 0;
  CUtensorMap ma;
  memset(&ma, 0, sizeof(ma));
  const bool abf = g.a_bf16 != 0;
  // 256-row stages: fp32 rows of 128 bytes (converted to bf16 hi/lo tiles) or
  // bf16 rows of 64 bytes (read by the MMAs as they land)
  if (!encode_2d(&ma, abf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                 abf ? 2 : 4, g.A, (uint64_t)g.a_cols_total, (uint64_t)g.a_rows_total,
                 (uint64_t)g.lda, OBK, OUNIT,
                 abf ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B))
    return cudaErrorInvalidValue;
  const size_t smem = omega_smem(g.L) + 64;
  cudaError_t e = abf ? launch_omega2_kernel<true>(ma, P, Gc, smem, s)
                      : launch_omega2_kernel<false>(ma, P, Gc, smem, s);
  if (e != cudaSuccess) return e;
  // the two CTAs of a pair form two interleaved stream-K problems (row halves)
  for (int r = 0; r < 2; ++r) {
    TcParams Q = P;
    Q.uoff = r * OUNIT;
    Q.wadd = r;
    e = launch_tc_reduce(Q, (int)Gc, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_tc_omega(const TcGemm& g, cudaStream_t s) {
  if (!tc_supported(g.L) || g.form != 0 || !g.omega) return cudaErrorInvalidValue;
  if (device_sm_count() >= 2) return launch_tc_omega2(g, s);
  if (g.a_bf16) return cudaErrorNotSupported;   // the 1-CTA kernel takes fp32 A only
  int64_t tiles, kiters, total, G;
  int maxseg;
  sk_plan(g.rows, g.K, OUNIT, OBK, device_sm_count(), &tiles, &kiters, &total, &G, &maxseg);
  TcParams P;
  P.rows = g.rows;
  P.K = g.K;
  P.bm = OUNIT;
  P.ustride = OUNIT;
  P.uoff = 0;
  P.wmul = 1;
  P.wadd = 0;
  P.L = g.L;
  P.lvalid = g.lvalid;
  P.qoff = g.col0 / 4;
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
  CUtensorMap ma;
  memset(&ma, 0, sizeof(ma));
  if (!encode_2d(&ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g.A, (uint64_t)g.a_cols_total,
                 (uint64_t)g.a_rows_total, (uint64_t)g.lda, OBK, OUNIT,
                 CU_TENSOR_MAP_SWIZZLE_128B))
    return cudaErrorInvalidValue;
  const size_t smem = omega_smem(g.L);
  cudaError_t e = cudaFuncSetAttribute(tc_omega_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int tr = trace_begin(RSVD_TRACE_A_OMEGA, s);
  tc_omega_kernel<<<(unsigned)G, OTHREADS, smem, s>>>(ma, P);
  count_launch();
  trace_end(tr, s);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_tc_reduce(P, (int)G, s);
}

}  // namespace rsvd
