// Inline-PTX helpers shared by the tcgen05 GEMM kernels: mbarriers with
// bounded waits, TMA tile loads, tensor-memory (TMEM) loads and stores, MMA
// issue and commit, shared-memory matrix descriptors.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "common.cuh"

namespace rsvd {

// Parameters of one persistent stream-K GEMM launch and of its boundary reduce.
struct TcParams {
  int64_t rows, K;
  int bm;          // output rows per stream-K unit (128, or 256 for two M-tiles)
  int L, lvalid;
  uint64_t seed;
  int64_t tiles, kiters, total;
  int maxseg;
  float* part;
  // final outputs: tiles covered by one CTA are written by its epilogue,
  // tiles split between CTAs by tc_reduce_kernel
  float* out;
  int64_t ldo;
  int ncols;
  __nv_bfloat16* out_hi;
  __nv_bfloat16* out_lo;
  int64_t ldt;
  const int* skip;
  int* d_info;
  // unit u covers rows u ustride + uoff .. + bm; stream-K worker c is CTA
  // wmul c + wadd (ustride = bm, uoff = 0, wmul = 1, wadd = 0 for one CTA per worker)
  int64_t ustride;
  int uoff, wmul, wadd;
  int qoff = 0;    // Omega: Philox quad index of the first output column (column / 4)
  // bounded accumulation runs (tc_unit_kernel): when > 0, a TMEM accumulator
  // takes at most `drain` K-chunks; the epilogue then adds it into the CTA's
  // partial tile in fp32 (round to nearest) and the next run starts afresh
  int drain = 0;
};

// Fixed-order sum of the stream-K partials of the tiles split between CTAs
// (k_tc.cu); G = number of CTAs of the GEMM launch.
cudaError_t launch_tc_reduce(const TcParams& P, int G, cudaStream_t s);

// 2-D tensor map (cuTensorMapEncodeTiled through the runtime's driver entry
// point); false when the driver call is unavailable or rejects the layout.
bool encode_2d(CUtensorMap* map, CUtensorMapDataType dt, int elem, const void* base,
               uint64_t inner, uint64_t outer, uint64_t pitch_elems, uint32_t box_inner,
               uint32_t box_outer, CUtensorMapSwizzle sw);

// Stream-K plan: units of bm rows, K in chunks of bk; G CTAs; maxseg = the
// largest number of unit segments one CTA touches.
void sk_plan(int64_t rows, int64_t K, int bm, int bk, int G_hint, int64_t* tiles, int64_t* kiters,
             int64_t* total, int64_t* G, int* maxseg);

namespace tc {

constexpr long long WAIT_LIMIT = 2000000000LL;   // cycles (~1 s)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
// try_wait with a suspend-time hint: the waiting thread sleeps in hardware
// until the phase completes or about 20 us pass, instead of spinning and
// taking issue slots from the working warps.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the CTA aborted or the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                          int* d_info) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*abort_flag) return false;
    if (clock64() - t0 > WAIT_LIMIT) {
      *abort_flag = 1;
      set_info(d_info, RSVD_ERR_TIMEOUT);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// TMA tile load with an L2 cache-eviction policy (createpolicy): streaming
// operands are loaded evict-first, operands re-read by many CTAs evict-last.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tma_load_2d_hint(void* dst, const CUtensorMap* map, uint64_t* bar,
                                                 int x, int y, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      ".L2::cache_hint [%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y), "l"(policy)
      : "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, "
      "%10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
      "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]),
      "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
        "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// D[tmem] (+)= A[tmem] * B[smem desc], kind::f16 (bf16 inputs, fp32 accumulate).
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// D[tmem] (+)= A[smem desc] * B[smem desc], kind::f16 (bf16 in, fp32 accumulate).
__device__ __forceinline__ void mma_ss(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Byte offset of the 16-byte chunk c (0..3) of row r in a K-major tile of
// 64-byte rows with the 64-byte swizzle (8-row groups of 512 bytes): the layout
// TMA writes with CU_TENSOR_MAP_SWIZZLE_64B and sw64_desc describes.
__device__ __forceinline__ uint32_t sw64_off(uint32_t r, uint32_t c) {
  return r * 64u + ((c ^ ((r >> 1) & 3u)) << 4);
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle, 8-row groups of
// 512 bytes (SBO), version 1 (bit 46), layout code 4 in bits 61-63.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                 // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512u >> 4) << 32;        // stride byte offset
  d |= (uint64_t)1u << 46;                 // descriptor version
  d |= (uint64_t)4u << 61;                 // SWIZZLE_64B
  return d;
}
// Instruction descriptor: D f32, A bf16, B bf16, both K-major, N and M.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi_elem), "f"(lo_elem));
  return r;
}

// 32 fp32 values of one A row -> 16 hi words and 16 lo words (2 bf16 each).
__device__ __forceinline__ void split_row(const float (&x)[32], uint32_t (&hi)[16],
                                          uint32_t (&lo)[16]) {
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const float a = x[2 * e], b = x[2 * e + 1];
    const uint32_t h = pack_bf16x2(a, b);
    const float ha = __uint_as_float(h << 16), hb = __uint_as_float(h & 0xFFFF0000u);
    hi[e] = h;
    lo[e] = pack_bf16x2(a - ha, b - hb);
  }
}

}  // namespace tc
}  // namespace rsvd
