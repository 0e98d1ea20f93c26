// FP8 E4M3 with power-of-two block scales (the sketch of RSVD_PREC_FP8).
//
// A block of 32 values along the contraction gets the scale 2^k,
// k = ceil(log2(amax / 448)), 448 the largest finite E4M3 value; each value
// x / 2^k is rounded to the nearest E4M3 value (ties to the even code,
// saturating at 448) and multiplied by 2^k again.  With amax = f 2^e,
// f in [0.5, 1) (frexpf), amax / 448 = (f / 0.875) 2^(e - 9), so k = e - 8
// when f > 0.875 and k = e - 9 otherwise: the scale is exact, and so is the
// dequantised value (at most four significant bits), which bf16 holds exactly.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

namespace rsvd {

__device__ __forceinline__ int e4m3_block_exp(float amax) {
  if (!(amax > 0.f)) return 0;
  int e;
  const float f = frexpf(amax, &e);
  return f > 0.875f ? e - 8 : e - 9;
}

// x / 2^k to E4M3 and back, times 2^k (a pair; both entries of the block).
__device__ __forceinline__ float2 e4m3_deq2(float a, float b, float inv, float sc) {
  const __nv_fp8x2_storage_t q =
      __nv_cvt_float2_to_fp8x2(make_float2(a * inv, b * inv), __NV_SATFINITE, __NV_E4M3);
  const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2(q, __NV_E4M3);
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&h));
  return make_float2(f.x * sc, f.y * sc);
}

// The 32 values of a block, quantised, as 16 words of two bf16 each (exact).
__device__ __forceinline__ void e4m3_block_bf16(const float (&x)[32], uint32_t (&w)[16]) {
  float amax = 0.f;
#pragma unroll
  for (int i = 0; i < 32; ++i) amax = fmaxf(amax, fabsf(x[i]));
  const int k = e4m3_block_exp(amax);
  const float inv = ldexpf(1.f, -k), sc = ldexpf(1.f, k);
#pragma unroll
  for (int e = 0; e < 16; ++e) {
    const float2 d = e4m3_deq2(x[2 * e], x[2 * e + 1], inv, sc);
    const __nv_bfloat162 p = __floats2bfloat162_rn(d.x, d.y);
    w[e] = *reinterpret_cast<const uint32_t*>(&p);
  }
}

}  // namespace rsvd
