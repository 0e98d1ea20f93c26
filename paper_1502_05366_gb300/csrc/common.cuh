// Shared device helpers for the randomized QB / RSVD / ID / CUR kernels.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "rsvd.h"

#define RSVD_CUDA_TRY(expr)                                   \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return RSVD_ERR_CUDA;              \
  } while (0)

#define RSVD_LAUNCH_CHECK()                                   \
  do {                                                        \
    cudaError_t _e = cudaGetLastError();                      \
    if (_e != cudaSuccess) return RSVD_ERR_CUDA;              \
  } while (0)

namespace rsvd {

// Host-side count of kernel launches made by the library (tracing aid), and
// CUDA-event records around selected kernels when tracing is enabled.
void count_launch();
int trace_begin(int cls, cudaStream_t s);
void trace_end(int idx, cudaStream_t s);

// First device-side error wins; later ones are dropped.
__device__ __forceinline__ void set_info(int* d_info, int code) {
  if (d_info) atomicCAS(d_info, 0, code);
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  One round maps counter
// (c0, c1, c2, c3) with key (k0, k1) to
//   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl constants
// 0x9E3779B9, 0xBB67AE85 between rounds.
// ---------------------------------------------------------------------------
struct Words4 {
  uint32_t x0, x1, x2, x3;
};

__device__ __forceinline__ Words4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t p0 = (uint64_t)0xD2511F53u * c0;   // one wide multiply each
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
    const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
    const uint32_t n0 = hi1 ^ c1 ^ k0;
    const uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return Words4{c0, c1, c2, c3};
}

// Counter layout of Omega: (row i, column quad j/4, tag, batch); key = seed.
__device__ __forceinline__ Words4 omega_words(uint64_t seed, uint32_t row, uint32_t quad,
                                              uint32_t tag = 0, uint32_t batch = 0) {
  return philox4x32_10(row, quad, tag, batch, (uint32_t)(seed & 0xffffffffu),
                       (uint32_t)(seed >> 32));
}

// u = (2*(x >> 9) + 1) * 2^-24: odd multiples of 2^-24 in (0, 1), exact in fp32.
// In single precision it is formed without an integer conversion: the float
// with exponent 0 and mantissa x >> 9 is 1 + (x >> 9) 2^-23, and subtracting
// 1 - 2^-24 leaves (2 (x >> 9) + 1) 2^-24, exactly representable, so exact.
__device__ __forceinline__ float word_to_uniform_f(uint32_t x) {
  return __uint_as_float(0x3f800000u | (x >> 9)) - 0x1.fffffep-1f;
}
__device__ __forceinline__ double word_to_uniform_d(uint32_t x) {
  return (double)(2u * (x >> 9) + 1u) * 5.9604644775390625e-8;
}

// Box-Muller (Box & Muller 1958) on the four words: (x0,x1) -> z0, z1 and
// (x2,x3) -> z2, z3.  Single precision with the hardware approximations
// __log2f and __sincosf (the values feed bf16 Omega entries, 8 significant
// bits): r = sqrt(-2 ln u0) (minus2log_f); the angle 2 pi u1 is taken as
// 2 pi (u1 - 1/2) in [-pi, pi), where __sincosf is accurate, and the sign of
// sin and cos flipped back (cos(x + pi) = -cos x, sin(x + pi) = -sin x).
// -2 ln u for u in (0, 1): the Taylor series of ln(1 - v), v = 1 - u (exact in
// fp32 for these u), when v <= 1/8 (truncation below 2^-24 relative), else
// -2 ln 2 log2 u with the hardware log2 (whose absolute error would dominate
// near u = 1).
__device__ __forceinline__ float minus2log_f(float u) {
  const float v = 1.0f - u;
  if (v <= 0.125f) {
    float p = 1.0f / 7.0f;
    p = fmaf(p, v, 1.0f / 6.0f);
    p = fmaf(p, v, 0.2f);
    p = fmaf(p, v, 0.25f);
    p = fmaf(p, v, 1.0f / 3.0f);
    p = fmaf(p, v, 0.5f);
    p = fmaf(p, v, 1.0f);
    return 2.0f * v * p;
  }
  return -1.3862943611198906f * __log2f(u);
}

// sqrt(x) for the Box-Muller radius (x = -2 ln u >= 2^-23 > 0) as x rsqrt(x):
// a few ulp, far below the bf16 rounding that follows.
__device__ __forceinline__ float bm_sqrt(float x) { return x * rsqrtf(x); }

__device__ __forceinline__ void gauss4_f(const Words4& w, float z[4]) {
  const float r0 = bm_sqrt(minus2log_f(word_to_uniform_f(w.x0)));
  const float r1 = bm_sqrt(minus2log_f(word_to_uniform_f(w.x2)));
  float s0, c0, s1, c1;
  __sincosf(6.283185307179586f * (word_to_uniform_f(w.x1) - 0.5f), &s0, &c0);
  __sincosf(6.283185307179586f * (word_to_uniform_f(w.x3) - 0.5f), &s1, &c1);
  z[0] = -r0 * c0;
  z[1] = -r0 * s0;
  z[2] = -r1 * c1;
  z[3] = -r1 * s1;
}

__device__ __forceinline__ void gauss4_d(const Words4& w, double z[4]) {
  const double r0 = sqrt(-2.0 * log(word_to_uniform_d(w.x0)));
  const double r1 = sqrt(-2.0 * log(word_to_uniform_d(w.x2)));
  double s0, c0, s1, c1;
  sincospi(2.0 * word_to_uniform_d(w.x1), &s0, &c0);
  sincospi(2.0 * word_to_uniform_d(w.x3), &s1, &c1);
  z[0] = r0 * c0;
  z[1] = r0 * s0;
  z[2] = r1 * c1;
  z[3] = r1 * s1;
}

// fp32 -> bf16 (nearest even) -> fp32.
__device__ __forceinline__ float round_bf16(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

// Omega entries for the quad (row, quad) in the arithmetic type T:
// double for FP64 inputs, bf16-rounded float for FP32 inputs.
template <typename T>
struct OmegaGen;

template <>
struct OmegaGen<float> {
  __device__ __forceinline__ static void quad(uint64_t seed, uint32_t row, uint32_t quad,
                                              float z[4], uint32_t tag = 0) {
    gauss4_f(omega_words(seed, row, quad, tag), z);
#pragma unroll
    for (int t = 0; t < 4; ++t) z[t] = round_bf16(z[t]);
  }
};

template <>
struct OmegaGen<double> {
  __device__ __forceinline__ static void quad(uint64_t seed, uint32_t row, uint32_t quad,
                                              double z[4], uint32_t tag = 0) {
    gauss4_d(omega_words(seed, row, quad, tag), z);
  }
};

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__host__ __device__ __forceinline__ int64_t ceil_div(int64_t a, int64_t b) {
  return (a + b - 1) / b;
}
__host__ __device__ __forceinline__ int64_t round_up(int64_t a, int64_t b) {
  return ceil_div(a, b) * b;
}

}  // namespace rsvd
