// Omega of the FP8 sketch (RSVD_PREC_FP8): the bf16 Gaussians of the Philox
// stream (as the FP32 path draws them), quantised to E4M3 with one
// power-of-two scale per block of 32 rows of each column (fp8.cuh), written
// either transposed as bf16 (the stored operand of the tensor-core sketch:
// row j of the output is column j of Omega; rows l .. L - 1 zero) or, for
// checking, as n x l floats.
#include "common.cuh"
#include "fp8.cuh"
#include "kernels.h"

namespace rsvd {

// One thread: columns 4 q .. 4 q + 3 over the 32-row block kb.
template <bool TRANS>
__global__ void __launch_bounds__(256) omega_fp8_kernel(int64_t n, int l, int L, uint64_t seed,
                                                        void* out, int64_t ld) {
  const int64_t nq = L / 4;
  const int64_t nb = (n + 31) / 32;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nq * nb) return;
  const int q = (int)(t % nq);
  const int64_t kb = t / nq;
  const int64_t k0 = kb * 32;
  const int kr = (int)min((int64_t)32, n - k0);
  float v[4][32];
#pragma unroll
  for (int r = 0; r < 32; ++r) {
    float z[4] = {0.f, 0.f, 0.f, 0.f};
    if (r < kr && 4 * q < l) OmegaGen<float>::quad(seed, (uint32_t)(k0 + r), (uint32_t)q, z);
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c][r] = (4 * q + c < l) ? z[c] : 0.f;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const int j = 4 * q + c;
    uint32_t w[16];
    e4m3_block_bf16(v[c], w);
    if (TRANS) {
      uint16_t* o = reinterpret_cast<uint16_t*>(out) + (int64_t)j * ld + k0;
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        if (2 * e < kr) o[2 * e] = (uint16_t)(w[e] & 0xffffu);
        if (2 * e + 1 < kr) o[2 * e + 1] = (uint16_t)(w[e] >> 16);
      }
    } else if (j < l) {
      float* o = reinterpret_cast<float*>(out);
#pragma unroll
      for (int e = 0; e < 16; ++e) {
        if (2 * e < kr) o[(k0 + 2 * e) * ld + j] = __uint_as_float(w[e] << 16);
        if (2 * e + 1 < kr) o[(k0 + 2 * e + 1) * ld + j] = __uint_as_float(w[e] & 0xffff0000u);
      }
    }
  }
}

cudaError_t launch_omega_fp8_t(int64_t n, int l, int L, uint64_t seed, uint16_t* out, int64_t ldt,
                               cudaStream_t s) {
  if (n < 1 || l < 1 || L % 4 != 0 || L < l) return cudaErrorInvalidValue;
  const int64_t total = (int64_t)(L / 4) * ((n + 31) / 32);
  omega_fp8_kernel<true><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(n, l, L, seed, out, ldt);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_omega_fp8(int64_t n, int l, uint64_t seed, float* out, int64_t ldo,
                             cudaStream_t s) {
  if (n < 1 || l < 1) return cudaErrorInvalidValue;
  const int L = (l + 3) & ~3;
  const int64_t total = (int64_t)(L / 4) * ((n + 31) / 32);
  omega_fp8_kernel<false><<<(unsigned)ceil_div(total, 256), 256, 0, s>>>(n, l, L, seed, out, ldo);
  count_launch();
  return cudaGetLastError();
}

}  // namespace rsvd
