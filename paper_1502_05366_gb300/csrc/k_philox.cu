// Materialisation of Omega and of its Philox words (checking aids: the sketch
// kernels generate the same values in-register and never store them), and of
// the left test matrix Omega~ (tag 1, Sec. 3.5), stored transposed (m x l) as
// the right-hand operand of the left sketch A^T Omega~^T.
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

template <typename T>
__global__ void omega_kernel(int64_t n, int l, uint64_t seed, T* __restrict__ Om, int64_t ldo,
                             uint32_t tag) {
  const int nq = (l + 3) / 4;
  const int64_t total = n * (int64_t)nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / nq;
    const int q = (int)(t - i * nq);
    T z[4];
    OmegaGen<T>::quad(seed, (uint32_t)i, (uint32_t)q, z, tag);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = 4 * q + c;
      if (j < l) Om[i * ldo + j] = z[c];
    }
  }
}

__global__ void omega_words_kernel(int64_t n, int l, uint64_t seed, uint32_t* __restrict__ out) {
  const int nq = (l + 3) / 4;
  const int64_t total = n * (int64_t)nq;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / nq;
    const int q = (int)(t - i * nq);
    const Words4 w = omega_words(seed, (uint32_t)i, (uint32_t)q);
    uint4 v = make_uint4(w.x0, w.x1, w.x2, w.x3);
    reinterpret_cast<uint4*>(out)[t] = v;
  }
}

static int grid_for(int64_t work, int threads) {
  int64_t b = ceil_div(work, threads);
  if (b > 65535LL * 8) b = 65535LL * 8;
  if (b < 1) b = 1;
  return (int)b;
}

template <typename T>
cudaError_t launch_omega(int64_t n, int l, uint64_t seed, T* Om, int64_t ldo, cudaStream_t s,
                         uint32_t tag) {
  const int64_t work = n * ((l + 3) / 4);
  omega_kernel<T><<<grid_for(work, 256), 256, 0, s>>>(n, l, seed, Om, ldo, tag);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_omega_words(int64_t n, int l, uint64_t seed, uint32_t* out, cudaStream_t s) {
  const int64_t work = n * ((l + 3) / 4);
  omega_words_kernel<<<grid_for(work, 256), 256, 0, s>>>(n, l, seed, out);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_omega<float>(int64_t, int, uint64_t, float*, int64_t, cudaStream_t,
                                         uint32_t);
template cudaError_t launch_omega<double>(int64_t, int, uint64_t, double*, int64_t, cudaStream_t,
                                          uint32_t);

}  // namespace rsvd
