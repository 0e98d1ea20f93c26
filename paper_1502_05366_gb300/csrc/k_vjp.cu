// Element-wise kernels of the reverse-mode derivative of Alg. 5 (the small
// l x l steps of the adjoint; the products with A and the tall products run on
// the GEMM kernels of the forward path).
//
// For X = Q R (thin QR, diag(R) > 0, Q^* Q = I) the cotangent of X given
// those of Q and R follows from dX = dQ R + Q dR with Q^* dQ skew and dR upper
// triangular:  g_X = (g_Q + Q sym(M)) R^{-*},  M = g_R R^* - Q^* g_Q,  where
// sym(M) keeps the upper triangle of M and mirrors its strictly upper part
// below the diagonal (sym_upper below).
//
// For the square SVD R = Uh diag(s) Vh^* with distinct s, writing
// dC = Uh^* dR Vh: ds = diag(dC) and, off the diagonal, (Uh^* dUh)_ij =
// F_ij (s_j dC_ij + s_i dC_ji), (Vh^* dVh)_ij = F_ij (s_i dC_ij + s_j dC_ji)
// with F_ij = 1 / (s_j^2 - s_i^2).  Collecting the coefficients of dC gives
// g_R = Uh X Vh^*,  X = diag(g_s) + (F o (Gu - Gu^*)) diag(s)
//                        + diag(s) (F o (Gv - Gv^*)),  Gu = Uh^* g_Uh,
// Gv = Vh^* g_Vh (svd_vjp_core below builds X).
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
inline unsigned grid_for(int64_t work) {
  int64_t b = ceil_div(work, 256);
  if (b > 65535LL * 8) b = 65535LL * 8;
  if (b < 1) b = 1;
  return (unsigned)b;
}
}  // namespace

// X (L x L, ld ldx): the l x l core of the square-SVD rule, zero padding.
// F_ij is formed as 1 / ((s_j - s_i)(s_j + s_i)) in double; equal singular
// values (F undefined) contribute nothing.
template <typename T>
__global__ void svd_vjp_core_kernel(int l, int L, int k, const double* __restrict__ s,
                                    const double* __restrict__ gs, const T* __restrict__ Gu,
                                    const T* __restrict__ Gv, int64_t ldg, T* __restrict__ X,
                                    int64_t ldx) {
  const int64_t total = (int64_t)L * L;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / L), j = (int)(t - (int64_t)(t / L) * L);
    double x = 0.0;
    if (i < l && j < l) {
      if (i == j) {
        x = (gs && i < k) ? gs[i] : 0.0;
      } else {
        const double si = s[i], sj = s[j];
        const double d = (sj - si) * (sj + si);
        if (d != 0.0) {
          const double f = 1.0 / d;
          const double du = (double)Gu[i * ldg + j] - (double)Gu[j * ldg + i];
          const double dv = (double)Gv[i * ldg + j] - (double)Gv[j * ldg + i];
          x = f * (du * sj + si * dv);
        }
      }
    }
    X[i * ldx + j] = (T)x;
  }
}

template <typename T>
cudaError_t launch_svd_vjp_core(int l, int L, int k, const double* s, const double* gs,
                                const T* Gu, const T* Gv, int64_t ldg, T* X, int64_t ldx,
                                cudaStream_t st) {
  svd_vjp_core_kernel<T><<<grid_for((int64_t)L * L), 256, 0, st>>>(l, L, k, s, gs, Gu, Gv, ldg,
                                                                    X, ldx);
  count_launch();
  return cudaGetLastError();
}

// out (L x L) = sym(P1 - P2) on the leading l x l block (P1 may be null),
// zero padding: out_ij = M_ij for i <= j, M_ji for i > j.
template <typename T>
__global__ void sym_upper_kernel(int l, int L, const T* __restrict__ P1,
                                 const T* __restrict__ P2, int64_t ldp, T* __restrict__ out,
                                 int64_t ldo) {
  const int64_t total = (int64_t)L * L;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / L), j = (int)(t - (int64_t)(t / L) * L);
    T v = T(0);
    if (i < l && j < l) {
      const int a = i <= j ? i : j, b = i <= j ? j : i;
      v = -P2[a * ldp + b];
      if (P1) v += P1[a * ldp + b];
    }
    out[i * ldo + j] = v;
  }
}

template <typename T>
cudaError_t launch_sym_upper(int l, int L, const T* P1, const T* P2, int64_t ldp, T* out,
                             int64_t ldo, cudaStream_t st) {
  sym_upper_kernel<T><<<grid_for((int64_t)L * L), 256, 0, st>>>(l, L, P1, P2, ldp, out, ldo);
  count_launch();
  return cudaGetLastError();
}

// dst(:, 0:cols) = scale * src(:, 0:cols), with the columns j whose sign
// entry is negative (signs may be null) negated once more.
template <typename T>
__global__ void pack_cols_kernel(int64_t rows, int cols, const T* __restrict__ src, int64_t lds,
                                 T* __restrict__ dst, int64_t ldd, T scale,
                                 const int* __restrict__ signs) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols;
    const int j = (int)(t - i * cols);
    T v = scale * src[i * lds + j];
    if (signs && signs[j] < 0) v = -v;
    dst[i * ldd + j] = v;
  }
}

template <typename T>
cudaError_t launch_pack_cols(int64_t rows, int cols, const T* src, int64_t lds, T* dst,
                             int64_t ldd, T scale, const int* signs, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  pack_cols_kernel<T><<<grid_for(rows * cols), 256, 0, st>>>(rows, cols, src, lds, dst, ldd,
                                                              scale, signs);
  count_launch();
  return cudaGetLastError();
}

template cudaError_t launch_svd_vjp_core<float>(int, int, int, const double*, const double*,
                                                const float*, const float*, int64_t, float*,
                                                int64_t, cudaStream_t);
template cudaError_t launch_svd_vjp_core<double>(int, int, int, const double*, const double*,
                                                 const double*, const double*, int64_t, double*,
                                                 int64_t, cudaStream_t);
template cudaError_t launch_sym_upper<float>(int, int, const float*, const float*, int64_t,
                                             float*, int64_t, cudaStream_t);
template cudaError_t launch_sym_upper<double>(int, int, const double*, const double*, int64_t,
                                              double*, int64_t, cudaStream_t);
template cudaError_t launch_pack_cols<float>(int64_t, int, const float*, int64_t, float*,
                                             int64_t, float, const int*, cudaStream_t);
template cudaError_t launch_pack_cols<double>(int64_t, int, const double*, int64_t, double*,
                                              int64_t, double, const int*, cudaStream_t);

}  // namespace rsvd
