// Small data-movement kernels: copies, transposes, the bf16 split of tensor-core
// operands, the sign rule of the SVD output, and the gathers of ID/CUR.
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

static unsigned grid1d(int64_t work, int threads = 256, int64_t cap = 16384) {
  int64_t b = ceil_div(work, threads);
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (unsigned)b;
}

template <typename TI, typename TO>
__global__ void copy2d_kernel(int64_t rows, int64_t cols, const TI* __restrict__ in,
                              int64_t ldi, TO* __restrict__ out, int64_t ldo) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols, j = t - i * cols;
    out[i * ldo + j] = (TO)in[i * ldi + j];
  }
}

template <typename TI, typename TO>
cudaError_t launch_copy2d(int64_t rows, int64_t cols, const TI* in, int64_t ldi, TO* out,
                          int64_t ldo, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  copy2d_kernel<TI, TO><<<grid1d(rows * cols), 256, 0, s>>>(rows, cols, in, ldi, out, ldo);
  count_launch();
  return cudaGetLastError();
}

// out (cols x rows) = in^T, through 32 x 32 shared tiles.
template <typename TI, typename TO>
__global__ void transpose_kernel(int64_t rows, int64_t cols, const TI* __restrict__ in,
                                 int64_t ldi, TO* __restrict__ out, int64_t ldo) {
  __shared__ TO tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t r = r0 + dy, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[dy][threadIdx.x] = (TO)in[r * ldi + c];
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t c = c0 + dy, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * ldo + r] = tile[threadIdx.x][dy];
  }
}

template <typename TI, typename TO>
cudaError_t launch_transpose(int64_t rows, int64_t cols, const TI* in, int64_t ldi, TO* out,
                             int64_t ldo, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(cols, 32), (unsigned)ceil_div(rows, 32));
  if (grid.y > 65535u) return cudaErrorInvalidConfiguration;
  transpose_kernel<TI, TO><<<grid, dim3(32, 8), 0, s>>>(rows, cols, in, ldi, out, ldo);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void fill_kernel(int64_t rows, int64_t cols, T* __restrict__ out, int64_t ldo,
                            T value) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols, j = t - i * cols;
    out[i * ldo + j] = value;
  }
}

template <typename T>
cudaError_t launch_fill(int64_t rows, int64_t cols, T* out, int64_t ldo, T value,
                        cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  fill_kernel<T><<<grid1d(rows * cols), 256, 0, s>>>(rows, cols, out, ldo, value);
  count_launch();
  return cudaGetLastError();
}

// X (rows x L, fp32) -> hi = bf16(X^T), lo = bf16(X^T - hi): two L x rows bf16
// arrays (ld ldt).  hi + lo carries 16 significant bits of each entry.
__global__ void split_transpose_kernel(int64_t rows, int cols, int L, const float* __restrict__ X,
                                       int64_t ldx, __nv_bfloat16* __restrict__ hi,
                                       __nv_bfloat16* __restrict__ lo, int64_t ldt) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int64_t r = r0 + dy;
    const int c = c0 + threadIdx.x;
    tile[dy][threadIdx.x] = (r < rows && c < cols) ? X[r * ldx + c] : 0.0f;
  }
  __syncthreads();
  for (int dy = threadIdx.y; dy < 32; dy += blockDim.y) {
    const int c = c0 + dy;
    const int64_t r = r0 + threadIdx.x;
    if (r < rows && c < L) {
      const float x = tile[threadIdx.x][dy];
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      hi[(int64_t)c * ldt + r] = h;
      lo[(int64_t)c * ldt + r] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
  }
}

cudaError_t launch_split_transpose(int64_t rows, int cols, int L, const float* X, int64_t ldx,
                                   void* hi, void* lo, int64_t ldt, cudaStream_t s) {
  if (rows <= 0 || L <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(L, 32));
  split_transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(rows, cols, L, X, ldx,
                                                      (__nv_bfloat16*)hi, (__nv_bfloat16*)lo,
                                                      ldt);
  count_launch();
  return cudaGetLastError();
}

// One block per column j of V: the entry of largest magnitude (lowest row on
// ties) decides the sign; then the column pair (U(:,j), V(:,j)) is scaled.
template <typename T>
__global__ void sign_find_kernel(int64_t n, const T* __restrict__ V, int64_t ldv,
                                 int* __restrict__ signs) {
  const int j = blockIdx.x;
  T best = T(-1);
  int64_t bi = 0x7fffffffffffffffLL;
  T bv = T(0);
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const T v = V[i * ldv + j];
    const T a = v < T(0) ? -v : v;
    if (a > best || (a == best && i < bi)) {
      best = a;
      bi = i;
      bv = v;
    }
  }
  __shared__ T sbest[256];
  __shared__ int64_t sidx[256];
  __shared__ T sval[256];
  sbest[threadIdx.x] = best;
  sidx[threadIdx.x] = bi;
  sval[threadIdx.x] = bv;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const T b2 = sbest[threadIdx.x + o];
      const int64_t i2 = sidx[threadIdx.x + o];
      if (b2 > sbest[threadIdx.x] || (b2 == sbest[threadIdx.x] && i2 < sidx[threadIdx.x])) {
        sbest[threadIdx.x] = b2;
        sidx[threadIdx.x] = i2;
        sval[threadIdx.x] = sval[threadIdx.x + o];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) signs[j] = (sval[0] < T(0)) ? -1 : 1;
}

template <typename T>
__global__ void sign_apply_kernel(int64_t rows, int k, T* __restrict__ X, int64_t ldx,
                                  const int* __restrict__ signs) {
  const int64_t total = rows * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    if (signs[j] < 0) X[i * ldx + j] = -X[i * ldx + j];
  }
}

template <typename T>
cudaError_t launch_sign_fix(int64_t m, int64_t n, int k, T* U, int64_t ldu, T* V, int64_t ldv,
                            int* signs, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  sign_find_kernel<T><<<k, 256, 0, s>>>(n, V, ldv, signs);
  count_launch();
  sign_apply_kernel<T><<<grid1d(m * k), 256, 0, s>>>(m, k, U, ldu, signs);
  count_launch();
  sign_apply_kernel<T><<<grid1d(n * k), 256, 0, s>>>(n, k, V, ldv, signs);
  count_launch();
  return cudaGetLastError();
}

// W (k x m doubles, row-major) = C^T with C = A(:, J[0:k]): W[i*m + r] = A[r, J[i]].
template <typename T>
__global__ void gather_ct_kernel(int64_t m, int k, const T* __restrict__ A, int64_t lda,
                                 const int32_t* __restrict__ J, double* __restrict__ W) {
  const int64_t total = m * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / m);
    const int64_t r = t - (int64_t)i * m;
    W[t] = (double)A[r * lda + J[i]];
  }
}

template <typename T>
cudaError_t launch_gather_ct(int64_t m, int k, const T* A, int64_t lda, const int32_t* J,
                             double* W, cudaStream_t s) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  gather_ct_kernel<T><<<grid1d(m * k), 256, 0, s>>>(m, k, A, lda, J, W);
  count_launch();
  return cudaGetLastError();
}

// Double-float planes of W = C^T (k x m), column-major (column r of C^T is
// row r of C): Wh[r*k + i] = A[r, J[i]], Wl = 0.
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename S>
__global__ void gather_ct_df_kernel(int64_t m, int k, const S* __restrict__ A, int64_t lda,
                                    const int32_t* __restrict__ J, float* __restrict__ Wh,
                                    float* __restrict__ Wl) {
  const int64_t total = m * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / k;
    const int i = (int)(t - r * k);
    Wh[t] = to_f32(A[r * lda + J[i]]);
    Wl[t] = 0.0f;
  }
}

cudaError_t launch_gather_ct_df(int64_t m, int k, const void* A, int64_t lda, int a_bf16,
                                const int32_t* J, double* W, cudaStream_t s) {
  if (m <= 0 || k <= 0) return cudaSuccess;
  float* Wh = reinterpret_cast<float*>(W);
  if (a_bf16)
    gather_ct_df_kernel<__nv_bfloat16><<<grid1d(m * k), 256, 0, s>>>(
        m, k, reinterpret_cast<const __nv_bfloat16*>(A), lda, J, Wh, Wh + m * k);
  else
    gather_ct_df_kernel<float><<<grid1d(m * k), 256, 0, s>>>(m, k, (const float*)A, lda, J, Wh,
                                                             Wh + m * k);
  count_launch();
  return cudaGetLastError();
}

template <typename T>
__global__ void gather_rows_kernel(int k, int64_t n, const T* __restrict__ A, int64_t lda,
                                   const int32_t* __restrict__ I, T* __restrict__ R,
                                   int64_t ldr) {
  const int64_t total = (int64_t)k * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n);
    const int64_t c = t - (int64_t)i * n;
    R[(int64_t)i * ldr + c] = A[(int64_t)I[i] * lda + c];
  }
}

template <typename T>
cudaError_t launch_gather_rows(int k, int64_t n, const T* A, int64_t lda, const int32_t* I,
                               T* R, int64_t ldr, cudaStream_t s) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  gather_rows_kernel<T><<<grid1d((int64_t)k * n), 256, 0, s>>>(k, n, A, lda, I, R, ldr);
  count_launch();
  return cudaGetLastError();
}

// R (k x n, fp32) = rows I of a bf16 A.
__global__ void gather_rows_bf16_kernel(int k, int64_t n, const __nv_bfloat16* __restrict__ A,
                                        int64_t lda, const int32_t* __restrict__ I,
                                        float* __restrict__ R, int64_t ldr) {
  const int64_t total = (int64_t)k * n;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / n);
    const int64_t c = t - (int64_t)i * n;
    R[(int64_t)i * ldr + c] = __bfloat162float(A[(int64_t)I[i] * lda + c]);
  }
}

cudaError_t launch_gather_rows_bf16(int k, int64_t n, const void* A, int64_t lda,
                                    const int32_t* I, float* R, int64_t ldr, cudaStream_t s) {
  if (k <= 0 || n <= 0) return cudaSuccess;
  gather_rows_bf16_kernel<<<grid1d((int64_t)k * n), 256, 0, s>>>(
      k, n, reinterpret_cast<const __nv_bfloat16*>(A), lda, I, R, ldr);
  count_launch();
  return cudaGetLastError();
}

// out[c, :] = X[idx[c], :] for c < count (rows of width cols).
template <typename T>
__global__ void gather_rows_perm_kernel(int64_t count, int cols, const T* __restrict__ X,
                                        int64_t ldx, const int32_t* __restrict__ idx,
                                        T* __restrict__ out, int64_t ldo) {
  const int64_t total = count * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = t / cols;
    const int j = (int)(t - c * cols);
    out[c * ldo + j] = X[(int64_t)idx[c] * ldx + j];
  }
}

template <typename T>
cudaError_t launch_gather_rows_by_perm(int64_t count, int cols, const T* X, int64_t ldx,
                                       const int32_t* idx, T* out, int64_t ldo,
                                       cudaStream_t s) {
  if (count <= 0 || cols <= 0) return cudaSuccess;
  gather_rows_perm_kernel<T><<<grid1d(count * cols), 256, 0, s>>>(count, cols, X, ldx, idx,
                                                                 out, ldo);
  count_launch();
  return cudaGetLastError();
}

// W (n x l doubles, column c of B = row c of Bt, contiguous) from Bt.
template <typename T>
cudaError_t launch_bt_to_w64(int64_t n, int l, const T* Bt, int64_t ldbt, double* W,
                             cudaStream_t s) {
  return launch_copy2d<T, double>(n, l, Bt, ldbt, W, l, s);
}

template <typename T>
__global__ void add_inplace_kernel(int64_t rows, int64_t cols, const T* __restrict__ X,
                                   int64_t ldx, T* __restrict__ Y, int64_t ldy) {
  const int64_t total = rows * cols;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / cols, j = t - i * cols;
    Y[i * ldy + j] += X[i * ldx + j];
  }
}

template <typename T>
cudaError_t launch_add_inplace(int64_t rows, int64_t cols, const T* X, int64_t ldx, T* Y,
                               int64_t ldy, cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  add_inplace_kernel<T><<<grid1d(rows * cols), 256, 0, s>>>(rows, cols, X, ldx, Y, ldy);
  count_launch();
  return cudaGetLastError();
}

// Copy used when the third CholeskyQR pass is skipped: runs only if *flag == 1.
template <typename T>
__global__ void cond_copy_kernel(const int* flag, const int* veto, int64_t count,
                                 const T* __restrict__ in, T* __restrict__ out) {
  if (*flag != 1 || (veto && *veto == 1)) return;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = in[t];
}

template <typename T>
cudaError_t launch_cond_copy(const int* flag, const int* veto, int64_t count, const T* in,
                             T* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  cond_copy_kernel<T><<<grid1d(count), 256, 0, s>>>(flag, veto, count, in, out);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_cond_copy<float>(const int*, const int*, int64_t, const float*,
                                             float*, cudaStream_t);

// Columns j < k of X (rows x k) scaled by 1/S[j] (S double; 0 stays 0).
template <typename T>
__global__ void scale_cols_kernel(int64_t rows, int k, T* __restrict__ X, int64_t ldx,
                                  const double* __restrict__ S) {
  const int64_t total = rows * k;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / k;
    const int j = (int)(t - i * k);
    const double sj = S[j];
    X[i * ldx + j] = sj > 0.0 ? (T)((double)X[i * ldx + j] / sj) : T(0);
  }
}

template <typename T>
cudaError_t launch_scale_cols(int64_t rows, int k, T* X, int64_t ldx, const double* S,
                              cudaStream_t s) {
  if (rows <= 0 || k <= 0) return cudaSuccess;
  scale_cols_kernel<T><<<grid1d(rows * k), 256, 0, s>>>(rows, k, X, ldx, S);
  count_launch();
  return cudaGetLastError();
}
template cudaError_t launch_scale_cols<float>(int64_t, int, float*, int64_t, const double*,
                                              cudaStream_t);
template cudaError_t launch_scale_cols<double>(int64_t, int, double*, int64_t, const double*,
                                               cudaStream_t);

__global__ void copy_i32_kernel(int64_t count, const int32_t* __restrict__ in,
                                int32_t* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x)
    out[t] = in[t];
}

cudaError_t launch_copy_i32(int64_t count, const int32_t* in, int32_t* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  copy_i32_kernel<<<grid1d(count), 256, 0, s>>>(count, in, out);
  count_launch();
  return cudaGetLastError();
}

__global__ void check_finite_kernel(int64_t count, const double* __restrict__ x, int* d_info) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
       t += (int64_t)gridDim.x * blockDim.x) {
    if (!isfinite(x[t])) set_info(d_info, RSVD_ERR_NUMERIC);
  }
}

cudaError_t launch_check_finite_d(int64_t count, const double* x, int* d_info,
                                  cudaStream_t s) {
  if (count <= 0 || !d_info) return cudaSuccess;
  check_finite_kernel<<<grid1d(count), 256, 0, s>>>(count, x, d_info);
  count_launch();
  return cudaGetLastError();
}

#define INST2(TI, TO)                                                                        \
  template cudaError_t launch_copy2d<TI, TO>(int64_t, int64_t, const TI*, int64_t, TO*,      \
                                             int64_t, cudaStream_t);                         \
  template cudaError_t launch_transpose<TI, TO>(int64_t, int64_t, const TI*, int64_t, TO*,   \
                                                int64_t, cudaStream_t);
INST2(float, float)
INST2(double, double)
INST2(float, double)
INST2(double, float)
#undef INST2

#define INST1(T)                                                                             \
  template cudaError_t launch_fill<T>(int64_t, int64_t, T*, int64_t, T, cudaStream_t);       \
  template cudaError_t launch_sign_fix<T>(int64_t, int64_t, int, T*, int64_t, T*, int64_t,   \
                                          int*, cudaStream_t);                               \
  template cudaError_t launch_gather_ct<T>(int64_t, int, const T*, int64_t, const int32_t*,  \
                                           double*, cudaStream_t);                           \
  template cudaError_t launch_gather_rows<T>(int, int64_t, const T*, int64_t,                \
                                             const int32_t*, T*, int64_t, cudaStream_t);     \
  template cudaError_t launch_gather_rows_by_perm<T>(int64_t, int, const T*, int64_t,        \
                                                     const int32_t*, T*, int64_t,            \
                                                     cudaStream_t);                          \
  template cudaError_t launch_bt_to_w64<T>(int64_t, int, const T*, int64_t, double*,         \
                                           cudaStream_t);                                    \
  template cudaError_t launch_add_inplace<T>(int64_t, int64_t, const T*, int64_t, T*,        \
                                             int64_t, cudaStream_t);
INST1(float)
INST1(double)
#undef INST1
template cudaError_t launch_fill<int>(int64_t, int64_t, int*, int64_t, int, cudaStream_t);

}  // namespace rsvd
