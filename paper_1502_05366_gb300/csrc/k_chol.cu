// Cholesky factor and inverse of the l x l Gram matrix for CholeskyQR.
//
// orth(X) (Sec. 2.1: an unpivoted QR whose Q is unique by diag(R) > 0) is
// computed as Q = X R^{-1} with G = X^T X = R^T R, repeated two or three times
// (CholeskyQR2/3).  A pass whose Gram has a pivot below tau * max(diag G),
// tau = 4 l eps, is redone with a diagonal shift (shifted CholeskyQR, Fukaya et
// al. 2020), the shift growing tenfold per retry; any shifted pass, or a second
// pass whose Gram is far from I, requests the third pass.  One CTA of 1024
// threads holds the matrix in shared memory (global memory beyond the limit).
#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int CT = 256;   // threads (a 255-register budget keeps the unrolled panel code in registers)
constexpr size_t SMEM_LIMIT = 212 * 1024;   // dynamic part; static arrays take <= 9 KB
template <typename T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ float eps_of<float>() { return 5.9604645e-8f; }
template <> __device__ __forceinline__ double eps_of<double>() { return 1.1102230246251565e-16; }
}  // namespace

// Global fallback when l x l does not fit in shared memory: the matrix plus a
// 32 x l block-row buffer for the blocked inverse.
size_t chol_scratch_bytes(int l, int elem) {
  const size_t b = (size_t)l * l * elem;
  return b <= SMEM_LIMIT ? 0 : b + (size_t)32 * l * elem;
}

template <typename T>
__device__ void block_max(T v, T* red, T* out) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nw = (blockDim.x * blockDim.y) / 32;
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  if (tid < 32) {
    T w = tid < nw ? red[tid] : T(0);
    for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
    if (tid == 0) *out = w;
  }
  __syncthreads();
}

template <typename T>
__device__ void write_identity_outputs(const CholArgs& a) {
  const int L = a.L;
  for (int i = threadIdx.y; i < L; i += blockDim.y)
  for (int c = threadIdx.x; c < L; c += blockDim.x) {
    const int t = i * L + c;
    const T v = (i == c) ? T(1) : T(0);
    if (a.R) ((T*)a.R)[t] = v;
    if (a.Rinv) ((T*)a.Rinv)[t] = v;
    if (a.Whi) {
      ((__nv_bfloat16*)a.Whi)[t] = __float2bfloat16_rn((float)v);
      ((__nv_bfloat16*)a.Wlo)[t] = __float2bfloat16_rn(0.0f);
      ((__nv_bfloat16*)a.Wlo2)[t] = __float2bfloat16_rn(0.0f);
    }
  }
}

// ---------------------------------------------------------------------------
// Blocked right-looking Cholesky G = R^T R on the l x l row-major matrix S
// (upper triangle used, R left there), panels of NB = 32 columns:
//   (a) the diagonal block is factored by warp 0 in registers (lane c holds
//       column c of the block; row j of R is shared by shuffles);
//   (b) the panel row block becomes R_pp^{-T} S_panel (one thread per column);
//   (c) the trailing upper triangle is updated with 4 x 4 register tiles.
// A pivot not above thr stops the factorization and records its column.
// ---------------------------------------------------------------------------
constexpr int NB = 32;

template <typename T>
__device__ void chol_blocked(T* S, int l, T thr, int* s_fail) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nthr = blockDim.x * blockDim.y;
  for (int p0 = 0; p0 < l; p0 += NB) {
    const int pb = min(NB, l - p0);
    if (warp == 0) {
      T d[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i)
        d[i] = (lane < pb && i <= lane) ? S[(p0 + i) * l + p0 + lane] : T(0);
      int failed = -1;
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) {
        if (jj < pb && failed < 0) {
          const T piv = __shfl_sync(0xffffffffu, d[jj], jj);
          if (!(piv > thr)) {
            failed = jj;
          } else {
            const T r = sqrt(piv);
            T rj = d[jj];
            if (lane == jj) rj = r;
            else if (lane > jj) rj = rj / r;
            d[jj] = rj;
#pragma unroll
            for (int i = jj + 1; i < NB; ++i) {
              const T ri = __shfl_sync(0xffffffffu, rj, i);
              if (lane >= i) d[i] -= ri * rj;
            }
          }
        }
      }
      if (failed < 0) {
#pragma unroll
        for (int i = 0; i < NB; ++i)
          if (lane < pb && i <= lane) S[(p0 + i) * l + p0 + lane] = d[i];
      } else if (lane == 0) {
        *s_fail = p0 + failed;
      }
    }
    __syncthreads();
    if (*s_fail >= 0) return;
    const int c0 = p0 + pb, nt = l - c0;
    if (nt <= 0) return;
    // (b) X = R_pp^{-T} S(p0:p0+pb, c0:l), forward substitution per column
    for (int c = c0 + tid; c < l; c += nthr) {
      T x[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i < pb) {
          T acc = S[(p0 + i) * l + c];
#pragma unroll
          for (int t = 0; t < i; ++t) acc -= S[(p0 + t) * l + p0 + i] * x[t];
          x[i] = acc / S[(p0 + i) * l + p0 + i];
        } else {
          x[i] = T(0);
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < pb) S[(p0 + i) * l + c] = x[i];
    }
    __syncthreads();
    // (c) trailing update of the upper triangle: S(i, c) -= sum_t X(t, i) X(t, c)
    const int nT = (nt + 3) / 4;
    for (int tt = tid; tt < nT * nT; tt += nthr) {
      const int ti = tt / nT, tc = tt - ti * nT;
      if (tc < ti) continue;
      const int i0 = c0 + 4 * ti, k0 = c0 + 4 * tc;
      T acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = T(0);
      for (int t = 0; t < pb; ++t) {
        const T* row = S + (p0 + t) * l;
        T xi[4], xc[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          xi[q] = (i0 + q < l) ? row[i0 + q] : T(0);
          xc[q] = (k0 + q < l) ? row[k0 + q] : T(0);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] = fma(xi[q], xc[w], acc[q][w]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int i = i0 + q, c = k0 + w;
          if (i < l && c < l && c >= i) S[i * l + c] -= acc[q][w];
        }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// In-place inverse of the upper-triangular R held in the upper triangle of S
// (l x l row-major), by block rows from the bottom:
//   T = E_I - R(I, I+1:) X(I+1:, :)   (E_I: rows of the identity)
//   X(I, :) = R_II^{-1} T             (back substitution, one thread per column)
// R_II is copied aside first since X(I, :) overwrites row block I.
// ---------------------------------------------------------------------------
template <typename T>
__device__ void inv_upper_blocked(T* S, int l, T* ttmp) {
  __shared__ T Rd[NB][NB + 1];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
  const int nb = (l + NB - 1) / NB;
  constexpr int MAXE = 32;   // ne <= 32 l <= MAXE * 256 threads for l <= 256
  for (int Ib = nb - 1; Ib >= 0; --Ib) {
    const int r0 = Ib * NB, rb = min(NB, l - r0);
    const int ncol = l - r0;
    const int ne = rb * ncol;
    for (int t = tid; t < NB * NB; t += nthr) {
      const int i = t / NB, c = t - i * NB;
      Rd[i][c] = (i < rb && c < rb && c >= i) ? S[(r0 + i) * l + r0 + c] : T(0);
    }
    if (ttmp) {   // large l: T through the global buffer
      for (int e = tid; e < ne; e += nthr) {
        const int i = r0 + e / ncol, c = r0 + e % ncol;
        T acc = (i == c) ? T(1) : T(0);
        for (int t = r0 + rb; t <= c; ++t) acc -= S[i * l + t] * S[t * l + c];
        ttmp[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < ne; e += nthr) S[(r0 + e / ncol) * l + r0 + e % ncol] = ttmp[e];
    } else {      // T into registers (at most MAXE elements per thread)
      T tv[MAXE];
#pragma unroll
      for (int u = 0; u < MAXE; ++u) {
        const int e = tid + u * nthr;
        tv[u] = T(0);
        if (e < ne) {
          const int i = r0 + e / ncol, c = r0 + e % ncol;
          T acc = (i == c) ? T(1) : T(0);
          for (int t = r0 + rb; t <= c; ++t) acc -= S[i * l + t] * S[t * l + c];
          tv[u] = acc;
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < MAXE; ++u) {
        const int e = tid + u * nthr;
        if (e < ne) S[(r0 + e / ncol) * l + r0 + e % ncol] = tv[u];
      }
    }
    __syncthreads();
    // X(I, c) = R_II^{-1} T(:, c)
    for (int c = r0 + tid; c < l; c += nthr) {
      T x[NB];
#pragma unroll
      for (int i = NB - 1; i >= 0; --i) {
        if (i < rb) {
          T acc = S[(r0 + i) * l + c];
#pragma unroll
          for (int t = i + 1; t < NB; ++t)
            if (t < rb) acc -= Rd[i][t] * x[t];
          x[i] = acc / Rd[i][i];
        } else {
          x[i] = T(0);
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < rb) S[(r0 + i) * l + c] = x[i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// fp32 variants on a padded shared-memory matrix (leading dimension ld, a
// multiple of 4 with ld % 32 == 4, zero padding), so that 4-wide rows load as
// one conflict-free float4 and every FMA-heavy phase runs on 4 x 4 register
// tiles spread over all threads.
// ---------------------------------------------------------------------------
__host__ __device__ inline int chol_ld(int l) {
  int ld = (l + 3) & ~3;
  while ((ld & 31) != 4) ld += 4;
  return ld;
}

// Upper-triangle tile (ti, tc), tc >= ti, of linear index u in row-major order
// over an nT x nT tile grid.
__device__ __forceinline__ void tri_tile(int u, int nT, int* ti, int* tc) {
  const float b = 2.0f * nT + 1.0f;
  int r = (int)((b - sqrtf(b * b - 8.0f * (float)u)) * 0.5f);
  if (r < 0) r = 0;
  if (r > nT - 1) r = nT - 1;
  while (r > 0 && r * nT - (r * (r - 1)) / 2 > u) --r;
  while (r + 1 < nT && (r + 1) * nT - ((r + 1) * r) / 2 <= u) ++r;
  *ti = r;
  *tc = r + (u - (r * nT - (r * (r - 1)) / 2));
}

// s_dinv (l floats, shared) receives 1 / R_ii for the solves.
__device__ void chol_tiled(float* S, int l, int ld, float thr, int* s_fail, float* s_dinv) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nthr = blockDim.x * blockDim.y;
  for (int p0 = 0; p0 < l; p0 += NB) {
    const int pb = min(NB, l - p0);
    if (warp == 0) {   // (a) diagonal block in registers (lane c holds column c)
      float d[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i)
        d[i] = (lane < pb && i <= lane) ? S[(p0 + i) * ld + p0 + lane] : 0.f;
      int failed = -1;
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) {
        if (jj < pb && failed < 0) {
          const float piv = __shfl_sync(0xffffffffu, d[jj], jj);
          if (!(piv > thr)) {
            failed = jj;
          } else {
            // one rsqrt on the pivot chain: R_jj = piv rsqrt(piv), R_jc = S_jc rsqrt(piv)
            const float rinv = rsqrtf(piv);
            float rj = d[jj];
            if (lane == jj) rj = piv * rinv;
            else if (lane > jj) rj = rj * rinv;
            d[jj] = rj;
            if (lane == jj) s_dinv[p0 + jj] = rinv;
#pragma unroll
            for (int i = jj + 1; i < NB; ++i) {
              const float ri = __shfl_sync(0xffffffffu, rj, i);
              if (lane >= i) d[i] -= ri * rj;
            }
          }
        }
      }
      if (failed < 0) {
#pragma unroll
        for (int i = 0; i < NB; ++i)
          if (lane < pb && i <= lane) S[(p0 + i) * ld + p0 + lane] = d[i];
      } else if (lane == 0) {
        *s_fail = p0 + failed;
      }
    }
    __syncthreads();
    if (*s_fail >= 0) return;
    const int c0 = p0 + pb, nt = l - c0;
    if (nt <= 0) return;
    // (b) X = R_pp^{-T} S(p0:p0+pb, c0:l), forward substitution per column
    for (int c = c0 + tid; c < l; c += nthr) {
      float x[NB];
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        if (i < pb) {
          float acc = S[(p0 + i) * ld + c];
#pragma unroll
          for (int t = 0; t < i; ++t) acc -= S[(p0 + t) * ld + p0 + i] * x[t];
          x[i] = acc * s_dinv[p0 + i];
        } else {
          x[i] = 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < pb) S[(p0 + i) * ld + c] = x[i];
    }
    __syncthreads();
    // (c) trailing upper triangle S(i, c) -= sum_t X(t, i) X(t, c), 4 x 4 tiles
    // over the upper-triangular tile grid only, float4 row loads
    const int nT = (nt + 3) / 4;
    const int ntiles = nT * (nT + 1) / 2;
    for (int u = tid; u < ntiles; u += nthr) {
      int ti, tc;
      tri_tile(u, nT, &ti, &tc);
      const int i0 = c0 + 4 * ti, k0 = c0 + 4 * tc;
      float acc[4][4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) acc[q][w] = 0.f;
#pragma unroll 4
      for (int t = 0; t < pb; ++t) {
        const float* row = S + (p0 + t) * ld;
        const float4 xi = *reinterpret_cast<const float4*>(row + i0);
        const float4 xc = *reinterpret_cast<const float4*>(row + k0);
        const float a4[4] = {xi.x, xi.y, xi.z, xi.w};
        const float b4[4] = {xc.x, xc.y, xc.z, xc.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] = fmaf(a4[q], b4[w], acc[q][w]);
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int i = i0 + q, c = k0 + w;
          if (i < l && c < l && c >= i) S[i * ld + c] -= acc[q][w];
        }
    }
    __syncthreads();
  }
}

// In-place inverse of the upper-triangular R in S (padded ld), block rows
// from the bottom:  T = E_I - R(I, I+1:) X(I+1:, :) with the product on 4 x 4
// register tiles (K range clipped to the tile's columns, X upper triangular),
// then X(I, :) = R_II^{-1} T by back substitution per column.
__device__ void inv_upper_tiled(float* S, int l, int ld, const float* s_dinv) {
  __shared__ float Rd[NB][NB + 1];
  const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
  // the strictly lower triangle holds Gram entries: zero it (X is upper triangular)
  for (int e = tid; e < l * l; e += nthr) {
    const int i = e / l, c = e - i * l;
    if (c < i) S[i * ld + c] = 0.f;
  }
  __syncthreads();
  const int nb = (l + NB - 1) / NB;
  for (int Ib = nb - 1; Ib >= 0; --Ib) {
    const int r0 = Ib * NB, rb = min(NB, l - r0);
    const int cs = r0 + rb;                 // first column of the off-diagonal part
    for (int t = tid; t < NB * NB; t += nthr) {
      const int i = t / NB, c = t - i * NB;
      Rd[i][c] = (i < rb && c < rb && c >= i) ? S[(r0 + i) * ld + r0 + c] : 0.f;
    }
    // T(i, c) = -sum_{t = cs}^{c} R(i, t) X(t, c) for c >= cs, in registers
    // (at most two 4 x 4 tiles per thread: 8 x ceil((l - cs) / 4) <= 2 nthr)
    const int nTc = (l - cs + 3) / 4;
    const int ntiles = (NB / 4) * nTc;
    float acc[2][4][4];
    int i0s[2], k0s[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int u = tid + h * nthr;
      i0s[h] = -1;
      k0s[h] = 0;
      if (u < ntiles) {
        const int ti = u / nTc, tc = u - ti * nTc;
        const int i0 = r0 + 4 * ti, k0 = cs + 4 * tc;
        i0s[h] = i0;
        k0s[h] = k0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[h][q][w] = 0.f;
        const int tmax = min(l, k0 + 4);
#pragma unroll 2
        for (int t = cs; t < tmax; ++t) {
          float a4[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) a4[q] = (i0 + q < r0 + rb) ? S[(i0 + q) * ld + t] : 0.f;
          const float4 xc = *reinterpret_cast<const float4*>(S + t * ld + k0);
          const float b4[4] = {xc.x, xc.y, xc.z, xc.w};
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[h][q][w] = fmaf(a4[q], b4[w], acc[h][q][w]);
        }
      }
    }
    __syncthreads();                          // R(I, I+1:) read by everyone before T lands
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (i0s[h] >= 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int i = i0s[h] + q, c = k0s[h] + w;
            if (i < r0 + rb && c < l) S[i * ld + c] = -acc[h][q][w];
          }
      }
    }
    // the diagonal block of T is the identity
    for (int t = tid; t < rb * rb; t += nthr) {
      const int i = t / rb, c = t - i * rb;
      S[(r0 + i) * ld + r0 + c] = (i == c) ? 1.f : 0.f;
    }
    __syncthreads();
    // X(I, c) = R_II^{-1} T(:, c)
    for (int c = r0 + tid; c < l; c += nthr) {
      float x[NB];
#pragma unroll
      for (int i = NB - 1; i >= 0; --i) {
        if (i < rb) {
          float acc2 = S[(r0 + i) * ld + c];
#pragma unroll
          for (int t = i + 1; t < NB; ++t)
            if (t < rb) acc2 -= Rd[i][t] * x[t];
          x[i] = acc2 * s_dinv[r0 + i];
        } else {
          x[i] = 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < NB; ++i)
        if (i < rb) S[(r0 + i) * ld + c] = x[i];
    }
    __syncthreads();
  }
}

// The body of chol_kernel for a matrix S of leading dimension ld; the shared-
// memory instance receives S derived from the kernel's shared array, so that
// after inlining every access to it compiles as a shared-memory access (a
// generic pointer that might alias global memory would serialise the loads).
template <typename T>
__device__ __forceinline__ void chol_body(const CholArgs& a, T* S, int ld, T* red, T& s_maxdiag,
                                          T& s_dev, int& s_fail, float* s_dinv) {
  const int l = a.l, L = a.L;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int tx = threadIdx.x, ty = threadIdx.y, nty = blockDim.y;
  const T* G = (const T*)a.G;
  const int64_t ldg = a.ldg;

  if (a.skip_idx >= 0 && a.flags && a.flags[a.skip_idx] == 1) {  // pass not needed: R = I
    write_identity_outputs<T>(a);
    return;
  }

  // scale of G and, on the second pass, its distance to I
  T md = T(0), dev = T(0);
  bool bad = false;
  for (int i = ty; i < l; i += nty)
    for (int c = tx; c < l; c += 32) {
      const T g = G[(int64_t)i * ldg + c];
      if (!isfinite(g)) bad = true;
      if (i == c) md = max(md, g);
      dev = max(dev, abs(g - (i == c ? T(1) : T(0))));
    }
  if (bad) set_info(a.d_info, RSVD_ERR_NUMERIC);
  block_max<T>(md, red, &s_maxdiag);
  block_max<T>(dev, red, &s_dev);
  const T maxdiag = s_maxdiag;
  if (!(maxdiag > T(0))) {                       // X = 0 or non-finite: no basis
    set_info(a.d_info, RSVD_ERR_NOT_SPD);
    write_identity_outputs<T>(a);
    return;
  }
  const T tau = T(4) * T(l) * eps_of<T>();
  T shift = T(0);
  int used_shift = 0;
  int fail = -1;
  for (int attempt = 0; attempt < 12; ++attempt) {
    for (int i = ty; i < l; i += nty)
      for (int c = tx; c < ld; c += 32)
        S[i * ld + c] = c < l ? G[(int64_t)i * ldg + c] + ((i == c) ? shift : T(0)) : T(0);
    if (tid == 0) s_fail = -1;
    __syncthreads();
    if (sizeof(T) == 4 && a.sld > 0)
      chol_tiled((float*)S, l, ld, (float)(tau * maxdiag), &s_fail, s_dinv);
    else
      chol_blocked<T>(S, l, tau * maxdiag, &s_fail);
    fail = s_fail;
    __syncthreads();
    if (fail < 0) break;
    shift = (shift == T(0)) ? tau * maxdiag : shift * T(10);
    used_shift = 1;
  }
  if (fail >= 0) {
    set_info(a.d_info, RSVD_ERR_NOT_SPD);
    write_identity_outputs<T>(a);
    return;
  }
  if (tid == 0 && a.flags) {
    if (a.pass == 1) {
      a.flags[1] = used_shift;
      // conditional second pass (inside the power scheme): only after a shift;
      // the third pass is skipped unless the second one asks for it
      a.flags[3] = used_shift ? 0 : 1;
      a.flags[2] = 1;
    } else if (a.pass == 2) {
      a.flags[1] |= used_shift;
      a.flags[0] = (a.flags[1] || T(l) * s_dev > T(0.5)) ? 1 : 0;
      a.flags[2] = 1 - a.flags[0];   // skip flag of the third pass
    }
  }
  // R out (identity on the padding)
  if (a.R) {
    T* R = (T*)a.R;
    for (int i = ty; i < L; i += nty)
      for (int c = tx; c < L; c += 32) {
        T v;
        if (i < l && c < l) v = (c >= i) ? S[i * ld + c] : T(0);
        else v = (i == c) ? T(1) : T(0);
        R[i * L + c] = v;
      }
  }
  if (sizeof(T) == 4 && a.sld > 0)
    inv_upper_tiled((float*)S, l, ld, s_dinv);
  else
    inv_upper_blocked<T>(S, l, a.scratch ? (T*)a.scratch + (size_t)l * l : nullptr);
  if (a.Rinv) {
    T* Ri = (T*)a.Rinv;
    for (int i = ty; i < L; i += nty)
      for (int c = tx; c < L; c += 32) {
        T v;
        if (i < l && c < l) v = (c >= i) ? S[i * ld + c] : T(0);
        else v = (i == c) ? T(1) : T(0);
        Ri[i * L + c] = v;
      }
  }
  if (a.Whi) {  // W^T with W = R^{-1}: Wt[j][kk] = Rinv[kk][j], three bf16 terms (24 bits)
    __nv_bfloat16* hi = (__nv_bfloat16*)a.Whi;
    __nv_bfloat16* lo = (__nv_bfloat16*)a.Wlo;
    __nv_bfloat16* lo2 = (__nv_bfloat16*)a.Wlo2;
    for (int j = ty; j < L; j += nty)
    for (int kk = tx; kk < L; kk += 32) {
      const int t = j * L + kk;
      float v;
      if (j < l && kk < l) v = (j >= kk) ? (float)S[kk * ld + j] : 0.0f;
      else v = (j == kk) ? 1.0f : 0.0f;
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      const float r1 = v - __bfloat162float(h);
      const __nv_bfloat16 mdl = __float2bfloat16_rn(r1);
      hi[t] = h;
      lo[t] = mdl;
      lo2[t] = __float2bfloat16_rn(r1 - __bfloat162float(mdl));
    }
  }
}

// S in shared memory (l x ld) ...
template <typename T>
__global__ void __launch_bounds__(CT) chol_kernel(CholArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ T red[32];
  __shared__ T s_maxdiag, s_dev;
  __shared__ int s_fail;
  __shared__ float s_dinv[256];   // 1 / R_ii of the fp32 tiled path (l <= 256 there)
  chol_body<T>(a, reinterpret_cast<T*>(dsm), a.sld > 0 ? a.sld : a.l, red, s_maxdiag, s_dev,
               s_fail, s_dinv);
}
// ... or in the global scratch (large l)
template <typename T>
__global__ void __launch_bounds__(CT) chol_kernel_global(CholArgs a) {
  __shared__ T red[32];
  __shared__ T s_maxdiag, s_dev;
  __shared__ int s_fail;
  chol_body<T>(a, (T*)a.scratch, a.l, red, s_maxdiag, s_dev, s_fail, nullptr);
}

// Racc <- R * Racc for upper-triangular L x L matrices (through tmp).
template <typename T>
__global__ void trmm_upper_kernel(int L, const T* __restrict__ R, const T* __restrict__ Racc,
                                  T* __restrict__ tmp) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < L * L; t += gridDim.x * blockDim.x) {
    const int i = t / L, c = t - i * L;
    T s = T(0);
    if (c >= i)
      for (int q = i; q <= c; ++q) s += R[i * L + q] * Racc[q * L + c];
    tmp[t] = s;
  }
}

template <typename T>
cudaError_t launch_chol(const CholArgs& a, cudaStream_t s) {
  const size_t bytes = (size_t)a.l * a.l * sizeof(T);
  CholArgs b = a;
  b.sld = 0;
  size_t dyn = 0;
  const size_t tiled = (size_t)a.l * chol_ld(a.l) * sizeof(float);
  if (sizeof(T) == 4 && tiled <= SMEM_LIMIT) {   // fp32 register-tiled path
    b.scratch = nullptr;
    b.sld = chol_ld(a.l);
    dyn = tiled;
  } else if (bytes <= SMEM_LIMIT) {
    b.scratch = nullptr;
    dyn = bytes;
  } else if (a.scratch == nullptr) {
    return cudaErrorInvalidValue;
  }
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(chol_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  const int tr_ = trace_begin(RSVD_TRACE_CHOL, s);
  if (b.scratch)
    chol_kernel_global<T><<<1, dim3(32, CT / 32), 0, s>>>(b);
  else
    chol_kernel<T><<<1, dim3(32, CT / 32), dyn, s>>>(b);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_trmm_upper(int L, const T* R, T* Racc, T* tmp, cudaStream_t s) {
  const int blocks = (L * L + 255) / 256;
  trmm_upper_kernel<T><<<blocks, 256, 0, s>>>(L, R, Racc, tmp);
  count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemcpyAsync(Racc, tmp, sizeof(T) * L * L, cudaMemcpyDeviceToDevice, s);
}

template cudaError_t launch_chol<float>(const CholArgs&, cudaStream_t);
template cudaError_t launch_chol<double>(const CholArgs&, cudaStream_t);
template cudaError_t launch_trmm_upper<float>(int, const float*, float*, float*, cudaStream_t);
template cudaError_t launch_trmm_upper<double>(int, const double*, double*, double*,
                                               cudaStream_t);

}  // namespace rsvd
