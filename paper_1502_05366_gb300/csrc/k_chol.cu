// Cholesky factor and inverse of the l x l Gram matrix for CholeskyQR.
//
// orth(X) (Sec. 2.1: an unpivoted QR whose Q is unique by diag(R) > 0) is
// computed as Q = X R^{-1} with G = X^T X = R^T R, repeated two or three times
// (CholeskyQR2/3).  A pass whose Gram has a pivot below tau * max(diag G),
// tau = 4 l eps, is redone with a diagonal shift (shifted CholeskyQR, Fukaya et
// al. 2020), the shift growing tenfold per retry; any shifted pass, or a second
// pass whose Gram is far from I, requests the third pass.  fp32 up to l = 224:
// one CTA of 384 threads on register tiles with the matrix in shared memory;
// fp32 beyond: a cooperative grid of 32 x 32 block tasks (chol_coop_kernel);
// fp64: one CTA of 256 threads (global memory beyond the shared-memory limit).
#include <algorithm>

#include "common.cuh"
#include "kernels.h"

namespace rsvd {

namespace {
constexpr int CT = 256;   // threads of the generic kernel (a 255-register budget keeps its unrolled panel code in registers)
constexpr size_t SMEM_LIMIT = 212 * 1024;   // dynamic part; static arrays take <= 9 KB
template <typename T> __device__ __forceinline__ T eps_of();
template <> __device__ __forceinline__ float eps_of<float>() { return 5.9604645e-8f; }
template <> __device__ __forceinline__ double eps_of<double>() { return 1.1102230246251565e-16; }
}  // namespace

// Global fallback when l x l does not fit in shared memory: the matrix plus a
// 32 x l block-row buffer for the blocked inverse.
size_t chol_coop_scratch_bytes(int l);
size_t chol_scratch_bytes(int l, int elem) {
  const size_t b = (size_t)l * l * elem;
  const size_t g = b <= SMEM_LIMIT ? 0 : b + (size_t)32 * l * elem;
  // fp32: the cooperative kernel's header, padded matrix and inverse
  if (elem == 4) return std::max(g, chol_coop_scratch_bytes(l));
  return g;
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

// Pass bookkeeping in a.flags after a successful factorization.  ldev is
// l * max |G - I| of this pass's Gram.
__device__ void chol_update_flags(const CholArgs& a, int used_shift, double ldev) {
  if (!a.flags) return;
  if (a.pass == 1) {
    a.flags[1] = used_shift;
    // conditional second pass (inside the power scheme): only after a shift;
    // the third pass is skipped unless the second one asks for it
    a.flags[3] = used_shift ? 0 : 1;
    a.flags[2] = 1;
  } else if (a.pass == 2) {
    a.flags[1] |= used_shift;
    a.flags[0] = (a.flags[1] || ldev > 0.5) ? 1 : 0;
    a.flags[2] = 1 - a.flags[0];   // skip flag of the third pass
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

// ---------------------------------------------------------------------------
// fp32 path for l <= 224: one CTA of 384 threads with the whole matrix in
// shared memory (leading dimension chf_ld(l), a multiple of 8 so that every
// 8-column group is one aligned pair of float4; zero padding columns).
//
// Factor (right-looking, panels of NB = 32 columns):
//   (a) warp 0 factors the diagonal block R_pp and forms its inverse D_p
//       (both in registers, one column per lane; the rows of R_pp and of D_p
//       are broadcast through shared memory);
//   (b) the panel row block becomes D_p^T S_panel (4 x 4 register tiles);
//   (c) the next diagonal block is updated by the worker warps and handed to
//       warp 0, which factors it while the workers update the rest of the
//       trailing upper triangle with 8 x 8 register tiles (lookahead).
// Inverse X = R^{-1}, block rows from the bottom:
//   T = -R(I, I+1:) X(I+1:, :)
//   X(I, I+1:) = D_I T,  X(I, I) = D_I   (4 x 4 register tiles).
// D_p is kept, transposed, in the strictly lower triangle of the diagonal
// block (1 / R_ii in s_dinv); no phase reads the lower triangle otherwise.
// ---------------------------------------------------------------------------
constexpr int CHF_T = 384;     // threads: one register tile each in every phase
constexpr int CHF_LMAX = 224;  // (b) and the inverse need 8 * ceil((l - 32) / 4) <= CHF_T
constexpr int CHF_DLD = 36;   // row stride of the current panel's D_p copy

__host__ __device__ inline int chf_ld(int l) {
  int ld = (l + 7) & ~7;
  while ((ld & 31) != 8) ld += 8;
  return ld;
}
inline size_t chf_smem(int l) {
  return (size_t)l * chf_ld(l) * sizeof(float) + (size_t)NB * CHF_DLD * sizeof(float);
}

__device__ __forceinline__ float4 lds4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}

// G (+ shift on the diagonal) into S; on the first load also the largest
// diagonal entry, the largest |G - I| entry and whether G is finite.
__device__ void chf_load(const CholArgs& a, float* S, int ld, float shift, float* md, float* dev,
                         bool* bad) {
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int l = a.l;
  const float* G = (const float*)a.G;
  const int64_t ldg = a.ldg;
  const int nq = ld / 4;
  const bool vec = (ldg % 4 == 0) && ((reinterpret_cast<uintptr_t>(G) & 15) == 0) &&
                   ldg >= ((l + 3) & ~3);
  const int ne = l * nq;
  if (vec) {
    // every 16-byte piece of G in flight at once (cp.async, zero-filled past
    // column l), then the scan and the shift in shared memory
    for (int e = tid; e < ne; e += nthr) {
      const int i = e / nq, c = 4 * (e - (e / nq) * nq);
      const int nbytes = c < l ? min(16, 4 * (l - c)) : 0;
      const float* g = G + (int64_t)i * ldg + (c < l ? c : 0);
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(S + i * ld + c);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(g), "r"(nbytes)
                   : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (md) {
      for (int e = tid; e < ne; e += nthr) {
        const int i = e / nq, c = 4 * (e - (e / nq) * nq);
        if (c >= l) continue;
        const float4 v = lds4(S + i * ld + c);
        const float w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int cc = c + w;
          if (cc < l) {
            if (!isfinite(w4[w])) *bad = true;
            if (cc == i) *md = fmaxf(*md, w4[w]);
            *dev = fmaxf(*dev, fabsf(w4[w] - (cc == i ? 1.f : 0.f)));
          }
        }
      }
    }
    if (shift != 0.f)
      for (int i = tid; i < l; i += nthr) S[i * ld + i] += shift;
    return;
  }
  for (int e0 = tid; e0 < ne; e0 += 8 * nthr) {
    float4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nthr;
      v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (e < ne) {
        const int i = e / nq, c = 4 * (e - (e / nq) * nq);
        if (c < l) {
          const float* g = G + (int64_t)i * ldg + c;
          if (vec) {
            v[u] = *reinterpret_cast<const float4*>(g);
          } else {
            v[u].x = g[0];
            if (c + 1 < l) v[u].y = g[1];
            if (c + 2 < l) v[u].z = g[2];
            if (c + 3 < l) v[u].w = g[3];
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * nthr;
      if (e < ne) {
        const int i = e / nq, c = 4 * (e - (e / nq) * nq);
        float w4[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          const int cc = c + w;
          if (cc >= l) {
            w4[w] = 0.f;
          } else {
            if (md) {
              if (!isfinite(w4[w])) *bad = true;
              if (cc == i) *md = fmaxf(*md, w4[w]);
              *dev = fmaxf(*dev, fabsf(w4[w] - (cc == i ? 1.f : 0.f)));
            }
            if (cc == i) w4[w] += shift;
          }
        }
        *reinterpret_cast<float4*>(S + i * ld + c) = make_float4(w4[0], w4[1], w4[2], w4[3]);
      }
    }
  }
}

// (a) by warp 0: R_pp in place (upper triangle, zeros below), D_p = R_pp^{-1}
// into Dc (row-major, zeros below the diagonal) and transposed into the
// strictly lower triangle of the block, 1 / R_ii into s_dinv.  Returns the
// failing column (relative to p0) or -1.
//
// Lane i owns row i of the block, unscaled: after step j the row holds
// S_i. - sum_{t <= j} R_ti R_t. / ... in the form  e_i = R_ii * (row i of R),
// so that step j needs only the raw pivot row e_j and rinv_j = 1 / sqrt(piv_j):
// R_ji R_jc = (e_ji rinv_j^2) e_jc.  Every row is scaled by its own rinv at the
// end.  The per-step chain is: pivot shuffle, rsqrt, two multiplies, the
// downdate of the next pivot; the exchange of the raw pivot row through shared
// memory overlaps the rsqrt.  The step loop is rolled with static register
// indices.
__device__ int chf_diag(float* S, int ld, int p0, int pb, float thr, float* Dc, float* s_dinv,
                        float* rowbuf) {
  const int lane = threadIdx.x & 31;
  float e[NB];
  const float* myrow = S + (p0 + lane) * ld + p0;
#pragma unroll
  for (int c4 = 0; c4 < NB / 4; ++c4) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < pb && 4 * c4 < pb) v = lds4(myrow + 4 * c4);
    e[4 * c4] = v.x; e[4 * c4 + 1] = v.y; e[4 * c4 + 2] = v.z; e[4 * c4 + 3] = v.w;
  }
  // columns beyond pb read as padding zeros or as the next rows: clear them
#pragma unroll
  for (int c = 0; c < NB; ++c) e[c] = (c < pb) ? e[c] : 0.f;
  float diag = lane < pb ? myrow[lane] : 1.f;
  float myrinv = 0.f;
  for (int jj = 0; jj < pb; ++jj) {
    float* rb = rowbuf + (jj & 1) * NB;
    if (lane == jj) {
#pragma unroll
      for (int c4 = 0; c4 < NB / 4; ++c4)
        *reinterpret_cast<float4*>(rb + 4 * c4) =
            make_float4(e[4 * c4], e[4 * c4 + 1], e[4 * c4 + 2], e[4 * c4 + 3]);
    }
    const float piv = __shfl_sync(0xffffffffu, diag, jj);
    if (!(piv > thr)) return jj;
    const float rinv = rsqrtf(piv);
    if (lane == jj) {
      myrinv = rinv;
      s_dinv[p0 + jj] = rinv;
    }
    __syncwarp();
    const float eji = rb[lane];
    const float coef = eji * (rinv * rinv);   // R_ji / R_jj^... : R_ji R_jc = coef e_jc
    if (lane > jj) {
      diag = fmaf(-coef, eji, diag);
#pragma unroll
      for (int c4 = 0; c4 < NB / 4; ++c4) {
        const float4 r4 = lds4(rb + 4 * c4);
        e[4 * c4] = fmaf(-coef, r4.x, e[4 * c4]);
        e[4 * c4 + 1] = fmaf(-coef, r4.y, e[4 * c4 + 1]);
        e[4 * c4 + 2] = fmaf(-coef, r4.z, e[4 * c4 + 2]);
        e[4 * c4 + 3] = fmaf(-coef, r4.w, e[4 * c4 + 3]);
      }
    }
  }
  // row i of R = rinv_i e_i on and above the diagonal, zeros below
  if (lane < pb) {
#pragma unroll
    for (int c4 = 0; c4 < NB / 4; ++c4) {
      if (4 * c4 < pb) {
        float w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) w[u] = (4 * c4 + u >= lane) ? e[4 * c4 + u] * myrinv : 0.f;
        *reinterpret_cast<float4*>(S + (p0 + lane) * ld + p0 + 4 * c4) =
            make_float4(w[0], w[1], w[2], w[3]);
      }
    }
  }
  __syncwarp();
  // D_p: lane c solves R_pp x = e_c from the bottom (x_t = 0 for t > c),
  // unrolled (a rolled loop with a run-time trip count measured 3x slower);
  // the term of x_{i+1}, the last one known, is added last
  float x[NB];
#pragma unroll
  for (int i = NB - 1; i >= 0; --i) {
    x[i] = 0.f;
    if (i < pb) {
      const float* row = S + (p0 + i) * ld + p0;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      float last = 0.f;
#pragma unroll
      for (int i4 = (i + 1) / 4; i4 < NB / 4; ++i4) {
        if (4 * i4 < pb) {
          const float4 r4 = lds4(row + 4 * i4);
          const float rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int t = 4 * i4 + w;
            if (t == i + 1) last = rr[w];
            else if (t > i + 1) acc[w] = fmaf(rr[w], x[t], acc[w]);
          }
        }
      }
      float sum = (acc[0] + acc[1]) + (acc[2] + acc[3]);
      if (i + 1 < NB) sum = fmaf(last, x[i + 1 < NB ? i + 1 : 0], sum);
      x[i] = ((lane == i ? 1.f : 0.f) - sum) * s_dinv[p0 + i];
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    Dc[i * CHF_DLD + lane] = x[i];
    if (i < lane && lane < pb) S[(p0 + lane) * ld + p0 + i] = x[i];
  }
  return -1;
}

// Full factorization; returns the failing column or -1 (uniform over the CTA).
// Lookahead: while other warps apply panel p's update to the trailing matrix,
// warp 0 applies it to the next diagonal block and factors that block.
__device__ int chf_factor(float* S, int l, int ld, float thr, float* Dc, float* s_dinv,
                          float* rowbuf, int* s_fail) {
  const int tid = threadIdx.x, warp = tid >> 5, nthr = blockDim.x;
  if (warp == 0) {
    const int f = chf_diag(S, ld, 0, min(NB, l), thr, Dc, s_dinv, rowbuf);
    if (tid == 0) *s_fail = f < 0 ? -1 : f;
  }
  __syncthreads();
  if (*s_fail >= 0) return *s_fail;
  for (int p0 = 0; p0 < l; p0 += NB) {
    const int pb = min(NB, l - p0);
    const int c0 = p0 + pb, nt = l - c0;
    if (nt <= 0) break;
    // (b) S(p, c0:) <- D_p^T S(p, c0:), 4 x 4 register tiles
    {
      const int ncq = (nt + 3) / 4;
      const bool have = tid < 8 * ncq;
      float acc[4][4];
      int i0 = 0, c = 0;
      if (have) {
        const int rg = tid / ncq;
        i0 = 4 * rg;
        c = c0 + 4 * (tid - rg * ncq);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int w = 0; w < 4; ++w) acc[q][w] = 0.f;
        const int tmax = min(pb, i0 + 4);
#pragma unroll 4
        for (int t = 0; t < tmax; ++t) {
          const float4 da = lds4(Dc + t * CHF_DLD + i0);
          const float4 s4 = lds4(S + (p0 + t) * ld + c);
          const float dv[4] = {da.x, da.y, da.z, da.w};
          const float sv[4] = {s4.x, s4.y, s4.z, s4.w};
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[q][w] = fmaf(dv[q], sv[w], acc[q][w]);
        }
      }
      __syncthreads();
      if (have) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (i0 + q < pb)
            *reinterpret_cast<float4*>(S + (p0 + i0 + q) * ld + c) =
                make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
      }
      __syncthreads();
    }
    const int nb1 = min(NB, nt);   // width of the next panel
    // the next diagonal block's update, spread over the worker warps (one
    // entry per thread and pass, the products added in the panel's row
    // order), handed to warp 0 through named barrier 1
    if ((warp & 3) != 0) {
      const int nwk = (nthr >> 5) - (nthr >> 7);
      const int wt = (warp - 1 - (warp >> 2)) * 32 + (tid & 31);
      for (int o = wt; o < nb1 * nb1; o += nwk * 32) {
        const int i = o / nb1, c = o - (o / nb1) * nb1;
        if (c < i) continue;
        float acc = 0.f;
        for (int t = 0; t < pb; ++t) {
          const float* row = S + (p0 + t) * ld + c0;
          acc = fmaf(row[i], row[c], acc);
        }
        S[(c0 + i) * ld + c0 + c] -= acc;
      }
      __threadfence_block();
      asm volatile("bar.arrive 1, %0;" ::"r"(nwk * 32 + 32) : "memory");
    }
    if (warp == 0) {
      asm volatile("bar.sync 1, %0;" ::"r"((nthr >> 5) * 32 - (nthr >> 7) * 32 + 32) : "memory");
      const int f = chf_diag(S, ld, c0, nb1, thr, Dc, s_dinv, rowbuf);
      if (tid == 0) *s_fail = f < 0 ? -1 : c0 + f;
    } else if ((warp & 3) != 0) {
      // (c) the rest of the trailing upper triangle, 8 x 8 tiles over the
      // upper tile grid; the tiles of the next diagonal block (tc < nbT) are
      // warp 0's.  Warps 4, 8, .. (warp 0's scheduler partition) stay idle so
      // that warp 0's dependent chain keeps its issue slots.
      const int nT = (nt + 7) / 8, nbT = (nb1 + 7) / 8;
      const int ntl = nT * (nT + 1) / 2;
      const int nwk = (nthr >> 5) - (nthr >> 7);          // working warps
      const int wk = warp - 1 - (warp >> 2);              // 0 .. nwk - 1
      for (int u = wk * 32 + (tid & 31); u < ntl; u += nwk * 32) {
        int ti, tc;
        tri_tile(u, nT, &ti, &tc);
        if (tc < nbT) continue;
        const int i0 = c0 + 8 * ti, k0 = c0 + 8 * tc;
        float acc[8][8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
#pragma unroll
          for (int w = 0; w < 8; ++w) acc[q][w] = 0.f;
#pragma unroll 2
        for (int t = 0; t < pb; ++t) {
          const float* row = S + (p0 + t) * ld;
          const float4 a0 = lds4(row + i0), a1 = lds4(row + i0 + 4);
          const float4 b0 = lds4(row + k0), b1 = lds4(row + k0 + 4);
          const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
          const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
          for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int w = 0; w < 8; ++w) acc[q][w] = fmaf(av[q], bv[w], acc[q][w]);
        }
        if (tc > ti) {   // off-diagonal tile: whole rows (padding columns receive 0)
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            if (i0 + q < l) {
              float4* o = reinterpret_cast<float4*>(S + (i0 + q) * ld + k0);
              float4 u0 = o[0], u1 = o[1];
              u0.x -= acc[q][0]; u0.y -= acc[q][1]; u0.z -= acc[q][2]; u0.w -= acc[q][3];
              u1.x -= acc[q][4]; u1.y -= acc[q][5]; u1.z -= acc[q][6]; u1.w -= acc[q][7];
              o[0] = u0;
              o[1] = u1;
            }
          }
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q)
#pragma unroll
            for (int w = 0; w < 8; ++w) {
              const int i = i0 + q, cc = k0 + w;
              if (i < l && cc < l && cc >= i) S[i * ld + cc] -= acc[q][w];
            }
        }
      }
    }
    __syncthreads();
    if (*s_fail >= 0) return *s_fail;
  }
  return -1;
}

// In-place X = R^{-1} (upper triangle of S), using the D_I blocks left by the
// factorization.
__device__ void chf_inverse(float* S, int l, int ld, const float* s_dinv) {
  const int tid = threadIdx.x;
  const int nb = (l + NB - 1) / NB;
  for (int Ib = nb - 1; Ib >= 0; --Ib) {
    const int r0 = Ib * NB, rb = min(NB, l - r0);
    const int cs = r0 + rb, ncol = l - cs;   // ncol > 0 only for full blocks
    if (ncol > 0) {
      // T(i, c) = -sum_{t = cs}^{c} R(i, t) X(t, c): 4 x 4 register tiles
      {
        const int ncq = (ncol + 3) / 4;
        const bool have = tid < 8 * ncq;
        float acc[4][4];
        int i0 = 0, k0 = 0;
        if (have) {
          const int rg = tid / ncq;
          i0 = r0 + 4 * rg;
          k0 = cs + 4 * (tid - rg * ncq);
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[q][w] = 0.f;
          for (int t = cs; t < k0; t += 4) {   // rows of X above the tile: all upper
            float ra[4][4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float4 r4 = lds4(S + (i0 + q) * ld + t);
              ra[q][0] = r4.x; ra[q][1] = r4.y; ra[q][2] = r4.z; ra[q][3] = r4.w;
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float4 x4 = lds4(S + (t + e) * ld + k0);
              const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
              for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int w = 0; w < 4; ++w) acc[q][w] = fmaf(ra[q][e], xv[w], acc[q][w]);
            }
          }
          const int te = min(l, k0 + 4);
          for (int t = k0; t < te; ++t) {       // the tile's own diagonal band
            const float4 x4 = lds4(S + t * ld + k0);
            const float xr[4] = {x4.x, x4.y, x4.z, x4.w};
            float xv[4];
#pragma unroll
            for (int w = 0; w < 4; ++w) xv[w] = (k0 + w >= t) ? xr[w] : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              const float r = S[(i0 + q) * ld + t];
#pragma unroll
              for (int w = 0; w < 4; ++w) acc[q][w] = fmaf(r, xv[w], acc[q][w]);
            }
          }
        }
        __syncthreads();
        if (have) {   // padding columns receive 0 (X is zero there)
#pragma unroll
          for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4*>(S + (i0 + q) * ld + k0) =
                make_float4(-acc[q][0], -acc[q][1], -acc[q][2], -acc[q][3]);
        }
        __syncthreads();
      }
      // X(i, c) = sum_{t >= i} D_I(i, t) T(t, c): 4 x 4 register tiles
      {
        const int ncq = (ncol + 3) / 4;
        const bool have = tid < 8 * ncq;
        float acc[4][4];
        int i0 = 0, c = 0;
        if (have) {
          const int rg = tid / ncq;
          i0 = 4 * rg;
          c = cs + 4 * (tid - rg * ncq);
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int w = 0; w < 4; ++w) acc[q][w] = 0.f;
          for (int t = i0; t < NB; ++t) {
            // D_I(i, t), i = i0 .. i0 + 3, sits at S(r0 + t, r0 + i) for t > i
            const float4 da = lds4(S + (r0 + t) * ld + r0 + i0);
            float dv[4] = {da.x, da.y, da.z, da.w};
            if (t < i0 + 4) {
              const float dd = s_dinv[r0 + t];
#pragma unroll
              for (int q = 0; q < 4; ++q)
                dv[q] = (t > i0 + q) ? dv[q] : ((t == i0 + q) ? dd : 0.f);
            }
            const float4 t4 = lds4(S + (r0 + t) * ld + c);
            const float tv[4] = {t4.x, t4.y, t4.z, t4.w};
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
              for (int w = 0; w < 4; ++w) acc[q][w] = fmaf(dv[q], tv[w], acc[q][w]);
          }
        }
        __syncthreads();
        if (have) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            *reinterpret_cast<float4*>(S + (r0 + i0 + q) * ld + c) =
                make_float4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
        }
      }
    }
    // X(I, I) = D_I into the block's upper triangle (D_I^T stays below)
    for (int e = tid; e < NB * NB; e += blockDim.x) {
      const int i = e >> 5, cc = e & 31;
      if (i < rb && cc < rb && cc >= i)
        S[(r0 + i) * ld + r0 + cc] = (cc == i) ? s_dinv[r0 + i] : S[(r0 + cc) * ld + r0 + i];
    }
    __syncthreads();
  }
}

// Upper triangle of S (identity on the padding up to L) to a row-major L x L
// fp32 matrix: one row per warp, four columns per lane (L % 4 == 0).
__device__ void chf_store_upper(const float* S, int l, int ld, int L, float* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < L; i += nw) {
    for (int c = 4 * lane; c < L; c += 128) {
      float v[4];
      if (i < l && c + 3 < ld) {
        const float4 s4 = lds4(S + i * ld + c);
        v[0] = s4.x; v[1] = s4.y; v[2] = s4.z; v[3] = s4.w;
      }
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        const int cc = c + w;
        if (i < l && cc < l) v[w] = cc >= i ? v[w] : 0.f;
        else v[w] = (i == cc) ? 1.f : 0.f;
      }
      *reinterpret_cast<float4*>(out + (size_t)i * L + c) = make_float4(v[0], v[1], v[2], v[3]);
    }
  }
}

// W^T with W = R^{-1} (Wt[j][kk] = X[kk][j]) as three bf16 terms: each warp
// takes 32 x 32 tiles; lane j reads column j of the tile (rows kk, coalesced
// across lanes) and writes its 32 consecutive entries of row j of Wt.
__device__ void chf_store_w(const float* S, int l, int ld, int L, __nv_bfloat16* hi,
                            __nv_bfloat16* lo, __nv_bfloat16* lo2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nt = (L + 31) / 32;
  for (int tt = warp; tt < nt * nt; tt += nw) {
    const int tj = tt / nt, tk = tt - tj * nt;
    const int j = 32 * tj + lane;
    if (j >= L) continue;
    for (int k8 = 0; k8 < 32; k8 += 8) {
      uint32_t ph[4], pm[4], pl[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float v2[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int kk = 32 * tk + k8 + 2 * h + e;
          float v;
          if (j < l && kk < l) v = (j >= kk) ? S[kk * ld + j] : 0.f;
          else v = (j == kk) ? 1.f : 0.f;
          v2[e] = v;
        }
        uint32_t w3[3][2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const __nv_bfloat16 b0 = __float2bfloat16_rn(v2[e]);
          const float r1 = v2[e] - __bfloat162float(b0);
          const __nv_bfloat16 b1 = __float2bfloat16_rn(r1);
          const __nv_bfloat16 b2 = __float2bfloat16_rn(r1 - __bfloat162float(b1));
          w3[0][e] = __bfloat16_as_ushort(b0);
          w3[1][e] = __bfloat16_as_ushort(b1);
          w3[2][e] = __bfloat16_as_ushort(b2);
        }
        ph[h] = w3[0][0] | (w3[0][1] << 16);
        pm[h] = w3[1][0] | (w3[1][1] << 16);
        pl[h] = w3[2][0] | (w3[2][1] << 16);
      }
      const int kb = 32 * tk + k8;
      if (kb + 8 <= L) {
        const size_t o = (size_t)j * L + kb;
        *reinterpret_cast<uint4*>(hi + o) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
        *reinterpret_cast<uint4*>(lo + o) = make_uint4(pm[0], pm[1], pm[2], pm[3]);
        *reinterpret_cast<uint4*>(lo2 + o) = make_uint4(pl[0], pl[1], pl[2], pl[3]);
      }
    }
  }
}

// The body of chol_kernel for a matrix S of leading dimension ld; the shared-
// memory instance receives S derived from the kernel's shared array, so that
// after inlining every access to it compiles as a shared-memory access (a
// generic pointer that might alias global memory would serialise the loads).
template <typename T>
__device__ __forceinline__ void chol_body(const CholArgs& a, T* S, int ld, T* red, T& s_maxdiag,
                                          T& s_dev, int& s_fail) {
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
  if (tid == 0) chol_update_flags(a, used_shift, (double)l * (double)s_dev);
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
  chol_body<T>(a, reinterpret_cast<T*>(dsm), a.l, red, s_maxdiag, s_dev, s_fail);
}
// ... or in the global scratch (large l)
template <typename T>
__global__ void __launch_bounds__(CT) chol_kernel_global(CholArgs a) {
  __shared__ T red[32];
  __shared__ T s_maxdiag, s_dev;
  __shared__ int s_fail;
  chol_body<T>(a, (T*)a.scratch, a.l, red, s_maxdiag, s_dev, s_fail);
}

// fp32, l <= 224: the register-tiled kernel on the padded shared-memory matrix
__global__ void __launch_bounds__(CHF_T, 1) chol_f32_kernel(CholArgs a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ float red[32];
  __shared__ float s_maxdiag, s_dev;
  __shared__ int s_fail;
  __shared__ float s_dinv[256];
  __shared__ __align__(16) float rowbuf[2 * NB];
  float* S = reinterpret_cast<float*>(dsm);
  const int l = a.l, L = a.L, ld = chf_ld(l);
  float* Dc = S + l * ld;
  if (a.skip_idx >= 0 && a.flags && a.flags[a.skip_idx] == 1) {  // pass not needed: R = I
    write_identity_outputs<float>(a);
    return;
  }
  float md = 0.f, dev = 0.f;
  bool bad = false;
  chf_load(a, S, ld, 0.f, &md, &dev, &bad);
  if (bad) set_info(a.d_info, RSVD_ERR_NUMERIC);
  block_max<float>(md, red, &s_maxdiag);
  block_max<float>(dev, red, &s_dev);
  const float maxdiag = s_maxdiag;
  if (!(maxdiag > 0.f)) {                        // X = 0 or non-finite: no basis
    set_info(a.d_info, RSVD_ERR_NOT_SPD);
    write_identity_outputs<float>(a);
    return;
  }
  const float tau = 4.f * (float)l * 5.9604645e-8f;
  float shift = 0.f;
  int used_shift = 0, fail = -1;
  for (int attempt = 0; attempt < 12; ++attempt) {
    if (attempt > 0) {
      __syncthreads();
      chf_load(a, S, ld, shift, nullptr, nullptr, nullptr);
    }
    __syncthreads();
    fail = chf_factor(S, l, ld, tau * maxdiag, Dc, s_dinv, rowbuf, &s_fail);
    __syncthreads();
    if (fail < 0) break;
    shift = (shift == 0.f) ? tau * maxdiag : shift * 10.f;
    used_shift = 1;
  }
  if (fail >= 0) {
    set_info(a.d_info, RSVD_ERR_NOT_SPD);
    write_identity_outputs<float>(a);
    return;
  }
  if (threadIdx.x == 0) chol_update_flags(a, used_shift, (double)l * (double)s_dev);
  if (a.R) chf_store_upper(S, l, ld, L, (float*)a.R);
  __syncthreads();                               // R read before the inverse overwrites it
  chf_inverse(S, l, ld, s_dinv);
  if (a.Rinv) chf_store_upper(S, l, ld, L, (float*)a.Rinv);
  if (a.Whi)
    chf_store_w(S, l, ld, L, (__nv_bfloat16*)a.Whi, (__nv_bfloat16*)a.Wlo,
                (__nv_bfloat16*)a.Wlo2);
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

// One CTA per problem of a batch: the factor and inverse of chol_kernel
// (shifted retries included) on the problem's l x l Gram, without the pass
// bookkeeping of CholeskyQR2/3 (the batched path always runs two passes).
// CHB_T = 128 threads: at the batch's widths (l <= 128) the panel solve has at
// most l - 32 <= 96 columns of work, so half of the generic kernel's 256
// threads would idle there, and at ~168 registers a thread three 128-thread
// CTAs fit on an SM against one of 256 (the 512-problem batch in ~1.2 waves
// instead of 3.5).
// The inverse keeps at most 32 elements of T per thread in registers, which
// covers ne <= NB * l for l <= 32 * CHB_T / NB.
constexpr int CHB_T = 128;
static_assert(32 * CHB_T >= NB * BATCH_LMAX, "inverse register capacity of the batched Cholesky");
__global__ void __launch_bounds__(CT) chol_batched_kernel(const BChol* __restrict__ tasks,
                                                          int* d_info) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ float red[32];
  __shared__ float s_maxdiag, s_dev;
  __shared__ int s_fail;
  const BChol tk = tasks[blockIdx.x];
  CholArgs a{};
  a.l = tk.l;
  a.L = tk.l;
  a.G = tk.G;
  a.ldg = tk.l;
  a.R = tk.R;
  a.Rinv = tk.Rinv;
  a.pass = 1;
  a.skip_idx = -1;
  a.d_info = d_info;
  chol_body<float>(a, reinterpret_cast<float*>(dsm), tk.l, red, s_maxdiag, s_dev, s_fail);
}

cudaError_t launch_chol_batched(const BChol* tasks, int batch, int lmax, int* d_info,
                                cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  if (lmax > BATCH_LMAX) return cudaErrorInvalidValue;
  const size_t dyn = (size_t)lmax * lmax * sizeof(float);
  if (dyn > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(chol_batched_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
  }
  const int tr_ = trace_begin(RSVD_TRACE_CHOL, s);
  chol_batched_kernel<<<batch, dim3(32, CHB_T / 32), dyn, s>>>(tasks, d_info);
  count_launch();
  trace_end(tr_, s);
  return cudaGetLastError();
}

// Racc <- R Racc per problem (upper triangular), one CTA each.
__global__ void trmm_batched_kernel(const BTrmm* __restrict__ tasks) {
  const BTrmm tk = tasks[blockIdx.x];
  const int l = tk.l;
  for (int t = threadIdx.x; t < l * l; t += blockDim.x) {
    const int i = t / l, c = t - (t / l) * l;
    float acc = 0.f;
    if (c >= i)
      for (int q = i; q <= c; ++q) acc = fmaf(tk.R[i * l + q], tk.Racc[q * l + c], acc);
    tk.tmp[t] = acc;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < l * l; t += blockDim.x) tk.Racc[t] = tk.tmp[t];
}

cudaError_t launch_trmm_batched(const BTrmm* tasks, int batch, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  trmm_batched_kernel<<<batch, 256, 0, s>>>(tasks);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cooperative blocked Cholesky and inverse of an fp32 Gram over many CTAs
// (l beyond the one-CTA shared-memory kernel, up to 1024).  The padded matrix
// lp x lp (lp = l rounded up to 32, identity on the padding) lives in the
// global scratch with its inverse X beside it; every phase is a set of 32 x 32
// block tasks spread over the grid, separated by bounded grid barriers:
//   D(k)   the diagonal block: R_kk by warp 0 in registers (lane c holds
//          column c; pivots not above thr stop the attempt), then
//          X_kk = R_kk^-1 by back substitution (lane c: column c);
//   P(k)   R_kj = X_kk^T A_kj for the blocks right of the diagonal;
//   U(k)   A_ij -= R_ki^T R_kj for k < i <= j; CTA 0 first updates block
//          (k+1, k+1) and factors it (D(k+1)), so one barrier per phase;
//   inverse, by block diagonals d = 1, 2, ..:
//          X_ij = -X_ii (sum over m = i+1..j of R_im X_mj), j = i + d.
// The shifted retries, the flags of CholeskyQR2/3 and the outputs are those of
// chol_body.  Every wait is bounded: on expiry RSVD_ERR_TIMEOUT is recorded and
// each CTA leaves at its next barrier.
// ---------------------------------------------------------------------------
#ifndef CHOL_COOP_MIN_L
#define CHOL_COOP_MIN_L 225               // below: the one-CTA shared-memory kernels
#endif
namespace {
constexpr int CC_T = 256;                 // threads per CTA
constexpr long long CC_SPIN = 4000000000LL;
constexpr int CC_ATTEMPTS = 12;          // shifted retries, as chol_body
struct CoopHdr {
  unsigned bar;                  // grid barrier counter
  unsigned md_bits;              // max diagonal of G (bits of a non-negative float)
  unsigned dev_bits;             // max |G - I|
  int bad;                       // a non-finite entry
  int fail[CC_ATTEMPTS];         // a pivot of the attempt was not above thr (one slot per
                                 // attempt: nothing is reset while another CTA may read it)
};
inline int coop_lp(int l) { return (l + 31) & ~31; }
}  // namespace

size_t chol_coop_scratch_bytes(int l) {
  const size_t lp = (size_t)coop_lp(l);
  return 256 + 2 * lp * lp * sizeof(float);
}

__device__ __forceinline__ unsigned cc_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// false when the wait ran out (the caller leaves)
__device__ bool cc_barrier(CoopHdr* h, unsigned target, int* d_info) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&h->bar, 1u);
    const long long t0 = clock64();
    int ok = 1;
    unsigned it = 0;
    while (cc_ld_acquire(&h->bar) < target) {
      __nanosleep(64);
      if (((++it) & 255u) == 0 && clock64() - t0 > CC_SPIN) {
        set_info(d_info, RSVD_ERR_TIMEOUT);
        ok = 0;
        break;
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// A 32 x 32 block (row-major in the lp-wide matrix M at block (bi, bj)) into
// shared memory, read through L2 (other CTAs wrote it before the barrier).
__device__ __forceinline__ void cc_load(float (*T)[33], const float* M, int lp, int bi, int bj) {
  for (int e = threadIdx.x; e < 1024; e += CC_T) {
    const int r = e >> 5, c = e & 31;
    T[r][c] = __ldcg(M + (size_t)(32 * bi + r) * lp + 32 * bj + c);
  }
}

// acc[w] = sum_t A[t][r] B[t][c0 + w]  (A^T B), thread: r = tid / 8, c0 = 4 (tid % 8)
__device__ __forceinline__ void cc_atb(const float (*A)[33], const float (*B)[33], float acc[4]) {
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
#pragma unroll 8
  for (int t = 0; t < 32; ++t) {
    const float a = A[t][r];
#pragma unroll
    for (int w = 0; w < 4; ++w) acc[w] = fmaf(a, B[t][c0 + w], acc[w]);
  }
}
// acc[w] += sum_t A[r][t] B[t][c0 + w]  (A B)
__device__ __forceinline__ void cc_ab(const float (*A)[33], const float (*B)[33], float acc[4]) {
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
#pragma unroll 8
  for (int t = 0; t < 32; ++t) {
    const float a = A[r][t];
#pragma unroll
    for (int w = 0; w < 4; ++w) acc[w] = fmaf(a, B[t][c0 + w], acc[w]);
  }
}
__device__ __forceinline__ void cc_store(float* M, int lp, int bi, int bj, const float acc[4]) {
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
  float* d = M + (size_t)(32 * bi + r) * lp + 32 * bj + c0;
  *reinterpret_cast<float4*>(d) = make_float4(acc[0], acc[1], acc[2], acc[3]);
}

// D(k): factor the (updated) diagonal block k, write R_kk into S and X_kk into
// X; on a pivot not above thr set *fail.  The whole CTA enters.
__device__ void cc_diag(float* S, float* X, int lp, int k, float thr, int* fail,
                        float (*Rs)[33]) {
  const int tid = threadIdx.x, lane = tid & 31;
  __syncthreads();
  if (tid < 32) {
    float d[32];
#pragma unroll
    for (int i = 0; i < 32; ++i)
      d[i] = (i <= lane) ? __ldcg(S + (size_t)(32 * k + i) * lp + 32 * k + lane) : 0.f;
    int failed = -1;
#pragma unroll
    for (int jj = 0; jj < 32; ++jj) {
      if (failed < 0) {
        const float piv = __shfl_sync(0xffffffffu, d[jj], jj);
        if (!(piv > thr)) {
          failed = jj;
        } else {
          const float r = sqrtf(piv);
          float rj = d[jj];
          if (lane == jj) rj = r;
          else if (lane > jj) rj = rj / r;
          d[jj] = rj;
#pragma unroll
          for (int i = jj + 1; i < 32; ++i) {
            const float ri = __shfl_sync(0xffffffffu, rj, i);
            if (lane >= i) d[i] -= ri * rj;
          }
        }
      }
    }
    if (failed >= 0) {
      if (lane == 0) atomicExch(fail, 1);
    } else {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        Rs[i][lane] = (i <= lane) ? d[i] : 0.f;
        if (i <= lane) S[(size_t)(32 * k + i) * lp + 32 * k + lane] = d[i];
      }
      __syncwarp();
      // column c = lane of X_kk = R_kk^-1: x_c = 1 / r_cc, then upward
      float x[32];
#pragma unroll
      for (int i = 31; i >= 0; --i) {
        if (i > lane) {
          x[i] = 0.f;
        } else if (i == lane) {
          x[i] = 1.f / Rs[i][i];
        } else {
          float acc = 0.f;
#pragma unroll
          for (int m = i + 1; m < 32; ++m)
            if (m <= lane) acc = fmaf(Rs[i][m], x[m], acc);
          x[i] = -acc / Rs[i][i];
        }
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) X[(size_t)(32 * k + i) * lp + 32 * k + lane] = x[i];
    }
  }
  __syncthreads();
}

__device__ void cc_identity_rows(const CholArgs& a) {
  const int L = a.L;
  for (int i = blockIdx.x; i < L; i += gridDim.x)
    for (int c = threadIdx.x; c < L; c += CC_T) {
      const size_t t = (size_t)i * L + c;
      const float v = (i == c) ? 1.f : 0.f;
      if (a.R) ((float*)a.R)[t] = v;
      if (a.Rinv) ((float*)a.Rinv)[t] = v;
      if (a.Whi) {
        ((__nv_bfloat16*)a.Whi)[t] = __float2bfloat16_rn(v);
        ((__nv_bfloat16*)a.Wlo)[t] = __float2bfloat16_rn(0.f);
        ((__nv_bfloat16*)a.Wlo2)[t] = __float2bfloat16_rn(0.f);
      }
    }
}

__global__ void __launch_bounds__(CC_T) chol_coop_kernel(CholArgs a, int lp) {
  __shared__ float As[32][33], Bs[32][33];
  __shared__ float s_red[2][CC_T / 32];
  __shared__ int s_bad;
  const int l = a.l, L = a.L, nb = lp / 32, G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  CoopHdr* h = reinterpret_cast<CoopHdr*>(a.scratch);
  float* S = reinterpret_cast<float*>(reinterpret_cast<char*>(a.scratch) + 256);
  float* X = S + (size_t)lp * lp;
  const float* Gm = (const float*)a.G;
  unsigned epoch = 0;
  if (a.skip_idx >= 0 && a.flags && a.flags[a.skip_idx] == 1) {   // pass not needed: R = I
    cc_identity_rows(a);
    return;
  }
  // scale of G, its distance to I and non-finite entries (rows over the CTAs)
  {
    float md = 0.f, dev = 0.f;
    int bad = 0;
    for (int i = b; i < l; i += G)
      for (int c = tid; c < l; c += CC_T) {
        const float g = Gm[(size_t)i * a.ldg + c];
        if (!isfinite(g)) bad = 1;
        if (i == c) md = fmaxf(md, g);
        dev = fmaxf(dev, fabsf(g - (i == c ? 1.f : 0.f)));
      }
    if (tid == 0) s_bad = 0;
    for (int o = 16; o > 0; o >>= 1) {
      md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
      dev = fmaxf(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    }
    __syncthreads();
    if (bad) s_bad = 1;
    if ((tid & 31) == 0) {
      s_red[0][tid >> 5] = md;
      s_red[1][tid >> 5] = dev;
    }
    __syncthreads();
    if (tid == 0) {
      for (int w = 1; w < CC_T / 32; ++w) {
        md = fmaxf(md, s_red[0][w]);
        dev = fmaxf(dev, s_red[1][w]);
      }
      atomicMax(&h->md_bits, __float_as_uint(md));
      atomicMax(&h->dev_bits, __float_as_uint(dev));
      if (s_bad) atomicOr(&h->bad, 1);
    }
  }
  if (!cc_barrier(h, ++epoch * G, a.d_info)) return;
  const float maxdiag = __uint_as_float(__ldcg(&h->md_bits));
  const float gdev = __uint_as_float(__ldcg(&h->dev_bits));
  if (b == 0 && tid == 0 && __ldcg(&h->bad)) set_info(a.d_info, RSVD_ERR_NUMERIC);
  if (!(maxdiag > 0.f)) {                        // X = 0 or non-finite: no basis
    if (b == 0 && tid == 0) set_info(a.d_info, RSVD_ERR_NOT_SPD);
    cc_identity_rows(a);
    return;
  }
  const float thr = 4.f * (float)l * 5.9604645e-8f * maxdiag;
  float shift = 0.f;
  int used_shift = 0;
  bool ok = false;
  for (int attempt = 0; attempt < CC_ATTEMPTS && !ok; ++attempt) {
    int* fail = &h->fail[attempt];
    // S = G + shift I, maxdiag on the padding's diagonal (above thr, decoupled
    // from the rest; its factor never reaches the outputs); X = 0
    for (int i = b; i < lp; i += G)
      for (int c = tid; c < lp; c += CC_T) {
        float v;
        if (i < l && c < l) v = Gm[(size_t)i * a.ldg + c] + ((i == c) ? shift : 0.f);
        else v = (i == c) ? maxdiag : 0.f;
        S[(size_t)i * lp + c] = v;
        X[(size_t)i * lp + c] = 0.f;
      }
    if (!cc_barrier(h, ++epoch * G, a.d_info)) return;
    if (b == 0) cc_diag(S, X, lp, 0, thr, fail, As);
    if (!cc_barrier(h, ++epoch * G, a.d_info)) return;
    ok = __ldcg(fail) == 0;
    for (int k = 0; ok && k + 1 < nb; ++k) {
      // P(k): R_kj = X_kk^T A_kj
      for (int j = k + 1 + b; j < nb; j += G) {
        cc_load(As, X, lp, k, k);
        cc_load(Bs, S, lp, k, j);
        __syncthreads();
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        cc_atb(As, Bs, acc);
        __syncthreads();
        cc_store(S, lp, k, j, acc);
      }
      if (!cc_barrier(h, ++epoch * G, a.d_info)) return;
      // U(k): A_ij -= R_ki^T R_kj, k < i <= j.  Task 0 is block (k+1, k+1):
      // CTA 0 updates it and factors it (D(k+1)) and takes nothing else; the
      // other tasks go to CTAs 1 .. G-1 (all to CTA 0 when G = 1)
      const int m = nb - k - 1;                  // trailing block rows
      const int ntask = m * (m + 1) / 2;
      const int first = (G == 1 || b == 0) ? 0 : b;
      const int stride = (G == 1) ? 1 : (b == 0 ? ntask : G - 1);
      for (int t = first; t < ntask; t += stride) {
        // task t -> (i, j): row-major over the upper triangle of the trailing blocks
        int i = 0, rem = t;
        while (rem >= m - i) {
          rem -= m - i;
          ++i;
        }
        const int bi = k + 1 + i, bj = bi + rem;
        cc_load(As, S, lp, k, bi);
        cc_load(Bs, S, lp, k, bj);
        __syncthreads();
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        cc_atb(As, Bs, acc);
        const int r = tid >> 3, c0 = (tid & 7) * 4;
        float* d = S + (size_t)(32 * bi + r) * lp + 32 * bj + c0;
        const float4 o = __ldcg(reinterpret_cast<const float4*>(d));
        __syncthreads();
        *reinterpret_cast<float4*>(d) =
            make_float4(o.x - acc[0], o.y - acc[1], o.z - acc[2], o.w - acc[3]);
        if (t == 0) cc_diag(S, X, lp, k + 1, thr, fail, As);
      }
      if (!cc_barrier(h, ++epoch * G, a.d_info)) return;
      ok = __ldcg(fail) == 0;
    }
    if (!ok) {
      shift = (shift == 0.f) ? thr : shift * 10.f;
      used_shift = 1;
    }
  }
  if (!ok) {
    if (b == 0 && tid == 0) set_info(a.d_info, RSVD_ERR_NOT_SPD);
    cc_identity_rows(a);
    return;
  }
  if (b == 0 && tid == 0) chol_update_flags(a, used_shift, (double)l * (double)gdev);
  // R out (identity on the padding)
  if (a.R)
    for (int i = b; i < L; i += G)
      for (int c = tid; c < L; c += CC_T) {
        float v;
        if (i < l && c < l) v = (c >= i) ? __ldcg(S + (size_t)i * lp + c) : 0.f;
        else v = (i == c) ? 1.f : 0.f;
        ((float*)a.R)[(size_t)i * L + c] = v;
      }
  // inverse by block diagonals
  for (int dg = 1; dg < nb; ++dg) {
    for (int i = b; i + dg < nb; i += G) {
      const int j = i + dg;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      for (int mm = i + 1; mm <= j; ++mm) {
        cc_load(As, S, lp, i, mm);
        cc_load(Bs, X, lp, mm, j);
        __syncthreads();
        cc_ab(As, Bs, acc);
        __syncthreads();
      }
      // X_ij = -X_ii T
      {
        const int r = tid >> 3, c0 = (tid & 7) * 4;
#pragma unroll
        for (int w = 0; w < 4; ++w) Bs[r][c0 + w] = acc[w];
      }
      cc_load(As, X, lp, i, i);
      __syncthreads();
      float o[4] = {0.f, 0.f, 0.f, 0.f};
      cc_ab(As, Bs, o);
      __syncthreads();
#pragma unroll
      for (int w = 0; w < 4; ++w) o[w] = -o[w];
      cc_store(X, lp, i, j, o);
    }
    if (!cc_barrier(h, ++epoch * G, a.d_info)) return;
  }
  if (a.Rinv)
    for (int i = b; i < L; i += G)
      for (int c = tid; c < L; c += CC_T) {
        float v;
        if (i < l && c < l) v = (c >= i) ? __ldcg(X + (size_t)i * lp + c) : 0.f;
        else v = (i == c) ? 1.f : 0.f;
        ((float*)a.Rinv)[(size_t)i * L + c] = v;
      }
  if (a.Whi)   // W^T with W = R^{-1}: Wt[j][kk] = X[kk][j], three bf16 terms
    for (int j = b; j < L; j += G)
      for (int kk = tid; kk < L; kk += CC_T) {
        float v;
        if (j < l && kk < l) v = (j >= kk) ? __ldcg(X + (size_t)kk * lp + j) : 0.f;
        else v = (j == kk) ? 1.f : 0.f;
        const __nv_bfloat16 hb = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(hb);
        const __nv_bfloat16 mb = __float2bfloat16_rn(r1);
        const size_t t = (size_t)j * L + kk;
        ((__nv_bfloat16*)a.Whi)[t] = hb;
        ((__nv_bfloat16*)a.Wlo)[t] = mb;
        ((__nv_bfloat16*)a.Wlo2)[t] = __float2bfloat16_rn(r1 - __bfloat162float(mb));
      }
}

static cudaError_t launch_chol_coop(const CholArgs& a, cudaStream_t s) {
  const int lp = coop_lp(a.l), nb = lp / 32;
  // one CTA per task of the widest phase, leaving room beside a running
  // cluster kernel (the Jacobi of the combined call)
  int G = nb * (nb - 1) / 2;
  const int sms = device_sm_count();
  if (G > sms - 16) G = sms - 16;
  if (G < 1) G = 1;
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_coop_kernel, CC_T, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  e = cudaMemsetAsync(a.scratch, 0, sizeof(CoopHdr), s);
  if (e != cudaSuccess) return e;
  CholArgs b = a;
  int lpv = lp;
  void* args[] = {(void*)&b, (void*)&lpv};
  return cudaLaunchCooperativeKernel((const void*)chol_coop_kernel, dim3((unsigned)G), dim3(CC_T),
                                     args, 0, s);
}

template <typename T>
cudaError_t launch_chol(const CholArgs& a, cudaStream_t s) {
  const size_t bytes = (size_t)a.l * a.l * sizeof(T);
  // the fp32 kernel: its matrix plus about 2 KB of static arrays in one CTA,
  // 16-byte R rows and W rows
  const bool f32 = sizeof(T) == 4 && a.l <= CHF_LMAX && chf_smem(a.l) + 2048 <= 232448 &&
                   a.L % 4 == 0 && (a.Whi == nullptr || a.L % 8 == 0);
  // fp32 beyond the one-CTA kernel's range: the cooperative kernel (its
  // scratch is part of every fp32 orth workspace)
  const bool coop = sizeof(T) == 4 && a.scratch != nullptr && a.l >= CHOL_COOP_MIN_L &&
                    a.l <= 1024;
  const int tr_ = trace_begin(RSVD_TRACE_CHOL, s);
  if (coop) {
    cudaError_t e = launch_chol_coop(a, s);
    if (e != cudaSuccess) return e;
  } else if (f32) {
    const size_t dyn = chf_smem(a.l);
    cudaError_t e = cudaFuncSetAttribute(chol_f32_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    chol_f32_kernel<<<1, CHF_T, dyn, s>>>(a);
  } else {
    CholArgs b = a;
    size_t dyn = 0;
    if (bytes <= SMEM_LIMIT) {
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
    if (b.scratch)
      chol_kernel_global<T><<<1, dim3(32, CT / 32), 0, s>>>(b);
    else
      chol_kernel<T><<<1, dim3(32, CT / 32), dyn, s>>>(b);
  }
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
