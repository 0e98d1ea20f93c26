// Host-side launchers of the library's kernels (internal; not part of the C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rsvd {

// ----- Philox / Omega (k_philox.cu) ----------------------------------------
// tag: the counter's third word (0 = Omega of the right sketch, 1 = the left
// test matrix Omega~ of Sec. 3.5, stored transposed: n here is its column count m)
template <typename T>
cudaError_t launch_omega(int64_t n, int l, uint64_t seed, T* Om, int64_t ldo, cudaStream_t s,
                         uint32_t tag = 0);
cudaError_t launch_omega_words(int64_t n, int l, uint64_t seed, uint32_t* out, cudaStream_t s);
// Omega of the FP8 sketch (k_fp8.cu): bf16 Gaussians quantised to E4M3 with a
// power-of-two scale per 32-row block of each column; transposed bf16 (L x ldt,
// rows >= l zero; L a multiple of 4) or n x l floats (checking aid).
cudaError_t launch_omega_fp8_t(int64_t n, int l, int L, uint64_t seed, uint16_t* out, int64_t ldt,
                               cudaStream_t s);
cudaError_t launch_omega_fp8(int64_t n, int l, uint64_t seed, float* out, int64_t ldo,
                             cudaStream_t s);

// ----- SIMT GEMMs (k_simt.cu) ----------------------------------------------
// C (M x N) = A (M x K) * B (K x N); B = Omega(seed) when B == nullptr, with
// columns >= nvalid of Omega set to zero.  Row-major, leading dimensions given.
template <typename T>
cudaError_t launch_gemm_nn(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda,
                           const T* B, int64_t ldb, T* C, int64_t ldc, uint64_t seed,
                           int64_t nvalid, cudaStream_t s);
// Partial products of C (M x N) = A^T B with A (K x M), B (K x N): split-K slab
// z writes P[z*M*ldp + i*ldp + j]; nsplit slabs of kchunk rows.
template <typename T>
cudaError_t launch_gemm_tn_partial(int64_t M, int64_t N, int64_t K, const T* A, int64_t lda,
                                   const T* B, int64_t ldb, T* P, int64_t ldp, int nsplit,
                                   int64_t kchunk, cudaStream_t s);
// out[i*ldo + j] = sum_z P[z*M*ldp + i*ldp + j] (fixed order), j < ncols.
template <typename T>
cudaError_t launch_reduce_slabs(int64_t M, int64_t ncols, int nsplit, const T* P, int64_t ldp,
                                T* out, int64_t ldo, cudaStream_t s);
// Choice of split-K for the TN GEMM so the grid covers the GPU.
void tn_split(int64_t M, int64_t N, int64_t K, int num_sms, int* nsplit, int64_t* kchunk);

// ----- small dense helpers (k_misc.cu) -------------------------------------
template <typename TI, typename TO>
cudaError_t launch_copy2d(int64_t rows, int64_t cols, const TI* in, int64_t ldi, TO* out,
                          int64_t ldo, cudaStream_t s);
template <typename TI, typename TO>
cudaError_t launch_transpose(int64_t rows, int64_t cols, const TI* in, int64_t ldi, TO* out,
                             int64_t ldo, cudaStream_t s);
template <typename T>
cudaError_t launch_fill(int64_t rows, int64_t cols, T* out, int64_t ldo, T value,
                        cudaStream_t s);
// X (rows x cols fp32) -> hi/lo bf16 of X^T padded to L x rows (zeros for
// columns >= cols): the stored-operand form of the tensor-core GEMMs.
cudaError_t launch_split_transpose(int64_t rows, int cols, int L, const float* X, int64_t ldx,
                                   void* hi, void* lo, int64_t ldt, cudaStream_t s);
// out = in when *flag == 1 and not (veto && *veto == 1), decided on the device.
template <typename T>
cudaError_t launch_cond_copy(const int* flag, const int* veto, int64_t count, const T* in,
                             T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_scale_cols(int64_t rows, int k, T* X, int64_t ldx, const double* S,
                              cudaStream_t s);
cudaError_t launch_copy_i32(int64_t count, const int32_t* in, int32_t* out, cudaStream_t s);
// Sign rule: s_j = sign of the largest-|.| entry of column j of V (n x k);
// then U(:, j) *= s_j, V(:, j) *= s_j.
template <typename T>
cudaError_t launch_sign_fix(int64_t m, int64_t n, int k, T* U, int64_t ldu, T* V,
                            int64_t ldv, int* signs, cudaStream_t s);
// Gathers for ID/CUR.
// W (k x m doubles, row-major) = C^T with C = A(:, J[0:k]): W[i*m + r] = A[r, J[i]].
template <typename T>
cudaError_t launch_gather_ct(int64_t m, int k, const T* A, int64_t lda, const int32_t* J,
                             double* W, cudaStream_t s);
// Double-float planes (hi = the fp32 or bf16 value, lo = 0) of the same W, column-
// major, in the working area W (2 k m floats).
cudaError_t launch_gather_ct_df(int64_t m, int k, const void* A, int64_t lda, int a_bf16,
                                const int32_t* J, double* W, cudaStream_t s);
// R (k x n, fp32) = rows I of a bf16 A (ld lda)
cudaError_t launch_gather_rows_bf16(int k, int64_t n, const void* A, int64_t lda,
                                    const int32_t* I, float* R, int64_t ldr, cudaStream_t s);
template <typename T>
cudaError_t launch_gather_rows(int k, int64_t n, const T* A, int64_t lda, const int32_t* I,
                               T* R, int64_t ldr, cudaStream_t s);
template <typename T>
cudaError_t launch_gather_rows_by_perm(int64_t count, int cols, const T* X, int64_t ldx,
                                       const int32_t* idx, T* out, int64_t ldo,
                                       cudaStream_t s);
template <typename T>
cudaError_t launch_bt_to_w64(int64_t n, int l, const T* Bt, int64_t ldbt, double* W,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_add_inplace(int64_t rows, int64_t cols, const T* X, int64_t ldx, T* Y,
                               int64_t ldy, cudaStream_t s);
cudaError_t launch_check_finite_d(int64_t count, const double* x, int* d_info, cudaStream_t s);

// ----- Cholesky + triangular inverse (k_chol.cu) ---------------------------
struct CholArgs {
  int l;          // true size
  int L;          // padded size (outputs are L x L, identity on the padding)
  const void* G;  // l x l Gram (ld ldg)
  int64_t ldg;
  void* R;        // L x L upper factor (ld L), may be null
  void* Rinv;     // L x L inverse of R (ld L), may be null
  void* Whi;      // L x L bf16: (Rinv)^T first term (tensor-core operand), may be null
  void* Wlo;      // L x L bf16 second term
  void* Wlo2;     // L x L bf16 third term
  void* scratch;  // global fallback storage when the matrix does not fit in smem
  int* flags;     // [0] third pass needed, [1] a shift was used, [2] skip pass 3,
                  // [3] skip pass 2 (conditional second pass)
  int pass;       // 1, 2 or 3
  int skip_idx;   // when >= 0 and flags[skip_idx] == 1: write R = I and return
  int* d_info;
};
template <typename T>
cudaError_t launch_chol(const CholArgs& a, cudaStream_t s);
template <typename T>
cudaError_t launch_trmm_upper(int L, const T* R, T* Racc, T* tmp, cudaStream_t s);
size_t chol_scratch_bytes(int l, int elem);

// ----- Jacobi SVD (k_jacobi.cu) --------------------------------------------
template <typename T>
cudaError_t launch_jacobi(int l, const T* M, int64_t ldm, T* Uh, int64_t lduh, double* Sh,
                          T* Vh, int64_t ldvh, T* scratch, int max_sweeps, int* d_info,
                          cudaStream_t s);
size_t jacobi_scratch_bytes(int l, int elem);
template <typename T>
cudaError_t launch_svd_finalize(int l, const T* P, int64_t ldp, const T* Uin, int64_t ldin, T* Uh,
                                int64_t lduh, double* Sh, T* Vh, int64_t ldvh, int* d_info,
                                cudaStream_t s);

// ----- CPQR / ID (k_cpqr.cu) -----------------------------------------------
struct CpqrArgs {
  int r;            // rows of the sketch
  int64_t n;        // columns
  int k;            // steps
  double* W;        // r x n row-major, element (i, c) at W[i*n + c] (overwritten)
  int32_t* J;       // n permutation (output)
  int64_t* where;   // n scratch: position of each original column
  double* gaps;     // k (may be null)
  double* pval;     // 2 * 1024 * 2 scratch (best, second per CTA)
  int64_t* pidx;    // 2 * 1024 scratch
  double* nrm;      // 2n scratch: residual norms^2 (-1 once pivoted), last exact norms^2
  double* diagR;    // k: diagonal of S (the Householder betas)
  unsigned* bar;    // 1 counter, zeroed by the launcher
  int* d_info;
  int tpc;          // set by the launcher: threads per column (FP64 kernel)
  int nrm_local;    // set by the launcher: residual norms in shared memory (double-float kernel)
  long long spin_limit;  // set by the launcher: bound of each grid-barrier wait (SM clocks)
  int withhold;     // set by the launcher: CTA 0 skips its first arrival (test aid)
  // Tolerance mode (Sec. 2.6): with tol2 > 0 the factorisation stops before
  // step j >= 1 once the sum of the residual column norms^2, ||S22(j)||_F^2,
  // is below tol2 (at the latest after k steps); *k_out (device) receives the
  // number of steps taken.  psum: 2 * 1024 doubles of per-CTA partial sums.
  double tol2;
  int* k_out;
  double* psum;
};
cudaError_t launch_cpqr(const CpqrArgs& a, int* grid_out, cudaStream_t s);
// Double-float arithmetic on the same working area reinterpreted as two float
// planes, hi then lo, each r x n COLUMN-major (ld r); used for sketches of
// FP32 data, r <= 1024.
cudaError_t launch_cpqr_df(const CpqrArgs& a, int* grid_out, cudaStream_t s);
// S11 as k x k float2 pairs followed by k float2 reciprocals of its diagonal
// (S11 must hold k*k + k doubles), S12 as k x (n-k) float2 pairs.
cudaError_t launch_id_extract_df(int r, int64_t n, int k, const double* W, const int32_t* J,
                                 const double* diagR, double* S11, double* S12, cudaStream_t s);
// Back substitution S11 x = rhs for ncols right-hand sides in double-float
// (kk <= 1024; S11 in the layout written by launch_id_extract_df or
// launch_upper_to_df); rhs(i, c) = rhs[i*rs_i + c*rs_c] (float2 pairs or
// floats), out(i, c) = out[i*os_i + c*os_c].
template <typename TR, typename TO>
cudaError_t launch_upper_solve_df(int kk, int64_t ncols, const double* S11, const TR* rhs,
                                  int64_t rs_i, int64_t rs_c, TO* out, int64_t os_i,
                                  int64_t os_c, int* d_info, cudaStream_t s);
// Upper-triangular R (R(i, t) = R[i*ldr + t]) into that layout (kk*kk + kk
// float2 in S11).
template <typename T>
cudaError_t launch_upper_to_df(int kk, const T* R, int64_t ldr, double* S11, cudaStream_t s);
size_t cpqr_scratch_bytes(int64_t n);
// Largest triangle the many-right-hand-side solve handles (one 32-thread block
// of kk doubles each in 220 KB of shared memory).
constexpr int UPPER_SOLVE_MAX_K = 880;
// Upper-triangular solve for many right-hand sides:
//   for c < ncols: U x = rhs(:, c), out(:, c) = x; U(i, t) = Ug[i*us_i + t*us_t].
template <typename TR, typename TO>
cudaError_t launch_upper_solve(int kk, int64_t ncols, const double* Ug, int64_t us_i,
                               int64_t us_t, const TR* rhs, int64_t rs_i, int64_t rs_c,
                               TO* out, int64_t os_i, int64_t os_c, int* d_info,
                               cudaStream_t s);
// S11 (k x k, column-major dense) and S12 columns from the CPQR working array.
cudaError_t launch_id_extract(int r, int64_t n, int k, const double* W, const int32_t* J,
                              const double* diagR, double* S11, double* S12, cudaStream_t s);

// ----- tcgen05 tensor-core GEMMs (k_tc.cu) ---------------------------------
struct TcGemm {
  int form;             // 0: Y = A W (A rows x K), 1: Z = A^T W (A K x rows)
  int omega;            // form 0 only: W = Omega(seed) generated in-kernel
  uint64_t seed;
  int64_t rows;         // output rows (M): rows of A (form 0) or columns of A (form 1)
  int64_t K;            // contraction length
  int L;                // output columns (multiple of 16; above 256 launch_tc_gemm runs
                        // column chunks of at most 256)
  int lvalid;           // Omega columns >= lvalid are zero
  int col0;             // Omega: global index of output column 0 (a multiple of 4; the
                        // column chunks of L > 256 start at 256, 512, ..)
  const float* A;       // source, row-major, 16-byte aligned rows: fp32 (lda % 4 == 0) or,
                        // with a_bf16, bf16 values (lda % 8 == 0) behind this pointer
  int64_t lda;          // elements
  int a_bf16;           // A holds bf16: one product per W term (a0 exact), half the bytes
  int64_t a_rows_total; // rows of the A tensor (form 0: rows, form 1: K)
  int64_t a_cols_total; // cols of the A tensor (form 0: K, form 1: rows)
  int wterms;           // stored W: 1 (hi: one product a0 w0), 2 (hi, lo) or 3 (hi, mid, lo)
  int gram;             // form 1 with W = split of A itself: adds the lo*lo product
  const void* Whi;      // L x K bf16 (K contiguous): leading term of W^T (stored W only)
  const void* Wlo;      // second term
  const void* Wlo2;     // third term (wterms == 3)
  int64_t ldw;          // elements, multiple of 8
  float* part;          // stream-K partial tiles (workspace, tc_part_bytes)
  float* out;           // fp32 output rows x ncols (ld ldo)
  int64_t ldo;
  int ncols;
  void* out_hi;         // optional: bf16 hi/lo of out^T (L x rows, ld ldt); padding zero
  void* out_lo;
  int64_t ldt;
  const int* skip;      // when non-null and *skip == 1 the launch does nothing
  int* d_info;
  int drain;            // stored-operand passes: K-chunks per TMEM accumulation run
                        // (0 = one run per stream-K segment); see tc_unit_kernel
  int q8;               // form 0, one stored W term: every 32-value K-chunk of each A
                        // row quantised to E4M3 with its power-of-two scale (fp8.cuh)
                        // before the product (the FP8 sketch; W = its quantised Omega^T)
};
size_t tc_part_bytes(int64_t rows, int64_t K, int L);
cudaError_t launch_tc_gemm(const TcGemm& g, cudaStream_t s);
// Y = A Omega with two M-tiles per CTA sharing each generated Omega stage
// (k_omega.cu); called by launch_tc_gemm for form 0 with omega set.
cudaError_t launch_tc_omega(const TcGemm& g, cudaStream_t s);
// Stored-operand GEMMs (wterms 1 or 2, no Gram) on 256-row units, two M-tiles
// per CTA sharing each W stage (k_tc2.cu); called by launch_tc_gemm.
bool tc_unit_supported(const TcGemm& g);
cudaError_t launch_tc_unit(const TcGemm& g, cudaStream_t s);
bool tc_supported(int L);
int device_sm_count();

// ----- batched problems (k_batched.cu, k_chol.cu, k_jacobi.cu) -------------
// One GEMM of a batch: C (M x N, ld ldc) = op(A) W with op(A) = A (M x K, ld
// lda) or, with transA, A^T for A stored K x M (ld lda); W is K x N (ld ldw)
// or, when null, the Omega of problem `batch` (bf16-rounded Gaussians, Philox
// counter (row, column / 4, 0, batch)).  Only the first ncol columns are
// written.
struct BGemm {
  const float* A;
  int64_t lda;
  const float* W;
  int64_t ldw;
  float* C;
  int64_t ldc;
  int M, N, K, ncol;
  int transA;
  int batch;
};
// tasks: (gemm index, first output row), one CTA each, all of one block height
// `rows` = bgemm_rows(N) of their GEMMs (64, 128 or 256)
cudaError_t launch_bgemm(const BGemm* gemms, const int2* tasks, int ntasks, int rows,
                         uint64_t seed, cudaStream_t s);
int bgemm_rows(int N);
constexpr int BATCH_LMAX = 128;     // largest sketch width of the batched path
// Cholesky R^T R = G and R^-1 of one l x l Gram per CTA (the shifted CholeskyQR
// factorisation of chol_kernel); R, Rinv l x l (ld l)
struct BChol {
  const float* G;
  float* R;
  float* Rinv;
  int l;
};
cudaError_t launch_chol_batched(const BChol* tasks, int batch, int lmax, int* d_info,
                                cudaStream_t s);
// out[e] = sum_{s < nslice} part[s * count + e] (fixed order), one CTA per problem
struct BSum {
  const float* part;
  float* out;
  int nslice;
  int count;
};
cudaError_t launch_sum_batched(const BSum* tasks, int batch, cudaStream_t s);
// Racc <- R Racc (upper triangular l x l) per problem, through tmp
struct BTrmm {
  const float* R;
  float* Racc;
  float* tmp;
  int l;
};
cudaError_t launch_trmm_batched(const BTrmm* tasks, int batch, cudaStream_t s);
// SVD of one l x l core M per CTA: M = Uh diag(Sh) Vh^T (Jacobi for the left
// vectors, sigma_j = ||M^T u_j||, sorted descending); Uj is working storage
struct BSvd {
  const float* M;
  float* Uj;
  float* Uh;
  float* Vh;
  double* Sh;
  int l;
};
cudaError_t launch_small_svd_batched(const BSvd* tasks, int batch, int lmax, int max_sweeps,
                                     int* d_info, cudaStream_t s);
// Sign rule per problem (largest |entry| of each v_j positive, lowest index on
// ties) applied to U (m x k) and V (n x k), and S[0:k] = Sh[0:k]
struct BSign {
  float* U;
  float* V;
  double* S;
  const double* Sh;
  int64_t m, n;
  int k;
};
cudaError_t launch_sign_batched(const BSign* tasks, int batch, cudaStream_t s);

// ----- grouped tensor-core passes of the batched path (k_tc_group.cu) -----
constexpr int TG_NMAX = 128;      // widest MMA N: round_up(l, 16) <= BATCH_LMAX
// One problem of a grouped pass: C (M x ncol, ld ldc) = A W (form 0) or A^T W
// (form 1); A and the bf16 terms of W^T through the launch's tensor maps.
struct TgProb {
  float* C;
  int64_t ldc;
  int M;          // output rows
  int K;          // contraction length
  int ncol;       // output columns (l)
  int N;          // MMA width, round_up(l, 16) <= TG_NMAX
};
struct TgTask {   // one 128-row output tile of one problem
  int prob, r0;
};
struct TgPad {    // rows x cols fp32 copied from pitch lds to pitch ldd
  const float* src;
  float* dst;
  int64_t rows, cols, lds, ldd;
};
struct TgSplit {  // W (rows x l, ld ldw) -> bf16 hi / lo (/ lo2) of W^T (N x ldt); Omega^T: W = null
  const float* W;
  int64_t ldw;
  uint16_t* hi;
  uint16_t* lo;
  uint16_t* lo2;  // third term (R^-1), or null
  int64_t rows, ldt;
  int l, N, batch;
};
// Tensor maps of one problem (A, then up to three bf16 terms of W^T) for form
// 0 / 1; A with pitch ldap (a multiple of 4), W^T with pitch ldt (a multiple of 8).
bool tg_encode_maps(int form, int nwt, const float* Ap, int64_t m, int64_t n, int64_t ldap,
                    const void* whi, const void* wlo, const void* wlo2, int64_t K, int N,
                    int64_t ldt, CUtensorMap out[4]);
// nwt: 1 = one bf16 term of W (Omega, bf16-exact), 2 = hi and lo, 3 = R^-1's
// three terms; gram: W is A itself (nwt 2, the a1 w1 product kept).
// maps: 4 per problem, 64-byte aligned, in device memory.
cudaError_t launch_tc_group(int form, int nwt, bool gram, const TgProb* probs,
                            const TgTask* tasks, int ntasks, const CUtensorMap* maps, int* d_info,
                            cudaStream_t s);
// chunks: (job, first row), 32 rows each
cudaError_t launch_pad_rows_batched(const TgPad* jobs, const int2* chunks, int nchunks,
                                    cudaStream_t s);
cudaError_t launch_split_t_batched(const TgSplit* jobs, const int2* chunks, int nchunks,
                                   cudaStream_t s);
cudaError_t launch_omega_t_batched(const TgSplit* jobs, const int2* chunks, int nchunks,
                                   uint64_t seed, cudaStream_t s);

// ----- adjoint of Alg. 5 (k_vjp.cu) ---------------------------------------
// X (L x L) = diag(gs) + (F o (Gu - Gu^T)) diag(s) + diag(s) (F o (Gv - Gv^T)),
// F_ij = 1 / (s_j^2 - s_i^2), on the leading l x l block (gs: k entries, may
// be null); zero padding.
template <typename T>
cudaError_t launch_svd_vjp_core(int l, int L, int k, const double* s, const double* gs,
                                const T* Gu, const T* Gv, int64_t ldg, T* X, int64_t ldx,
                                cudaStream_t st);
// out (L x L) = sym(P1 - P2): upper triangle of M = P1 - P2 mirrored below
// (P1 may be null); zero padding.
template <typename T>
cudaError_t launch_sym_upper(int l, int L, const T* P1, const T* P2, int64_t ldp, T* out,
                             int64_t ldo, cudaStream_t st);
// dst(:, 0:cols) = scale * src(:, 0:cols), columns with signs[j] < 0 negated
// once more (signs may be null).
template <typename T>
cudaError_t launch_pack_cols(int64_t rows, int cols, const T* src, int64_t lds, T* dst,
                             int64_t ldd, T scale, const int* signs, cudaStream_t st);

// ----- blocked adaptive QB (k_adaptive.cu) --------------------------------
// X (rows x cols, ld ldx) <- X - Q Bt^T with Q rows x K (ld ldq) and Bt cols x K
// (ld ldb); K = 0 leaves X unwritten.  With sumsq set, sumsq[t] (t <
// rank_update_tiles(rows, cols)) receives the sum of squares of the updated
// entries of tile t.
int64_t rank_update_tiles(int64_t rows, int64_t cols);
template <typename T>
cudaError_t launch_rank_update(int64_t rows, int64_t cols, T* X, int64_t ldx, const T* Q,
                               int64_t ldq, const T* Bt, int64_t ldb, int K, double* sumsq,
                               cudaStream_t s);
// *out = sqrt(sum_t parts[t]) in a fixed order; non-finite -> RSVD_ERR_NUMERIC.
cudaError_t launch_sumsq_finish(int64_t nparts, const double* parts, double* out, int* d_info,
                                cudaStream_t s);

}  // namespace rsvd
