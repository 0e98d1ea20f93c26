/*
 * rsvd.h - C ABI of the GB300 (sm_103a) randomized QB / RSVD / ID / CUR library.
 *
 * The operations are those of Voronin & Martinsson, "RSVDPACK: an implementation
 * of randomized algorithms for computing the singular value, interpolative, and
 * CUR decompositions of matrices on multi-core and GPU architectures":
 *   - randomized range finder with the power scheme (Fig. 1 steps 1-3, Sec. 3.2,
 *     Alg. 5 first part),
 *   - the QB step B = Q^* A (Fig. 1 step 4; realised as Bt = A^* Q as in Alg. 5),
 *   - the small SVD of B through the QR of Bt (Alg. 5, "RSVD version II"),
 *   - the randomized ID from B (Sec. 3.5, last part; Sec. 2.4; Alg. 1),
 *   - the CUR through the two-sided ID (Sec. 2.5, Sec. 3.6; Alg. 2 and 3).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Matrices are dense and ROW-MAJOR: element (i, j) of an r x c matrix X with
 * leading dimension ldx sits at X[i*ldx + j], ldx >= c.  Indices are 0-based.
 * l = k + p is the sketch width.  "dtype" is an rsvd_dtype naming the element
 * type of A; floating outputs have the same type as A for RSVD_F64 (double) and
 * are float for RSVD_F32 and RSVD_BF16.  Singular values are always double.
 *
 * RSVD_BF16 (A stored as bf16, the mixed-precision path): accepted by the
 * whole-path calls (rsvd_qb, rsvd_svd, rsvd_id, rsvd_cur, rsvd_svd_id_cur,
 * rsvd_svd_id_cur_host) and by rsvd_sample / rsvd_apply, on the tensor-core
 * path only: A 16-byte aligned with lda % 8 == 0, precision RSVD_PREC_TC or
 * RSVD_PREC_MIXED,
 * l rounded up to 16 <= 1024; otherwise RSVD_ERR_UNSUPPORTED.  The bf16 values of A are
 * exact tensor-core operands: each pass over A issues one product per term of
 * its right-hand operand and reads 2 bytes per entry.  All other arithmetic
 * (Gram, CholeskyQR, small SVD, pivoted QR, solves) is the FP32 path's.
 *
 * Ownership: every pointer is caller-owned DEVICE memory on the current CUDA
 * device, except `opts` (host memory, may be NULL for defaults).  The library
 * allocates nothing, never synchronises the host with the device, and enqueues
 * all work on `stream` (a cudaStream_t; NULL = legacy default stream).  Scratch
 * space is the caller's `work` buffer of `work_bytes` bytes, 256-byte aligned,
 * sized by the matching *_workspace_size() query; its contents on entry do not
 * matter and on exit are undefined.
 *
 * Errors: argument errors are reported synchronously by the return value and
 * nothing is launched (RSVD_ERR_INVALID_ARG, RSVD_ERR_WORKSPACE,
 * RSVD_ERR_UNSUPPORTED); a failed launch returns RSVD_ERR_CUDA.  Numerical
 * failures detected on the device (Cholesky breakdown, Jacobi non-convergence,
 * non-finite values, a bounded wait that ran out) are written, as an
 * rsvd_status value, into the caller's device integer *d_info, which the call
 * first resets to 0 in stream order; outputs are then unspecified.  d_info may
 * be NULL when the caller does not want the code.
 *
 * Randomness: Omega is never stored.  Its entries are Gaussian samples
 * generated inside the kernels from the Philox4x32-10 counter stream (Salmon et
 * al., SC'11) keyed by `seed`, with counter (row i, column j / 4, tag 0, 0) and
 * the Box-Muller transform on words (x0,x1) -> columns 4q, 4q+1 and (x2,x3) ->
 * 4q+2, 4q+3, uniforms u = (2*(x >> 9) + 1) * 2^-24.  For RSVD_F64 inputs the
 * samples are computed in double; for RSVD_F32 inputs in float and rounded to
 * bf16 (nearest even), so the tensor cores consume them exactly.  Results are
 * reproducible for a given seed, sizes and GPU.
 */
#ifndef RSVD_H
#define RSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RSVD_OK = 0,
  RSVD_ERR_INVALID_ARG = 1,    /* bad size, leading dimension, pointer or option  */
  RSVD_ERR_WORKSPACE = 2,      /* work_bytes below the *_workspace_size() value    */
  RSVD_ERR_CUDA = 3,           /* a CUDA runtime/driver call or launch failed       */
  RSVD_ERR_UNSUPPORTED = 4,    /* valid request outside what this build implements  */
  RSVD_ERR_NOT_SPD = 5,        /* device: Gram matrix not positive definite         */
  RSVD_ERR_NO_CONVERGENCE = 6, /* device: Jacobi SVD exceeded max_sweeps            */
  RSVD_ERR_NUMERIC = 7,        /* device: NaN or Inf met                            */
  RSVD_ERR_TIMEOUT = 8         /* device: a bounded wait ran out                    */
} rsvd_status;

typedef enum { RSVD_F32 = 0, RSVD_F64 = 1, RSVD_BF16 = 2 } rsvd_dtype;

typedef enum {
  RSVD_PREC_TC = 0,   /* FP32 inputs: tcgen05 tensor-core products of bf16 splits
                         (two-term split of each fp32 operand, fp32 accumulation) */
  RSVD_PREC_SIMT = 1, /* FP32 inputs: plain fp32 FMA kernels (slower; cross-check) */
  RSVD_PREC_MIXED = 2,/* FP32 or BF16 inputs, tensor cores: the passes of the power
                         scheme (Z = A^T Y, Y = A Z) take one bf16 term of A and of the
                         stored operand, one product per K-step; the sketch
                         Y = A Omega, the orthonormalisations and Bt = A^T Q keep the
                         RSVD_PREC_TC arithmetic (the subspace iteration tolerates
                         bf16 rounding, the projection onto it does not) */
  RSVD_PREC_FP8 = 3   /* FP32 or BF16 inputs, tensor cores: the sketch Y = A Omega
                         takes A and Omega quantised to FP8 E4M3 (round to nearest
                         even, saturating at 448) with one power-of-two scale per
                         block of 32 entries along the contraction, 2^ceil(log2(
                         amax / 448)) (the block-scaled 8-bit format); a scaled
                         E4M3 value is exact in bf16, so the products run as bf16
                         tensor-core products with fp32 accumulation and give the
                         FP8 sketch's values.  Omega is rounded to bf16 before its
                         quantisation (as on the FP32 path) and its quantised
                         transpose is generated once per call into the workspace.
                         Every other product as RSVD_PREC_TC. */
} rsvd_precision;

/* Options.  Pass NULL for the defaults set by rsvd_opts_default(). */
typedef struct {
  int s;           /* orthonormalisation frequency of the power scheme (Alg. 5):
                      orth before the product number t (t = 0, 1, ...) when
                      t mod s == 0; default 1 (orth before every product)        */
  int max_sweeps;  /* sweep limit of the one-sided Jacobi SVD; default 30        */
  int precision;   /* rsvd_precision; default RSVD_PREC_TC                        */
  int reserved[13];/* must be zero                                                */
} rsvd_opts;

/* Fills *opts with the defaults.  Host only. */
void rsvd_opts_default(rsvd_opts* opts);

/* Static string naming a status code.  Host only. */
const char* rsvd_status_string(int status);

/* Library version (major*10000 + minor*100 + patch). */
int rsvd_version(void);

/* -------------------------------------------------------------------------
 * Workspace queries.  Return the byte count the matching call needs, or 0
 * when the arguments are invalid or outside the call's supported sizes (the
 * call itself then returns RSVD_ERR_INVALID_ARG or RSVD_ERR_UNSUPPORTED).
 * Host only; nothing is launched.
 * ------------------------------------------------------------------------- */
size_t rsvd_qb_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                              const rsvd_opts* opts);
size_t rsvd_svd_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                               const rsvd_opts* opts);
size_t rsvd_id_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                              const rsvd_opts* opts);
size_t rsvd_cur_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                               const rsvd_opts* opts);
size_t rsvd_svd_id_cur_workspace_size(int64_t m, int64_t n, int k, int p, int q,
                                      int dtype, const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_qb - randomized range finder and QB step (Alg. 5 up to Bt = A^* Q;
 * Fig. 1 steps 1-4; power scheme of Sec. 3.2).
 *   Y = A Omega; for j = 1..q: Y <- orth(Y), Z = A^* Y, Z <- orth(Z), Y = A Z
 *   (orth placement by opts->s); Q = orth(Y); Bt = A^* Q.
 * In:  A  m x n (dtype), lda >= n; 1 <= k, p >= 0, l = k+p <= min(m, n), q >= 0.
 * Out: Q  m x l, orthonormal columns (ldq >= l);
 *      Bt n x l = B^* with B = Q^* A (ldbt >= l).
 * orth is an unpivoted QR whose Q is unique by diag(R) > 0 (CholeskyQR with
 * an adaptive shift and two or three passes).
 * ------------------------------------------------------------------------- */
rsvd_status rsvd_qb(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                    const void* A, int64_t lda, void* Q, int64_t ldq, void* Bt,
                    int64_t ldbt, void* work, size_t work_bytes, int* d_info,
                    void* stream, const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_svd - rank-k approximate SVD A ~ U diag(S) V^T by Alg. 5 (RSVD version
 * II, Sec. 3.4): QB step, [Qh, Rh] = qr(Bt), Rh = Uh Sigma Vh^T (one-sided
 * Jacobi), U = Q Vh(:, 1:k), V = Qh Uh(:, 1:k).
 * Out: U m x k (ldu >= k), S k singular values in descending order (double),
 *      V n x k (ldv >= k).  Each pair (u_j, v_j) is signed so that the entry of
 *      largest magnitude of v_j is positive (ties: lowest row index).
 * ------------------------------------------------------------------------- */
rsvd_status rsvd_svd(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                     const void* A, int64_t lda, void* U, int64_t ldu, double* S,
                     void* V, int64_t ldv, void* work, size_t work_bytes, int* d_info,
                     void* stream, const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_id - rank-k column interpolative decomposition through the QB step
 * (Sec. 3.5, last part): k steps of column-pivoted Householder QR (pivot =
 * largest residual column norm, ties to the lowest column index, LAPACK-style
 * exchanges) of B = Bt^T (l x n), T = S11^{-1} S12 by back substitution.  The
 * arithmetic is FP64 for RSVD_F64 A and double-float (hi + lo float pairs,
 * about 48 significant bits, compensated dot products) for RSVD_F32 and
 * RSVD_BF16 A, with the reflector scalars in FP64.
 * Out: J  n int32, the column permutation; J[0:k] is the skeleton;
 *      T  k x (n-k) (ldt >= n-k): A(:, J[k+c]) ~ sum_i A(:, J[i]) T[i][c].
 * Sizes: k < n and k <= 880 (the triangular solve for T holds 32 right-hand
 * sides of k doubles in one CTA's shared memory); a larger k returns
 * RSVD_ERR_UNSUPPORTED.  The same
 * bound holds for every call that forms an ID or a CUR (rsvd_cur,
 * rsvd_svd_id_cur, the tolerance calls' kmax, rsvd_id_left, rsvd_cpqr_id*).
 * ------------------------------------------------------------------------- */
rsvd_status rsvd_id(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                    const void* A, int64_t lda, int32_t* J, void* T, int64_t ldt,
                    void* work, size_t work_bytes, int* d_info, void* stream,
                    const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * Tolerance mode (Sec. 2.6; Sec. 4, "TOL"): the rank is chosen from the
 * result instead of fixed in advance.  The sketch is built with
 * l = kmax + p columns; the host learns the rank through one synchronisation
 * with `stream`, so these three calls cannot be captured in a CUDA graph.
 * `rank` is HOST memory.  tol must be positive and finite.
 *
 * rsvd_svd_tol - rsvd_svd with k = kmax, then *rank = the number of computed
 *   singular values above tol (at least 1): sigma_{rank+1} <= tol.  U, S, V
 *   are written for all kmax columns; the first *rank form the result.
 *   Workspace: rsvd_svd_workspace_size(m, n, kmax, p, q, dtype, opts).
 *
 * rsvd_id_tol - rsvd_id whose pivoted QR of B (l x n) stops before step
 *   j >= 1 as soon as ||S22(j)||_F < tol (the Frobenius norm of the
 *   residual block, i.e. the root of the sum of the residual column norms^2
 *   that the pivoting tracks), at the latest after kmax steps; *rank = the
 *   number of steps taken, and J, T are the ID of that rank (T is
 *   rank x (n - rank), ldt >= n - 1).  1 <= kmax < n.
 *
 * rsvd_cur_tol - rsvd_cur on the column ID of rsvd_id_tol: the row ID of
 *   C = A(:, Jc) takes *rank steps.  Jc, Ir hold kmax entries and U kmax x kmax
 *   (ldu >= kmax); the first *rank (rows and columns) are written.
 *   kmax < min(m, n).
 *
 * Errors as rsvd_id / rsvd_cur; a device failure recorded in *d_info (the
 * call has synchronised, so it can be read at once) leaves *rank = 0 for the
 * ID and CUR calls.
 * ------------------------------------------------------------------------- */
size_t rsvd_id_tol_workspace_size(int64_t m, int64_t n, int kmax, int p, int q, int dtype,
                                  const rsvd_opts* opts);
size_t rsvd_cur_tol_workspace_size(int64_t m, int64_t n, int kmax, int p, int q, int dtype,
                                   const rsvd_opts* opts);
rsvd_status rsvd_svd_tol(int64_t m, int64_t n, int kmax, int p, int q, double tol, uint64_t seed,
                         int dtype, const void* A, int64_t lda, void* U, int64_t ldu, double* S,
                         void* V, int64_t ldv, int* rank, void* work, size_t work_bytes,
                         int* d_info, void* stream, const rsvd_opts* opts);
rsvd_status rsvd_id_tol(int64_t m, int64_t n, int kmax, int p, int q, double tol, uint64_t seed,
                        int dtype, const void* A, int64_t lda, int32_t* J, void* T, int64_t ldt,
                        int* rank, void* work, size_t work_bytes, int* d_info, void* stream,
                        const rsvd_opts* opts);
rsvd_status rsvd_cur_tol(int64_t m, int64_t n, int kmax, int p, int q, double tol, uint64_t seed,
                         int dtype, const void* A, int64_t lda, int32_t* Jc, int32_t* Ir, void* U,
                         int64_t ldu, int* rank, void* work, size_t work_bytes, int* d_info,
                         void* stream, const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_id_left - rank-k column ID from the LEFT sketch (Sec. 3.5, Alg. 6):
 *   Y = Omega~ A (A^* A)^q, Omega~ l x m Gaussian (l = k + p), orthonormalised
 *   before every product (Y <- (A orth(Y^*))^*, then (A^* orth(Y^*))^*; the
 *   s option is not used), then k steps of the pivoted QR of Y (l x n) as in
 *   rsvd_id and T = S11^{-1} S12.  Omega~^* is the Philox stream of `seed`
 *   with counter (row i < m, column j / 4, tag 1, 0), values as for Omega.
 *   It is generated once into the workspace (m x l), not re-drawn per tile.
 * Out: J n int32 (J[0:k] skeleton); T k x (n-k) (ldt >= n-k).
 * ------------------------------------------------------------------------- */
size_t rsvd_id_left_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                                   const rsvd_opts* opts);
rsvd_status rsvd_id_left(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                         const void* A, int64_t lda, int32_t* J, void* T, int64_t ldt, void* work,
                         size_t work_bytes, int* d_info, void* stream, const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_cur - rank-k CUR A ~ A(:, Jc) U A(Ir, :) (Sec. 3.6; Alg. 2, 3): the
 * randomized ID above, then a k-step pivoted QR of C^* with C = A(:, Jc)
 * (row ID), R = A(Ir, :), and U = V^* R^dagger with R^dagger = Q_R R_R^{-T}
 * from the QR of R^*.
 * Out: Jc k int32, Ir k int32, U k x k (ldu >= k).
 * ------------------------------------------------------------------------- */
rsvd_status rsvd_cur(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                     const void* A, int64_t lda, int32_t* Jc, int32_t* Ir, void* U,
                     int64_t ldu, void* work, size_t work_bytes, int* d_info,
                     void* stream, const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_svd_id_cur - RSVD, ID and CUR from ONE sketch: one QB step feeds the
 * small SVD (as rsvd_svd), the ID (as rsvd_id) and the CUR (as rsvd_cur).
 * Any output group may be skipped by passing NULL for all its pointers
 * (U,S,V | J,T | Jc,Ir,Ucur).  Outputs as in the three calls above.
 * ------------------------------------------------------------------------- */
rsvd_status rsvd_svd_id_cur(int64_t m, int64_t n, int k, int p, int q, uint64_t seed,
                            int dtype, const void* A, int64_t lda,
                            void* U, int64_t ldu, double* S, void* V, int64_t ldv,
                            int32_t* J, void* T, int64_t ldt,
                            int32_t* Jc, int32_t* Ir, void* Ucur, int64_t lducur,
                            void* work, size_t work_bytes, int* d_info, void* stream,
                            const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_svd_id_cur_host - rsvd_svd_id_cur with A in host memory.
 * A_host (m x lda, same layout as A; page-locked for the copy to overlap) is
 * copied into the caller's device buffer A, which holds A on return.  On the
 * tensor-core path the copy runs in row chunks on an auxiliary stream and the
 * sketch Y = A Omega (Fig. 1 step 2; its rows are independent) processes each
 * chunk as it lands; the later passes need all of A.  Workspace size as
 * rsvd_svd_id_cur_workspace_size.  Outputs and errors as rsvd_svd_id_cur;
 * RSVD_ERR_INVALID_ARG when A_host is NULL.
 * ------------------------------------------------------------------------- */
rsvd_status rsvd_svd_id_cur_host(int64_t m, int64_t n, int k, int p, int q, uint64_t seed,
                                 int dtype, const void* A_host, void* A, int64_t lda,
                                 void* U, int64_t ldu, double* S, void* V, int64_t ldv,
                                 int32_t* J, void* T, int64_t ldt,
                                 int32_t* Jc, int32_t* Ir, void* Ucur, int64_t lducur,
                                 void* work, size_t work_bytes, int* d_info, void* stream,
                                 const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_qb_adaptive - blocked randomized QB to a tolerance (Alg. 7, "QB2";
 * Sec. 3.3; the rank is not fixed in advance, Sec. 2.6 / Sec. 4 "TOL" mode).
 *
 * Block t = 0, 1, ... of b columns:
 *   Omega_t (n x b) from the Philox stream keyed by seed + t (counters as for
 *     Omega above);
 *   Q_t = orth of the range finder with q power iterations (and the s of
 *     opts) applied to the CURRENT A;
 *   Q_t <- orth(Q_t - Qbar Qbar^* Q_t), Qbar = [Q_0 .. Q_{t-1}];
 *   B_t = Q_t^* A, stored as Bt_t = A^* Q_t (n x b);
 *   A <- A - Q_t B_t, then resid[t+1] = ||A||_F.
 * The loop stops after the first block with resid[t+1] < tol, tol = eps
 * (relative == 0) or eps * ||A_in||_F (relative != 0), or after M blocks, or
 * when a device failure was recorded in *d_info.  The paper's ||A|| is read as
 * the Frobenius norm.
 *
 * dtype: RSVD_F32 (tensor-core or SIMT path as for rsvd_qb; RSVD_PREC_MIXED
 *        applies to the power scheme) or RSVD_F64; RSVD_BF16 gives
 *        RSVD_ERR_UNSUPPORTED (A is updated in its own storage type).
 * A:     m x n (lda >= n), device, READ AND OVERWRITTEN: on return it holds the
 *        residual A_in - Q B of the blocks computed.  Pass a copy to keep A.
 * Q:     m x (b M) capacity (ldq >= b M); columns [0, *rank) receive Qbar,
 *        orthonormal.  Bt: n x (b M) capacity (ldbt >= b M); columns
 *        [0, *rank) receive B^* = A_in^* Qbar.  Other columns are not written.
 * resid: device double[M + 1]: resid[0] = ||A_in||_F, resid[t] = ||A||_F after
 *        block t; entries past *rank / b are not written.
 * rank:  HOST int, set to b times the number of blocks computed.
 * Sizes: 1 <= b <= 1024, M >= 1, b M <= min(m, n), 0 <= q <= 64, eps >= 0.
 * Errors: as the other calls (RSVD_ERR_INVALID_ARG, RSVD_ERR_WORKSPACE with
 * nothing launched); device failures in *d_info.
 * Unlike every other call, this one SYNCHRONISES the host with `stream` once
 * per block (and once more for a relative tolerance): the stopping test reads
 * the residual norm on the host, so the call cannot be captured in a CUDA
 * graph.
 * ------------------------------------------------------------------------- */
size_t rsvd_qb_adaptive_workspace_size(int64_t m, int64_t n, int b, int M, int q, int dtype,
                                       const rsvd_opts* opts);
rsvd_status rsvd_qb_adaptive(int64_t m, int64_t n, int b, int M, int q, double eps,
                             int relative, uint64_t seed, int dtype, void* A, int64_t lda,
                             void* Q, int64_t ldq, void* Bt, int64_t ldbt, double* resid,
                             int* rank, void* work, size_t work_bytes, int* d_info,
                             void* stream, const rsvd_opts* opts);

/* -------------------------------------------------------------------------
 * rsvd_svd_vjp - reverse-mode derivative of rsvd_svd (Alg. 5 with the orth of
 * every power step, s = 1) with Omega held fixed and the sign rule treated as
 * constant: given the cotangents gU (m x k), gS (k doubles) and gV (n x k) of
 * the outputs U, S, V, writes gA (m x n, ldga >= n) = the cotangent of A.
 * Nothing needs to be kept from the forward call: this call replays the
 * forward path from A and `seed` (every orthonormalisation a full CholeskyQR,
 * so each Q is orthonormal to working precision) and keeps its factors in the
 * workspace, then applies the adjoints in reverse order: of the products with
 * A and A^*, of the thin QR X = Q R (diag(R) > 0), and of the square SVD of
 * R-hat with its 1 / (s_j^2 - s_i^2) coupling (distinct singular values; equal
 * ones contribute nothing).  U (m x k), S (k) and V (n x k) receive the
 * replayed forward outputs when non-NULL.
 * dtype: RSVD_F32 (tensor-core or SIMT path as rsvd_svd) or RSVD_F64;
 * RSVD_BF16 gives RSVD_ERR_UNSUPPORTED.  gU, gS, gV must be non-NULL (pass
 * zeros for an output the loss does not use).
 * ------------------------------------------------------------------------- */
size_t rsvd_svd_vjp_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                                   const rsvd_opts* opts);
rsvd_status rsvd_svd_vjp(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                         const void* A, int64_t lda, const void* gU, int64_t ldgu,
                         const double* gS, const void* gV, int64_t ldgv, void* gA, int64_t ldga,
                         void* U, int64_t ldu, double* S, void* V, int64_t ldv, void* work,
                         size_t work_bytes, int* d_info, void* stream, const rsvd_opts* opts);

/* =========================================================================
 * Step-level entry points (one per step of the path; same conventions).
 * ========================================================================= */

/* Omega itself, n x l (ldo >= l), exactly as the sketch kernels generate it
 * (Fig. 1 step 1): double for RSVD_F64, float holding bf16 values for RSVD_F32.
 * Intended for checking the stream; the path never stores Omega. */
rsvd_status rsvd_omega(int64_t n, int l, uint64_t seed, int dtype, void* Omega,
                       int64_t ldo, void* stream);

/* Omega of the FP8 sketch (RSVD_PREC_FP8), n x l floats (ldo >= l): the bf16
 * Omega of rsvd_omega quantised to E4M3 with one power-of-two scale per block
 * of 32 rows of each column, times that scale, exactly as the sketch uses it.
 * Intended for checking. */
rsvd_status rsvd_omega_fp8(int64_t n, int l, uint64_t seed, float* Omega, int64_t ldo,
                           void* stream);

/* The raw Philox4x32-10 words behind Omega: out is n x ceil(l/4) x 4 uint32,
 * word t of counter (i, q, 0, 0) at out[(i*ceil(l/4) + q)*4 + t]. */
rsvd_status rsvd_omega_words(int64_t n, int l, uint64_t seed, uint32_t* out,
                             void* stream);

size_t rsvd_sample_workspace_size(int64_t m, int64_t n, int l, int dtype,
                                  const rsvd_opts* opts);
/* Sample matrix Y = A Omega (Fig. 1 step 2), Y m x l (ldy >= l). */
rsvd_status rsvd_sample(int64_t m, int64_t n, int l, uint64_t seed, int dtype,
                        const void* A, int64_t lda, void* Y, int64_t ldy, void* work,
                        size_t work_bytes, void* stream, const rsvd_opts* opts);

size_t rsvd_apply_workspace_size(int64_t m, int64_t n, int l, int dtype,
                                 const rsvd_opts* opts);
/* Power-scheme half steps (Sec. 3.2):
 *   trans = 0: Y = A X with X n x l (ldx >= l), Y m x l (ldy >= l);
 *   trans = 1: Y = A^* X with X m x l, Y n x l.
 * X and Y have A's floating type (float for RSVD_F32). */
rsvd_status rsvd_apply(int64_t m, int64_t n, int l, int trans, int dtype, const void* A,
                       int64_t lda, const void* X, int64_t ldx, void* Y, int64_t ldy,
                       void* work, size_t work_bytes, void* stream,
                       const rsvd_opts* opts);

size_t rsvd_orth_workspace_size(int64_t rows, int l, int dtype, const rsvd_opts* opts);
/* orth(X) (Sec. 2.1): X rows x l (rows >= l) -> Q rows x l with orthonormal
 * columns and upper-triangular R (l x l, ldr >= l; may be NULL) with X = Q R,
 * diag(R) > 0.  Q may alias X only when ldq == ldx. */
rsvd_status rsvd_orth(int64_t rows, int l, int dtype, const void* X, int64_t ldx,
                      void* Q, int64_t ldq, void* R, int64_t ldr, void* work,
                      size_t work_bytes, int* d_info, void* stream,
                      const rsvd_opts* opts);

size_t rsvd_small_svd_workspace_size(int l, int dtype, const rsvd_opts* opts);
/* SVD of a small square matrix M (l x l, ldm >= l) by one-sided Jacobi
 * (the core step of Alg. 5): M = Uh diag(Sh) Vh^T with Sh descending.
 * Uh, Vh l x l (ld >= l); Sh l doubles. */
rsvd_status rsvd_small_svd(int l, int dtype, const void* M, int64_t ldm, void* Uh,
                           int64_t lduh, double* Sh, void* Vh, int64_t ldvh, void* work,
                           size_t work_bytes, int* d_info, void* stream,
                           const rsvd_opts* opts);

size_t rsvd_cpqr_workspace_size(int r, int64_t n, int k);
/* Column ID of an explicit matrix (Sec. 2.3, 2.4; Alg. 1): M r x n in double
 * (ldm >= n), k steps of the pivoted QR described at rsvd_id.
 * Out: J n int32; T k x (n-k) double (ldt >= n-k); gaps (may be NULL) k
 * doubles, (nu1 - nu2) / nu1 of the two largest residual norms at each step
 * (+inf when one candidate remains). */
rsvd_status rsvd_cpqr_id(int r, int64_t n, int k, const double* M, int64_t ldm,
                         int32_t* J, double* T, int64_t ldt, double* gaps, void* work,
                         size_t work_bytes, int* d_info, void* stream);

size_t rsvd_cpqr_f32_workspace_size(int r, int64_t n, int k);
/* rsvd_cpqr_id for an FP32 matrix M (r x n floats, ldm >= n), in the
 * arithmetic of the FP32 rsvd_id / rsvd_cur path: the entries are carried as
 * double-float pairs (about 48 significant bits; dot products compensated),
 * residual norms, reflector scalars and the triangular solve in FP64.
 * Out: J n int32; T k x (n-k) float (ldt >= n-k); gaps as rsvd_cpqr_id.
 * Errors as rsvd_cpqr_id. */
rsvd_status rsvd_cpqr_id_f32(int r, int64_t n, int k, const float* M, int64_t ldm,
                             int32_t* J, float* T, int64_t ldt, double* gaps, void* work,
                             size_t work_bytes, int* d_info, void* stream);

/* -------------------------------------------------------------------------
 * rsvd_small_svd_noalloc - rsvd_small_svd without a caller workspace.
 * The paper has no counterpart: this is an interface for callers that cannot
 * allocate device memory or pass a workspace (cudaMalloc/cudaFree synchronise
 * the device, and some host frameworks own the whole device-memory budget).
 * Same arguments and results as rsvd_small_svd minus work/work_bytes.  Its
 * scratch is one static device array of RSVD_NOALLOC_SCRATCH_BYTES per GPU
 * (held until the process exits), shared by all calls: calls that overlap on
 * the GPU race and must be serialised by the caller.  The first call on a
 * device looks up the array's address (make it before any stream capture);
 * the address is kept for the life of the process, so the entry point must not
 * be called on a device after a cudaDeviceReset of that device.
 * Sizes whose scratch need exceeds the array (l above 512 in FP64, about 720
 * in FP32) return RSVD_ERR_WORKSPACE; nothing is allocated.
 * ------------------------------------------------------------------------- */
#define RSVD_NOALLOC_SCRATCH_BYTES (16u << 20)
rsvd_status rsvd_small_svd_noalloc(int l, int dtype, const void* M, int64_t ldm, void* Uh,
                                   int64_t lduh, double* Sh, void* Vh, int64_t ldvh,
                                   int* d_info, void* stream, const rsvd_opts* opts);

/* =========================================================================
 * Tracing aids (host only; not part of the paper's method).
 * ========================================================================= */

/* Kernel classes timed when tracing is enabled. */
enum {
  RSVD_TRACE_A_OMEGA = 0, /* sketch Y = A Omega (tensor cores, Omega in-kernel)      */
  RSVD_TRACE_A_W = 1,     /* power step Y = A Z (tensor cores)                       */
  RSVD_TRACE_AT_W = 2,    /* power step Z = A^T Y and QB step Bt = A^T Q             */
  RSVD_TRACE_GRAM = 3,    /* Gram X^T X of CholeskyQR                                */
  RSVD_TRACE_APPLY = 4,   /* X R^-1 of CholeskyQR                                    */
  RSVD_TRACE_REDUCE = 5,  /* fixed-order sum of the stream-K partial tiles           */
  RSVD_TRACE_CPQR = 6,    /* column-pivoted QR of ID / CUR                           */
  RSVD_TRACE_JACOBI = 7,  /* one-sided Jacobi SVD of the l x l core                  */
  RSVD_TRACE_CHOL = 8,    /* Cholesky factor and inverse of CholeskyQR               */
  RSVD_TRACE_SOLVE = 9,   /* triangular solves of ID / CUR                           */
  RSVD_TRACE_SIMT = 10,   /* SIMT GEMMs (lift, CUR products, FP64 path)              */
  RSVD_TRACE_CLASSES = 11
};

/* Turns on (1) or off (0) CUDA-event timing of the classes above.  While on,
 * every traced launch records a start and an end event on its own stream. */
rsvd_status rsvd_trace_enable(int enable);

/* Synchronises with the recorded events, writes per class the summed duration
 * in milliseconds and the number of launches (arrays of nclass entries), and
 * clears the records.  Returns RSVD_TRACE_CLASSES, or -1 on bad arguments. */
int rsvd_trace_read(double* ms, int64_t* launches, int nclass);

/* Number of kernels the library has launched since it was loaded. */
int64_t rsvd_kernel_launch_count(void);

/* Test aid for the failure path of the bounded waits (host only; not part of
 * the paper's method).  While `cycles` > 0, every grid-barrier wait of the
 * pivoted-QR kernels (rsvd_id, rsvd_cur, rsvd_cpqr_id, rsvd_cpqr_id_f32 and the
 * combined calls) gives up after `cycles` SM clock cycles instead of about
 * 2 s; with `withhold` non-zero, CTA 0 also withholds its arrival at the first
 * barrier, so that every CTA's wait runs out: each records RSVD_ERR_TIMEOUT in
 * *d_info and returns, nothing is left running and the context stays usable.
 * cycles = 0 restores the defaults (withhold is then ignored).  Affects the
 * launches enqueued after it by any thread.  RSVD_ERR_INVALID_ARG when
 * cycles < 0. */
rsvd_status rsvd_test_set_barrier_wait(long long cycles, int withhold);

/* ------------------------------------------------------------------------
 * Batched RSVD of many small FP32 matrices of different sizes (Alg. 5 for each
 * problem: the power scheme with orthonormalisation before every product,
 * s = 1, then the SVD of B through the QR of Bt).  Every step is one launch
 * over the whole batch, so a batch of hundreds of problems costs a few dozen
 * launches instead of a few dozen per problem.
 *
 * items (HOST array of `batch` entries) gives, per problem i:
 *   m, n     A_i is m x n, row-major with leading dimension n, at A + a_off;
 *   k        rank; l = k + p must satisfy l <= min(m, n) and l <= 128;
 *   u_off    U_i (m x k, row-major, leading dimension k) at U + u_off;
 *   v_off    V_i (n x k, leading dimension k) at V + v_off;
 *   s_off    S_i (k doubles, descending) at S + s_off.
 * A, U, V, S are device buffers holding all problems at the given element
 * offsets; outputs must not overlap.  Omega of problem i is the Philox stream
 * of `seed` with the problem index as the counter's batch word (counter (row,
 * column / 4, 0, i)), rounded to bf16 as on the FP32 path.  The passes over A
 * and the CholeskyQR steps of the power scheme run as grouped tcgen05 launches
 * (bf16 split products, fp32 accumulation, as rsvd_svd's tensor-core path);
 * the final orthonormalisations of Y and Bt and the lifts of U and V are plain
 * fp32 products, the l x l factorisations fp32 with the CholeskyQR shift
 * fallback.
 * Sign rule and ordering as rsvd_svd.  The work buffer (256-byte aligned)
 * holds per-problem scratch and the task tables, which are copied from the
 * host with cudaMemcpyAsync on `stream` (no host synchronisation).
 * Errors: RSVD_ERR_INVALID_ARG (a bad item, size or pointer),
 * RSVD_ERR_WORKSPACE, RSVD_ERR_CUDA; device failures in *d_info.
 * ------------------------------------------------------------------------ */
typedef struct {
  int64_t m, n;
  int k;
  int64_t a_off, u_off, v_off, s_off;
} rsvd_batch_item;

size_t rsvd_svd_batched_workspace_size(int batch, const rsvd_batch_item* items, int p, int q);
/* The choices of the batched path's tile autotuner so far in this process
 * (not part of the paper's method).  The plain fp32 GEMMs of the batch
 * (Gram slices, applies and lifts of the final orthonormalisations, and the
 * passes over A when the tensor-core grouped passes do not apply) run on
 * blocks of 64, 128 or 256 output rows; the first call that meets a class
 * (kind: 0 pass over A, 1 Gram slice, 2 apply, 3 lift, 4 sketch; and width N)
 * times every valid height on its own GEMMs of the class and keeps the
 * fastest.  That call synchronises its stream once per new class; later calls
 * do not.  Every height gives bit-identical results.  Writes up to `cap`
 * entries: kind, width, chosen rows, and ms[3 i + h] the time of height
 * 64 << h (-1 when not valid); returns the number of classes. */
int rsvd_batched_tuning(int cap, int* kind, int* width, int* rows, float* ms);
rsvd_status rsvd_svd_batched(int batch, const rsvd_batch_item* items, int p, int q,
                             uint64_t seed, const float* A, float* U, double* S, float* V,
                             void* work, size_t work_bytes, int* d_info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RSVD_H */
