// Reverse-mode derivative of the randomized SVD (Alg. 5, s = 1) with Omega
// held fixed: rsvd_svd_vjp.
//
// Nothing is kept between the forward call and this one but A and the seed:
// the call first replays the forward path, keeping in its workspace the
// factors the backward needs (the Q and R of every orthonormalisation, the
// QR of Bt, the small SVD and the sign rule), then runs the backward in
// reverse order.  Every orthonormalisation of the replay is a full CholeskyQR
// (two or three passes), so each Q is orthonormal to working precision, as
// the QR rule requires.
//
// Backward, with X = Q R rules and the square-SVD rule of k_vjp.cu:
//   g_U, g_V <- g_U, g_V with the sign rule's flips;
//   g_Vh(:, :k) = Q^* g_U,   g_Q = g_U Vh(:, :k)^*      (U = Q Vh(:, :k))
//   g_Uh(:, :k) = Qh^* g_V,  g_Qh = g_V Uh(:, :k)^*     (V = Qh Uh(:, :k))
//   g_Rh = square-SVD rule;  g_Bt = QR rule (Qh, Rh)
//   Bt = A^* Q:   g_A += Q g_Bt^*,  g_Q += A g_Bt;   g_Y = QR rule (Q, Rq)
//   then for each power step, last first:
//     Y = A Qz:   g_A += g_Y Qz^*,  g_Qz = A^* g_Y;  g_Z = QR rule (Qz, Rz)
//     Z = A^* Qy: g_A += Qy g_Z^*,  g_Qy = A g_Z;    g_Y = QR rule (Qy, Ry)
//   Y0 = A Omega: g_A += g_Y Omega^*.
// The rank-l contributions to g_A are packed side by side (2q + 2 pairs of
// m x l and n x l factors) and applied in one rank update of the m x n g_A.
// Products with A and A^* run on the forward path's GEMM kernels (tensor
// cores with split operands on the FP32 path), the l x l steps on the SIMT
// kernels, the solves with R^* in double-float (FP32 path) or FP64.
#include "engine.cuh"

namespace rsvd {

template <typename T>
static rsvd_status run_svd_vjp(Ctx& c, const Opts& o, bool tc, int64_t m, int64_t n, int k,
                               int p, int q, uint64_t seed, const T* A, int64_t lda,
                               const T* gU, int64_t ldgu, const double* gS, const T* gV,
                               int64_t ldgv, T* gA, int64_t ldga, T* Uo, int64_t ldu,
                               double* So, T* Vo, int64_t ldv) {
  Engine<T> e(c, o, tc);
  const int l = k + p, L = padL(l);
  const int K = (2 * q + 2) * l;   // width of the packed rank update
  auto b = e.take_qb(m, n, L);
  auto sb = e.take_svd(l, L, k);
  std::vector<T*> Qy(q), Ry(q), Qz(q), Rz(q);
  for (int i = 0; i < q; ++i) {
    Qy[i] = c.template take<T>((size_t)m * L);
    Ry[i] = c.template take<T>((size_t)L * L);
    Qz[i] = c.template take<T>((size_t)n * L);
    Rz[i] = c.template take<T>((size_t)L * L);
  }
  T* Rq = c.template take<T>((size_t)L * L);
  T* Rh = c.template take<T>((size_t)L * L);
  T* Om = c.template take<T>((size_t)n * L);
  T* U = Uo ? Uo : c.template take<T>((size_t)m * k);
  T* V = Vo ? Vo : c.template take<T>((size_t)n * k);
  double* S = So ? So : c.template take<double>((size_t)k);
  if (!Uo) ldu = k;
  if (!Vo) ldv = k;
  T* gUs = c.template take<T>((size_t)m * k);
  T* gVs = c.template take<T>((size_t)n * k);
  T* sq[13];
  for (int i = 0; i < 13; ++i) sq[i] = c.template take<T>((size_t)L * L);
  T *gVh = sq[0], *gUh = sq[1], *Gu = sq[2], *Gv = sq[3], *X = sq[4], *T1 = sq[5],
    *gRh = sq[6], *VhT = sq[7], *UhkT = sq[8], *VhkT = sq[9], *RT = sq[10], *P1 = sq[11],
    *P2 = sq[12];
  T* symM = c.template take<T>((size_t)L * L);
  double* Rdf = c.template take<double>((size_t)L * L + L);
  T* gQ = c.template take<T>((size_t)m * L);
  T* tm = c.template take<T>((size_t)m * L);
  T* gY = c.template take<T>((size_t)m * L);
  T* Gm = c.template take<T>((size_t)m * L);
  T* gQh = c.template take<T>((size_t)n * L);
  T* gBt = c.template take<T>((size_t)n * L);
  T* tn = c.template take<T>((size_t)n * L);
  T* gZ = c.template take<T>((size_t)n * L);
  T* Gn = c.template take<T>((size_t)n * L);
  typename Engine<T>::Split sm{}, sn{};
  if (tc) {
    sm = e.take_split(L, m);
    sn = e.take_split(L, n);
  }
  // split-K slabs of the SIMT transposed products (l rows; k or l columns;
  // contractions over m, n or l)
  size_t se = 0;
  for (int nc : {k, l})
    for (int64_t kk : {m, n, (int64_t)l}) {
      int ns;
      int64_t kc;
      tn_split(l, nc, kk, e.sms, &ns, &kc);
      se = std::max(se, (size_t)ns * l * nc);
    }
  T* tslabs = c.template take<T>(se);
  T* Xcat = c.template take<T>((size_t)m * K);
  T* Wcat = c.template take<T>((size_t)n * K);
  if (c.dry) return RSVD_OK;
  if (c.off > c.cap) return RSVD_ERR_WORKSPACE;
  cudaStream_t st = c.stream;
  const bool abf = c.abf != 0;
  rsvd_status r;

  // ------------------------------ helpers ---------------------------------
  // out (rows x L) = A W, W n x L (zero padding)
  auto mulA = [&](const T* W, T* out) -> rsvd_status {
    if (tc)
      LK(launch_split_transpose(n, l, L, (const float*)W, L, sn.hi, sn.lo, sn.ld, st));
    return e.gemm_n(m, n, L, A, lda, m, n, false, 0, L, tc ? &sn : nullptr, W, L, out, L, L,
                    nullptr, b.part, nullptr, abf);
  };
  // out (n x L) = A^* X, X m x L
  auto mulAt = [&](const T* Xm, T* out) -> rsvd_status {
    if (tc)
      LK(launch_split_transpose(m, l, L, (const float*)Xm, L, sm.hi, sm.lo, sm.ld, st));
    return e.gemm_t(n, m, L, A, lda, tc ? &sm : nullptr, Xm, L, out, L, L, nullptr, b.part,
                    b.slabs, nullptr, false, abf);
  };
  // out (l x ncols, ld ldo) = P(:, :l)^* B with P rows x L, B rows x ncols (ld ldb).
  // The l x l steps touch only the leading l x l blocks: the padding of the
  // small SVD's factors is never read.
  auto tnp = [&](int64_t rows, const T* P, const T* B, int64_t ldb, int ncols, T* out,
                 int64_t ldo) -> rsvd_status {
    int ns;
    int64_t kc;
    tn_split(l, ncols, rows, e.sms, &ns, &kc);
    LK(launch_gemm_tn_partial<T>(l, ncols, rows, P, L, B, ldb, tslabs, ncols, ns, kc, st));
    LK(launch_reduce_slabs<T>(l, ncols, ns, tslabs, ncols, out, ldo, st));
    return RSVD_OK;
  };
  // out (M x N) = P (M x Kk) B (Kk x N)
  auto nn = [&](int64_t M, int N, int Kk, const T* P, int64_t ldp, const T* B, int64_t ldb,
                T* out, int64_t ldo) -> rsvd_status {
    LK(launch_gemm_nn<T>(M, N, Kk, P, ldp, B, ldb, out, ldo, 0, N, st));
    return RSVD_OK;
  };
  // g_X (rows x L) = (g_Q + Q sym(g_R R^* - Q^* g_Q)) R^{-*} (g_R may be null)
  auto qr_vjp = [&](int64_t rows, const T* Qm, const T* R, const T* gQm, const T* gR, T* G,
                    T* gX) -> rsvd_status {
    rsvd_status s2 = tnp(rows, Qm, gQm, L, l, P2, L);
    if (s2 != RSVD_OK) return s2;
    if (gR) {
      LK(launch_transpose<T, T>(l, l, R, L, RT, L, st));
      s2 = nn(l, l, l, gR, L, RT, L, P1, L);
      if (s2 != RSVD_OK) return s2;
    }
    LK(launch_sym_upper<T>(l, L, gR ? P1 : nullptr, P2, L, symM, L, st));
    // Q's padding columns and sym's padding are zero: G has zero padding too
    s2 = nn(rows, L, L, Qm, L, symM, L, G, L);
    if (s2 != RSVD_OK) return s2;
    LK(launch_add_inplace<T>(rows, L, gQm, L, G, L, st));
    LK(launch_fill<T>(rows, L, gX, L, T(0), st));
    // rows of g_X: R x = G(c, :)^*, i.e. g_X = G R^{-*}
    if (sizeof(T) == 4) {
      LK(launch_upper_to_df<float>(l, (const float*)R, L, Rdf, st));
      LK(launch_upper_solve_df<float, float>(l, rows, Rdf, (const float*)G, 1, L, (float*)gX, 1,
                                             L, c.d_info, st));
    } else {
      LK(launch_upper_solve<double, double>(l, rows, (const double*)R, L, 1, (const double*)G, 1,
                                            L, (double*)gX, 1, L, c.d_info, st));
    }
    return RSVD_OK;
  };
  int npair = 0;
  auto pair = [&](const T* Xm, const T* Wn) -> rsvd_status {
    LK(launch_pack_cols<T>(m, l, Xm, L, Xcat + (size_t)npair * l, K, T(-1), nullptr, st));
    LK(launch_pack_cols<T>(n, l, Wn, L, Wcat + (size_t)npair * l, K, T(1), nullptr, st));
    ++npair;
    return RSVD_OK;
  };
#define RUN(x)                    \
  do {                            \
    r = (x);                      \
    if (r != RSVD_OK) return r;   \
  } while (0)

  // ---------------------- forward replay (Alg. 5) -------------------------
  reset_info(c);
  if (!tc) LK(launch_fill<T>(m, L, b.Y, L, T(0), st));
  RUN(e.gemm_n(m, n, L, A, lda, m, n, true, seed, l, nullptr, nullptr, 0, b.Y, L, L, &b.ys,
               b.part, nullptr, abf));
  for (int i = 0; i < q; ++i) {
    RUN(e.orth(m, l, L, b.Y, b.Ytmp, &b.ys, b.ob, b.part, b.slabs, true, true));
    std::swap(b.Y, b.Ytmp);
    LK(launch_copy2d<T, T>(m, L, b.Y, L, Qy[i], L, st));
    LK(launch_copy2d<T, T>(L, L, b.ob.Racc, L, Ry[i], L, st));
    RUN(e.gemm_t(n, m, L, A, lda, &b.ys, b.Y, L, b.Z, L, L, &b.zs, b.part, b.slabs, nullptr,
                 false, abf));
    RUN(e.orth(n, l, L, b.Z, b.Ztmp, &b.zs, b.ob, b.part, b.slabs, true, true));
    std::swap(b.Z, b.Ztmp);
    LK(launch_copy2d<T, T>(n, L, b.Z, L, Qz[i], L, st));
    LK(launch_copy2d<T, T>(L, L, b.ob.Racc, L, Rz[i], L, st));
    RUN(e.gemm_n(m, n, L, A, lda, m, n, false, 0, L, &b.zs, b.Z, L, b.Y, L, L, &b.ys, b.part,
                 nullptr, abf));
  }
  RUN(e.orth(m, l, L, b.Y, b.Ytmp, &b.ys, b.ob, b.part, b.slabs, true, true));
  std::swap(b.Y, b.Ytmp);                         // b.Y = Q
  LK(launch_copy2d<T, T>(L, L, b.ob.Racc, L, Rq, L, st));
  RUN(e.gemm_t(n, m, L, A, lda, &b.ys, b.Y, L, b.Z, L, L, &b.zs, b.part, b.slabs, nullptr,
               false, abf, kDrainQB));            // b.Z = Bt
  RUN(e.svd_prep(b, sb, n, l));                   // b.Ztmp = Qh, Racc = Rh
  LK(launch_copy2d<T, T>(L, L, b.ob.Racc, L, Rh, L, st));
  RUN(e.small_svd_jacobi(l, b.ob.Racc, L, sb, st));
  RUN(e.svd_finish(b, sb, m, n, k, l, U, ldu, S, V, ldv));
  const T* Q = b.Y;
  const T* Qh = b.Ztmp;
  const T* Uh = sb.Uh;
  const T* Vh = sb.Vh;

  // ------------------------------ backward --------------------------------
  LK(launch_pack_cols<T>(m, k, gU, ldgu, gUs, k, T(1), sb.signs, st));
  LK(launch_pack_cols<T>(n, k, gV, ldgv, gVs, k, T(1), sb.signs, st));
  LK(launch_fill<T>(L, L, gVh, L, T(0), st));
  LK(launch_fill<T>(L, L, gUh, L, T(0), st));
  LK(launch_fill<T>(m, L, gQ, L, T(0), st));
  LK(launch_fill<T>(n, L, gQh, L, T(0), st));
  RUN(tnp(m, Q, gUs, k, k, gVh, L));              // g_Vh(:, :k) = Q^* g_U
  LK(launch_transpose<T, T>(l, k, Vh, L, VhkT, L, st));
  RUN(nn(m, l, k, gUs, k, VhkT, L, gQ, L));        // g_Q = g_U Vh(:, :k)^*
  RUN(tnp(n, Qh, gVs, k, k, gUh, L));             // g_Uh(:, :k) = Qh^* g_V
  LK(launch_transpose<T, T>(l, k, Uh, L, UhkT, L, st));
  RUN(nn(n, l, k, gVs, k, UhkT, L, gQh, L));       // g_Qh = g_V Uh(:, :k)^*
  // square-SVD rule: g_Rh = Uh X Vh^*
  RUN(tnp(l, Uh, gUh, L, l, Gu, L));
  RUN(tnp(l, Vh, gVh, L, l, Gv, L));
  LK(launch_svd_vjp_core<T>(l, L, k, sb.Sh, gS, Gu, Gv, L, X, L, st));
  RUN(nn(l, l, l, Uh, L, X, L, T1, L));
  LK(launch_transpose<T, T>(l, l, Vh, L, VhT, L, st));
  RUN(nn(l, l, l, T1, L, VhT, L, gRh, L));
  // [Qh, Rh] = qr(Bt)
  RUN(qr_vjp(n, Qh, Rh, gQh, gRh, Gn, gBt));
  // Bt = A^* Q
  RUN(pair(Q, gBt));
  RUN(mulA(gBt, tm));
  LK(launch_add_inplace<T>(m, L, tm, L, gQ, L, st));
  RUN(qr_vjp(m, Q, Rq, gQ, nullptr, Gm, gY));      // Q = orth(Y)
  for (int i = q - 1; i >= 0; --i) {
    RUN(pair(gY, Qz[i]));                          // Y = A Qz
    RUN(mulAt(gY, tn));
    RUN(qr_vjp(n, Qz[i], Rz[i], tn, nullptr, Gn, gZ));
    RUN(pair(Qy[i], gZ));                          // Z = A^* Qy
    RUN(mulA(gZ, tm));
    RUN(qr_vjp(m, Qy[i], Ry[i], tm, nullptr, Gm, gY));
  }
  // Y0 = A Omega: Omega as the sketch kernels draw it
  LK(launch_fill<T>(n, L, Om, L, T(0), st));
  LK(launch_omega<T>(n, l, seed, Om, L, st));
  RUN(pair(gY, Om));
  // g_A = sum of the pairs X W^*: g_A <- 0 - (-Xcat) Wcat^*
  LK(cudaMemset2DAsync(gA, sizeof(T) * ldga, 0, sizeof(T) * n, m, st));
  LK(launch_rank_update<T>(m, n, gA, ldga, Xcat, K, Wcat, K, K, nullptr, st));
#undef RUN
  return RSVD_OK;
}

static bool vjp_args_ok(int64_t m, int64_t n, int k, int p, int q, int dtype) {
  if (dtype != RSVD_F32 && dtype != RSVD_F64) return false;
  return base_args_ok(m, n, k, p, q, dtype);
}

template <typename T>
static size_t vjp_size(const Opts& o, bool tc, int64_t m, int64_t n, int k, int p, int q) {
  Ctx c;
  c.dry = true;
  run_svd_vjp<T>(c, o, tc, m, n, k, p, q, 0, nullptr, n, nullptr, k, nullptr, nullptr, k,
                 nullptr, n, nullptr, k, nullptr, nullptr, k);
  return c.off + 256;
}

}  // namespace rsvd

using namespace rsvd;

extern "C" {

size_t rsvd_svd_vjp_workspace_size(int64_t m, int64_t n, int k, int p, int q, int dtype,
                                   const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o) || !vjp_args_ok(m, n, k, p, q, dtype)) return 0;
  if (dtype == RSVD_F64) return vjp_size<double>(o, false, m, n, k, p, q);
  const bool tc = want_tc(dtype, o, k + p, nullptr, 0);
  if (o.precision == RSVD_PREC_FP8 && !tc) return 0;   // FP8 sketch: tensor cores only
  const size_t s1 = vjp_size<float>(o, false, m, n, k, p, q);
  const size_t s2 = tc ? vjp_size<float>(o, true, m, n, k, p, q) : 0;
  return s1 > s2 ? s1 : s2;
}

rsvd_status rsvd_svd_vjp(int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int dtype,
                         const void* A, int64_t lda, const void* gU, int64_t ldgu,
                         const double* gS, const void* gV, int64_t ldgv, void* gA, int64_t ldga,
                         void* U, int64_t ldu, double* S, void* V, int64_t ldv, void* work,
                         size_t work_bytes, int* d_info, void* stream, const rsvd_opts* opts) {
  Opts o;
  if (!read_opts(opts, &o)) return RSVD_ERR_INVALID_ARG;
  if (dtype == RSVD_BF16) return RSVD_ERR_UNSUPPORTED;
  if (!vjp_args_ok(m, n, k, p, q, dtype)) return RSVD_ERR_INVALID_ARG;
  if (!A || lda < n || !gU || ldgu < k || !gS || !gV || ldgv < k || !gA || ldga < n)
    return RSVD_ERR_INVALID_ARG;
  if ((U && ldu < k) || (V && ldv < k)) return RSVD_ERR_INVALID_ARG;
  if (!work && work_bytes) return RSVD_ERR_INVALID_ARG;
  if (work && ((uintptr_t)work & 15u)) return RSVD_ERR_INVALID_ARG;
  if (rsvd_svd_vjp_workspace_size(m, n, k, p, q, dtype, opts) > work_bytes)
    return RSVD_ERR_WORKSPACE;
  Ctx c;
  c.dry = false;
  c.base = (char*)work;
  c.cap = work_bytes;
  c.stream = (cudaStream_t)stream;
  c.d_info = d_info;
  rsvd_status st;
  if (dtype == RSVD_F64) {
    st = run_svd_vjp<double>(c, o, false, m, n, k, p, q, seed, (const double*)A, lda,
                             (const double*)gU, ldgu, gS, (const double*)gV, ldgv, (double*)gA,
                             ldga, (double*)U, ldu, S, (double*)V, ldv);
  } else {
    const bool tc = want_tc(dtype, o, k + p, A, lda);
    st = run_svd_vjp<float>(c, o, tc, m, n, k, p, q, seed, (const float*)A, lda,
                            (const float*)gU, ldgu, gS, (const float*)gV, ldgv, (float*)gA, ldga,
                            (float*)U, ldu, S, (float*)V, ldv);
  }
  if (st == RSVD_OK && c.err != cudaSuccess) st = RSVD_ERR_CUDA;
  return st;
}

}  // extern "C"
