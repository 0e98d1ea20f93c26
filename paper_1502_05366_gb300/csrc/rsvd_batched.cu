// rsvd_svd_batched: the RSVD of Alg. 5 (QB through the power scheme with
// orthonormalisation before every product, s = 1; B's SVD through the QR of
// Bt) for a batch of small FP32 problems of different sizes.  Each step is one
// launch over the whole batch: grouped GEMM tasks (k_batched.cu), one CTA per
// problem for the l x l factorisations (k_chol.cu, k_jacobi.cu).  The task
// tables are built on the host from the problem sizes and copied into the
// workspace once per call.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "rsvd.h"

namespace rsvd {

namespace {

struct Carve {   // workspace carving; dry when base is null
  char* base = nullptr;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T) + 16;
    return p;
  }
};

struct ProbBufs {
  float *Y, *Yt, *Z, *Zt, *G, *Gpart, *R, *Rinv, *Racc, *tmp, *Uj, *Uh, *Vh;
  double* Sh;
  // grouped tensor-core passes: A at a 16-byte pitch, the bf16 operands
  float* Ap;
  uint16_t *Oh, *Yh, *Yl, *Zh, *Zl;   // Omega^T; hi / lo of Y^T and of Z^T
};

// A Gram of a tall sample runs as one GEMM per slice of this many rows (split
// K), so that a stage has several tasks per problem; the slices are summed in
// order.
constexpr int GRAM_SLICE = 512;
inline int gram_slices(int64_t rows) { return (int)((rows + GRAM_SLICE - 1) / GRAM_SLICE); }

enum StageKind { ST_GEMM, ST_CHOL, ST_TRMM, ST_SVD, ST_SIGN, ST_SUM, ST_TCG, ST_PAD, ST_SPLIT,
                 ST_OMT };
struct Stage {
  int kind;
  int first, count;   // into the table of the kind (gemm: tasks; others: problems; pad /
                      // split / omega: chunks; grouped tensor-core pass: tasks)
  int rows;           // gemm: block height of the tasks
  int first2 = 0;     // grouped pass: first problem record (and its 3 tensor maps)
  int form = 0, nwt = 0;
};

struct Plan {
  std::vector<BGemm> gemms;
  std::vector<int2> tasks;
  std::vector<BChol> chols;
  std::vector<BTrmm> trmms;
  std::vector<BSvd> svds;
  std::vector<BSign> signs;
  std::vector<BSum> sums;
  std::vector<Stage> stages;
  int lmax = 0;
  // grouped tensor-core passes
  std::vector<TgProb> tgp;
  std::vector<TgTask> tgt;
  std::vector<CUtensorMap> tgm;
  std::vector<TgPad> pads;
  std::vector<TgSplit> splits;
  std::vector<int2> chunks;   // pad, split and omega chunks: (job, first row)
  bool map_fail = false;      // a tensor map could not be encoded
};

bool items_ok(int batch, const rsvd_batch_item* it, int p, int q) {
  if (batch < 1 || !it || p < 0 || q < 0 || q > 64) return false;
  for (int i = 0; i < batch; ++i) {
    const int64_t l = (int64_t)it[i].k + p;
    if (it[i].k < 1 || it[i].m < 1 || it[i].n < 1) return false;
    if (l > it[i].m || l > it[i].n || l > BATCH_LMAX) return false;
    if (it[i].m > 0x7fffffffLL || it[i].n > 0x7fffffffLL) return false;
    if (it[i].a_off < 0 || it[i].u_off < 0 || it[i].v_off < 0 || it[i].s_off < 0) return false;
  }
  return true;
}

// One GEMM per problem; tasks over blocks of output rows whose height follows
// the width, one launch per height.
void add_gemm_stage(Plan& P, const std::vector<BGemm>& gs) {
  const int g0 = (int)P.gemms.size();
  for (const BGemm& g : gs) P.gemms.push_back(g);
  for (int rows = 64; rows <= 256; rows *= 2) {
    Stage st{ST_GEMM, (int)P.tasks.size(), 0, rows};
    for (int i = 0; i < (int)gs.size(); ++i) {
      if (bgemm_rows(gs[i].N) != rows) continue;
      for (int r0 = 0; r0 < gs[i].M; r0 += rows) P.tasks.push_back(make_int2(g0 + i, r0));
    }
    st.count = (int)P.tasks.size() - st.first;
    if (st.count > 0) P.stages.push_back(st);
  }
}

BGemm gemm_of(const float* A, int64_t lda, int transA, const float* W, int64_t ldw, float* C,
              int64_t ldc, int64_t M, int N, int64_t K, int ncol, int batch) {
  BGemm g;
  g.A = A;
  g.lda = lda;
  g.W = W;
  g.ldw = ldw;
  g.C = C;
  g.ldc = ldc;
  g.M = (int)M;
  g.N = N;
  g.K = (int)K;
  g.ncol = ncol;
  g.transA = transA;
  g.batch = batch;
  return g;
}

inline int tg_n(int l) { return (l + 15) & ~15; }
inline int64_t pad4(int64_t x) { return (x + 3) & ~(int64_t)3; }
inline int64_t pad8(int64_t x) { return (x + 7) & ~(int64_t)7; }

// Chunks of 32 rows of each job (rows[i]) appended to P.chunks; returns the
// stage's (first, count).
void add_chunks(Plan& P, int first_job, const std::vector<int64_t>& rows, int kind) {
  Stage st{kind, (int)P.chunks.size(), 0, 0};
  for (size_t i = 0; i < rows.size(); ++i)
    for (int64_t r0 = 0; r0 < rows[i]; r0 += 32) P.chunks.push_back(make_int2(first_job + (int)i, (int)r0));
  st.count = (int)P.chunks.size() - st.first;
  if (st.count > 0) P.stages.push_back(st);
}

// W^T split (hi, lo) of every problem's X (rows x l, ld l): Y (rows m) or Z (rows n).
void add_split(Plan& P, int batch, const rsvd_batch_item* it, int p, std::vector<ProbBufs>& b,
               bool on_z) {
  const int j0 = (int)P.splits.size();
  std::vector<int64_t> rows;
  for (int i = 0; i < batch; ++i) {
    const int l = it[i].k + p;
    const int64_t rr = on_z ? it[i].n : it[i].m;
    TgSplit sp;
    sp.W = on_z ? b[i].Z : b[i].Y;
    sp.ldw = l;
    sp.hi = on_z ? b[i].Zh : b[i].Yh;
    sp.lo = on_z ? b[i].Zl : b[i].Yl;
    sp.rows = rr;
    sp.ldt = pad8(rr);
    sp.l = l;
    sp.N = tg_n(l);
    sp.batch = i;
    P.splits.push_back(sp);
    rows.push_back(rr);
  }
  add_chunks(P, j0, rows, ST_SPLIT);
}

// One grouped tensor-core pass over every problem's A: form 0 C = A W (W^T
// from Omega^T when omega, else the split of Z), form 1 C = A^T W (W^T the
// split of Y).  Output C = Y (form 0) or Z (form 1).  Tasks ordered by
// decreasing contraction length, so that the CTAs' round-robin shares are even.
void add_tc_pass(Plan& P, int batch, const rsvd_batch_item* it, int p, std::vector<ProbBufs>& b,
                 int form, bool omega, bool encode) {
  Stage st{ST_TCG, (int)P.tgt.size(), 0, 0};
  st.first2 = (int)P.tgp.size();
  st.form = form;
  st.nwt = omega ? 1 : 2;
  std::vector<TgTask> tasks;
  std::vector<int> cost;
  for (int i = 0; i < batch; ++i) {
    const int l = it[i].k + p;
    const int64_t m = it[i].m, n = it[i].n;
    TgProb pr;
    pr.C = form == 0 ? b[i].Y : b[i].Z;
    pr.ldc = l;
    pr.M = (int)(form == 0 ? m : n);
    pr.K = (int)(form == 0 ? n : m);
    pr.ncol = l;
    pr.N = tg_n(l);
    P.tgp.push_back(pr);
    CUtensorMap mp[3];
    memset(mp, 0, sizeof(mp));
    if (encode) {
      const uint16_t* whi = form == 1 ? b[i].Yh : (omega ? b[i].Oh : b[i].Zh);
      const uint16_t* wlo = form == 1 ? b[i].Yl : (omega ? nullptr : b[i].Zl);
      if (!tg_encode_maps(form, st.nwt, b[i].Ap, m, n, pad4(n), whi, wlo, pr.K, pr.N,
                          pad8(pr.K), mp))
        P.map_fail = true;
    }
    for (int t = 0; t < 3; ++t) P.tgm.push_back(mp[t]);
    for (int r0 = 0; r0 < pr.M; r0 += 128) {
      tasks.push_back(TgTask{i, r0});
      cost.push_back(pr.K);
    }
  }
  std::vector<int> order(tasks.size());
  for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  for (int t : order) P.tgt.push_back(tasks[t]);
  st.count = (int)P.tgt.size() - st.first;
  if (st.count > 0) P.stages.push_back(st);
}

// CholeskyQR2 of X (rows x l per problem, ld l) in place, through Xt; with
// want_R the triangular factor R = R2 R1 ends in Racc.
void add_orth(Plan& P, int batch, const rsvd_batch_item* it, int p, std::vector<ProbBufs>& b,
              bool on_z, bool want_R) {
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<BGemm> gram, apply;
    Stage sc{ST_CHOL, (int)P.chols.size(), batch, 0};
    Stage ss{ST_SUM, (int)P.sums.size(), batch, 0};
    for (int i = 0; i < batch; ++i) {
      const int l = it[i].k + p;
      const int64_t rows = on_z ? it[i].n : it[i].m;
      float* X = on_z ? b[i].Z : b[i].Y;
      float* Xt = on_z ? b[i].Zt : b[i].Yt;
      const float* src = pass == 0 ? X : Xt;
      float* dst = pass == 0 ? Xt : X;
      // G = sum over row slices of X_s^T X_s (split K)
      const int ns = gram_slices(rows);
      for (int sl = 0; sl < ns; ++sl) {
        const int64_t r0 = (int64_t)sl * GRAM_SLICE;
        const int64_t rs = std::min<int64_t>(GRAM_SLICE, rows - r0);
        gram.push_back(gemm_of(src ? src + r0 * l : nullptr, l, 1, src ? src + r0 * l : nullptr, l,
                               b[i].Gpart ? b[i].Gpart + (int64_t)sl * l * l : nullptr, l, l, l,
                               rs, l, i));
      }
      BSum su;
      su.part = b[i].Gpart;
      su.out = b[i].G;
      su.nslice = ns;
      su.count = l * l;
      P.sums.push_back(su);
      BChol c;
      c.G = b[i].G;
      c.R = (want_R && pass == 0) ? b[i].Racc : b[i].R;
      c.Rinv = b[i].Rinv;
      c.l = l;
      P.chols.push_back(c);
      apply.push_back(gemm_of(src, l, 0, b[i].Rinv, l, dst, l, rows, l, l, l, i));
    }
    add_gemm_stage(P, gram);
    P.stages.push_back(ss);
    P.stages.push_back(sc);
    add_gemm_stage(P, apply);
  }
  if (want_R) {
    Stage st{ST_TRMM, (int)P.trmms.size(), batch, 0};
    for (int i = 0; i < batch; ++i) {
      BTrmm t;
      t.R = b[i].R;
      t.Racc = b[i].Racc;
      t.tmp = b[i].tmp;
      t.l = it[i].k + p;
      P.trmms.push_back(t);
    }
    P.stages.push_back(st);
  }
}

// Carves the per-problem buffers and the plan; returns the workspace bytes.
size_t build(int batch, const rsvd_batch_item* it, int p, int q, const float* A, float* U,
             double* S, float* V, char* base, Plan& P, char** tables, bool tc) {
  Carve cv;
  cv.base = base;
  std::vector<ProbBufs> b(batch);
  const bool enc = base != nullptr;   // tensor maps need the device addresses
  for (int i = 0; i < batch; ++i) {
    const int64_t m = it[i].m, n = it[i].n;
    const int l = it[i].k + p;
    P.lmax = std::max(P.lmax, l);
    b[i].Y = cv.take<float>((size_t)m * l);
    b[i].Yt = cv.take<float>((size_t)m * l);
    b[i].Z = cv.take<float>((size_t)n * l);
    b[i].Zt = cv.take<float>((size_t)n * l);
    b[i].G = cv.take<float>((size_t)l * l);
    b[i].Gpart = cv.take<float>((size_t)gram_slices(std::max(m, n)) * l * l);
    b[i].R = cv.take<float>((size_t)l * l);
    b[i].Rinv = cv.take<float>((size_t)l * l);
    b[i].Racc = cv.take<float>((size_t)l * l);
    b[i].tmp = cv.take<float>((size_t)l * l);
    b[i].Uj = cv.take<float>((size_t)l * l);
    b[i].Uh = cv.take<float>((size_t)l * l);
    b[i].Vh = cv.take<float>((size_t)l * l);
    b[i].Sh = cv.take<double>((size_t)l);
    b[i].Ap = nullptr;
    b[i].Oh = b[i].Yh = b[i].Yl = b[i].Zh = b[i].Zl = nullptr;
    if (tc) {
      const int N = tg_n(l);
      b[i].Ap = cv.take<float>((size_t)m * pad4(n));
      b[i].Oh = cv.take<uint16_t>((size_t)N * pad8(n));
      b[i].Yh = cv.take<uint16_t>((size_t)N * pad8(m));
      b[i].Yl = cv.take<uint16_t>((size_t)N * pad8(m));
      b[i].Zh = cv.take<uint16_t>((size_t)N * pad8(n));
      b[i].Zl = cv.take<uint16_t>((size_t)N * pad8(n));
    }
  }
  if (tc) {
    // A at a 16-byte pitch, then Omega^T of every problem
    std::vector<int64_t> rows;
    for (int i = 0; i < batch; ++i) {
      TgPad pd;
      pd.src = A ? A + it[i].a_off : nullptr;
      pd.dst = b[i].Ap;
      pd.rows = it[i].m;
      pd.cols = it[i].n;
      pd.lds = it[i].n;
      pd.ldd = pad4(it[i].n);
      P.pads.push_back(pd);
      rows.push_back(it[i].m);
    }
    add_chunks(P, 0, rows, ST_PAD);
    rows.clear();
    const int j0 = (int)P.splits.size();
    for (int i = 0; i < batch; ++i) {
      const int l = it[i].k + p;
      TgSplit sp;
      sp.W = nullptr;
      sp.ldw = 0;
      sp.hi = b[i].Oh;
      sp.lo = nullptr;
      sp.rows = it[i].n;
      sp.ldt = pad8(it[i].n);
      sp.l = l;
      sp.N = tg_n(l);
      sp.batch = i;
      P.splits.push_back(sp);
      rows.push_back(it[i].n);
    }
    add_chunks(P, j0, rows, ST_OMT);
  }
  // Y = A Omega (Sec. 3.1, Fig. 1 step 2)
  std::vector<BGemm> gs;
  if (tc) {
    add_tc_pass(P, batch, it, p, b, 0, true, enc);
  } else {
    for (int i = 0; i < batch; ++i) {
      const int l = it[i].k + p;
      gs.push_back(gemm_of(A ? A + it[i].a_off : nullptr, it[i].n, 0, nullptr, 0, b[i].Y, l,
                           it[i].m, l, it[i].n, l, i));
    }
    add_gemm_stage(P, gs);
  }
  // power scheme, orthonormalising before every product (Alg. 5, s = 1)
  for (int j = 0; j < q; ++j) {
    add_orth(P, batch, it, p, b, false, false);
    gs.clear();
    if (tc) {                           // Z = A^T Y
      add_split(P, batch, it, p, b, false);
      add_tc_pass(P, batch, it, p, b, 1, false, enc);
    } else {
      for (int i = 0; i < batch; ++i) {
        const int l = it[i].k + p;
        gs.push_back(gemm_of(A ? A + it[i].a_off : nullptr, it[i].n, 1, b[i].Y, l, b[i].Z, l,
                             it[i].n, l, it[i].m, l, i));
      }
      add_gemm_stage(P, gs);
    }
    add_orth(P, batch, it, p, b, true, false);
    gs.clear();
    if (tc) {                           // Y = A Z
      add_split(P, batch, it, p, b, true);
      add_tc_pass(P, batch, it, p, b, 0, false, enc);
    } else {
      for (int i = 0; i < batch; ++i) {
        const int l = it[i].k + p;
        gs.push_back(gemm_of(A ? A + it[i].a_off : nullptr, it[i].n, 0, b[i].Z, l, b[i].Y, l,
                             it[i].m, l, it[i].n, l, i));
      }
      add_gemm_stage(P, gs);
    }
  }
  add_orth(P, batch, it, p, b, false, false);   // Q = orth(Y)
  gs.clear();
  if (tc) {                                     // Bt = A^T Q
    add_split(P, batch, it, p, b, false);
    add_tc_pass(P, batch, it, p, b, 1, false, enc);
  } else {
    for (int i = 0; i < batch; ++i) {
      const int l = it[i].k + p;
      gs.push_back(gemm_of(A ? A + it[i].a_off : nullptr, it[i].n, 1, b[i].Y, l, b[i].Z, l,
                           it[i].n, l, it[i].m, l, i));
    }
    add_gemm_stage(P, gs);
  }
  add_orth(P, batch, it, p, b, true, true);     // Bt = Qh Rh
  {
    Stage st{ST_SVD, (int)P.svds.size(), batch, 0};   // Rh = Uh diag(Sh) Vh^T
    for (int i = 0; i < batch; ++i) {
      BSvd s;
      s.M = b[i].Racc;
      s.Uj = b[i].Uj;
      s.Uh = b[i].Uh;
      s.Vh = b[i].Vh;
      s.Sh = b[i].Sh;
      s.l = it[i].k + p;
      P.svds.push_back(s);
    }
    P.stages.push_back(st);
  }
  gs.clear();
  for (int i = 0; i < batch; ++i) {   // U = Q Vh(:, :k), V = Qh Uh(:, :k)
    const int l = it[i].k + p, k = it[i].k;
    gs.push_back(gemm_of(b[i].Y, l, 0, b[i].Vh, l, U ? U + it[i].u_off : nullptr, k, it[i].m, k,
                         l, k, i));
    gs.push_back(gemm_of(b[i].Z, l, 0, b[i].Uh, l, V ? V + it[i].v_off : nullptr, k, it[i].n, k,
                         l, k, i));
  }
  add_gemm_stage(P, gs);
  {
    Stage st{ST_SIGN, (int)P.signs.size(), batch, 0};
    for (int i = 0; i < batch; ++i) {
      BSign s;
      s.U = U ? U + it[i].u_off : nullptr;
      s.V = V ? V + it[i].v_off : nullptr;
      s.S = S ? S + it[i].s_off : nullptr;
      s.Sh = b[i].Sh;
      s.m = it[i].m;
      s.n = it[i].n;
      s.k = it[i].k;
      P.signs.push_back(s);
    }
    P.stages.push_back(st);
  }
  // the tables themselves
  *tables = cv.base ? cv.base + ((cv.off + 255) & ~(size_t)255) : nullptr;
  cv.take<BGemm>(P.gemms.size());
  cv.take<int2>(P.tasks.size());
  cv.take<BChol>(P.chols.size());
  cv.take<BTrmm>(P.trmms.size());
  cv.take<BSvd>(P.svds.size());
  cv.take<BSign>(P.signs.size());
  cv.take<BSum>(P.sums.size());
  cv.take<TgProb>(P.tgp.size());
  cv.take<TgTask>(P.tgt.size());
  cv.take<CUtensorMap>(P.tgm.size());
  cv.take<TgPad>(P.pads.size());
  cv.take<TgSplit>(P.splits.size());
  cv.take<int2>(P.chunks.size());
  return cv.off + 256;
}

}  // namespace

}  // namespace rsvd

using namespace rsvd;

extern "C" {

size_t rsvd_svd_batched_workspace_size(int batch, const rsvd_batch_item* items, int p, int q) {
  if (!items_ok(batch, items, p, q)) return 0;
  Plan P;
  char* tables = nullptr;
  return build(batch, items, p, q, nullptr, nullptr, nullptr, nullptr, nullptr, P, &tables,
               true);
}

rsvd_status rsvd_svd_batched(int batch, const rsvd_batch_item* items, int p, int q,
                             uint64_t seed, const float* A, float* U, double* S, float* V,
                             void* work, size_t work_bytes, int* d_info, void* stream) {
  if (!items_ok(batch, items, p, q) || !A || !U || !S || !V) return RSVD_ERR_INVALID_ARG;
  if (!work || ((uintptr_t)work & 255u)) return RSVD_ERR_INVALID_ARG;
  Plan dry;
  char* t0 = nullptr;
  const size_t need = build(batch, items, p, q, nullptr, nullptr, nullptr, nullptr, nullptr, dry,
                            &t0, true);
  if (need > work_bytes) return RSVD_ERR_WORKSPACE;
  Plan P;
  char* tables = nullptr;
  build(batch, items, p, q, A, U, S, V, (char*)work, P, &tables, true);
  if (P.map_fail) return RSVD_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (d_info && cudaMemsetAsync(d_info, 0, sizeof(int), s) != cudaSuccess) return RSVD_ERR_CUDA;
  // upload the tables (same carving as in build)
  Carve cv;
  cv.base = (char*)work;
  cv.off = (size_t)(tables - (char*)work);
  BGemm* dg = cv.take<BGemm>(P.gemms.size());
  int2* dt = cv.take<int2>(P.tasks.size());
  BChol* dc = cv.take<BChol>(P.chols.size());
  BTrmm* dm = cv.take<BTrmm>(P.trmms.size());
  BSvd* dv = cv.take<BSvd>(P.svds.size());
  BSign* dsg = cv.take<BSign>(P.signs.size());
  BSum* dsu = cv.take<BSum>(P.sums.size());
  TgProb* dtp = cv.take<TgProb>(P.tgp.size());
  TgTask* dtt = cv.take<TgTask>(P.tgt.size());
  CUtensorMap* dtm = cv.take<CUtensorMap>(P.tgm.size());
  TgPad* dpd = cv.take<TgPad>(P.pads.size());
  TgSplit* dsp = cv.take<TgSplit>(P.splits.size());
  int2* dch = cv.take<int2>(P.chunks.size());
#define UPLOAD(dst, vec)                                                                 \
  if (!vec.empty() && cudaMemcpyAsync(dst, vec.data(), vec.size() * sizeof(vec[0]),      \
                                      cudaMemcpyHostToDevice, s) != cudaSuccess)         \
    return RSVD_ERR_CUDA;
  UPLOAD(dg, P.gemms);
  UPLOAD(dt, P.tasks);
  UPLOAD(dc, P.chols);
  UPLOAD(dm, P.trmms);
  UPLOAD(dv, P.svds);
  UPLOAD(dsg, P.signs);
  UPLOAD(dsu, P.sums);
  UPLOAD(dtp, P.tgp);
  UPLOAD(dtt, P.tgt);
  UPLOAD(dtm, P.tgm);
  UPLOAD(dpd, P.pads);
  UPLOAD(dsp, P.splits);
  UPLOAD(dch, P.chunks);
#undef UPLOAD
  for (const Stage& st : P.stages) {
    cudaError_t e = cudaSuccess;
    switch (st.kind) {
      case ST_GEMM: e = launch_bgemm(dg, dt + st.first, st.count, st.rows, seed, s); break;
      case ST_CHOL: e = launch_chol_batched(dc + st.first, st.count, P.lmax, d_info, s); break;
      case ST_TRMM: e = launch_trmm_batched(dm + st.first, st.count, s); break;
      case ST_SVD:
        e = launch_small_svd_batched(dv + st.first, st.count, P.lmax, 30, d_info, s);
        break;
      case ST_SIGN: e = launch_sign_batched(dsg + st.first, st.count, s); break;
      case ST_SUM: e = launch_sum_batched(dsu + st.first, st.count, s); break;
      case ST_TCG:
        e = launch_tc_group(st.form, st.nwt, dtp + st.first2, dtt + st.first, st.count,
                            dtm + 3 * (int64_t)st.first2, d_info, s);
        break;
      case ST_PAD: e = launch_pad_rows_batched(dpd, dch + st.first, st.count, s); break;
      case ST_SPLIT: e = launch_split_t_batched(dsp, dch + st.first, st.count, s); break;
      case ST_OMT: e = launch_omega_t_batched(dsp, dch + st.first, st.count, seed, s); break;
      default: break;
    }
    if (e != cudaSuccess) return RSVD_ERR_CUDA;
  }
  return RSVD_OK;
}

}  // extern "C"
