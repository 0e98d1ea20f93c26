// rsvd_svd_batched: the RSVD of Alg. 5 (QB through the power scheme with
// orthonormalisation before every product, s = 1; B's SVD through the QR of
// Bt) for a batch of small FP32 problems of different sizes.  Each step is one
// launch over the whole batch: grouped GEMM tasks (k_batched.cu), one CTA per
// problem for the l x l factorisations (k_chol.cu, k_jacobi.cu).  The task
// tables are built on the host from the problem sizes and copied into the
// workspace once per call.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
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
  uint16_t* Rw[3];                    // R^-1 in three bf16 terms (transposed)
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
  std::vector<int> gkind;     // tuner class kind of every SIMT GEMM
  int64_t tune_cap = 0;       // tasks of all SIMT GEMMs at the smallest height
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

// ---------------------------------------------------------------------------
// Tile autotuner of the grouped SIMT GEMM (bgemm_kernel): a task is a block of
// 64, 128 or 256 output rows by 128, 64 or 32 columns.  The block height of
// every GEMM class (kind: sketch or pass over A, Gram slice, apply, lift; and
// its width N) is measured the first time a call meets the class: each valid
// height runs the class's GEMMs of that call (CUDA events, after one warm-up
// launch) and the fastest is kept for the life of the process.  Every height
// computes each output entry by the same sequence of fused multiply-adds, so
// the choice changes the time only, never the result.
// ---------------------------------------------------------------------------
enum GemmKind { GK_PASS = 0, GK_GRAM = 1, GK_APPLY = 2, GK_LIFT = 3, GK_SKETCH = 4 };
struct TuneEntry {
  int rows;
  float ms[3];   // measured time of heights 64, 128, 256 (-1: not valid)
};
std::mutex g_tune_mu;
std::map<std::pair<int, int>, TuneEntry> g_tune;   // (kind, N) -> choice

inline bool rows_valid(int rows, int N) { return N <= 8192 / rows; }
int tuned_rows(int kind, int N) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto f = g_tune.find(std::make_pair(kind, N));
  return f != g_tune.end() ? f->second.rows : bgemm_rows(N);
}

// One GEMM per problem; tasks over blocks of output rows, one launch per
// block height; the height of each GEMM is the tuner's choice for its class.
void add_gemm_stage(Plan& P, const std::vector<BGemm>& gs, int kind) {
  const int g0 = (int)P.gemms.size();
  for (const BGemm& g : gs) P.gemms.push_back(g);
  std::vector<int> h(gs.size());
  for (size_t i = 0; i < gs.size(); ++i) {
    h[i] = tuned_rows(kind, gs[i].N);
    P.gkind.push_back(kind);
    P.tune_cap += (gs[i].M + 63) / 64;
  }
  for (int rows = 64; rows <= 256; rows *= 2) {
    Stage st{ST_GEMM, (int)P.tasks.size(), 0, rows};
    for (int i = 0; i < (int)gs.size(); ++i) {
      if (h[i] != rows) continue;
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
    sp.lo2 = nullptr;
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

// One grouped tensor-core launch: C_i = A_i W_i (form 0) or A_i^T W_i (form 1)
// per problem, W_i^T in nwt bf16 terms (w[0..nwt)).  Tasks ordered by
// decreasing contraction length, so that the CTAs' round-robin shares are even.
struct TcSpec {
  const float* A;
  int64_t arows, acols, lda;   // A as stored (row-major, pitch lda: a multiple of 4)
  const uint16_t* w[3];
  int64_t ldt;                 // pitch of the W^T terms (a multiple of 8)
  float* C;
  int64_t ldc;
  int M, K, ncol, N;
};
void add_tc_stage(Plan& P, int form, int nwt, bool gram, const std::vector<TcSpec>& specs,
                  bool encode) {
  Stage st{ST_TCG, (int)P.tgt.size(), 0, 0};
  st.first2 = (int)P.tgp.size();
  st.form = form;
  st.nwt = nwt;
  st.rows = gram ? 1 : 0;
  std::vector<TgTask> tasks;
  std::vector<int> cost;
  for (size_t i = 0; i < specs.size(); ++i) {
    const TcSpec& sp = specs[i];
    TgProb pr;
    pr.C = sp.C;
    pr.ldc = sp.ldc;
    pr.M = sp.M;
    pr.K = sp.K;
    pr.ncol = sp.ncol;
    pr.N = sp.N;
    P.tgp.push_back(pr);
    CUtensorMap mp[4];
    memset(mp, 0, sizeof(mp));
    if (encode && !tg_encode_maps(form, nwt, sp.A, sp.arows, sp.acols, sp.lda, sp.w[0], sp.w[1],
                                  sp.w[2], sp.K, sp.N, sp.ldt, mp))
      P.map_fail = true;
    for (int t = 0; t < 4; ++t) P.tgm.push_back(mp[t]);
    for (int r0 = 0; r0 < pr.M; r0 += 128) {
      tasks.push_back(TgTask{(int)i, r0});
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

// One pass over every problem's A (A at its 16-byte pitch copy): form 0
// C = A W (W^T from Omega^T when omega, else the split of Z), form 1
// C = A^T W (W^T the split of Y); C = Y (form 0) or Z (form 1).
void add_tc_pass(Plan& P, int batch, const rsvd_batch_item* it, int p, std::vector<ProbBufs>& b,
                 int form, bool omega, bool encode) {
  std::vector<TcSpec> specs;
  for (int i = 0; i < batch; ++i) {
    const int l = it[i].k + p;
    const int64_t m = it[i].m, n = it[i].n;
    TcSpec sp;
    sp.A = b[i].Ap;
    sp.arows = m;
    sp.acols = n;
    sp.lda = pad4(n);
    sp.w[0] = form == 1 ? b[i].Yh : (omega ? b[i].Oh : b[i].Zh);
    sp.w[1] = form == 1 ? b[i].Yl : (omega ? nullptr : b[i].Zl);
    sp.w[2] = nullptr;
    sp.C = form == 0 ? b[i].Y : b[i].Z;
    sp.ldc = l;
    sp.M = (int)(form == 0 ? m : n);
    sp.K = (int)(form == 0 ? n : m);
    sp.ldt = pad8(sp.K);
    sp.ncol = l;
    sp.N = tg_n(l);
    specs.push_back(sp);
  }
  add_tc_stage(P, form, omega ? 1 : 2, false, specs, encode);
}

// R^-1 of every problem in three bf16 terms, transposed: row j of the split
// is column j of R^-1.
void add_rinv_split(Plan& P, int batch, const rsvd_batch_item* it, int p,
                    std::vector<ProbBufs>& b) {
  const int j0 = (int)P.splits.size();
  std::vector<int64_t> rows;
  for (int i = 0; i < batch; ++i) {
    const int l = it[i].k + p;
    TgSplit sp;
    sp.W = b[i].Rinv;
    sp.ldw = l;
    sp.hi = b[i].Rw[0];
    sp.lo = b[i].Rw[1];
    sp.lo2 = b[i].Rw[2];
    sp.rows = l;
    sp.ldt = pad8(l);
    sp.l = l;
    sp.N = tg_n(l);
    sp.batch = i;
    P.splits.push_back(sp);
    rows.push_back(l);
  }
  add_chunks(P, j0, rows, ST_SPLIT);
}

// CholeskyQR2 on the tensor cores: per pass the split of the current X, the
// Gram X^T X, the Cholesky factor and inverse (one CTA a problem), the split
// of R^-1, the apply X R^-1.  X has pitch l (a multiple of 4: TMA).
void add_orth_tc(Plan& P, int batch, const rsvd_batch_item* it, int p, std::vector<ProbBufs>& b,
                 bool on_z, bool want_R, bool encode) {
  for (int pass = 0; pass < 2; ++pass) {
    // split of src
    {
      const int j0 = (int)P.splits.size();
      std::vector<int64_t> rows;
      for (int i = 0; i < batch; ++i) {
        const int l = it[i].k + p;
        const int64_t rr = on_z ? it[i].n : it[i].m;
        TgSplit sp;
        sp.W = pass == 0 ? (on_z ? b[i].Z : b[i].Y) : (on_z ? b[i].Zt : b[i].Yt);
        sp.ldw = l;
        sp.hi = on_z ? b[i].Zh : b[i].Yh;
        sp.lo = on_z ? b[i].Zl : b[i].Yl;
        sp.lo2 = nullptr;
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
    std::vector<TcSpec> gram, apply;
    Stage sc{ST_CHOL, (int)P.chols.size(), batch, 0};
    for (int i = 0; i < batch; ++i) {
      const int l = it[i].k + p;
      const int64_t rr = on_z ? it[i].n : it[i].m;
      float* X = on_z ? b[i].Z : b[i].Y;
      float* Xt = on_z ? b[i].Zt : b[i].Yt;
      float* src = pass == 0 ? X : Xt;
      float* dst = pass == 0 ? Xt : X;
      TcSpec g;
      g.A = src;
      g.arows = rr;
      g.acols = l;
      g.lda = l;
      g.w[0] = on_z ? b[i].Zh : b[i].Yh;
      g.w[1] = on_z ? b[i].Zl : b[i].Yl;
      g.w[2] = nullptr;
      g.ldt = pad8(rr);
      g.C = b[i].G;
      g.ldc = l;
      g.M = l;
      g.K = (int)rr;
      g.ncol = l;
      g.N = tg_n(l);
      gram.push_back(g);
      BChol c;
      c.G = b[i].G;
      c.R = (want_R && pass == 0) ? b[i].Racc : b[i].R;
      c.Rinv = b[i].Rinv;
      c.l = l;
      P.chols.push_back(c);
      TcSpec a;
      a.A = src;
      a.arows = rr;
      a.acols = l;
      a.lda = l;
      a.w[0] = b[i].Rw[0];
      a.w[1] = b[i].Rw[1];
      a.w[2] = b[i].Rw[2];
      a.ldt = pad8(l);
      a.C = dst;
      a.ldc = l;
      a.M = (int)rr;
      a.K = l;
      a.ncol = l;
      a.N = tg_n(l);
      apply.push_back(a);
    }
    add_tc_stage(P, 1, 2, true, gram, encode);
    P.stages.push_back(sc);
    add_rinv_split(P, batch, it, p, b);
    add_tc_stage(P, 0, 3, false, apply, encode);
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
    add_gemm_stage(P, gram, GK_GRAM);
    P.stages.push_back(ss);
    P.stages.push_back(sc);
    add_gemm_stage(P, apply, GK_APPLY);
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
      for (int t = 0; t < 3; ++t) b[i].Rw[t] = cv.take<uint16_t>((size_t)N * pad8(l));
    } else {
      for (int t = 0; t < 3; ++t) b[i].Rw[t] = nullptr;
    }
  }
  // the CholeskyQR steps take TMA maps of the samples, whose pitch (l
  // floats) must be a multiple of 16 bytes
  bool tc_orth = tc;
  for (int i = 0; i < batch && tc_orth; ++i) tc_orth = ((it[i].k + p) % 4) == 0;
  // the orthonormalisations of the power scheme only need a well-conditioned
  // basis of the span: tensor cores; Q and Qh, which the returned U and V are
  // lifted from, keep fp32 products
  auto orth = [&](bool on_z, bool want_R, bool final_q) {
    if (tc_orth && !final_q)
      add_orth_tc(P, batch, it, p, b, on_z, want_R, enc);
    else
      add_orth(P, batch, it, p, b, on_z, want_R);
  };
  if (tc) {
    // A at a 16-byte pitch (a copy unless the problem's rows already are:
    // n a multiple of 4 and A_i 16-byte aligned), then Omega^T of every problem
    std::vector<int64_t> rows;
    const int j0p = (int)P.pads.size();
    for (int i = 0; i < batch; ++i) {
      const float* Ai = A ? A + it[i].a_off : nullptr;
      if (Ai && it[i].n % 4 == 0 && ((uintptr_t)Ai & 15u) == 0) {
        b[i].Ap = const_cast<float*>(Ai);   // read in place (TMA loads only)
        continue;
      }
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
    add_chunks(P, j0p, rows, ST_PAD);
    rows.clear();
    const int j0 = (int)P.splits.size();
    for (int i = 0; i < batch; ++i) {
      const int l = it[i].k + p;
      TgSplit sp;
      sp.W = nullptr;
      sp.ldw = 0;
      sp.hi = b[i].Oh;
      sp.lo = nullptr;
      sp.lo2 = nullptr;
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
    add_gemm_stage(P, gs, GK_SKETCH);
  }
  // power scheme, orthonormalising before every product (Alg. 5, s = 1)
  for (int j = 0; j < q; ++j) {
    orth(false, false, false);
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
      add_gemm_stage(P, gs, GK_PASS);
    }
    orth(true, false, false);
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
      add_gemm_stage(P, gs, GK_PASS);
    }
  }
  orth(false, false, true);                     // Q = orth(Y)
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
    add_gemm_stage(P, gs, GK_PASS);
  }
  orth(true, true, true);                       // Bt = Qh Rh
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
  // U = Q Vh(:, :k), V = Qh Uh(:, :k): plain fp32 (the returned vectors keep
  // 24 bits; the split products hold Q to 16)
  for (int i = 0; i < batch; ++i) {
    const int l = it[i].k + p, k = it[i].k;
    gs.push_back(gemm_of(b[i].Y, l, 0, b[i].Vh, l, U ? U + it[i].u_off : nullptr, k, it[i].m, k,
                         l, k, i));
    gs.push_back(gemm_of(b[i].Z, l, 0, b[i].Uh, l, V ? V + it[i].v_off : nullptr, k, it[i].n, k,
                         l, k, i));
  }
  add_gemm_stage(P, gs, GK_LIFT);

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
  cv.take<int2>((size_t)std::max<int64_t>((int64_t)P.tasks.size(), P.tune_cap));   // any heights
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
  cv.take<int2>((size_t)P.tune_cap);   // the tuner's candidate task lists
  return cv.off + 256;
}

}  // namespace

}  // namespace rsvd

using namespace rsvd;

extern "C" {

int rsvd_batched_tuning(int cap, int* kind, int* width, int* rows, float* ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int i = 0;
  for (const auto& kv : g_tune) {
    if (i < cap) {
      if (kind) kind[i] = kv.first.first;
      if (width) width[i] = kv.first.second;
      if (rows) rows[i] = kv.second.rows;
      if (ms)
        for (int h = 0; h < 3; ++h) ms[3 * i + h] = kv.second.ms[h];
    }
    ++i;
  }
  return i;
}

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
  int2* dt = cv.take<int2>((size_t)std::max<int64_t>((int64_t)P.tasks.size(), P.tune_cap));
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
  int2* dtune = cv.take<int2>((size_t)P.tune_cap);
  // classes of SIMT GEMMs not tuned yet: time each valid block height on this
  // call's GEMMs of the class, keep the fastest, then rebuild the plan with
  // the choices (the tables are uploaded again below)
  {
    std::map<std::pair<int, int>, std::vector<int>> todo;
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      for (size_t g = 0; g < P.gemms.size(); ++g) {
        const auto key = std::make_pair(P.gkind[g], P.gemms[g].N);
        if (!g_tune.count(key)) todo[key].push_back((int)g);
      }
    }
    if (!todo.empty()) {
      cudaEvent_t e0, e1;
      if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return RSVD_ERR_CUDA;
      std::vector<std::pair<std::pair<int, int>, TuneEntry>> found;
      for (const auto& kv : todo) {
        TuneEntry te;
        te.rows = bgemm_rows(kv.first.second);
        float best = -1.f;
        for (int hi = 0; hi < 3; ++hi) {
          const int rows = 64 << hi;
          te.ms[hi] = -1.f;
          if (!rows_valid(rows, kv.first.second)) continue;
          std::vector<int2> tl;
          for (int g : kv.second)
            for (int r0 = 0; r0 < P.gemms[g].M; r0 += rows) tl.push_back(make_int2(g, r0));
          if (tl.empty() || (int64_t)tl.size() > P.tune_cap) continue;
          if (cudaMemcpyAsync(dtune, tl.data(), tl.size() * sizeof(int2), cudaMemcpyHostToDevice,
                              s) != cudaSuccess ||
              launch_bgemm(dg, dtune, (int)tl.size(), rows, seed, s) != cudaSuccess ||
              cudaEventRecord(e0, s) != cudaSuccess ||
              launch_bgemm(dg, dtune, (int)tl.size(), rows, seed, s) != cudaSuccess ||
              cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return RSVD_ERR_CUDA;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          te.ms[hi] = ms;
          if (best < 0.f || ms < best) {
            best = ms;
            te.rows = rows;
          }
        }
        found.push_back(std::make_pair(kv.first, te));
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (const auto& f : found) g_tune.emplace(f.first, f.second);
      }
      // the plan again, with the tuned heights (same tables, same carving)
      Plan P2;
      char* tables2 = nullptr;
      build(batch, items, p, q, A, U, S, V, (char*)work, P2, &tables2, true);
      if (P2.map_fail || tables2 != tables || (int64_t)P2.tasks.size() > P.tune_cap)
        return RSVD_ERR_CUDA;
      if (!P2.tasks.empty() &&
          cudaMemcpyAsync(dt, P2.tasks.data(), P2.tasks.size() * sizeof(int2),
                          cudaMemcpyHostToDevice, s) != cudaSuccess)
        return RSVD_ERR_CUDA;
      P.stages = P2.stages;
      P.tasks = P2.tasks;
    }
  }
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
        e = launch_tc_group(st.form, st.nwt, st.rows != 0, dtp + st.first2, dtt + st.first,
                            st.count, dtm + 4 * (int64_t)st.first2, d_info, s);
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
