"""Parity at the full size of the bench workload: A = 50000 x 20000 fp32 (the C2
recipe: sigma_j = 1/j for j <= 2000 plus 1e-4 N(0,1) noise), k = 200, p = 20,
q = 2, through the call bench.py times (one Plan on the tensor-core path) and
the same kernels at the same sizes (rs.sample, rs.qb), on outputs the oracle
computes one by one:

* 16 rows of the sketch Y = A Omega against those rows of A times Omega (the
  kernels' own Omega: bar 2e-4; the oracle's Omega, which differs by rare bf16
  rounding flips: bar 3e-4).  At n = 20000 the fp32 accumulation runs over 5x
  the contraction of the 2e-5 / 1e-4 small-size bars.
* 16 rows of Bt = A^T Q against the matching columns of A times the library's
  own Q, contraction over m = 50000 (bar 5e-4; 3e-5 at K <= 4096).
* The k singular values of the plan against LAPACK's on the library's own B
  (host FP64): per index 3e-4.  Weyl bounds the difference by the absolute
  error of the small SVD (~1e-6 ||B||), and sigma_k sits in the noise bulk
  near 0.035 ||B||.
* The plan's ID pivots against the oracle's CPQR fed the library's own B: the
  same at every step before the first whose oracle gap is <= 1e-6; where all
  k match, T against the oracle's T (fp32 output: bar 1e-5).

* The whole path against the FP64 oracle itself (oracle.rsvd and oracle.rcur on
  the same stored A promoted to float64, the same seed and the bf16 rounding of
  Omega): singular values per index (1e-5 above the noise edge, where sigma_i
  exceeds twice the noise's spectral norm; a documented looser bar in the
  noise bulk), reconstruction errors within 1 %, ID and CUR indices identical
  before the first oracle step whose pivot gap is <= 1e-6, CUR error within 1 %.

Collected after the other parity files (file name): it builds the 4 GB matrix,
the slowest setup of the suite.
"""
import numpy as np
import pytest

from oracle import philox, rsvd as orc
from synth import config, make_matrix_torch, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def c2():
    cfg = config("c2_f32_50000x20000")
    A = make_matrix_torch(cfg["m"], cfg["n"], spectrum(cfg["spectrum"], cfg["r"]),
                          noise=cfg["noise"], seed=cfg["a_seed"], dtype=cfg["dtype"], device=DEV)
    torch.cuda.synchronize()
    yield cfg, A
    del A
    torch.cuda.empty_cache()


def _rows(X, idx):
    return X[torch.as_tensor(idx, device=X.device)].double().cpu().numpy()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


IDX_M = [0, 1, 4097, 12345, 24999, 25000, 31337, 40000, 44444, 47000, 49151, 49152, 49900,
         49997, 49998, 49999]
IDX_N = [0, 1, 255, 256, 4096, 7777, 9999, 10000, 12288, 15000, 17001, 19455, 19456, 19800,
         19998, 19999]


def test_fullsize_sketch_rows(c2):
    cfg, A = c2
    n, l, seed = cfg["n"], cfg["k"] + cfg["p"], cfg["omega_seed"]
    Y = rs.sample(A, l, seed)
    Ar = _rows(A, IDX_M)
    Yr = _rows(Y, IDX_M)
    Om_gpu = rs.omega(n, l, seed, torch.float32, DEV).double().cpu().numpy()
    assert _rel(Yr, Ar @ Om_gpu) <= 2e-4
    assert _rel(Yr, Ar @ philox.omega(n, l, seed, "bf16")) <= 3e-4


def test_fullsize_plan_against_its_own_sketch(c2):
    cfg, A = c2
    m, n, k, p, q, seed = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["q"], cfg["omega_seed"]
    plan = rs.Plan(m, n, k, p, q, torch.float32, DEV)
    plan.run(A, seed)
    torch.cuda.synchronize()
    rs.check_info(plan.info, "plan")
    Q, Bt = rs.qb(A, k, p, q, seed)
    Qn = Q.double().cpu().numpy()
    Btn = Bt.double().cpu().numpy()
    # Bt = A^T Q on sampled rows (columns of A)
    Acols = A[:, torch.as_tensor(IDX_N, device=DEV)].double().cpu().numpy()
    assert _rel(Btn[IDX_N], Acols.T @ Qn) <= 5e-4
    # singular values of the plan against LAPACK on the same B
    s_host = np.linalg.svd(Btn, compute_uv=False)[:k]
    S = plan.S.cpu().numpy()
    assert np.all(np.diff(S) <= 0)
    assert np.max(np.abs(S - s_host) / s_host) <= 3e-4
    # ID pivots against the oracle's CPQR of the same B
    J = plan.J.cpu().numpy()
    assert sorted(J.tolist()) == list(range(n))
    Jo, To, gaps = orc.id_from_matrix(Btn.T, k)
    t = 0
    while t < k and J[t] == Jo[t]:
        t += 1
    first_small = next((i for i, g in enumerate(gaps) if g <= 1e-6), k)
    assert t >= min(first_small, k), (t, first_small)
    if t >= k:
        # the same k pivots make the same LAPACK-style exchanges, so both T are
        # indexed by the same order of J[k:]
        assert np.array_equal(J, Jo)
        assert _rel(plan.T.double().cpu().numpy(), To) <= 1e-5


def _rel_err_cur_blocked(A64, Jc, Ir, U, block=5000):
    """||A - A(:, Jc) U A(Ir, :)||_F / ||A||_F in FP64, row block by row block."""
    CU = A64[:, Jc] @ U
    R = A64[Ir, :]
    num = den = 0.0
    for i0 in range(0, A64.shape[0], block):
        Ab = A64[i0:i0 + block]
        D = Ab - CU[i0:i0 + block] @ R
        num += float(np.sum(D * D))
        den += float(np.sum(Ab * Ab))
    return np.sqrt(num / den)


def test_fullsize_whole_path_against_the_oracle(c2):
    """The bench's call (one Plan: SVD, ID and CUR from one sketch) against the
    oracle's Alg. 5, ID and CUR run in FP64 on the same matrix and Omega."""
    cfg, A = c2
    m, n, k, p, q, seed = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["q"], cfg["omega_seed"]
    plan = rs.Plan(m, n, k, p, q, torch.float32, DEV)
    plan.run(A, seed)
    torch.cuda.synchronize()
    rs.check_info(plan.info, "plan")
    A64 = A.cpu().numpy().astype(np.float64)
    Uo, So, Vo, _ = orc.rsvd(A64, k, p, q, seed, rounding="bf16")
    Jco, Iro, Ucuro, Jo, To, cgaps, rgaps = orc.rcur(A64, k, p, q, seed, rounding="bf16")
    S = plan.S.cpu().numpy()
    rel = np.abs(S - So) / So
    # noise edge: the 1e-4 N(0,1) noise has spectral norm ~1e-4 (sqrt(m) + sqrt(n))
    edge = 2.0 * cfg["noise"] * (np.sqrt(m) + np.sqrt(n))
    top = So > edge                  # sigma_j = 1/j: the first 14 at this size
    assert top.sum() >= 10 and top[:top.sum()].all()
    print("sigma rel err: above edge (%d) max %.2e; bulk max %.2e median %.2e"
          % (top.sum(), rel[top].max(), rel[~top].max(), np.median(rel[~top])))
    assert rel[top].max() <= 1e-5, rel[top].max()
    assert rel.max() <= 1e-4, rel.max()
    e_gpu = orc.rel_err_svd(A64, plan.U.double().cpu().numpy(), S, plan.V.double().cpu().numpy())
    e_orc = orc.rel_err_svd(A64, Uo, So, Vo)
    assert abs(e_gpu - e_orc) <= 0.01 * e_orc, (e_gpu, e_orc)
    # ID pivots: identical before the first oracle gap <= 1e-6
    J = plan.J.cpu().numpy()
    t = 0
    while t < k and J[t] == Jo[t]:
        t += 1
    first_small = next((i for i, g in enumerate(cgaps) if g <= 1e-6), k)
    print("ID pivots: %d of %d match; first oracle gap <= 1e-6 at %d" % (t, k, first_small))
    assert t >= min(first_small, k), (t, first_small)
    # CUR: row pivots by the same rule (when every column pivot matched), error within 1 %
    Ir = plan.Ir.cpu().numpy()
    if t >= k:
        tr = 0
        while tr < k and Ir[tr] == Iro[tr]:
            tr += 1
        first_small_r = next((i for i, g in enumerate(rgaps) if g <= 1e-6), k)
        print("CUR row pivots: %d of %d match; first oracle gap <= 1e-6 at %d"
              % (tr, k, first_small_r))
        assert tr >= min(first_small_r, k), (tr, first_small_r)
    c_gpu = _rel_err_cur_blocked(A64, plan.Jc.cpu().numpy(), Ir, plan.Ucur.double().cpu().numpy())
    c_orc = _rel_err_cur_blocked(A64, Jco, Iro, Ucuro)
    assert abs(c_gpu - c_orc) <= 0.01 * c_orc, (c_gpu, c_orc)
