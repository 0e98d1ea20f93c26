"""GPU parity of the tolerance modes (Sec. 2.6; Sec. 4 TOL mode) and of the
left-sketch ID (Sec. 3.5, Alg. 6) against the oracle's id_tol, svd_rank_tol,
cur_from_id and rid_left, through the C ABI.

Bars:
* ranks equal the oracle's: each tolerance sits between two of the oracle's
  residual norms ||S22(j)||_F (or singular values) that differ by orders of
  magnitude, so FP32 rounding (~1e-5 relative) cannot move the decision;
* pivots identical at every step before the first oracle step whose gap
  (nu1 - nu2) / nu1 is <= 1e-6, as for the fixed-rank ID;
* T, the CUR's U and the reconstruction errors within 1 % of the oracle's
  errors (relative error of the factorisation, in FP64 on the host).
"""
import numpy as np
import pytest

from oracle import rsvd as orc
from synth import make_matrix_np, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def _matched_prefix(J, Jo, gaps):
    t = 0
    while t < len(gaps) and t < len(J) and J[t] == Jo[t]:
        t += 1
    first_small = next((i for i, g in enumerate(gaps) if g <= 1e-6), len(gaps))
    return t, first_small


def _stepped(m, n, r, seed, dtype, noise=1e-7):
    """Rank-r matrix with a logspace(0, -2) spectrum plus small noise: the
    residual norms drop by orders of magnitude after r pivoted-QR steps."""
    sig = np.logspace(0.0, -2.0, r)
    return make_matrix_np(m, n, sig, noise=noise, seed=seed, dtype=dtype)


CASES = [("f32", "float32", 1200, 900, 30), ("f64", "float64", 1000, 700, 24),
         ("f32_ragged", "float32", 1001, 777, 13)]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_id_tol_rank_and_pivots(case):
    _, dtype, m, n, r = case
    kmax, p, q, seed = r + 10, 8, 1, 0x7001
    A = _stepped(m, n, r, 11 + m, dtype)
    A64 = A.astype(np.float64)
    rounding = "f64" if dtype == "float64" else "bf16"
    tdt = torch.float64 if dtype == "float64" else torch.float32
    Qo, Bto = orc.qb(A64, kmax, p, q, seed, rounding=rounding)
    for tol in (1e-3, None):
        if tol is None:
            # a tolerance in the smooth part: between the oracle's norms after
            # r // 2 and r // 2 + 1 steps (geometric mean)
            _, _, _, norms = orc.id_tol(Bto.T, 1.0)
            j = r // 2
            tol = float(np.sqrt(norms[j] * norms[j + 1]))
        Jo, To, ko, norms = orc.id_tol(Bto.T, tol)
        assert 1 <= ko <= kmax
        J, T, k = rs.id_tol(_dev(A, tdt), kmax, p, q, tol, seed)
        assert k == ko, (k, ko, norms[:ko + 2], tol)
        J = J.cpu().numpy()
        _, _, gaps = orc.id_from_matrix(Bto.T, k)
        t, first_small = _matched_prefix(J, Jo, gaps)
        assert t >= min(first_small, k), (t, first_small)
        assert sorted(J.tolist()) == list(range(n))
        if t >= k:
            e = orc.rel_err_id(A64, J, T.double().cpu().numpy(), k)
            eo = orc.rel_err_id(A64, Jo, To, k)
            assert abs(e - eo) <= 0.01 * eo + 1e-12, (e, eo)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_cur_tol(dtype):
    m, n, r = 1100, 800, 20
    kmax, p, q, seed, tol = 32, 8, 1, 0x7002, 1e-3
    A = _stepped(m, n, r, 5, dtype)
    A64 = A.astype(np.float64)
    rounding = "f64" if dtype == "float64" else "bf16"
    tdt = torch.float64 if dtype == "float64" else torch.float32
    _, Bto = orc.qb(A64, kmax, p, q, seed, rounding=rounding)
    Jo, To, ko, _ = orc.id_tol(Bto.T, tol)
    Io, Uo, rgaps = orc.cur_from_id(A64, Jo, To, ko)
    Jc, Ir, U, k = rs.cur_tol(_dev(A, tdt), kmax, p, q, tol, seed)
    assert k == ko == r
    _, _, cgaps = orc.id_from_matrix(Bto.T, k)
    Jc, Ir = Jc.cpu().numpy(), Ir.cpu().numpy()
    t, first_small = _matched_prefix(Jc, Jo[:k], cgaps)
    assert t >= min(first_small, k)
    if t >= k:
        tr, first_small_r = _matched_prefix(Ir, Io, rgaps)
        assert tr >= min(first_small_r, k)
        e = orc.rel_err_cur(A64, Jc, Ir, U.double().cpu().numpy())
        eo = orc.rel_err_cur(A64, Jo[:k], Io, Uo)
        assert abs(e - eo) <= 0.01 * eo + 1e-10, (e, eo)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_svd_tol(dtype):
    m, n = 1500, 1000
    kmax, p, q, seed = 60, 10, 2, 0x7003
    # sigma_j = exp(-j / 10): tol = exp(-3.55) sits between sigma_35 and sigma_36
    A = make_matrix_np(m, n, np.exp(-np.arange(1, n + 1) / 10.0), seed=8, dtype=dtype)
    A64 = A.astype(np.float64)
    rounding = "f64" if dtype == "float64" else "bf16"
    tdt = torch.float64 if dtype == "float64" else torch.float32
    tol = float(np.exp(-3.55))
    Uo, So, Vo, _ = orc.rsvd(A64, kmax, p, q, seed, rounding=rounding)
    ko = orc.svd_rank_tol(So, tol)
    U, S, V = rs.svd_tol(_dev(A, tdt), kmax, p, q, tol, seed)
    assert S.numel() == ko == 35
    S = S.cpu().numpy()
    bar = 1e-10 if dtype == "float64" else 1e-5
    assert np.max(np.abs(S - So[:ko]) / So[:ko]) <= bar
    e = orc.rel_err_svd(A64, U.double().cpu().numpy(), S, V.double().cpu().numpy())
    eo = orc.rel_err_svd(A64, Uo[:, :ko], So[:ko], Vo[:, :ko])
    assert abs(e - eo) <= 0.01 * eo, (e, eo)


LEFT = [("f32_q0", "float32", 900, 700, 20, 8, 0), ("f32_q2", "float32", 1300, 1000, 30, 10, 2),
        ("f64_q1", "float64", 1000, 800, 25, 8, 1), ("f32_ragged_q1", "float32", 1001, 513, 13, 5, 1)]


@pytest.mark.parametrize("case", LEFT, ids=[c[0] for c in LEFT])
def test_id_left_sketch(case):
    _, dtype, m, n, k, p, q = case
    seed = 0x7004 + q
    A = make_matrix_np(m, n, spectrum("logspace3", n), noise=1e-6, seed=m + n, dtype=dtype)
    A64 = A.astype(np.float64)
    rounding = "f64" if dtype == "float64" else "bf16"
    tdt = torch.float64 if dtype == "float64" else torch.float32
    J, T = rs.id_left(_dev(A, tdt), k, p, q, seed)
    J, T = J.cpu().numpy(), T.double().cpu().numpy()
    Jo, To, gaps, _ = orc.rid_left(A64, k, p, q, seed, rounding=rounding)
    t, first_small = _matched_prefix(J, Jo, gaps)
    assert t >= min(first_small, k), (t, first_small)
    assert sorted(J.tolist()) == list(range(n))
    if t >= k:
        e = orc.rel_err_id(A64, J, T, k)
        eo = orc.rel_err_id(A64, Jo, To, k)
        assert abs(e - eo) <= 0.01 * eo + 1e-12, (e, eo)
