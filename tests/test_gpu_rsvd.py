"""End-to-end GPU parity of rsvd_qb / rsvd_svd / rsvd_id / rsvd_cur against the oracle.

Bars (from the workload statement; "relative 1e-5" is per index i <= k, "within
1 %" is on ||A - U S V^T||_F / ||A||_F in FP64):
* top-k singular values: relative 1e-5 (FP32 paths), 1e-10 (FP64);
* reconstruction error ||A - U S V^T||_F / ||A||_F within 1 % of the oracle's;
* ID / CUR indices identical at every step before the first one whose pivot
  gap (nu1 - nu2) / nu1 is <= 1e-6 (oracle gaps); and identical everywhere when
  the oracle's CPQR is fed the GPU's own B (decoupled check).
"""
import numpy as np
import pytest

from oracle import rsvd as orc
from synth import make_matrix_np, spectrum, low_rank_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def _matched_prefix(J, Jo, gaps):
    t = 0
    while t < len(gaps) and J[t] == Jo[t]:
        t += 1
    first_small = next((i for i, g in enumerate(gaps) if g <= 1e-6), len(gaps))
    return t, first_small


CASES = [
    # name, m, n, k, p, q, spectrum, noise, dtype, precision
    ("c1_f64_full", 2000, 1000, 50, 10, 1, "exp20", 0.0, "float64", None),
    ("c2_like_f32", 3000, 2000, 40, 10, 2, "inv", 1e-4, "float32", "tc"),
    ("c2_like_f32_simt", 3000, 2000, 40, 10, 2, "inv", 1e-4, "float32", "simt"),
    ("c5_like_f32", 2048, 1024, 64, 16, 2, "sqrtgap64", 0.0, "float32", "tc"),
    ("ragged_f32", 1001, 777, 13, 5, 1, "logspace3", 1e-5, "float32", "tc"),
    ("q0_p0_f32", 900, 600, 20, 0, 0, "logspace4", 0.0, "float32", "tc"),
    ("k1_f64", 300, 200, 1, 4, 2, "logspace2", 0.0, "float64", None),
    # short and wide A (m < n): the contraction of Bt = A^T Q runs over the short side
    ("wide_f32", 700, 1900, 30, 10, 1, "logspace3", 1e-5, "float32", "tc"),
    ("wide_ragged_f32", 517, 2049, 37, 11, 2, "inv", 1e-4, "float32", "tc"),
    # l = m: Q is square and B = Q^T A keeps all of A
    ("l_eq_m_f64", 60, 500, 50, 10, 1, "logspace2", 0.0, "float64", None),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_svd_id_cur_parity(case):
    name, m, n, k, p, q, spec, noise, dtype, prec = case
    r = min(m, n) if spec != "inv" else min(2000, m, n)
    sig = spectrum(spec, r)
    A = make_matrix_np(m, n, sig, noise=noise, seed=0xA000 + m, dtype=dtype)
    A64 = A.astype(np.float64)
    seed = 0x5EED + k
    rounding = "f64" if dtype == "float64" else "bf16"
    opts = rs.make_opts(precision=rs.PREC_SIMT) if prec == "simt" else None
    tdt = torch.float64 if dtype == "float64" else torch.float32
    out = rs.svd_id_cur(_dev(A, tdt), k, p, q, seed, opts)
    S = out["S"].cpu().numpy()
    U = out["U"].double().cpu().numpy()
    V = out["V"].double().cpu().numpy()
    Uo, So, Vo, _ = orc.rsvd(A64, k, p, q, seed, rounding=rounding)
    tol = 1e-10 if dtype == "float64" else 1e-5
    rel = np.abs(S - So) / So
    assert np.max(rel) <= tol, (name, np.max(rel), np.argmax(rel))
    e_gpu = orc.rel_err_svd(A64, U, S, V)
    e_orc = orc.rel_err_svd(A64, Uo, So, Vo)
    assert abs(e_gpu - e_orc) <= 0.01 * e_orc + 1e-12, (e_gpu, e_orc)
    ortho_tol = 1e-12 if dtype == "float64" else 5e-5
    assert np.linalg.norm(U.T @ U - np.eye(k)) <= ortho_tol
    assert np.linalg.norm(V.T @ V - np.eye(k)) <= ortho_tol
    # sign rule on the GPU output: the largest |entry| of each v_j is positive
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(k)] > 0)
    # singular vectors agree with the oracle up to the accuracy of sigma gaps
    cosu = np.abs(np.sum(U * Uo, axis=0))
    gap = np.minimum(np.abs(np.diff(np.r_[np.inf, So])), np.abs(np.diff(np.r_[So, 0.0])))
    well = gap / So > 1e-2
    assert np.all(cosu[well] > 1 - 1e-4)

    # ---- ID ----
    J = out["J"].cpu().numpy()
    T = out["T"].double().cpu().numpy()
    Jo, To, gaps, (Qo, Bto) = orc.rid(A64, k, p, q, seed, rounding=rounding)
    t, first_small = _matched_prefix(J, Jo, gaps)
    assert t >= min(first_small, k), (name, t, first_small)
    assert sorted(J.tolist()) == list(range(n))            # a permutation
    e_id = orc.rel_err_id(A64, J, T, k)
    e_id_o = orc.rel_err_id(A64, Jo, To, k)
    if t >= k:
        assert abs(e_id - e_id_o) <= 0.01 * e_id_o + 1e-12
    # ---- CUR ----
    Jc = out["Jc"].cpu().numpy()
    Ir = out["Ir"].cpu().numpy()
    Uc = out["Ucur"].double().cpu().numpy()
    assert np.array_equal(Jc, J[:k])
    Jco, Iro, Uco, _, _, _, rgaps = orc.rcur(A64, k, p, q, seed, rounding=rounding)
    if t >= k:
        tr, first_small_r = _matched_prefix(Ir, Iro, rgaps)
        assert tr >= min(first_small_r, k)
        if tr >= k:
            e_c = orc.rel_err_cur(A64, Jc, Ir, Uc)
            e_co = orc.rel_err_cur(A64, Jco, Iro, Uco)
            assert abs(e_c - e_co) <= 0.01 * e_co + 1e-10, (e_c, e_co)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_decoupled_cpqr_on_gpu_sketch(dtype):
    """The oracle's CPQR fed the GPU's own B = Q^T A must pick the same pivots."""
    m, n, k, p, q = 1500, 1200, 30, 10, 1
    A = make_matrix_np(m, n, spectrum("logspace3", n), noise=1e-6, seed=3, dtype=dtype)
    tdt = torch.float64 if dtype == "float64" else torch.float32
    Q, Bt = rs.qb(_dev(A, tdt), k, p, q, 77)
    J, T = rs.id(_dev(A, tdt), k, p, q, 77)
    B = Bt.double().cpu().numpy().T
    Jo, To, gaps = orc.id_from_matrix(B, k)
    J = J.cpu().numpy()
    t, first_small = _matched_prefix(J, Jo, gaps)
    assert t >= min(first_small, k)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("q", [0, 2])
def test_exact_rank_recovery(dtype, q):
    m, n, rank = 800, 600, 9
    A = low_rank_np(m, n, rank, seed=5, dtype=dtype)
    tdt = torch.float64 if dtype == "float64" else torch.float32
    Q, Bt = rs.qb(_dev(A, tdt), 10, 4, q, 11)
    Qn, Btn = Q.double().cpu().numpy(), Bt.double().cpu().numpy()
    err = np.linalg.norm(A - Qn @ Btn.T) / np.linalg.norm(A)
    # FP32 tensor-core products carry 16-bit splits: noise ~2^-17 per product
    assert err <= (1e-12 if dtype == "float64" else 5e-5), err
    assert np.linalg.norm(Qn.T @ Qn - np.eye(14)) <= (1e-12 if dtype == "float64" else 5e-5)


def test_qb_matches_oracle_subspace():
    m, n, k, p, q = 2500, 1800, 48, 16, 2
    A = make_matrix_np(m, n, spectrum("sqrtgap64", n), seed=9, dtype="float32")
    Q, Bt = rs.qb(_dev(A, torch.float32), k, p, q, 5)
    Qo, Bto = orc.qb(A.astype(np.float64), k, p, q, 5, rounding="bf16")
    Qn = Q.double().cpu().numpy()
    # same subspace: the projectors agree on the dominant directions
    P = Qn.T @ Qo
    sv = np.linalg.svd(P, compute_uv=False)
    assert sv[k - 1] > 1 - 1e-4
    Btn = Bt.double().cpu().numpy()
    assert abs(np.linalg.norm(Btn) - np.linalg.norm(Bto)) <= 1e-5 * np.linalg.norm(Bto)


def test_determinism_same_seed():
    A = make_matrix_np(1200, 900, spectrum("logspace3", 900), noise=1e-5, seed=2,
                       dtype="float32")
    At = _dev(A, torch.float32)
    a = rs.svd_id_cur(At, 20, 8, 2, 42)
    b = rs.svd_id_cur(At, 20, 8, 2, 42)
    for key in a:
        assert torch.equal(a[key], b[key]), key


def test_invalid_arguments_rejected():
    A = torch.zeros(100, 50, device=DEV)
    with pytest.raises(rs.RsvdError) as e:
        rs.svd(A, 0, 5, 1, 1)
    assert e.value.code == 1
    with pytest.raises(rs.RsvdError):
        rs.svd(A, 40, 20, 1, 1)      # l > n


def test_zero_matrix_reports_not_spd():
    A = torch.zeros(300, 200, device=DEV)
    with pytest.raises(rs.RsvdError) as e:
        rs.svd(A, 5, 5, 1, 1)
    assert e.value.code in (5, 7)


@pytest.mark.parametrize("dtype", ["float32", "float64"])
def test_host_input_entry_point(dtype):
    """rsvd_svd_id_cur_host: A copied from page-locked host memory (in row
    chunks behind the sketch on the FP32 path) gives the device call's results
    and leaves A in the device buffer."""
    m, n, k, p, q = 3000, 2000, 40, 10, 2
    A = make_matrix_np(m, n, spectrum("inv", 2000), noise=1e-4, seed=21, dtype=dtype)
    tdt = torch.float64 if dtype == "float64" else torch.float32
    A_dev = _dev(A, tdt)
    plan = rs.Plan(m, n, k, p, q, tdt, DEV)
    plan.run(A_dev, 99)
    torch.cuda.synchronize()
    rs.check_info(plan.info)
    S_d, J_d = plan.S.clone(), plan.J.clone()
    A_host = torch.from_numpy(np.ascontiguousarray(A)).to(tdt).pin_memory()
    A_dev2 = torch.empty_like(A_dev)
    plan.run_host(A_host, A_dev2, 99)
    torch.cuda.synchronize()
    rs.check_info(plan.info)
    assert torch.equal(A_dev2, A_dev)
    tol = 1e-10 if dtype == "float64" else 1e-5
    rel = (plan.S - S_d).abs() / S_d
    assert rel.max().item() <= tol
    assert torch.equal(plan.J[:k], J_d[:k])
