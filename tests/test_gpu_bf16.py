"""GPU parity of the BF16-storage path (A held as bf16, RSVD_BF16) against the oracle.

The oracle runs on the stored bf16 values of A promoted to FP64, so parity is
about the algorithm, not about the bf16 rounding of A (which is measured
separately against the FP32 path, at equal relative error).

Tolerances: the bf16 values of A and Omega are exact tensor-core operands and
their products are exact in the fp32 accumulators, so the sketch Y = A Omega
carries only fp32 accumulation error (~1e-6 relative); the stored right-hand
operands (Y, Z, Q) keep two bf16 terms as on the FP32 path (2^-17 per
product).  The whole-path bars are those of the FP32 path.
"""
import numpy as np
import pytest

from oracle import philox, rsvd as orc
from synth import make_matrix_np, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _bf16(x):
    """(device bf16 tensor, the same values as a float64 array)."""
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t.to(DEV), t.double().numpy()


def _elem_err(Y, ref, absprod):
    """max over entries of |Y - ref| / (|A| |W|): each entry against the error
    bound of its own dot product; entries whose bound is zero must be zero."""
    d = np.abs(np.asarray(Y, dtype=np.float64) - ref)
    den = np.asarray(absprod, dtype=np.float64)
    assert np.all(d[den == 0] == 0)
    nz = den > 0
    return float(np.max(d[nz] / den[nz])) if nz.any() else 0.0


# lda % 8 == 0; the last shape is ragged against the 512- and 256-row units
SHAPES = [(1000, 800, 60), (4096, 2048, 220), (1001, 776, 13), (257, 296, 64),
          (16411, 4104, 220)]


@pytest.mark.parametrize("m,n,l", SHAPES)
def test_sample_bf16(m, n, l):
    rng = np.random.default_rng(3 * m + n + l)
    Ab, A64 = _bf16(rng.standard_normal((m, n)))
    seed = 77 + l
    Y = rs.sample(Ab, l, seed).cpu().numpy()
    # against the kernels' own Omega: only fp32 accumulation error
    Om_gpu = rs.omega(n, l, seed, torch.float32, DEV).double().cpu().numpy()
    assert _rel(Y, A64 @ Om_gpu) <= 1e-5
    # element-wise: exact products, fp32 accumulation only
    e = _elem_err(Y, A64 @ Om_gpu, np.abs(A64) @ np.abs(Om_gpu))
    assert e <= 1e-5, e
    # against the oracle's Omega (rare bf16 rounding flips of a Gaussian)
    assert _rel(Y, A64 @ philox.omega(n, l, seed, "bf16")) <= 1e-4


@pytest.mark.parametrize("m,n,l", SHAPES)
@pytest.mark.parametrize("trans", [0, 1])
def test_apply_bf16(m, n, l, trans):
    rng = np.random.default_rng(5 * m + n + l + trans)
    Ab, A64 = _bf16(rng.standard_normal((m, n)))
    X = rng.standard_normal((m if trans else n, l)).astype(np.float32)
    Y = rs.apply(Ab, torch.from_numpy(X).to(DEV), trans).cpu().numpy()
    X64 = X.astype(np.float64)
    ref = (A64.T @ X64) if trans else (A64 @ X64)
    assert _rel(Y, ref) <= 3e-5, _rel(Y, ref)
    # element-wise: two bf16 terms of X (2^-16 per product) and fp32 accumulation
    a, x = np.abs(A64), np.abs(X64)
    e = _elem_err(Y, ref, (a.T @ x) if trans else (a @ x))
    assert e <= 5e-5, e


def _matched_prefix(J, Jo, gaps):
    t = 0
    while t < len(gaps) and J[t] == Jo[t]:
        t += 1
    first_small = next((i for i, g in enumerate(gaps) if g <= 1e-6), len(gaps))
    return t, first_small


CASES = [
    # name, m, n, k, p, q, spectrum, noise
    ("c2_like_bf16", 3000, 2000, 40, 10, 2, "inv", 1e-4),
    ("c5_like_bf16", 2048, 1024, 64, 16, 2, "sqrtgap64", 0.0),
    ("ragged_bf16", 1001, 776, 13, 5, 1, "logspace3", 1e-5),
    ("wide_bf16", 520, 2048, 37, 11, 2, "inv", 1e-4),      # m < n
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_svd_id_cur_parity_bf16(case):
    name, m, n, k, p, q, spec, noise = case
    r = min(m, n) if spec != "inv" else min(2000, m, n)
    A32 = make_matrix_np(m, n, spectrum(spec, r), noise=noise, seed=0xB000 + m, dtype="float32")
    Ab, A64 = _bf16(A32)
    seed = 0x5EED + k
    out = rs.svd_id_cur(Ab, k, p, q, seed)
    S = out["S"].cpu().numpy()
    U = out["U"].double().cpu().numpy()
    V = out["V"].double().cpu().numpy()
    Uo, So, Vo, _ = orc.rsvd(A64, k, p, q, seed, rounding="bf16")
    rel = np.abs(S - So) / So
    assert np.max(rel) <= 1e-5, (name, np.max(rel), np.argmax(rel))
    e_gpu = orc.rel_err_svd(A64, U, S, V)
    e_orc = orc.rel_err_svd(A64, Uo, So, Vo)
    assert abs(e_gpu - e_orc) <= 0.01 * e_orc + 1e-12, (e_gpu, e_orc)
    assert np.linalg.norm(U.T @ U - np.eye(k)) <= 5e-5
    assert np.linalg.norm(V.T @ V - np.eye(k)) <= 5e-5
    J = out["J"].cpu().numpy()
    T = out["T"].double().cpu().numpy()
    Jo, To, gaps, _ = orc.rid(A64, k, p, q, seed, rounding="bf16")
    t, first_small = _matched_prefix(J, Jo, gaps)
    assert t >= min(first_small, k), (name, t, first_small)
    assert sorted(J.tolist()) == list(range(n))
    if t >= k:
        e_id = orc.rel_err_id(A64, J, T, k)
        e_id_o = orc.rel_err_id(A64, Jo, To, k)
        assert abs(e_id - e_id_o) <= 0.01 * e_id_o + 1e-12
        Jc = out["Jc"].cpu().numpy()
        Ir = out["Ir"].cpu().numpy()
        Uc = out["Ucur"].double().cpu().numpy()
        assert np.array_equal(Jc, J[:k])
        Jco, Iro, Uco, _, _, _, rgaps = orc.rcur(A64, k, p, q, seed, rounding="bf16")
        tr, first_small_r = _matched_prefix(Ir, Iro, rgaps)
        assert tr >= min(first_small_r, k)
        if tr >= k:
            e_c = orc.rel_err_cur(A64, Jc, Ir, Uc)
            e_co = orc.rel_err_cur(A64, Jco, Iro, Uco)
            assert abs(e_c - e_co) <= 0.01 * e_co + 1e-10, (e_c, e_co)


def test_bf16_storage_equal_error_to_fp32():
    """On a matrix with a noise tail above the bf16 rounding of A, the BF16
    path reaches the FP32 path's relative error (within 1 %) on the FP32 A."""
    m, n, k, p, q = 4000, 2496, 50, 10, 2
    A32 = make_matrix_np(m, n, spectrum("inv", 2000), noise=1e-4, seed=41, dtype="float32")
    A64 = A32.astype(np.float64)
    o32 = rs.svd_id_cur(torch.from_numpy(A32).to(DEV), k, p, q, 9)
    Ab, _ = _bf16(A32)
    o16 = rs.svd_id_cur(Ab, k, p, q, 9)
    e32 = orc.rel_err_svd(A64, o32["U"].double().cpu().numpy(), o32["S"].cpu().numpy(),
                          o32["V"].double().cpu().numpy())
    e16 = orc.rel_err_svd(A64, o16["U"].double().cpu().numpy(), o16["S"].cpu().numpy(),
                          o16["V"].double().cpu().numpy())
    assert abs(e16 - e32) <= 0.01 * e32, (e16, e32)


def test_bf16_host_input_entry_point():
    m, n, k, p, q = 3000, 2000, 40, 10, 2
    A32 = make_matrix_np(m, n, spectrum("inv", 2000), noise=1e-4, seed=23, dtype="float32")
    Ab, _ = _bf16(A32)
    plan = rs.Plan(m, n, k, p, q, torch.bfloat16, DEV)
    plan.run(Ab, 5)
    torch.cuda.synchronize()
    rs.check_info(plan.info)
    S_d, J_d = plan.S.clone(), plan.J.clone()
    A_host = Ab.cpu().pin_memory()
    A_dev2 = torch.empty_like(Ab)
    plan.run_host(A_host, A_dev2, 5)
    torch.cuda.synchronize()
    rs.check_info(plan.info)
    assert torch.equal(A_dev2, Ab)
    assert ((plan.S - S_d).abs() / S_d).max().item() <= 1e-5
    assert torch.equal(plan.J[:k], J_d[:k])


def test_bf16_unsupported_forms():
    Ab = torch.zeros(300, 200, dtype=torch.bfloat16, device=DEV)
    with pytest.raises(rs.RsvdError) as e:
        rs.svd(Ab, 5, 5, 1, 1, rs.make_opts(precision=rs.PREC_SIMT))
    assert e.value.code in (1, 4)
    # rows not 16-byte aligned (lda % 8 != 0): not TMA-addressable
    Ab2 = torch.zeros(300, 203, dtype=torch.bfloat16, device=DEV)
    with pytest.raises(rs.RsvdError) as e:
        rs.svd(Ab2, 5, 5, 1, 1)
    assert e.value.code in (1, 4)


# ---------------------------------------------------------------------------
# RSVD_PREC_MIXED: single-term bf16 products in the power scheme
# ---------------------------------------------------------------------------
MIXED_CASES = [
    # name, m, n, k, p, q, spectrum, noise, storage
    ("c2_like_mixed_f32", 3000, 2000, 40, 10, 2, "inv", 1e-4, "float32"),
    ("c2_like_mixed_bf16", 3000, 2000, 40, 10, 2, "inv", 1e-4, "bfloat16"),
    ("c5_like_mixed_f32", 2048, 1024, 64, 16, 2, "sqrtgap64", 0.0, "float32"),
]


@pytest.mark.parametrize("case", MIXED_CASES, ids=[c[0] for c in MIXED_CASES])
def test_mixed_precision_power_scheme(case):
    """The power scheme in single-term bf16 products perturbs the basis by
    ~2^-9 per iteration; the Ritz values of the final (split-precision)
    projection then move by about its square (quadratic in the subspace
    angle).  Bars: sigma relative 1e-4 against the oracle, reconstruction
    error within 1 % of the oracle's, and of the TC path's."""
    name, m, n, k, p, q, spec, noise, storage = case
    r = min(m, n) if spec != "inv" else min(2000, n)
    A32 = make_matrix_np(m, n, spectrum(spec, r), noise=noise, seed=0xC000 + m, dtype="float32")
    if storage == "bfloat16":
        Ad, A64 = _bf16(A32)
    else:
        Ad, A64 = torch.from_numpy(A32).to(DEV), A32.astype(np.float64)
    seed = 0x5EED + k
    mixed = rs.make_opts(precision=rs.PREC_MIXED)
    U, S, V = (t.double().cpu().numpy() for t in rs.svd(Ad, k, p, q, seed, mixed))
    Ut, St, Vt = (t.double().cpu().numpy() for t in rs.svd(Ad, k, p, q, seed))
    Uo, So, Vo, _ = orc.rsvd(A64, k, p, q, seed, rounding="bf16")
    rel = np.abs(S - So) / So
    print(name, "mixed sigma max rel %.2e, TC %.2e" % (rel.max(), (np.abs(St - So) / So).max()))
    assert rel.max() <= 1e-4, (name, rel.max())
    e_m = orc.rel_err_svd(A64, U, S, V)
    e_o = orc.rel_err_svd(A64, Uo, So, Vo)
    e_t = orc.rel_err_svd(A64, Ut, St, Vt)
    assert abs(e_m - e_o) <= 0.01 * e_o + 1e-12, (e_m, e_o)
    assert abs(e_m - e_t) <= 0.01 * e_t + 1e-12, (e_m, e_t)
    assert np.linalg.norm(U.T @ U - np.eye(k)) <= 5e-5
