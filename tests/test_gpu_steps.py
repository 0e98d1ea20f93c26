"""GPU parity of each step of the path against the FP64 oracle (through the C ABI).

Tolerances, from the arithmetic: the FP32 tensor-core path splits each fp32
operand into two bf16 terms (16 significant bits, unit roundoff 2^-16 per
term product) with fp32 accumulation, so a product entry carries a relative
error of order 2^-16 / sqrt(terms) ~ 1e-5 in the worst case and ~1e-6 in the
Frobenius mean; the SIMT FP32 path is plain fp32 (~1e-6); FP64 is ~1e-13.
"""
import numpy as np
import pytest

from oracle import philox, rsvd as orc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

rs = pytest.importorskip("paper_1502_05366_gb300")

DEV = "cuda:0"
SIMT = None


def _simt():
    return rs.make_opts(precision=rs.PREC_SIMT)


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def _elem_err(Y, ref, absprod):
    """max over entries of |Y - ref| / (|A| |W|): every entry against the error
    bound of its own dot product.  The split products and the fp32 sums err in
    proportion to the sum of the absolute term products, so a wrong tile, a
    stale padded column or a dropped stream-K contribution shows up at full
    size however small the entry is.  Entries whose bound is zero must be
    exactly zero."""
    d = np.abs(np.asarray(Y, dtype=np.float64) - ref)
    den = np.asarray(absprod, dtype=np.float64)
    assert np.all(d[den == 0] == 0)
    nz = den > 0
    return float(np.max(d[nz] / den[nz])) if nz.any() else 0.0


# Element-wise bars relative to |A| |W| (worst case of the arithmetic):
# Omega is bf16-exact and A carries two bf16 terms (2^-16 per product) plus fp32
# accumulation: 2e-5; a stored operand adds its own dropped terms: 5e-5; FP64: 1e-12.
ELEM_TC_SAMPLE, ELEM_TC_APPLY, ELEM_F64 = 2e-5, 5e-5, 1e-12


# ---------------------------------------------------------------------------
# Philox / Omega: integer words bit-exact, Gaussians within rounding
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n,l,seed", [(1000, 60, 0x5EED + 1), (777, 13, 3), (1, 1, 0),
                                      (4096, 224, (1 << 40) + 5)])
def test_omega_words_bit_exact(n, l, seed):
    w = rs.omega_words(n, l, seed, device=DEV).cpu().numpy().view(np.uint32)
    ref = philox.omega_words(n, l, seed)
    assert np.array_equal(w, ref)


def test_omega_f64_matches():
    n, l, seed = 2000, 61, 99
    g = rs.omega(n, l, seed, torch.float64, DEV).cpu().numpy()
    ref = philox.omega(n, l, seed, "f64")
    assert np.max(np.abs(g - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_omega_f32_bf16_rounding():
    n, l, seed = 20000, 220, 0x5EED + 2
    g = rs.omega(n, l, seed, torch.float32, DEV).cpu().numpy().astype(np.float64)
    ref = philox.omega(n, l, seed, "bf16")
    bits = g.astype(np.float32).view(np.uint32)
    assert np.all(bits & np.uint32(0xFFFF) == 0)          # bf16-exact entries
    diff = g != ref
    frac = diff.mean()
    # the kernels' fp32 Box-Muller (hardware log2 / sincos approximations, errors
    # ~1e-6 relative) differs from the FP64 oracle by a few fp32 ulps; a bf16
    # rounding flip needs the value within that distance of a rounding boundary:
    # rare, and one bf16 ulp each
    assert frac < 1e-3, frac
    if diff.any():
        # one bf16 ulp, plus an absolute 1e-5 for values near zero, where the
        # absolute error of the hardware sin / cos dominates the relative one
        assert np.all(np.abs(g[diff] - ref[diff]) <= 2.0 ** -7 * np.abs(ref[diff]) + 1e-5)


def test_omega_f32_distribution():
    """The kernels' fp32 Gaussians themselves: moments and a Kolmogorov-Smirnov test."""
    import scipy.stats as st
    z = rs.omega(20000, 200, 0x5EED + 9, torch.float32, DEV).double().cpu().numpy().ravel()
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    # bf16 rounding adds variance of about (2^-9)^2 / 3 relative: far below 5 sigma
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3) < 5 * np.sqrt(96 / n)
    # compare with the bf16-rounded normal CDF steps: a KS test on a subsample
    assert st.kstest(z[:100000], "norm").pvalue > 1e-4 or \
        st.kstest(z[:100000] + np.random.default_rng(0).uniform(-2**-9, 2**-9, 100000) *
                  np.abs(z[:100000]), "norm").pvalue > 1e-4


# ---------------------------------------------------------------------------
# sample Y = A Omega and the power half steps
# ---------------------------------------------------------------------------
# the last shape: m and n not multiples of the 512-row super-unit or the 256-row
# unit, and long enough contractions that stream-K splits them across CTAs
SHAPES = [(300, 200, 24), (1000, 777, 60), (517, 1290, 17), (129, 33, 16), (2048, 4096, 220),
          (16411, 4099, 220)]


@pytest.mark.parametrize("m,n,l", SHAPES)
@pytest.mark.parametrize("mode", ["tc", "simt", "f64"])
def test_sample(m, n, l, mode):
    rng = np.random.default_rng(m + n + l)
    A = rng.standard_normal((m, n))
    seed = 1234 + l
    if mode == "f64":
        Y = rs.sample(_dev(A, torch.float64), l, seed).cpu().numpy()
        Om = philox.omega(n, l, seed, "f64")
        ref = A @ Om
        assert _rel(Y, ref) <= 1e-13
        assert _elem_err(Y, ref, np.abs(A) @ np.abs(Om)) <= ELEM_F64
    else:
        A32 = A.astype(np.float32)
        opts = _simt() if mode == "simt" else None
        Y = rs.sample(_dev(A32, torch.float32), l, seed, opts).cpu().numpy()
        # GEMM arithmetic against the kernels' own Omega (same device function) ...
        Om_gpu = rs.omega(n, l, seed, torch.float32, DEV).double().cpu().numpy()
        ref = A32.astype(np.float64) @ Om_gpu
        tol = 2e-5 if mode == "tc" else 2e-6
        assert _rel(Y, ref) <= tol, _rel(Y, ref)
        if mode == "tc":
            e = _elem_err(Y, ref, np.abs(A32.astype(np.float64)) @ np.abs(Om_gpu))
            assert e <= ELEM_TC_SAMPLE, e
        # ... and against the oracle's Omega, which differs by rare bf16 flips
        ref_o = A32.astype(np.float64) @ philox.omega(n, l, seed, "bf16")
        assert _rel(Y, ref_o) <= 1e-4, _rel(Y, ref_o)


@pytest.mark.parametrize("m,n,l", SHAPES)
@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("mode", ["tc", "simt", "f64"])
def test_apply(m, n, l, trans, mode):
    rng = np.random.default_rng(7 * m + n + l + trans)
    A = rng.standard_normal((m, n))
    X = rng.standard_normal((m if trans else n, l))
    ref = (A.T @ X) if trans else (A @ X)
    if mode == "f64":
        Y = rs.apply(_dev(A, torch.float64), _dev(X, torch.float64), trans).cpu().numpy()
        assert _rel(Y, ref) <= 1e-13
        absprod = (np.abs(A).T @ np.abs(X)) if trans else (np.abs(A) @ np.abs(X))
        assert _elem_err(Y, ref, absprod) <= ELEM_F64
    else:
        opts = _simt() if mode == "simt" else None
        A32, X32 = A.astype(np.float32), X.astype(np.float32)
        ref = (A32.astype(np.float64).T @ X32) if trans else (A32.astype(np.float64) @ X32)
        Y = rs.apply(_dev(A32, torch.float32), _dev(X32, torch.float32), trans, opts).cpu().numpy()
        tol = 3e-5 if mode == "tc" else 2e-6
        assert _rel(Y, ref) <= tol, _rel(Y, ref)
        if mode == "tc":
            a, x = np.abs(A32.astype(np.float64)), np.abs(X32.astype(np.float64))
            e = _elem_err(Y, ref, (a.T @ x) if trans else (a @ x))
            assert e <= ELEM_TC_APPLY, e


# ---------------------------------------------------------------------------
# orth (CholeskyQR2/3) against the Householder Q of the oracle
# ---------------------------------------------------------------------------
# l = 300, 550 and 1000 take the cooperative multi-CTA Cholesky (fp32, l > 224);
# kappa = 1e6 drives its shifted retries
@pytest.mark.parametrize("rows,l", [(500, 40), (3000, 220), (129, 17), (64, 64), (20000, 96),
                                    (4000, 300), (6000, 550), (8000, 1000)])
@pytest.mark.parametrize("mode", ["tc", "simt", "f64"])
@pytest.mark.parametrize("cond", [1e1, 1e3, 1e6])
def test_orth(rows, l, mode, cond):
    rng = np.random.default_rng(rows + l)
    G, _ = np.linalg.qr(rng.standard_normal((rows, l)))
    H, _ = np.linalg.qr(rng.standard_normal((l, l)))
    X = (G * np.logspace(0, -np.log10(cond), l)) @ H
    if mode == "f64":
        Q, R = rs.orth(_dev(X, torch.float64))
        Qn, Rn = Q.cpu().numpy(), R.cpu().numpy()
        Qo, Ro = orc.qr_pos(X)
        assert np.linalg.norm(Qn.T @ Qn - np.eye(l)) <= 1e-12
        assert _rel(Qn @ Rn, X) <= 1e-13
        assert np.max(np.abs(Qn - Qo)) <= 1e-10 * cond
    else:
        X32 = X.astype(np.float32)
        opts = _simt() if mode == "simt" else None
        Q, R = rs.orth(_dev(X32, torch.float32), opts)
        Qn, Rn = Q.double().cpu().numpy(), R.double().cpu().numpy()
        Qo, Ro = orc.qr_pos(X32.astype(np.float64))
        orth_err = np.linalg.norm(Qn.T @ Qn - np.eye(l), 2)
        res = _rel(Qn @ Rn, X32)
        # fp32 CholeskyQR3 reaches O(u) orthogonality for kappa well below 1/u;
        # kappa = 1e6 is within 20x of 1/u = 1.7e7 and gets a looser bar.  There
        # the first pass needs the shift 4 l u max(diag G), which grows with l,
        # and the orthogonality the third pass leaves grows about as l^2
        # (measured 1.7e-5, 4.3e-5, 2.3e-4, 1.0e-3 at l = 220, 300, 550, 1000,
        # the same with the one-CTA and the cooperative Cholesky)
        tol = 1e-5 if cond < 1e6 else 1e-4 * max(1.0, l / 220.0) ** 2
        assert orth_err <= tol, (orth_err, res)
        assert res <= 3e-5, (orth_err, res)
        assert np.all(np.diag(Rn) > 0)
        assert np.allclose(np.tril(Rn, -1), 0)
        # Q is unique (diag R > 0); its columns agree with Householder's
        assert np.max(np.abs(Qn - Qo)) <= 5e-4 * max(1.0, cond / 1e3)


# ---------------------------------------------------------------------------
# small SVD (one-sided Jacobi)
# ---------------------------------------------------------------------------
# 224: the 8-CTA cluster kernel (fp32); 300, 550, 672: the 16-CTA cluster
# kernel (fp32; 672 is its largest size); 700: the one-CTA kernel beyond it
@pytest.mark.parametrize("l", [1, 2, 17, 60, 224, 300, 550, 672, 700])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_small_svd(l, dtype):
    if dtype == torch.float64 and l > 300:
        pytest.skip("the FP64 kernel is covered to l = 300")
    rng = np.random.default_rng(l)
    # upper-triangular core with a prescribed spectrum (as R-hat of Alg. 5 is)
    G1, _ = np.linalg.qr(rng.standard_normal((l, l)))
    G2, _ = np.linalg.qr(rng.standard_normal((l, l)))
    M = np.linalg.qr((G1 * np.logspace(0, -3, l)) @ G2.T)[1]
    Mt = M.astype(np.float32).astype(np.float64) if dtype == torch.float32 else M
    Uh, Sh, Vh = rs.small_svd(_dev(Mt, dtype))
    Uh, Sh, Vh = Uh.double().cpu().numpy(), Sh.cpu().numpy(), Vh.double().cpu().numpy()
    s_ref = np.linalg.svd(Mt, compute_uv=False)
    tol = 2e-6 if dtype == torch.float32 else 1e-13
    assert np.max(np.abs(Sh - s_ref) / s_ref) <= tol * 10
    assert np.all(np.diff(Sh) <= 0)
    # one-sided Jacobi stops once every pair has |x_a . x_b| <= sqrt(l) eps
    # ||x_a|| ||x_b||, so each off-diagonal entry of Uh^T Uh is bounded by
    # sqrt(l) eps and the Frobenius norm over l^2 entries by l^1.5 eps
    eps = 5.9604645e-8 if dtype == torch.float32 else 1.1102230246251565e-16
    assert np.linalg.norm(Uh.T @ Uh - np.eye(l)) <= max(tol * 100, l ** 1.5 * eps)
    assert _rel((Uh * Sh) @ Vh.T, Mt) <= tol * 50


def test_small_svd_closed_forms():
    M = np.diag([0.5, -3.0, 2.0, 1e-3])
    Uh, Sh, Vh = rs.small_svd(_dev(M, torch.float64))
    assert np.allclose(Sh.cpu().numpy(), [3.0, 2.0, 0.5, 1e-3], rtol=1e-15)
    a, b, d = 3.0, 4.0, 2.0
    M = np.array([[a, b], [0.0, d]])
    s = a * a + b * b + d * d
    s1 = np.sqrt((s + np.sqrt(s * s - 4 * (a * d) ** 2)) / 2)
    s2 = np.sqrt((s - np.sqrt(s * s - 4 * (a * d) ** 2)) / 2)
    _, Sh, _ = rs.small_svd(_dev(M, torch.float64))
    assert np.allclose(Sh.cpu().numpy(), [s1, s2], rtol=1e-14)


# ---------------------------------------------------------------------------
# CPQR / ID of an explicit matrix: pivots bit-exact, T close
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("r,n,k", [(20, 50, 10), (60, 1000, 50), (220, 5000, 200), (8, 9, 8),
                                   (33, 4097, 1)])
def test_cpqr_id(r, n, k):
    rng = np.random.default_rng(r * n + k)
    M = rng.standard_normal((r, n)) * np.logspace(0, -4, n)[rng.permutation(n)]
    J, T, gaps = rs.cpqr_id(_dev(M, torch.float64), k)
    J, T, gaps = J.cpu().numpy(), T.cpu().numpy(), gaps.cpu().numpy()
    Jo, To, go = orc.id_from_matrix(M, k)
    assert np.array_equal(J[:k], Jo[:k])
    assert np.array_equal(J, Jo)
    assert np.allclose(gaps[go < np.inf], go[go < np.inf], rtol=1e-9, atol=1e-12)
    if n > k:
        assert np.max(np.abs(T - To)) <= 1e-9 * max(1.0, np.max(np.abs(To)))


@pytest.mark.parametrize("r,n,k", [(20, 50, 10), (60, 1000, 50), (220, 5000, 200), (8, 9, 8),
                                   (33, 4097, 1), (200, 20011, 200), (300, 1500, 280),
                                   (600, 3001, 550)])
def test_cpqr_id_f32_double_float(r, n, k):
    """The double-float CPQR of the FP32 path against the FP64 oracle on the same
    fp32 matrix: pivots identical, gaps to 1e-9, T to fp32 rounding."""
    rng = np.random.default_rng(r * n + k + 1)
    M = (rng.standard_normal((r, n)) * np.logspace(0, -4, n)[rng.permutation(n)]).astype(np.float32)
    J, T, gaps = rs.cpqr_id(_dev(M, torch.float32), k)
    J, T, gaps = J.cpu().numpy(), T.double().cpu().numpy(), gaps.cpu().numpy()
    Jo, To, go = orc.id_from_matrix(M.astype(np.float64), k)
    assert np.array_equal(J, Jo)
    assert np.allclose(gaps[go < np.inf], go[go < np.inf], rtol=1e-9, atol=1e-12)
    if n > k:
        assert np.max(np.abs(T - To)) <= 1e-6 * max(1.0, np.max(np.abs(To)))


def test_cpqr_golden_worked_example():
    import os
    M = np.array([[3, 0, 1, 0], [4, 0, 0, 2]], dtype=np.float64)
    J, T, _ = rs.cpqr_id(_dev(M, torch.float64), 2)
    assert list(J.cpu().numpy()) == [0, 3, 2, 1]
    assert np.allclose(T.cpu().numpy(), [[1 / 3, 0], [-2 / 3, 0]], atol=1e-14)
    assert os.path.exists(os.path.join(os.path.dirname(__file__), "golden",
                                       "cpqr_worked_example.txt"))
