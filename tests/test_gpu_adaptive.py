"""GPU parity of the blocked adaptive QB to a tolerance (Alg. 7, rsvd_qb_adaptive)
against the oracle's qb_blocked on the same seeded inputs.

Inputs: stepped spectra (one level per block of b singular values, a flat
floor beyond) so that every block's span is well separated from the rest and
the stopping block is decided with a margin: the tolerance sits at the
geometric mean of two consecutive closed-form tail norms.

Tolerances (FP32 paths): the GPU updates A in fp32, so each residual carries
~1e-7 ||A_in||_F of rounding; residual norms are compared at 1e-3 relative
(they are >= 1e-3 ||A_in||_F here).  Q is orthonormal to the CholeskyQR2 level
(bar 5e-5); B = Q^* A_in to fp32 accumulation (1e-5 ||A_in||_F).  The spans of
every prefix of blocks agree with the oracle's to 1e-2 (projector distance):
the kernels draw the Gaussians of Omega in fp32 and the oracle in fp64, so a
few entries round to the neighbouring bf16 value (one bf16 ulp), and with no
oversampling inside a block (p = 0) such flips alone move a block's span by up
to 1.2e-3 on the oracle itself, while they move the residual norms by 3e-5.
FP64 path (Omega in double on both sides): residuals and spans at 1e-9.
"""
import numpy as np
import pytest

from oracle import rsvd as orc
from synth import make_matrix_np

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"

LEVELS = [1.0, 0.3, 0.1, 0.03, 0.01, 3e-3, 1e-3, 3e-4]
FLOOR = 1e-5


def _stepped(b, r):
    s = np.concatenate([np.full(b, v) for v in LEVELS] + [np.full(r - b * len(LEVELS), FLOOR)])
    return s


def _tails(sig, b, M):
    return [float(np.sqrt(np.sum(sig[b * j:] ** 2))) for j in range(M + 1)]


def _proj_dist(Q1, Q2):
    """||Q1 Q1^T - Q2 Q2^T||_F for orthonormal Q1, Q2 of the same width."""
    r = Q1.shape[1]
    c = np.linalg.norm(Q1.T @ Q2) ** 2
    return float(np.sqrt(max(2.0 * r - 2.0 * c, 0.0)))


CASES = [
    # name, m, n, b, M, q, dtype, precision, stop after block
    ("f32_tc", 3000, 2000, 32, 8, 1, "float32", "tc", 5),
    ("f32_tc_q2_ragged", 2501, 1777, 24, 8, 2, "float32", "tc", 3),
    ("f32_simt", 1500, 1000, 16, 8, 1, "float32", "simt", 4),
    ("f64", 1500, 1000, 20, 8, 1, "float64", "simt", 6),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_qb_adaptive_parity(case):
    name, m, n, b, M, q, dtype, prec, stop = case
    r = min(m, n)
    sig = _stepped(b, r)
    A_np = make_matrix_np(m, n, sig, noise=0.0, seed=0xAD00 + m, dtype=dtype)
    A64 = A_np.astype(np.float64)
    tails = _tails(sig, b, M)
    tol_abs = float(np.sqrt(tails[stop - 1] * tails[stop]))
    nA = float(np.linalg.norm(A64))
    eps = tol_abs / nA
    seed = 0x5EED + b
    opts = rs.make_opts(precision=rs.PREC_SIMT if prec == "simt" else rs.PREC_TC)
    A = torch.from_numpy(A_np).to(DEV)
    Q, Bt, resid = rs.qb_adaptive(A, b, M, q, eps, seed, relative=True, opts=opts)
    assert torch.equal(A, torch.from_numpy(A_np).to(DEV))     # the caller's A is kept
    Qg = Q.double().cpu().numpy()
    Btg = Bt.double().cpu().numpy()
    rg = resid.cpu().numpy()
    rounding = "f64" if dtype == "float64" else "bf16"
    Qo, Bto, ro = orc.qb_blocked(A64, b, M, q, eps, seed, rounding=rounding, relative=True)
    f64 = dtype == "float64"
    bar = 1e-9 if f64 else 1e-3
    span_bar = 1e-9 if f64 else 1e-2
    assert Qg.shape[1] == Qo.shape[1] == b * stop, (name, Qg.shape, Qo.shape, rg, ro)
    assert len(rg) == len(ro) == stop + 1
    assert abs(rg[0] - ro[0]) <= (1e-12 if f64 else 1e-6) * ro[0]
    assert np.all(np.abs(rg - ro) <= bar * np.asarray(ro)), (name, rg, ro)
    assert np.linalg.norm(Qg.T @ Qg - np.eye(b * stop)) <= (1e-12 if f64 else 5e-5)
    assert np.linalg.norm(Btg - A64.T @ Qg) <= (1e-12 if f64 else 1e-5) * nA
    for j in range(1, stop + 1):
        d = _proj_dist(Qg[:, :b * j], Qo[:, :b * j])
        assert d <= span_bar, (name, j, d)


def test_qb_adaptive_overwrites_a_with_the_residual():
    m, n, b, M = 2000, 1200, 32, 4
    sig = _stepped(b, 1200)
    A_np = make_matrix_np(m, n, sig, noise=0.0, seed=0xAD10, dtype="float32")
    A = torch.from_numpy(A_np).to(DEV)
    Q, Bt, resid = rs.qb_adaptive(A, b, M, 1, 0.0, 3, relative=False, overwrite=True)
    assert Q.shape[1] == b * M and len(resid) == M + 1
    A64 = A_np.astype(np.float64)
    Qg, Btg = Q.double().cpu().numpy(), Bt.double().cpu().numpy()
    R = A.double().cpu().numpy()
    assert np.linalg.norm(R - (A64 - Qg @ Btg.T)) <= 1e-5 * np.linalg.norm(A64)
    assert abs(np.linalg.norm(R) - resid[-1].item()) <= 1e-5 * resid[-1].item()
    # Pythagoras over the blocks (Q orthonormal), on the squares: in fp32 the
    # difference ||A||^2 - ||B||^2 carries ~1e-6 ||A||^2 of rounding
    nA2 = float(np.sum(A64 * A64))
    rg = resid.cpu().numpy()
    for j in range(1, M + 1):
        want2 = nA2 - np.linalg.norm(Btg[:, :b * j]) ** 2
        assert abs(rg[j] ** 2 - want2) <= 1e-3 * rg[j] ** 2 + 1e-5 * nA2, (j, rg[j] ** 2, want2)


def test_qb_adaptive_absolute_tolerance_and_block_limit():
    m, n, b, M = 2048, 1024, 16, 5
    sig = _stepped(b, 1024)
    A_np = make_matrix_np(m, n, sig, noise=0.0, seed=0xAD20, dtype="float32")
    A = torch.from_numpy(A_np).to(DEV)
    tails = _tails(sig, b, M)
    # absolute tolerance between tails[2] and tails[3]: three blocks
    Q, Bt, resid = rs.qb_adaptive(A, b, M, 1, float(np.sqrt(tails[2] * tails[3])), 7,
                                  relative=False)
    assert Q.shape[1] == 3 * b and len(resid) == 4
    # eps = 0: never met, M blocks
    Q, Bt, resid = rs.qb_adaptive(A, b, M, 1, 0.0, 7, relative=False)
    assert Q.shape[1] == M * b and len(resid) == M + 1
    # a tolerance above ||A||_F still computes one block (the test follows the block)
    Q, Bt, resid = rs.qb_adaptive(A, b, M, 1, 2.0, 7, relative=True)
    assert Q.shape[1] == b


def _rank_3b(b, dtype):
    rng = np.random.default_rng(31)
    return (rng.standard_normal((1200, 3 * b)) @ rng.standard_normal((3 * b, 900))).astype(dtype)


def test_qb_adaptive_exact_low_rank_f64():
    """FP64 A of exact rank 3b: three blocks capture it (the oracle leaves
    1.3e-13 ||A||_F); bar 1e-10."""
    b = 8
    A = torch.from_numpy(_rank_3b(b, np.float64)).to(DEV)
    Q, Bt, resid = rs.qb_adaptive(A, b, 10, 0, 1e-8, 5, relative=True)
    assert Q.shape[1] == 3 * b, resid
    assert resid[3].item() <= 1e-10 * resid[0].item()


def test_qb_adaptive_low_rank_f32_floor():
    """The same product rounded to fp32 on the tensor-core path.  Its passes
    multiply A as two bf16 terms (2^-17 relative per entry), and a block sketch
    with p = 0 amplifies that by the condition of A Omega_t: the residual after
    the third block sits at ~1e-3 ||A||_F (1.1e-3 when the oracle's products
    take the same two-term A; 1.5e-5 for the oracle in FP64 on this
    fp32-rounded input), and a fourth block takes it below the 1e-4 tolerance."""
    b = 8
    A = torch.from_numpy(_rank_3b(b, np.float32)).to(DEV)
    Q, Bt, resid = rs.qb_adaptive(A, b, 10, 0, 1e-4, 5, relative=True)
    assert Q.shape[1] in (3 * b, 4 * b), resid
    assert resid[3].item() <= 1e-2 * resid[0].item()
    assert resid[-1].item() < 1e-4 * resid[0].item()
    assert resid[2].item() >= 0.5 * resid[0].item()


def test_qb_adaptive_argument_errors():
    A = torch.zeros(300, 200, device=DEV)
    with pytest.raises(rs.RsvdError) as e:
        rs.qb_adaptive(A, 64, 4, 1, 1e-3, 1)              # b M > min(m, n)
    assert e.value.code == 1
    with pytest.raises(rs.RsvdError) as e:
        rs.qb_adaptive(A, 16, 4, 1, -1.0, 1)              # eps < 0
    assert e.value.code == 1
    with pytest.raises(rs.RsvdError) as e:
        rs.qb_adaptive(A, 16, 4, 1, float("nan"), 1)
    assert e.value.code == 1
    with pytest.raises(rs.RsvdError) as e:
        rs.qb_adaptive(A.to(torch.bfloat16), 16, 4, 1, 1e-3, 1)
    assert e.value.code in (1, 4)
