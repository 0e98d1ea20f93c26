"""GPU parity of the adjoint of Alg. 5 (rsvd_svd_vjp and the torch.autograd
Function around it) against the oracle, through the C ABI.

* rsvd_vjp of the oracle (FP64, Omega fixed, the same seed and bf16 rounding of
  Omega as the FP32 kernels) on the same A and the same cotangents: element by
  element, |gA - gA_oracle| <= tol * max |gA_oracle|, and the relative
  Frobenius error.  FP64 path: 1e-9.  FP32 path: each product carries two bf16
  terms (2^-16 relative) and the QR rules divide by R, whose condition number
  grows with the spread of the sketched spectrum, so the bar is 2e-3 of the
  largest entry (1e-3 in the Frobenius norm) at the differentiable workload
  (spectrum j^-1/2 with a 10x gap at j = 64).
* The differentiable workload (m = 8192, n = 4096, k = 64, p = 16, q = 2): the
  loss sum(S) + ||A - U diag(S) V^T||_F^2 through svd_autograd; A.grad against
  (1) the oracle's rsvd_vjp of the same cotangents plus the loss's direct term
  2 (A - U S V^T) (bars as above), (2) FP64 central differences of the
  oracle's loss on 64 random unit rank-1 directions D: |<g, D> - fd| within
  2e-3 of ||g||_F / sqrt(m n), the size of <g, D> for a random D, (3) the
  gradient of the same loss through the exact SVD, sum_i u_i v_i^T +
  2 (A - A_k), built from the generator's own singular vectors (the 10x gap
  and q = 2 make the randomized top-64 subspace exact to ~(0.09)^5; bar 1e-2
  in the Frobenius norm).
"""
import numpy as np
import pytest

from oracle import rsvd as orc
from synth import config, make_matrix_np, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"


def _dev(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


SMALL = [("f64_q1", "float64", 300, 200, 10, 5, 1), ("f64_q2", "float64", 257, 190, 12, 4, 2),
         ("f32_q0", "float32", 600, 400, 16, 8, 0), ("f32_q2", "float32", 1200, 700, 24, 8, 2)]


@pytest.mark.parametrize("case", SMALL, ids=[c[0] for c in SMALL])
def test_vjp_matches_oracle_on_random_cotangents(case):
    _, dtype, m, n, k, p, q = case
    seed = 0x6A00 + q
    A = make_matrix_np(m, n, spectrum("logspace2", n), noise=1e-4, seed=m, dtype=dtype)
    A64 = A.astype(np.float64)
    rng = np.random.default_rng(m + n)
    gU, gS, gV = rng.standard_normal((m, k)), rng.standard_normal(k), rng.standard_normal((n, k))
    rounding = "f64" if dtype == "float64" else "bf16"
    gAo, (Uo, So, Vo) = orc.rsvd_vjp(A64, k, p, q, seed, gU, gS, gV, rounding=rounding)
    tdt = torch.float64 if dtype == "float64" else torch.float32
    gA, U, S, V = rs.svd_vjp(_dev(A, tdt), k, p, q, seed, _dev(gU, tdt), torch.from_numpy(gS).to(DEV),
                             _dev(gV, tdt), with_outputs=True)
    gA = gA.double().cpu().numpy()
    tol = 1e-9 if dtype == "float64" else 2e-3
    err = np.max(np.abs(gA - gAo)) / np.max(np.abs(gAo))
    fro = np.linalg.norm(gA - gAo) / np.linalg.norm(gAo)
    print("%s: max %.2e fro %.2e" % (case[0], err, fro))
    assert err <= tol, (err, fro)
    assert fro <= tol / 2, (err, fro)
    s_bar = 1e-10 if dtype == "float64" else 1e-5
    assert np.max(np.abs(S.cpu().numpy() - So) / So) <= s_bar


@pytest.fixture(scope="module")
def c5():
    cfg = config("c5_f32_8192x4096")
    m, n = cfg["m"], cfg["n"]
    A, Ug, Vg = make_matrix_np(m, n, spectrum(cfg["spectrum"], cfg["r"]), noise=cfg["noise"],
                               seed=cfg["a_seed"], dtype=cfg["dtype"], factors=True)
    k = cfg["k"]
    return cfg, A, Ug[:, :k].copy(), Vg[:, :k].copy()


def _loss_and_cotangents(A64, U, S, V):
    """loss = sum(S) + ||A - U diag(S) V^T||_F^2, its direct gradient in A and
    the cotangents of U, S, V (FP64)."""
    R = A64 - (U * S[None, :]) @ V.T
    loss = float(np.sum(S) + np.sum(R * R))
    gU = -2.0 * (R @ V) * S[None, :]
    gV = -2.0 * (R.T @ U) * S[None, :]
    gS = 1.0 - 2.0 * np.einsum("ij,ij->j", U, R @ V)
    return loss, 2.0 * R, gU, gS, gV


def test_c5_loss_gradient(c5):
    cfg, A, Ue, Ve = c5
    m, n, k, p, q, seed = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["q"], cfg["omega_seed"]
    A64 = A.astype(np.float64)
    At = _dev(A, torch.float32).requires_grad_(True)
    U, S, V = rs.svd_autograd(At, k, p, q, seed)
    R = At - (U * S.float()[None, :]) @ V.T
    loss = S.sum() + (R * R).sum()
    loss.backward()
    g = At.grad.double().cpu().numpy()

    # (1) the oracle: rsvd_vjp of the loss's cotangents plus its direct term
    Uo, So, Vo, _ = orc.rsvd(A64, k, p, q, seed, rounding="bf16")
    _, direct, gUo, gSo, gVo = _loss_and_cotangents(A64, Uo, So, Vo)
    gAo, _ = orc.rsvd_vjp(A64, k, p, q, seed, gUo, gSo, gVo, rounding="bf16")
    go = gAo + direct
    err = np.max(np.abs(g - go)) / np.max(np.abs(go))
    fro = np.linalg.norm(g - go) / np.linalg.norm(go)
    print("C5 loss gradient vs oracle: max %.2e fro %.2e" % (err, fro))
    assert err <= 2e-3 and fro <= 1e-3, (err, fro)

    # (2) FP64 central differences of the oracle's loss on 64 rank-1 directions
    rng = np.random.default_rng(64)
    h = 1e-5

    def f(Ap):
        U2, S2, V2, _ = orc.rsvd(Ap, k, p, q, seed, rounding="bf16")
        return _loss_and_cotangents(Ap, U2, S2, V2)[0]

    # a random unit rank-1 direction meets g at about ||g||_F / sqrt(m n)
    scale = np.linalg.norm(g) / np.sqrt(m * n)
    worst = 0.0
    for _ in range(64):
        x = rng.standard_normal(m)
        y = rng.standard_normal(n)
        x /= np.linalg.norm(x)
        y /= np.linalg.norm(y)
        D = np.outer(x, y)
        fd = (f(A64 + h * D) - f(A64 - h * D)) / (2 * h)
        worst = max(worst, abs(x @ g @ y - fd) / scale)
    print("C5 central differences: worst |<g, D> - fd| / (||g||_F / sqrt(mn)) = %.2e" % worst)
    assert worst <= 2e-3, worst

    # (3) the same loss through the exact SVD (the generator's singular vectors)
    sig = spectrum(cfg["spectrum"], cfg["r"])
    Ak = (Ue * sig[None, :k]) @ Ve.T
    gfull = Ue @ Ve.T + 2.0 * (A64 - Ak)
    fro_full = np.linalg.norm(g - gfull) / np.linalg.norm(gfull)
    print("C5 vs exact-SVD gradient: fro %.2e" % fro_full)
    assert fro_full <= 1e-2, fro_full


def test_vjp_rejects_bf16_and_bad_arguments():
    A = torch.zeros(100, 80, device=DEV, dtype=torch.bfloat16)
    with pytest.raises(rs.RsvdError) as e:
        rs.svd_vjp(A, 5, 5, 1, 1, None, None, None)
    assert e.value.code in (1, 4)
    A = torch.zeros(100, 80, device=DEV)
    with pytest.raises(rs.RsvdError):
        rs.svd_vjp(A, 60, 40, 1, 1, None, None, None)       # l > n
