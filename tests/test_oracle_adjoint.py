"""Pins of the oracle's reverse-mode derivative of Alg. 5 (Omega fixed) to facts
outside it:

* FP64 central differences of the forward oracle (rsvd), on 64 random
  directions for each q: <g_A, dA> = d/dh <g, f(A + h dA)> at h = 0;
* the QR and square-SVD rules on their own, against central differences;
* the closed form d sigma_i / dA = u_i v_i^* of the exact SVD, which the RSVD
  reaches when l = n (Q then spans range(A) for every nearby A).
"""
import numpy as np
import pytest

from oracle import rsvd as orc
from synth import make_matrix_np, spectrum

H = 1e-6


def _fd(f, X, d):
    return (f(X + H * d) - f(X - H * d)) / (2 * H)


@pytest.mark.parametrize("shape", [(12, 5), (7, 7), (30, 1)])
def test_qr_rule_central_differences(shape):
    rng = np.random.default_rng(sum(shape))
    X = rng.standard_normal(shape)
    c = shape[1]
    gQ = rng.standard_normal(shape)
    gR = np.triu(rng.standard_normal((c, c)))
    Q, R = orc.qr_pos(X)
    g = orc.qr_pos_vjp(Q, R, gQ, gR)

    def f(Xp):
        Q2, R2 = orc.qr_pos(Xp)
        return np.sum(gQ * Q2) + np.sum(gR * R2)

    for _ in range(4):
        d = rng.standard_normal(shape)
        assert np.sum(g * d) == pytest.approx(_fd(f, X, d), rel=1e-6, abs=1e-9)


def test_square_svd_rule_central_differences():
    rng = np.random.default_rng(5)
    Rm = rng.standard_normal((6, 6))
    Uh, S, VhT = np.linalg.svd(Rm)
    Vh = VhT.T
    gUh, gS, gVh = rng.standard_normal((6, 6)), rng.standard_normal(6), rng.standard_normal((6, 6))
    g = orc.svd_square_vjp(Uh, S, Vh, gUh, gS, gVh)

    def f(Rp):
        U2, S2, V2T = np.linalg.svd(Rp)
        sg = np.sign(np.sum(U2 * Uh, axis=0))       # follow the base's sign choice
        return np.sum(gUh * U2 * sg) + np.sum(gS * S2) + np.sum(gVh * V2T.T * sg)

    for _ in range(4):
        d = rng.standard_normal((6, 6))
        assert np.sum(g * d) == pytest.approx(_fd(f, Rm, d), rel=1e-6)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_rsvd_adjoint_central_differences_64_directions(q):
    m, n, k, p, seed = 60, 40, 6, 4, 7
    A = make_matrix_np(m, n, spectrum("inv", 40), noise=1e-3, seed=3, dtype="float64")
    rng = np.random.default_rng(100 + q)
    gU, gS, gV = rng.standard_normal((m, k)), rng.standard_normal(k), rng.standard_normal((n, k))
    gA, (U, S, V) = orc.rsvd_vjp(A, k, p, q, seed, gU, gS, gV)
    U0, S0, V0, _ = orc.rsvd(A, k, p, q, seed)
    assert np.array_equal(S, S0) and np.allclose(U, U0, atol=1e-14) and np.allclose(V, V0, atol=1e-14)

    def f(Ap):
        U2, S2, V2, _ = orc.rsvd(Ap, k, p, q, seed)
        return np.sum(gU * U2) + np.sum(gS * S2) + np.sum(gV * V2)

    worst = 0.0
    for _ in range(64):
        d = rng.standard_normal((m, n))
        d /= np.linalg.norm(d)
        fd = _fd(f, A, d)
        worst = max(worst, abs(np.sum(gA * d) - fd) / max(abs(fd), 1e-6))
    assert worst <= 1e-6, worst


def test_singular_value_gradient_is_u_v_when_l_equals_n():
    m, n, k = 50, 30, 5
    A = make_matrix_np(m, n, spectrum("logspace2", 30), noise=0.0, seed=9, dtype="float64")
    Ue, Se, VeT = np.linalg.svd(A, full_matrices=False)
    for i in (0, 2, 4):
        gS = np.zeros(k)
        gS[i] = 1.0
        gA, _ = orc.rsvd_vjp(A, k, n - k, 1, 11, np.zeros((m, k)), gS, np.zeros((n, k)))
        assert np.linalg.norm(gA - np.outer(Ue[:, i], VeT[i])) <= 1e-9
