"""Pins of the oracle's one-sided Jacobi SVD (oracle/jacobi.py) against what
the mathematics fixes: the pair schedule, closed forms (diagonal and 2 x 2
triangular matrices), prescribed singular values of U diag(sigma) V^T, LAPACK's
singular values on well-conditioned matrices (a library routine computing the
same quantity), and rank deficiency."""
import numpy as np
import pytest

from oracle.jacobi import _rounds, svd_jacobi


def _check_factorisation(R, U, S, V, tol):
    l = R.shape[0]
    assert np.all(np.diff(S) <= 0) and np.all(S >= 0)
    assert np.linalg.norm(U @ np.diag(S) @ V.T - R) <= tol * max(np.linalg.norm(R), 1e-300)
    assert np.linalg.norm(U.T @ U - np.eye(l)) <= tol * l
    assert np.linalg.norm(V.T @ V - np.eye(l)) <= tol * l


@pytest.mark.parametrize("l", list(range(1, 14)))
def test_round_robin_covers_every_pair_once(l):
    seen = []
    for I, J in _rounds(l):
        cols = list(I) + list(J)
        assert len(set(cols)) == len(cols)            # a round's pairs share no column
        seen += [(int(i), int(j)) for i, j in zip(I, J)]
    assert sorted(seen) == [(i, j) for i in range(l) for j in range(i + 1, l)]


def test_diagonal_with_signs():
    d = np.array([3.0, -5.0, 0.5, 2.0, -0.25])
    U, S, V = svd_jacobi(np.diag(d))
    assert np.array_equal(S, np.sort(np.abs(d))[::-1])
    _check_factorisation(np.diag(d), U, S, V, 1e-15)


@pytest.mark.parametrize("a,b,d", [(1.0, 2.0, 3.0), (2.0, -1.0, 0.5), (1.0, 1e-8, 1.0),
                                   (4.0, 0.0, 4.0)])
def test_two_by_two_closed_form(a, b, d):
    # sigma_1,2 = (P +- Q) / 2 with P = sqrt((a + d)^2 + b^2), Q = sqrt((a - d)^2 + b^2):
    # sigma_1 sigma_2 = (P^2 - Q^2) / 4 = |a d| and sigma_1^2 + sigma_2^2 =
    # (P^2 + Q^2) / 2 = a^2 + b^2 + d^2, the determinant and trace of R^T R
    R = np.array([[a, b], [0.0, d]])
    P, Q = np.hypot(a + d, b), np.hypot(a - d, b)
    s1, s2 = (P + Q) / 2, abs(P - Q) / 2
    U, S, V = svd_jacobi(R)
    assert np.allclose(S, [s1, s2], rtol=1e-14, atol=0)
    _check_factorisation(R, U, S, V, 1e-14)


@pytest.mark.parametrize("l,kind", [(40, "flat"), (80, "graded"), (120, "cluster")])
def test_prescribed_singular_values(l, kind):
    rng = np.random.default_rng(l)
    j = np.arange(l, dtype=np.float64)
    sig = {"flat": 1.0 + j / l,
           "graded": 10.0 ** (-8.0 * j / (l - 1)),
           "cluster": np.where(j < l // 2, 1.0, 1.0 + 1e-9 * j)}[kind]
    sig = np.sort(sig)[::-1]
    Q1, _ = np.linalg.qr(rng.standard_normal((l, l)))
    Q2, _ = np.linalg.qr(rng.standard_normal((l, l)))
    R = (Q1 * sig[None, :]) @ Q2.T
    U, S, V = svd_jacobi(R)
    assert np.max(np.abs(S - sig)) <= 1e-13 * sig[0]
    _check_factorisation(R, U, S, V, 1e-13)


@pytest.mark.parametrize("l", [7, 64, 150])
def test_lapack_singular_values_well_conditioned(l):
    rng = np.random.default_rng(100 + l)
    R = np.triu(rng.standard_normal((l, l))) + 4.0 * np.eye(l)
    U, S, V = svd_jacobi(R)
    S0 = np.linalg.svd(R, compute_uv=False)
    assert np.max(np.abs(S - S0) / S0) <= 1e-12
    _check_factorisation(R, U, S, V, 1e-13)


def test_rank_deficient():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((30, 5)) @ rng.standard_normal((5, 30))
    U, S, V = svd_jacobi(X)
    assert np.all(S[5:] <= 1e-13 * S[0])
    assert np.all(S[:5] > 1e-3 * S[0])
    _check_factorisation(X, U, S, V, 1e-13)
    U0, S0, V0 = svd_jacobi(np.zeros((6, 6)))
    assert np.array_equal(S0, np.zeros(6))
    assert np.allclose(U0.T @ U0, np.eye(6), atol=1e-15)
