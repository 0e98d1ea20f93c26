"""Pins for the oracle's orth / QB / RSVD (CPU only).

Independent checks: closed forms (diagonal and 2x2 singular values), exact
recovery of matrices of rank <= l (the range lemma of Sec. 3), prescribed
spectra, interlacing, the Eckart-Young lower bound (Thm. of Sec. 2.2), brute
force through the eigenvalues of A^T A on tiny inputs, the Halko-Martinsson-
Tropp expected Frobenius bound (quoted in Sec. 3.4 through the paper's
reference), and the effect of the power scheme (Sec. 3.2).
"""
import numpy as np
import pytest

from oracle import philox, rsvd
from synth import spectrum, make_matrix_np, low_rank_np


def test_qr_pos_properties_and_gram_schmidt():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((300, 40))
    Q, R = rsvd.qr_pos(Y)
    assert np.linalg.norm(Q.T @ Q - np.eye(40)) <= 1e-13
    assert np.linalg.norm(Q @ R - Y) / np.linalg.norm(Y) <= 1e-14
    assert np.all(np.diag(R) >= 0)
    assert np.allclose(np.triu(R), R)
    # classical Gram-Schmidt twice gives the same unique Q (diag R > 0)
    G = np.zeros_like(Y)
    for j in range(Y.shape[1]):
        v = Y[:, j].copy()
        for _ in range(2):
            v -= G[:, :j] @ (G[:, :j].T @ v)
        G[:, j] = v / np.linalg.norm(v)
    assert np.max(np.abs(G - Q)) <= 1e-12


def test_diagonal_closed_form():
    A = np.zeros((7, 5))
    A[[0, 1, 2, 3, 4], [0, 1, 2, 3, 4]] = [0.5, -3.0, 2.0, 0.0, -1.0]
    U, S, V, _ = rsvd.rsvd(A, k=3, p=2, q=1, seed=3)
    assert np.allclose(S, [3.0, 2.0, 1.0], rtol=0, atol=1e-14)
    # sign rule: the largest entry of each v_j is positive; u_j follows
    for j, (col, sgn) in enumerate([(1, -1.0), (2, 1.0), (4, -1.0)]):
        assert V[col, j] == pytest.approx(1.0, abs=1e-14)
        assert U[col, j] == pytest.approx(sgn, abs=1e-14)


def test_two_by_two_closed_form():
    a, b, d = 3.0, 4.0, 2.0
    A = np.array([[a, b], [0.0, d], [0.0, 0.0]])
    s = a * a + b * b + d * d
    det = a * d
    s1 = np.sqrt((s + np.sqrt(s * s - 4 * det * det)) / 2)
    s2 = np.sqrt((s - np.sqrt(s * s - 4 * det * det)) / 2)
    _, S, _, _ = rsvd.rsvd(A, k=2, p=0, q=0, seed=1)
    assert np.allclose(S, [s1, s2], rtol=1e-14)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_exact_recovery_rank_le_l(q):
    A = low_rank_np(120, 80, rank=9, seed=2)
    Q, Bt = rsvd.qb(A, k=10, p=2, q=q, seed=11)
    err = np.linalg.norm(A - Q @ Bt.T) / np.linalg.norm(A)
    assert err <= 1e-12
    U, S, V, _ = rsvd.rsvd(A, k=9, p=3, q=q, seed=11)
    assert rsvd.rel_err_svd(A, U, S, V) <= 1e-12


def test_prescribed_spectrum_and_orthonormal_factors():
    sig = spectrum("exp20", 200)
    A = make_matrix_np(400, 200, sig, seed=5)
    # (sigma_61 / sigma_10)^(2(2q+1)) ~ 1e-11 for q = 2 sets the expected accuracy
    U, S, V, _ = rsvd.rsvd(A, k=30, p=30, q=2, seed=7)
    assert np.max(np.abs(S[:10] - sig[:10]) / sig[:10]) <= 1e-8
    assert np.linalg.norm(U.T @ U - np.eye(30)) <= 1e-13
    assert np.linalg.norm(V.T @ V - np.eye(30)) <= 1e-13


def test_interlacing_and_eckart_young():
    sig = spectrum("logspace2", 150)
    A = make_matrix_np(300, 150, sig, seed=9)
    k, p = 20, 5
    Q, Bt = rsvd.qb(A, k, p, q=0, seed=4)
    sb = np.linalg.svd(Bt, compute_uv=False)
    assert np.all(sb <= sig[:k + p] * (1 + 1e-13))
    U, S, V, _ = rsvd.rsvd(A, k, p, q=0, seed=4)
    D = A - (U * S) @ V.T
    assert np.linalg.norm(D) >= np.sqrt(np.sum(sig[k:] ** 2)) * (1 - 1e-12)
    assert np.linalg.norm(D, 2) >= sig[k] * (1 - 1e-12)


def test_brute_force_tiny_against_eigenvalues():
    rng = np.random.default_rng(12)
    for _ in range(5):
        A = rng.standard_normal((8, 6))
        _, S, _, _ = rsvd.rsvd(A, k=6, p=0, q=0, seed=int(rng.integers(1 << 30)))
        ev = np.sqrt(np.sort(np.linalg.eigvalsh(A.T @ A))[::-1])
        assert np.allclose(S, ev, rtol=1e-12)


def test_hmt_expected_frobenius_bound():
    """E ||A - Q Q^T A||_F <= (1 + k/(p-1))^{1/2} (sum_{j>k} sigma_j^2)^{1/2}, q = 0."""
    sig = spectrum("logspace1", 120)
    A = make_matrix_np(200, 120, sig, seed=21)
    k, p = 10, 5
    errs = []
    for s in range(60):
        Q = rsvd.range_finder(A, k + p, 0, seed=500 + s)
        errs.append(np.linalg.norm(A - Q @ (Q.T @ A)))
    bound = np.sqrt(1 + k / (p - 1)) * np.sqrt(np.sum(sig[k:] ** 2))
    assert np.mean(errs) <= bound


def test_power_scheme_reduces_error():
    sig = spectrum("logspace0.5", 200)          # slowly decaying, type I of Sec. 5
    A = make_matrix_np(300, 200, sig, seed=31)
    e = []
    for q in (0, 1, 2):
        U, S, V, _ = rsvd.rsvd(A, k=20, p=5, q=q, seed=8)
        e.append(np.linalg.norm(A - (U * S) @ V.T, 2))
    assert e[2] <= e[1] <= e[0]
    # Sec. 3.4: ||A - U S V^T||_2 <= (k n)^(1/(2(2q+1))) sigma_{k+1}, and >= sigma_{k+1}
    for q in (0, 1, 2):
        assert sig[20] * (1 - 1e-12) <= e[q] <= (20 * 200) ** (1 / (2 * (2 * q + 1))) * sig[20]


def test_orth_frequency_s_same_subspace():
    sig = spectrum("exp20", 100)
    A = make_matrix_np(150, 100, sig, seed=41)
    Q1 = rsvd.range_finder(A, 12, 2, seed=6, s=1)
    Q2 = rsvd.range_finder(A, 12, 2, seed=6, s=2)
    # same subspace in exact arithmetic: projectors agree closely
    assert np.linalg.norm(Q1 @ Q1.T - Q2 @ Q2.T) <= 1e-8


def test_omega_rounding_consumed():
    A = make_matrix_np(60, 40, spectrum("exp20", 40), seed=1, dtype="float32")
    Om = philox.omega(40, 12, seed=2, rounding="bf16")
    Q1 = rsvd.range_finder(A, 12, 1, seed=2, rounding="bf16")
    Q2 = rsvd.range_finder(A, 12, 1, seed=0, Omega=Om)
    assert np.array_equal(Q1, Q2)
