"""Pins of the oracle's QB3 (Alg. 8) and left-sketch randomized ID (Sec. 3.5,
Alg. 6 with the power scheme) to facts outside the oracle:

QB3
* one block is the fixed-rank QB with p = 0 and the same Omega;
* in exact arithmetic every block's power scheme keeps span((A A^*)^q A Omega_t)
  and the projection loop keeps the union of the spans, so span(Q) equals the
  span of the joint sketch (A A^*)^q A [Omega_0 ... Omega_{M-1}] (here on a
  spectrum where that sketch is well conditioned);
* the Eckart-Young tail bounds its error from below.

Left-sketch ID
* for A of exact rank k the sketch keeps the column dependencies, so the ID is
  exact;
* no rank-k ID beats sigma_{k+1} (spectral norm);
* the orthonormalisations between products do not change the row space of
  Omega~ A (A^* A)^q.

Tolerance modes (Sec. 2.6)
* the ID's residual A(:, J[k:]) - A(:, J[:k]) T equals Q2 S22, so its Frobenius
  norm is ||S22||_F, and k is the first step that brings it below TOL;
* an exactly rank-r matrix needs r steps;
* the SVD truncated at sigma_{k+1} <= TOL on a QB with ||A - Q B|| < eps errs
  by at most eps + TOL (spectral norm; triangle inequality and Eckart-Young).
"""
import numpy as np
import pytest

from oracle import philox, rsvd as orc
from synth import make_matrix_np, spectrum


def _proj_dist(Q1, Q2):
    r = Q1.shape[1]
    return float(np.sqrt(max(2.0 * r - 2.0 * np.linalg.norm(Q1.T @ Q2) ** 2, 0.0)))


def test_qb3_one_block_is_the_fixed_rank_qb():
    A = make_matrix_np(200, 150, spectrum("inv", 150), noise=1e-4, seed=21, dtype="float64")
    for q in (0, 1, 2):
        Q3, Bt3 = orc.qb_blocked_parallel(A, 24, 1, q, 17)
        Q0, Bt0 = orc.qb(A, 24, 0, q, 17)
        assert np.allclose(Q3, Q0, atol=1e-12) and np.allclose(Bt3, Bt0, atol=1e-12)


@pytest.mark.parametrize("q", [0, 1])
def test_qb3_span_is_the_joint_sketch(q):
    # sigma from 1 to 0.1: (A A^*)^q A Omega stays well conditioned for q <= 1
    A = make_matrix_np(240, 160, spectrum("logspace1", 160), noise=0.0, seed=22,
                       dtype="float64")
    b, M, seed = 10, 5, 40
    Q3, Bt3 = orc.qb_blocked_parallel(A, b, M, q, seed)
    Om = np.hstack([philox.omega(160, b, seed + t) for t in range(M)])
    Y = A @ Om
    for _ in range(q):
        Y = A @ (A.T @ Y)
    Qj = orc.orth(Y)
    assert np.linalg.norm(Q3.T @ Q3 - np.eye(b * M)) <= 1e-12
    assert _proj_dist(Q3, Qj) <= 1e-9
    assert np.allclose(Bt3, A.T @ Q3, atol=1e-13)


def test_qb3_eckart_young():
    sig = np.exp(-np.arange(1, 121) / 10.0)
    A = make_matrix_np(200, 120, sig, noise=0.0, seed=23, dtype="float64")
    b, M = 8, 4
    Q, Bt = orc.qb_blocked_parallel(A, b, M, 2, 9)
    err = np.linalg.norm(A - Q @ Bt.T)
    tail = np.sqrt(np.sum(sig[b * M:] ** 2))
    assert tail * (1 - 1e-12) <= err <= 1.5 * tail


def test_left_id_exact_rank():
    k, p = 12, 6
    rng = np.random.default_rng(24)
    A = rng.standard_normal((150, k)) @ rng.standard_normal((k, 110))
    for q in (0, 1):
        J, T, gaps, Y = orc.rid_left(A, k, p, q, 5)
        assert Y.shape == (k + p, 110)
        assert sorted(J.tolist()) == list(range(110))
        assert orc.rel_err_id(A, J, T, k) <= 1e-10


def test_left_id_bounded_below_by_sigma_k1():
    A = make_matrix_np(220, 160, spectrum("inv", 160), noise=1e-3, seed=25, dtype="float64")
    s = np.linalg.svd(A, compute_uv=False)
    k, p = 20, 8
    for q in (0, 2):
        J, T, _, _ = orc.rid_left(A, k, p, q, 6)
        V = orc.interpolation_matrix_t(J, T, k)
        E = A - A[:, J[:k]] @ V
        assert np.linalg.norm(E, 2) >= s[k] * (1 - 1e-12)
        assert np.linalg.norm(E) >= np.sqrt(np.sum(s[k:] ** 2)) * (1 - 1e-12)


def test_left_sketch_row_space_unchanged_by_orth():
    A = make_matrix_np(180, 140, spectrum("logspace1", 140), noise=0.0, seed=26,
                       dtype="float64")
    k, p, q, seed = 15, 5, 1, 8
    _, _, _, Y = orc.rid_left(A, k, p, q, seed)
    OmT = philox.omega(180, k + p, seed, tag=philox.TAG_OMEGA_LEFT)
    Yplain = OmT.T @ A @ np.linalg.matrix_power(A.T @ A, q)
    assert _proj_dist(orc.orth(Y.T), orc.orth(Yplain.T)) <= 1e-9


def test_left_omega_is_its_own_stream():
    a = philox.omega(64, 8, 3, tag=philox.TAG_OMEGA_LEFT)
    b = philox.omega(64, 8, 3)
    assert not np.allclose(a, b)
    # the same counters with tag 1 instead of 0: the words differ in every quad
    wa = philox.omega_words(64, 8, 3, tag=philox.TAG_OMEGA_LEFT)
    wb = philox.omega_words(64, 8, 3)
    assert np.all(np.any(wa != wb, axis=2))


# ---------------------------------------------------------------------------
# Tolerance mode of the ID and of the SVD (Sec. 2.6)
# ---------------------------------------------------------------------------
def test_id_tol_residual_is_s22_and_k_is_minimal():
    A = make_matrix_np(120, 90, spectrum("logspace4", 90), noise=0.0, seed=27, dtype="float64")
    for tol in (1e-1, 1e-2, 1e-3):
        J, T, k, norms = orc.id_tol(A, tol * np.linalg.norm(A))
        # the ID's residual equals ||S22||_F: A(:, J[k:]) - A(:, J[:k]) T = Q2 S22
        E = A[:, J[k:]] - A[:, J[:k]] @ T
        assert np.linalg.norm(E) == pytest.approx(norms[k], rel=1e-8, abs=1e-13)
        assert norms[k] < tol * np.linalg.norm(A) <= norms[k - 1]
        # the first k pivots of the full factorization (which gave the norms)
        # are those of the k-step ID
        Jfull = orc.cpqr(A, min(A.shape))[0]
        assert np.array_equal(J[:k], Jfull[:k])
    assert norms[0] == pytest.approx(np.linalg.norm(A), rel=1e-14)


def test_id_tol_exact_rank():
    rng = np.random.default_rng(28)
    A = rng.standard_normal((80, 7)) @ rng.standard_normal((7, 60))
    J, T, k, norms = orc.id_tol(A, 1e-9 * np.linalg.norm(A))
    assert k == 7 and norms[6] > 1e-3 * norms[0]


def test_svd_to_tolerance_on_an_adaptive_qb():
    # ||A - U_k S_k V_k^*||_2 <= ||A - Q B||_2 + sigma_{k+1}(B) <= eps + tol
    A = make_matrix_np(200, 150, spectrum("logspace3", 150), noise=0.0, seed=29,
                       dtype="float64")
    eps, tol = 1e-2, 3e-2
    Q, Bt, resid = orc.qb_blocked(A, 10, 15, 1, eps, 4)
    Qh, Rh = orc.qr_pos(Bt)
    Uh, S, VhT = np.linalg.svd(Rh)
    k = orc.svd_rank_tol(S, tol)
    assert S[k - 1] > tol >= (S[k] if k < S.size else 0.0)
    U = Q @ VhT.T[:, :k]
    V = Qh @ Uh[:, :k]
    err = np.linalg.norm(A - U @ np.diag(S[:k]) @ V.T, 2)
    assert err <= eps + tol
    assert err >= np.linalg.svd(A, compute_uv=False)[k] * (1 - 1e-12)
