"""Pins of the oracle's blocked adaptive QB (Alg. 7, Sec. 3.3) to facts that do
not come from the oracle itself:

* the lemma of Sec. 3.3: on exit Q has orthonormal columns, B = Q^* A_in and the
  residual is (I - Q Q^*) A_in;
* Pythagoras: ||A^(j)||_F^2 = ||A_in||_F^2 - ||B_1..j||_F^2 when Q is orthonormal;
* Eckart-Young: no rank-(b j) projection beats the tail of the spectrum, and
  the power scheme on a decaying spectrum comes close to it;
* stepped spectra with gaps at multiples of b, where the stopping block follows
  from the closed-form tail norms;
* an exactly rank-3b matrix is captured by three blocks;
* one block is the fixed-rank QB with p = 0 and the same Omega.
"""
import numpy as np
import pytest

from oracle import rsvd as orc
from synth import make_matrix_np, spectrum


def _stepped(b, levels, tail, r):
    s = np.concatenate([np.full(b, v) for v in levels] + [np.full(r - b * len(levels), tail)])
    return s


def test_lemma_orthonormal_projector_and_b():
    A = make_matrix_np(240, 180, spectrum("inv", 180), noise=1e-3, seed=11, dtype="float64")
    Q, Bt, resid = orc.qb_blocked(A, 12, 6, 1, 0.0, 7)
    assert Q.shape == (240, 72) and Bt.shape == (180, 72) and len(resid) == 7
    assert np.linalg.norm(Q.T @ Q - np.eye(72)) <= 1e-12
    # B = Q^* A_in although each block was taken from the updated residual
    assert np.linalg.norm(Bt - A.T @ Q) <= 1e-12 * np.linalg.norm(A)
    # the final residual is (I - Q Q^*) A_in
    R = A - Q @ (Q.T @ A)
    assert abs(np.linalg.norm(R) - resid[-1]) <= 1e-12 * np.linalg.norm(A)
    assert np.linalg.norm(A - Q @ Bt.T - R) <= 1e-12 * np.linalg.norm(A)


def test_pythagoras_of_the_residuals():
    A = make_matrix_np(200, 150, spectrum("logspace3", 150), noise=0.0, seed=12,
                       dtype="float64")
    b = 10
    Q, Bt, resid = orc.qb_blocked(A, b, 5, 0, 0.0, 3)
    nA2 = np.linalg.norm(A) ** 2
    assert resid[0] == pytest.approx(np.sqrt(nA2), rel=1e-14)
    for j in range(1, len(resid)):
        assert resid[j] ** 2 == pytest.approx(nA2 - np.linalg.norm(Bt[:, :b * j]) ** 2,
                                              rel=1e-9, abs=1e-12 * nA2)
    assert all(resid[j + 1] <= resid[j] for j in range(len(resid) - 1))


def test_eckart_young_bound_and_near_optimality():
    sig = np.exp(-np.arange(1, 161) / 8.0)
    A = make_matrix_np(300, 160, sig, noise=0.0, seed=13, dtype="float64")
    b = 8
    Q, Bt, resid = orc.qb_blocked(A, b, 6, 2, 0.0, 21)
    for j in range(1, len(resid)):
        tail = np.sqrt(np.sum(sig[b * j:] ** 2))
        assert resid[j] >= tail * (1 - 1e-12)
        # q = 2 stays within 8 % of the tail here (p = 0 inside a block); a
        # power scheme run on A_in instead of the residual reaches 1.9x and 5x
        assert resid[j] <= 1.15 * tail, (j, resid[j], tail)


@pytest.mark.parametrize("relative", [False, True])
def test_stops_at_the_first_block_below_tolerance(relative):
    b, r = 8, 120
    sig = _stepped(b, [1.0, 1e-2, 1e-4], 1e-7, r)
    A = make_matrix_np(200, r, sig, noise=0.0, seed=14, dtype="float64")
    tails = [np.sqrt(np.sum(sig[b * j:] ** 2)) for j in range(8)]
    nA = np.linalg.norm(A)
    # stops after blocks 1, 2, 3, and never (the flat 1e-7 tail keeps every
    # later residual above half of tails[3]): M = 7 blocks
    for tol_abs in (3 * tails[1], 3 * tails[2], 3 * tails[3], 0.5 * tails[3]):
        eps = tol_abs / nA if relative else tol_abs
        want = next((j for j in range(1, 8) if tails[j] < tol_abs), 7)
        Q, Bt, resid = orc.qb_blocked(A, b, 7, 1, eps, 5, relative=relative)
        assert Q.shape[1] == b * want, (tol_abs, want, resid)
        assert resid[-1] < tol_abs or want == 7
        assert all(x >= tol_abs for x in resid[1:-1])


def test_exact_rank_captured_by_three_blocks():
    b = 6
    rng = np.random.default_rng(15)
    A = rng.standard_normal((150, 3 * b)) @ rng.standard_normal((3 * b, 110))
    Q, Bt, resid = orc.qb_blocked(A, b, 10, 0, 1e-10, 9, relative=True)
    assert Q.shape[1] == 3 * b
    assert resid[3] <= 1e-12 * resid[0]
    assert resid[2] >= 1e-3 * resid[0]


def test_one_block_is_the_fixed_rank_qb():
    A = make_matrix_np(180, 120, spectrum("inv", 120), noise=1e-4, seed=16, dtype="float64")
    for q in (0, 2):
        Q1, Bt1, resid = orc.qb_blocked(A, 20, 1, q, 0.0, 33)
        Q0, Bt0 = orc.qb(A, 20, 0, q, 33)
        assert np.allclose(Q1, Q0, atol=1e-12) and np.allclose(Bt1, Bt0, atol=1e-12)
        assert len(resid) == 2


def test_block_omegas_come_from_consecutive_seeds():
    from oracle import philox
    A = make_matrix_np(100, 80, spectrum("inv", 80), noise=0.0, seed=17, dtype="float64")
    b = 5
    Q, Bt, resid = orc.qb_blocked(A, b, 3, 0, 0.0, 40)
    # block 1 (0-based) with q = 0 spans the re-projected (I - Q_0 Q_0^*) A Omega(seed + 1)
    A1 = A - Q[:, :b] @ Bt[:, :b].T
    Y = A1 @ philox.omega(80, b, 41)
    Y = Y - Q[:, :b] @ (Q[:, :b].T @ Y)
    P = orc.orth(Y)
    assert np.linalg.norm(P @ P.T - Q[:, b:2 * b] @ Q[:, b:2 * b].T) <= 1e-10
