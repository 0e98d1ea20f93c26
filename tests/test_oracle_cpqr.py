"""Pins for the oracle's column-pivoted QR, ID and CUR (CPU only).

Independent checks: a hand-worked example (tests/golden), the error identity
||A - C V^*|| = ||S22|| (Sec. 2.3, 2.4), identity columns of V^* at the
skeleton, C = Q1 S11, brute-force greedy pivots through least-squares
projections, the tie-break rule, exact recovery at exact rank, the two-sided ID
error equal to the column ID error (Sec. 2.5), the CUR normal equations
(U R - V^*) R^T = 0 (Sec. 2.5, Alg. 3), and the ID-from-QB bound of Sec. 3.5.
"""
import os

import numpy as np
import pytest

from oracle import rsvd
from synth import spectrum, make_matrix_np, low_rank_np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    i = 0
    while i < len(lines):
        tag = lines[i][0]
        if tag in ("M", "S", "T"):
            r, c = int(lines[i][1]), int(lines[i][2])
            out[tag] = np.array([[float(x) for x in lines[i + 1 + t]] for t in range(r)])
            assert out[tag].shape == (r, c)
            i += 1 + r
        elif tag == "K":
            out["K"] = int(lines[i][1])
            i += 1
        elif tag == "J":
            out["J"] = np.array([int(x) for x in lines[i][1:]])
            i += 1
        else:
            raise ValueError(tag)
    return out


def test_hand_worked_example():
    g = _read_golden("cpqr_worked_example.txt")
    perm, S, _, _ = rsvd.cpqr(g["M"], g["K"])
    assert np.array_equal(perm, g["J"])
    assert np.allclose(S, g["S"], atol=1e-14)
    J, T, _ = rsvd.id_from_matrix(g["M"], g["K"])
    assert np.allclose(T, g["T"], atol=1e-14)


def test_id_error_equals_s22():
    rng = np.random.default_rng(0)
    M = rng.standard_normal((30, 50)) @ np.diag(np.logspace(0, -3, 50))
    for k in (1, 5, 12):
        perm, S, S22, _ = rsvd.cpqr(M, k)
        J, T, _ = rsvd.id_from_matrix(M, k)
        err = np.linalg.norm(M - M[:, J[:k]] @ rsvd.interpolation_matrix_t(J, T, k))
        assert err == pytest.approx(np.linalg.norm(S22), rel=1e-10)
        Vs = rsvd.interpolation_matrix_t(J, T, k)
        assert np.array_equal(Vs[:, J[:k]], np.eye(k))
        # C = A(:, J(1:k)) = Q1 S11: norms of C's columns equal those of S11's columns
        assert np.allclose(np.linalg.norm(M[:, J[:k]], axis=0),
                           np.linalg.norm(S[:, :k], axis=0), rtol=1e-12)
        assert abs(S[0, 0]) == pytest.approx(np.max(np.linalg.norm(M, axis=0)), rel=1e-14)


def test_greedy_pivots_brute_force():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((6, 9))
    k = 5
    perm, _, _, _ = rsvd.cpqr(M, k)
    chosen = []
    for t in range(k):
        best, bestc = -1.0, None
        for c in range(M.shape[1]):
            if c in chosen:
                continue
            v = M[:, c]
            if chosen:
                B = M[:, chosen]
                coef, *_ = np.linalg.lstsq(B, v, rcond=None)
                v = v - B @ coef
            nv = np.linalg.norm(v)
            if nv > best * (1 + 1e-12):
                best, bestc = nv, c
        chosen.append(bestc)
    assert list(perm[:k]) == chosen


def test_tie_break_lowest_original_index():
    rng = np.random.default_rng(2)
    base = rng.standard_normal((4, 3))
    M = np.concatenate([base[:, [0]], base[:, [1]], base, base[:, [2]]], axis=1)
    # columns (0, 2) and (1, 3) and (4, 5) are duplicates; all norms present twice
    perm, _, _, _ = rsvd.cpqr(M, 3)
    norms = np.linalg.norm(M, axis=0)
    first = int(np.argmax(norms))          # lowest index among the maxima
    assert perm[0] == first


def test_exact_rank_recovery():
    A = low_rank_np(40, 60, rank=7, seed=3)
    J, T, _ = rsvd.id_from_matrix(A, 7)
    assert rsvd.rel_err_id(A, J, T, 7) <= 1e-12


def test_two_sided_id_error_equals_column_id_error():
    A = make_matrix_np(80, 60, spectrum("logspace3", 60), seed=4)
    k = 10
    J, T, _ = rsvd.id_from_matrix(A, k)
    C = A[:, J[:k]]
    Jr, _, _, _ = rsvd.cpqr(C.T, k)
    I = Jr[:k]
    W = C @ np.linalg.inv(C[I, :])          # C = W C(I, :), exact for rank-k C
    Vs = rsvd.interpolation_matrix_t(J, T, k)
    two_sided = W @ A[np.ix_(I, J[:k])] @ Vs
    assert np.linalg.norm(two_sided - C @ Vs) <= 1e-10 * np.linalg.norm(A)


def test_cur_normal_equations_and_error_order():
    A = make_matrix_np(120, 90, spectrum("logspace3", 90), seed=5)
    k = 12
    Jc, Ir, U, J, T, _, _ = rsvd.rcur(A, k, p=6, q=2, seed=9)
    R = A[Ir, :]
    Vs = rsvd.interpolation_matrix_t(J, T, k)
    assert np.linalg.norm((U @ R - Vs) @ R.T) <= 1e-10 * np.linalg.norm(Vs) * np.linalg.norm(R)
    e_id = rsvd.rel_err_id(A, J, T, k)
    e_cur = rsvd.rel_err_cur(A, Jc, Ir, U)
    Us, S, Vv, _ = rsvd.rsvd(A, k, p=6, q=2, seed=9)
    e_svd = rsvd.rel_err_svd(A, Us, S, Vv)
    assert e_svd <= e_id * (1 + 1e-12)     # truncated SVD is optimal (Sec. 2.2)
    assert e_cur < 50 * e_id


def test_id_from_qb_bound():
    """Sec. 3.5: ||A(:,J(1:k)) V^* - A|| <= [1 + sqrt(1 + 4k(n-k))] ||A - Q B||."""
    A = make_matrix_np(150, 100, spectrum("logspace2", 100), seed=6)
    k, p = 15, 5
    J, T, _, (Q, Bt) = rsvd.rid(A, k, p, q=1, seed=3)
    eps = np.linalg.norm(A - Q @ Bt.T, 2)
    err = np.linalg.norm(A - A[:, J[:k]] @ rsvd.interpolation_matrix_t(J, T, k), 2)
    assert err <= (1 + np.sqrt(1 + 4 * k * (100 - k))) * eps
