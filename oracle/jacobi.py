"""One-sided Jacobi SVD of a small square matrix in FP64 (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Alg. 5 ends with the SVD of the l x l triangular factor R-hat of the QR of
B^*; the paper calls a library SVD there and fixes no method.  The oracle
computes it by the one-sided Jacobi method (Hestenes 1958): plane rotations
applied to pairs of columns of M = R-hat until every pair is orthogonal to
working precision, so that M V = W has orthogonal columns, sigma_j = ||w_j||,
u_j = w_j / sigma_j and R-hat = U diag(sigma) V^T.

Rotation for a pair (i, j) with a = ||m_i||^2, b = ||m_j||^2, g = m_i . m_j
(Rutishauser's formulas for the symmetric 2 x 2 eigenproblem [[a, g], [g, b]]):
    zeta = (b - a) / (2 g),  t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
    c = 1 / sqrt(1 + t^2),   s = c t,
    m_i <- c m_i - s m_j,    m_j <- s m_i + c m_j   (the same on V's columns),
which makes the new pair orthogonal.  A pair is rotated while
|g| > tol sqrt(a b), tol = l * 2^-52 (the stopping rule of Demmel & Veselic
1992).  Pairs are visited in the round-robin (tournament) order of Brent & Luk
1985: each of the l - 1 rounds of a sweep pairs every column with another one
exactly once, and the pairs of a round share no column, so their rotations
commute and are applied together.
"""
import numpy as np

EPS = 2.0 ** -52


def _rounds(l):
    """The l' - 1 rounds of disjoint pairs (i, j), i < j, covering every pair of
    0 .. l'-1 once (l' = l rounded up to even; index l' - 1 >= l is a dummy)."""
    lp = l + (l & 1)
    ring = list(range(lp))
    out = []
    for _ in range(lp - 1):
        pairs = [(ring[t], ring[lp - 1 - t]) for t in range(lp // 2)]
        pairs = [(min(i, j), max(i, j)) for i, j in pairs if i < l and j < l]
        out.append((np.array([p[0] for p in pairs], dtype=np.int64),
                    np.array([p[1] for p in pairs], dtype=np.int64)))
        ring = [ring[0]] + [ring[-1]] + ring[1:-1]        # rotate all but the first
    return out


def svd_jacobi(R, max_sweeps=60):
    """(U, S, V) with R = U diag(S) V^T, S descending, U and V orthogonal (l x l).

    Columns of zero norm (R rank-deficient) give sigma = 0; their u_j complete
    the others to an orthonormal basis (Householder QR of [U_nonzero, I]).
    """
    M = np.array(R, dtype=np.float64)
    l = M.shape[1]
    assert M.shape == (l, l)
    # the columns of M and of V are kept as the rows of Mt and Vt (contiguous)
    Mt = np.ascontiguousarray(M.T)
    Vt = np.eye(l)
    tol = l * EPS
    rounds = _rounds(l)
    for _ in range(max_sweeps):
        rotated = False
        for I, J in rounds:
            if I.size == 0:
                continue
            mi, mj = Mt[I], Mt[J]
            a = np.einsum("ij,ij->i", mi, mi)
            b = np.einsum("ij,ij->i", mj, mj)
            g = np.einsum("ij,ij->i", mi, mj)
            act = np.abs(g) > tol * np.sqrt(a * b)
            if not act.any():
                continue
            rotated = True
            I, J, a, b, g = I[act], J[act], a[act], b[act], g[act]
            mi, mj = mi[act], mj[act]
            zeta = (b - a) / (2.0 * g)
            t = np.where(zeta >= 0, 1.0, -1.0) / (np.abs(zeta) + np.sqrt(1.0 + zeta * zeta))
            c = (1.0 / np.sqrt(1.0 + t * t))[:, None]
            s = c * t[:, None]
            Mt[I], Mt[J] = c * mi - s * mj, s * mi + c * mj
            vi, vj = Vt[I], Vt[J]
            Vt[I], Vt[J] = c * vi - s * vj, s * vi + c * vj
        if not rotated:
            break
    else:
        raise RuntimeError("one-sided Jacobi: no convergence in %d sweeps" % max_sweeps)
    M, V = Mt.T, Vt.T
    S = np.sqrt(np.einsum("ij,ij->j", M, M))
    order = np.argsort(-S, kind="stable")
    S, M, V = S[order], M[:, order], V[:, order]
    nz = S > 0
    U = np.zeros_like(M)
    U[:, nz] = M[:, nz] / S[nz][None, :]
    r = int(nz.sum())
    if r < l:
        Qc, _ = np.linalg.qr(np.hstack([U[:, :r], np.eye(l)]))
        U[:, r:] = Qc[:, r:l]
    return U, S, V
