"""Plain FP64 reference of the randomized QB / RSVD / ID / CUR path (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Every function takes the
stored input promoted to float64 and follows the paper's steps in the paper's
order; library primitives (matmul, LAPACK Householder QR, triangular solve)
serve as single steps, and the SVD of the l x l core is the one-sided Jacobi
method of ``oracle/jacobi.py``.  Nothing here is blocked, fused or
reordered.

Readings of points the paper leaves open (each is also taken by the CUDA side):
* orth(Y) is the Q of a Householder QR with diag(R) >= 0 (Sec. 2.1 defines orth
  as an unpivoted QR; the sign makes Q unique).
* The power scheme re-orthonormalises before every product with A or A^T
  (s = 1 in Alg. 5; Sec. 3.2); general s follows Alg. 5's mod tests.
* Singular values are returned in descending order; each pair (u_j, v_j) is
  sign-flipped so that the entry of largest magnitude of v_j is positive
  (ties: lowest index).
* Column-pivoted QR runs k steps only; the pivot is the column of largest
  exactly recomputed residual norm, ties broken by the lowest original column
  index; columns are exchanged like LAPACK (pivot position j <-> p).
* T = S11^{-1} S12 by plain back substitution (Sec. 3.5 mentions an unspecified
  "stabilized version"; it is not used).
"""
import numpy as np
import scipy.linalg as sla

from . import philox
from .jacobi import svd_jacobi


# ---------------------------------------------------------------------------
# orth: unpivoted QR (Sec. 2.1 notation; Fig. 1 step 3)
# ---------------------------------------------------------------------------
def qr_pos(Y):
    """Economic Householder QR of Y (m x l, m >= l) with diag(R) >= 0."""
    Q, R = np.linalg.qr(np.asarray(Y, dtype=np.float64), mode="reduced")
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :], R * d[:, None]


def orth(Y):
    return qr_pos(Y)[0]


# ---------------------------------------------------------------------------
# Range finder with the power scheme, and the QB step (Alg. 5; Sec. 3.2, 3.4)
# ---------------------------------------------------------------------------
def range_finder(A, l, q, seed, rounding="f64", s=1, Omega=None):
    """Q (m x l) with orthonormal columns spanning (A A^*)^q A Omega (Alg. 5)."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    if Omega is None:
        Omega = philox.omega(n, l, seed, rounding)
    Y = A @ Omega                                   # samples Y = A R
    for j in range(1, q + 1):
        if (2 * j - 2) % s == 0:
            Y = orth(Y)
        Z = A.T @ Y                                 # Z = A^* Y
        if (2 * j - 1) % s == 0:
            Z = orth(Z)
        Y = A @ Z                                   # Y = A Z
    return orth(Y)                                  # [Q, ~] = qr(Y, 0)


def qb(A, k, p, q, seed, rounding="f64", s=1, Omega=None):
    """Q (m x l) and Bt = A^* Q (n x l) = B^* with B = Q^* A (Alg. 5; Fig. 1 step 4)."""
    A = np.asarray(A, dtype=np.float64)
    Q = range_finder(A, k + p, q, seed, rounding, s, Omega)
    Bt = A.T @ Q
    return Q, Bt


# ---------------------------------------------------------------------------
# RSVD version II (Alg. 5; Sec. 3.4)
# ---------------------------------------------------------------------------
def normalize_signs(U, V):
    """Flip (u_j, v_j) so the largest-magnitude entry of v_j is positive."""
    U = U.copy()
    V = V.copy()
    for j in range(V.shape[1]):
        i = int(np.argmax(np.abs(V[:, j])))        # first maximum = lowest index
        if V[i, j] < 0:
            U[:, j] = -U[:, j]
            V[:, j] = -V[:, j]
    return U, V


def svd_from_qb(Q, Bt, k):
    """Steps after the QB step of Alg. 5: QR of Bt, SVD of the l x l R-hat, lift."""
    Qh, Rh = qr_pos(Bt)                             # [Q^, R^] = qr(Bt, 0)
    Uh, S, Vh = svd_jacobi(Rh)                      # R^ = U^ Sigma V^* (one-sided Jacobi)
    U = Q @ Vh[:, :k]                               # U_k = Q V^
    V = Qh @ Uh[:, :k]                              # V_k = Q^ U^
    U, V = normalize_signs(U, V)
    return U, S[:k].copy(), V, S


def rsvd(A, k, p, q, seed, rounding="f64", s=1, Omega=None):
    """Rank-k approximate SVD A ~ U diag(S) V^T by Alg. 5 (RSVD version II).

    Returns U (m x k), S (k,), V (n x k) and the l singular values of R-hat.
    """
    Q, Bt = qb(A, k, p, q, seed, rounding, s, Omega)
    return svd_from_qb(Q, Bt, k)


# ---------------------------------------------------------------------------
# Blocked adaptive QB to a tolerance (Alg. 7, "QB2"; Sec. 3.3)
# ---------------------------------------------------------------------------
def qb_blocked(A, b, M, q, eps, seed, rounding="f64", relative=False, s=1):
    """Alg. 7: Q and B built block by block from the updated residual of A.

    Block t (t = 0, 1, ...) draws its n x b Omega_t from the stream keyed by
    seed + t (the paper's randn(n, b) per block).  Its Q_t comes from the range
    finder with q power iterations applied to the CURRENT residual A, is
    re-projected against the earlier blocks and orthonormalised again; then
    B_t = Q_t^* A and A <- A - Q_t B_t.  The loop ends after the first block
    whose residual has ||A||_F < tol (tol = eps, or eps * ||A_in||_F when
    relative), or after M blocks.  The norm is the Frobenius norm (the paper
    writes ||A|| without naming one).

    Returns Q (m x b i), Bt = B^* (n x b i) and the residual norms
    [||A_in||_F, ||A^(1)||_F, ..., ||A^(i)||_F].
    """
    A = np.array(A, dtype=np.float64)               # the algorithm overwrites A
    n = A.shape[1]
    resid = [float(np.linalg.norm(A))]
    tol = eps * resid[0] if relative else eps
    Qs, Bts = [], []
    for t in range(M):
        Om = philox.omega(n, b, (seed + t) % (1 << 64), rounding)   # Omega_t = randn(n, b)
        Qt = range_finder(A, b, q, seed, rounding, s, Omega=Om)      # orth(A Omega_t), power scheme
        if Qs:
            Qbar = np.hstack(Qs)
            Qt = orth(Qt - Qbar @ (Qbar.T @ Qt))    # Q_t - sum_j Q_j Q_j^* Q_t, re-orthonormalised
        Bt = A.T @ Qt                               # B_t = Q_t^* A (stored transposed)
        A = A - Qt @ Bt.T                           # A <- A - Q_t B_t
        Qs.append(Qt)
        Bts.append(Bt)
        resid.append(float(np.linalg.norm(A)))
        if resid[-1] < tol:
            break
    return np.hstack(Qs), np.hstack(Bts), resid


def qb_blocked_parallel(A, b, M, q, seed, rounding="f64"):
    """Alg. 8: the approximate parallel blocked QB (fixed M blocks, A not updated).

    Every block sketches the ORIGINAL A with its own Omega_t (stream keyed by
    seed + t, as in qb_blocked) and runs its power scheme with orth between
    products; the blocks are then orthonormalised, projected one after the
    other against the blocks already accepted, orthonormalised again and
    appended; finally B = Q^* A.

    Returns Q (m x b M) and Bt = B^* (n x b M).
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    Ys = []
    for t in range(M):                              # first loop: independent blocks
        Om = philox.omega(n, b, (seed + t) % (1 << 64), rounding)
        Y = A @ Om                                  # Y_t = A Omega_t
        for _ in range(q):
            Qt = orth(Y)
            Y = A.T @ Qt                            # Y_t = A^* Q_t
            Qt = orth(Y)
            Y = A @ Qt                              # Y_t = A Q_t
        Ys.append(Y)
    Qs = [orth(Y) for Y in Ys]                      # second loop: Q_t = orth(Y_t)
    Q = np.zeros((A.shape[0], 0))
    for Qt in Qs:                                   # third loop: project, orth, append
        Qt = Qt - Q @ (Q.T @ Qt)
        Qt = orth(Qt)
        Q = np.hstack([Q, Qt])
    return Q, A.T @ Q                               # B = Q^* A


# ---------------------------------------------------------------------------
# Reverse-mode derivative of Alg. 5 with Omega fixed (differentiable RSVD)
# ---------------------------------------------------------------------------
def qr_pos_vjp(Q, R, gQ, gR):
    """Cotangent of X for X = Q R (thin QR, diag(R) > 0) given those of Q and R.

    From dX = dQ R + Q dR with Q^* dQ skew and dR upper triangular:
    g_X = (g_Q + Q sym(M)) R^{-*}, M = g_R R^* - Q^* g_Q, where sym(M) keeps
    the upper triangle of M and mirrors its strictly upper part below.
    """
    M = gR @ R.T - Q.T @ gQ
    symM = np.triu(M) + np.triu(M, 1).T
    return sla.solve_triangular(R, (gQ + Q @ symM).T, lower=False).T   # (R^{-1} Y^*)^*


def svd_square_vjp(Uh, S, Vh, gUh, gS, gVh):
    """Cotangent of R for the square SVD R = Uh diag(S) Vh^* (distinct S).

    With dC = Uh^* dR Vh: dS = diag(dC), and off the diagonal
    (Uh^* dUh)_ij = F_ij (s_j dC_ij + s_i dC_ji), (Vh^* dVh)_ij = F_ij (s_i dC_ij + s_j dC_ji),
    F_ij = 1 / (s_j^2 - s_i^2).  Collecting the coefficients of dC:
    g_R = Uh [diag(g_S) + (F o (Gu - Gu^*)) S + S (F o (Gv - Gv^*))] Vh^*,
    Gu = Uh^* g_Uh, Gv = Vh^* g_Vh.
    """
    s2 = S ** 2
    D = s2[None, :] - s2[:, None]                  # D_ij = s_j^2 - s_i^2
    np.fill_diagonal(D, 1.0)
    F = 1.0 / D
    np.fill_diagonal(F, 0.0)
    Gu = Uh.T @ gUh
    Gv = Vh.T @ gVh
    X = np.diag(gS) + (F * (Gu - Gu.T)) * S[None, :] + S[:, None] * (F * (Gv - Gv.T))
    return Uh @ X @ Vh.T


def rsvd_vjp(A, k, p, q, seed, gU, gS, gV, rounding="f64", Omega=None):
    """g_A for the map A -> (U, S, V) of Alg. 5 (s = 1) with Omega held fixed,
    given the cotangents of its outputs; the sign rule is treated as constant.

    The forward steps are those of rsvd(); the backward replays them in reverse
    with the adjoints of matmul, of orth (qr_pos_vjp with g_R = 0), of the QR of
    Bt and of the square SVD of R-hat (svd_square_vjp).

    Returns g_A (m x n) and the forward outputs (U, S, V).
    """
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    l = k + p
    if Omega is None:
        Omega = philox.omega(n, l, seed, rounding)
    # ---- forward, keeping what the backward needs ----
    tape = []                                      # ("orth", X, Q, R) | ("mulA", W) | ("mulAt", W)
    Y = A @ Omega
    tape.append(("mulA", Omega))
    for _ in range(q):
        Qy, Ry = qr_pos(Y)
        tape.append(("orth", Qy, Ry))
        Z = A.T @ Qy
        tape.append(("mulAt", Qy))
        Qz, Rz = qr_pos(Z)
        tape.append(("orth", Qz, Rz))
        Y = A @ Qz
        tape.append(("mulA", Qz))
    Q, Rq = qr_pos(Y)
    Bt = A.T @ Q
    Qh, Rh = qr_pos(Bt)
    Uh, S, Vh = svd_jacobi(Rh)
    U = Q @ Vh[:, :k]
    V = Qh @ Uh[:, :k]
    signs = np.ones(k)
    for j in range(k):
        i = int(np.argmax(np.abs(V[:, j])))
        if V[i, j] < 0:
            signs[j] = -1.0
    U = U * signs[None, :]
    V = V * signs[None, :]
    # ---- backward ----
    gU = np.asarray(gU, dtype=np.float64) * signs[None, :]
    gV = np.asarray(gV, dtype=np.float64) * signs[None, :]
    gA = np.zeros_like(A)
    gVh = np.zeros((l, l))
    gUh = np.zeros((l, l))
    gVh[:, :k] = Q.T @ gU                          # U = Q Vh(:, :k)
    gQ = gU @ Vh[:, :k].T
    gUh[:, :k] = Qh.T @ gV                         # V = Qh Uh(:, :k)
    gQh = gV @ Uh[:, :k].T
    gSfull = np.zeros(l)
    gSfull[:k] = gS
    gRh = svd_square_vjp(Uh, S, Vh, gUh, gSfull, gVh)
    gBt = qr_pos_vjp(Qh, Rh, gQh, gRh)             # [Qh, Rh] = qr(Bt)
    gA += Q @ gBt.T                                # Bt = A^* Q
    gQ += A @ gBt
    gY = qr_pos_vjp(Q, Rq, gQ, np.zeros_like(Rq))  # Q = orth(Y)
    for entry in reversed(tape):
        if entry[0] == "mulA":                     # Y = A W
            W = entry[1]
            gA += gY @ W.T
            gY = A.T @ gY                          # cotangent of W
        elif entry[0] == "mulAt":                  # Z = A^* W
            W = entry[1]
            gA += W @ gY.T
            gY = A @ gY
        else:                                      # Q_ = orth(X)
            _, Qo, Ro = entry
            gY = qr_pos_vjp(Qo, Ro, gY, np.zeros_like(Ro))
    return gA, (U, S[:k].copy(), V)


# ---------------------------------------------------------------------------
# Column-pivoted QR, k steps (Sec. 2.3; Alg. 1 first step)
# ---------------------------------------------------------------------------
def cpqr(M, ksteps):
    """k steps of Householder QR with column pivoting on M (r x n).

    Returns
      perm   int64 (n,): M[:, perm] ~ Q S, i.e. P = I(:, perm)
      S      (ksteps, n) float64: first ksteps rows of the triangular factor,
             columns in pivot (position) order; S[:, :ksteps] is upper triangular
      S22    (r - ksteps, n - ksteps): the remainder block after ksteps steps
      gaps   (ksteps,): relative gap (nu1 - nu2) / nu1 between the largest and
             second-largest residual column norms at each step (inf if single)
    """
    W = np.array(M, dtype=np.float64, copy=True)
    r, n = W.shape
    if not (0 <= ksteps <= min(r, n)):
        raise ValueError("ksteps out of range")
    perm = np.arange(n, dtype=np.int64)
    gaps = np.empty(ksteps)
    for j in range(ksteps):
        nrm2 = np.sum(W[j:, j:] ** 2, axis=0)       # exact residual norms^2
        vmax = nrm2.max()
        cand = np.flatnonzero(nrm2 == vmax)
        pos = j + int(cand[np.argmin(perm[j + cand])])
        if nrm2.size > 1:
            nu = np.sqrt(np.sort(nrm2)[::-1])
            gaps[j] = (nu[0] - nu[1]) / nu[0] if nu[0] > 0 else 0.0
        else:
            gaps[j] = np.inf
        if pos != j:                                # exchange positions j and pos
            W[:, [j, pos]] = W[:, [pos, j]]
            perm[[j, pos]] = perm[[pos, j]]
        x = W[j:, j].copy()
        normx = np.sqrt(np.sum(x * x))
        if normx == 0.0:
            continue
        beta = -normx if x[0] >= 0 else normx       # H x = beta e1
        v = x
        v[0] -= beta
        vv = np.dot(v, v)
        if vv > 0:
            W[j:, j:] -= np.outer(v, (2.0 / vv) * (v @ W[j:, j:]))
        W[j, j] = beta
        W[j + 1:, j] = 0.0
    return perm, W[:ksteps, :].copy(), W[ksteps:, ksteps:].copy(), gaps


# ---------------------------------------------------------------------------
# One-sided ID (Sec. 2.4; Alg. 1) and the QB-route randomized ID (Sec. 3.5)
# ---------------------------------------------------------------------------
def id_from_matrix(M, k):
    """Column ID of M: J (n,) and T = S11^{-1} S12 (k x (n-k))."""
    perm, S, _, gaps = cpqr(M, k)
    S11 = S[:, :k]
    S12 = S[:, k:]
    T = sla.solve_triangular(S11, S12, lower=False)
    return perm, T, gaps


def id_tol(M, tol):
    """Column ID of M to a tolerance (Sec. 2.6; Sec. 4, TOL mode): the fewest
    pivoted-QR steps k >= 1 after which ||S22||_F < tol (all min(r, n) steps
    when none does).  The paper's ||S22|| is read as the Frobenius norm, the
    root of the sum of the residual column norms that the pivoting tracks.

    The pivots of the first k steps do not depend on later steps, so one full
    factorization gives every ||S22(k)||_F = ||S[k:, k:]||_F; the ID itself is
    then the k-step one (later steps would reorder J[k:] and the columns of T).

    Returns J (n,), T (k x (n-k)), k and the norms ||S22(j)||_F, j = 0..min(r, n).
    """
    M = np.asarray(M, dtype=np.float64)
    kmax = min(M.shape)
    _, S, _, _ = cpqr(M, kmax)
    norms = np.array([np.linalg.norm(S[j:, j:]) for j in range(kmax)] + [0.0])
    k = next((j for j in range(1, kmax + 1) if norms[j] < tol), kmax)
    J, T, _ = id_from_matrix(M, k)
    return J, T, k, norms


def svd_rank_tol(S, tol):
    """Rank of the SVD to a tolerance (Sec. 2.6): the k with sigma_{k+1} <= tol,
    i.e. the number of singular values above tol (at least 1)."""
    S = np.asarray(S, dtype=np.float64)
    return max(1, int(np.sum(S > tol)))


def interpolation_matrix_t(J, T, k):
    """V^* = [I_k  T] P^T as a dense k x n array (Eq. for V in Sec. 2.4)."""
    n = J.size
    Vs = np.zeros((k, n))
    Vs[np.arange(k), J[:k]] = 1.0
    Vs[:, J[k:]] = T
    return Vs


def rid(A, k, p, q, seed, rounding="f64", s=1, Omega=None):
    """Randomized ID through the QB step: ID of B = Q^* A (Sec. 3.5, last part).

    Returns J (n,), T (k x (n-k)), pivot gaps, and (Q, Bt).
    """
    Q, Bt = qb(A, k, p, q, seed, rounding, s, Omega)
    J, T, gaps = id_from_matrix(Bt.T, k)
    return J, T, gaps, (Q, Bt)


# ---------------------------------------------------------------------------
# CUR through the two-sided ID (Sec. 2.5; Alg. 2, Alg. 3; Sec. 3.6)
# ---------------------------------------------------------------------------
def rid_left(A, k, p, q, seed, rounding="f64"):
    """Randomized ID from the left sketch Y = Omega~ A (A^* A)^q (Sec. 3.5, Alg. 6).

    Omega~ is (k + p) x m Gaussian: Omega~^* is the m x l stream of tag
    TAG_OMEGA_LEFT.  Between products the sample is orthonormalised as in the
    power scheme of Sec. 3.5: Y <- (A orth(Y^*))^*, then Y <- (A^* orth(Y^*))^*.
    The ID is that of Y (k steps of CPQR, T = S11^{-1} S12).

    Returns J (n,), T (k x (n-k)), pivot gaps, and Y (l x n).
    """
    A = np.asarray(A, dtype=np.float64)
    m = A.shape[0]
    l = k + p
    OmT = philox.omega(m, l, seed, rounding, tag=philox.TAG_OMEGA_LEFT)   # Omega~^*
    Y = (A.T @ OmT).T                               # Y = (A^* Omega~^*)^*, l x n
    for _ in range(q):
        Y = (A @ orth(Y.T)).T                       # l x m
        Y = (A.T @ orth(Y.T)).T                     # l x n
    J, T, gaps = id_from_matrix(Y, k)
    return J, T, gaps, Y


def cur_from_id(A, J, T, k):
    """Row ID of C = A(:, J[:k]) by k-step CPQR of C^*, then U = V^* R^dagger.

    R^dagger is taken through the Householder QR of R^* = Q_R R_R:
    R^dagger = Q_R R_R^{-T}.  Returns I (k,), U (k x k), row gaps.
    """
    A = np.asarray(A, dtype=np.float64)
    C = A[:, J[:k]]
    Jr, _, _, rgaps = cpqr(C.T, k)
    I = Jr[:k].copy()
    R = A[I, :]
    Vs = interpolation_matrix_t(J, T, k)
    QR_, RR = qr_pos(R.T)
    Mk = Vs @ QR_
    U = sla.solve_triangular(RR, Mk.T, lower=False).T   # U R_R^T = V^* Q_R
    return I, U, rgaps


def rcur(A, k, p, q, seed, rounding="f64", s=1, Omega=None):
    """Randomized CUR: A ~ A(:, Jc) U A(Ir, :).  Returns Jc (k,), Ir (k,), U,
    plus the full column permutation J, T and both gap arrays."""
    J, T, cgaps, _ = rid(A, k, p, q, seed, rounding, s, Omega)
    I, U, rgaps = cur_from_id(A, J, T, k)
    return J[:k].copy(), I, U, J, T, cgaps, rgaps


# ---------------------------------------------------------------------------
# Error measures used by the tests and the bench (plain definitions)
# ---------------------------------------------------------------------------
def rel_err_svd(A, U, S, V, block=4096):
    """||A - U diag(S) V^T||_F / ||A||_F in FP64, row block by row block."""
    A = np.asarray(A)
    num = 0.0
    den = 0.0
    VS = np.asarray(V, dtype=np.float64) * np.asarray(S, dtype=np.float64)[None, :]
    for i0 in range(0, A.shape[0], block):
        Ab = np.asarray(A[i0:i0 + block], dtype=np.float64)
        D = Ab - np.asarray(U[i0:i0 + block], dtype=np.float64) @ VS.T
        num += float(np.sum(D * D))
        den += float(np.sum(Ab * Ab))
    return np.sqrt(num / den)


def rel_err_id(A, J, T, k):
    A = np.asarray(A, dtype=np.float64)
    Vs = interpolation_matrix_t(J, T, k)
    D = A - A[:, J[:k]] @ Vs
    return np.linalg.norm(D) / np.linalg.norm(A)


def rel_err_cur(A, Jc, Ir, U):
    A = np.asarray(A, dtype=np.float64)
    D = A - A[:, Jc] @ U @ A[Ir, :]
    return np.linalg.norm(D) / np.linalg.norm(A)
