"""Sketch widths above 256 on the tensor-core path (the l = 550 case of the
BF16 workload needs them): the passes over A run in column chunks of at most
256, Omega's chunks taking its columns 256, 512, ..  Bars as on the FP32 path.
"""
import numpy as np
import pytest

from oracle import philox, rsvd as orc
from synth import make_matrix_np, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"


def _rel(a, b):
    return np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b)


def _bf16(x):
    t = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16)
    return t.to(DEV), t.double().numpy()


@pytest.mark.parametrize("storage", ["float32", "bfloat16"])
@pytest.mark.parametrize("l", [300, 520])
def test_sample_and_apply_wide(storage, l):
    m, n = 1500, 1200
    rng = np.random.default_rng(l)
    A = rng.standard_normal((m, n)).astype(np.float32)
    if storage == "bfloat16":
        Ad, A64 = _bf16(A)
    else:
        Ad, A64 = torch.from_numpy(A).to(DEV), A.astype(np.float64)
    seed = 99 + l
    Y = rs.sample(Ad, l, seed).cpu().numpy()
    Om = rs.omega(n, l, seed, torch.float32, DEV).double().cpu().numpy()
    assert _rel(Y, A64 @ Om) <= 2e-5
    assert _rel(Y, A64 @ philox.omega(n, l, seed, "bf16")) <= 1e-4
    for trans in (0, 1):
        X = rng.standard_normal((m if trans else n, l)).astype(np.float32)
        Yx = rs.apply(Ad, torch.from_numpy(X).to(DEV), trans).cpu().numpy()
        ref = (A64.T @ X.astype(np.float64)) if trans else (A64 @ X.astype(np.float64))
        assert _rel(Yx, ref) <= 3e-5, (trans, _rel(Yx, ref))


@pytest.mark.parametrize("storage", ["float32", "bfloat16"])
def test_svd_id_cur_wide(storage):
    m, n, k, p, q = 3000, 2000, 270, 20, 1
    A32 = make_matrix_np(m, n, spectrum("inv", 2000), noise=1e-4, seed=0xE000, dtype="float32")
    if storage == "bfloat16":
        Ad, A64 = _bf16(A32)
    else:
        Ad, A64 = torch.from_numpy(A32).to(DEV), A32.astype(np.float64)
    seed = 0x5EED + 3
    out = rs.svd_id_cur(Ad, k, p, q, seed)
    S = out["S"].cpu().numpy()
    U = out["U"].double().cpu().numpy()
    V = out["V"].double().cpu().numpy()
    Uo, So, Vo, _ = orc.rsvd(A64, k, p, q, seed, rounding="bf16")
    rel = np.abs(S - So) / So
    assert rel.max() <= 1e-5, (rel.max(), np.argmax(rel))
    e, eo = orc.rel_err_svd(A64, U, S, V), orc.rel_err_svd(A64, Uo, So, Vo)
    assert abs(e - eo) <= 0.01 * eo, (e, eo)
    # the right vectors of the small SVD are M^T u_j / sigma_j on the FP32 path,
    # so the Jacobi tolerance on u_j grows by sigma_1 / sigma_j: with k deep in
    # the noise bulk the orthogonality bar scales with sigma_1 / sigma_k
    cond = So[0] / So[k - 1]
    assert np.linalg.norm(U.T @ U - np.eye(k)) <= 5e-5 * cond, (np.linalg.norm(U.T @ U - np.eye(k)), cond)
    assert np.linalg.norm(V.T @ V - np.eye(k)) <= 5e-5 * cond
    J = out["J"].cpu().numpy()
    Jo, To, gaps, _ = orc.rid(A64, k, p, q, seed, rounding="bf16")
    t = 0
    while t < len(gaps) and J[t] == Jo[t]:
        t += 1
    first_small = next((i for i, g in enumerate(gaps) if g <= 1e-6), len(gaps))
    assert t >= min(first_small, k), (t, first_small)
    assert sorted(J.tolist()) == list(range(n))
