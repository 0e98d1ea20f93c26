"""Failure detection on the GPU, in forms that fault, trap or hang nothing.

Every device-side failure of the path is reported through *d_info (an
rsvd_status value) while the kernels return normally and the context stays
usable.  Each test provokes one failure from the host side and then checks
that an ordinary call right after it still gives the right answer:

* RSVD_ERR_NO_CONVERGENCE: the one-sided Jacobi SVD given a sweep limit of one
  on a core that needs several (the FP32 8-CTA cluster kernel, l = 60, and the
  FP64 kernel);
* RSVD_ERR_NUMERIC: a NaN planted in A (the Gram of the first CholeskyQR sees
  it);
* RSVD_ERR_TIMEOUT: the grid-barrier waits of the pivoted QR bounded to a few
  million clocks, with CTA 0 withholding its first arrival
  (rsvd_test_set_barrier_wait), so that every CTA's wait runs out and every CTA
  leaves; FP64 and double-float kernels.
"""
import numpy as np
import pytest

from oracle import rsvd as orc
from synth import make_matrix_np, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"

NO_CONVERGENCE, NUMERIC, TIMEOUT = 6, 7, 8


def _core(l, seed):
    rng = np.random.default_rng(seed)
    G1, _ = np.linalg.qr(rng.standard_normal((l, l)))
    G2, _ = np.linalg.qr(rng.standard_normal((l, l)))
    return np.linalg.qr((G1 * np.logspace(0, -3, l)) @ G2.T)[1]


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_jacobi_sweep_limit_reports_no_convergence(dtype):
    M = torch.from_numpy(_core(60, 5)).to(DEV, dtype)
    with pytest.raises(rs.RsvdError) as e:
        rs.small_svd(M, rs.make_opts(max_sweeps=1))
    assert e.value.code == NO_CONVERGENCE
    # the same core with the default limit converges
    _, Sh, _ = rs.small_svd(M)
    s_ref = np.linalg.svd(M.double().cpu().numpy(), compute_uv=False)
    tol = 2e-5 if dtype == torch.float32 else 1e-12
    assert np.max(np.abs(Sh.cpu().numpy() - s_ref) / s_ref) <= tol


def test_nan_in_a_reports_numeric():
    m, n, k, p, q = 600, 400, 20, 8, 1
    A = make_matrix_np(m, n, spectrum("logspace3", n), seed=3, dtype="float32")
    Ad = torch.from_numpy(A).to(DEV)
    Ad[123, 45] = float("nan")
    with pytest.raises(rs.RsvdError) as e:
        rs.svd(Ad, k, p, q, 0x5EED)
    assert e.value.code == NUMERIC
    # a clean call right after it
    Ad[123, 45] = float(A[123, 45])
    _, S, _ = rs.svd(Ad, k, p, q, 0x5EED)
    _, So, _, _ = orc.rsvd(A.astype(np.float64), k, p, q, 0x5EED, rounding="bf16")
    assert np.max(np.abs(S.cpu().numpy() - So) / So) <= 1e-5


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_cpqr_barrier_wait_runs_out(dtype):
    rng = np.random.default_rng(17)
    r, n, k = 60, 3000, 40
    M = rng.standard_normal((r, n)) * np.logspace(0, -3, n)[rng.permutation(n)]
    if dtype == torch.float32:
        M = M.astype(np.float32)
    Md = torch.from_numpy(M).to(DEV)
    rs.test_set_barrier_wait(2_000_000, withhold=True)     # ~1 ms at 2 GHz
    try:
        with pytest.raises(rs.RsvdError) as e:
            rs.cpqr_id(Md, k)
        assert e.value.code == TIMEOUT
    finally:
        rs.test_set_barrier_wait(0)
    # the default bound again: the same call completes with the oracle's pivots
    J, _, _ = rs.cpqr_id(Md, k)
    Jo, _, _ = orc.id_from_matrix(M.astype(np.float64), k)
    assert np.array_equal(J.cpu().numpy(), Jo)
