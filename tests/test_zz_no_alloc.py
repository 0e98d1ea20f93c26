"""rsvd_small_svd_noalloc against rsvd_small_svd, through the C ABI.

The no-allocation entry point serves callers that cannot allocate device
memory or hand over a workspace (cudaMalloc / cudaFree synchronise the device;
some host frameworks own the whole device-memory budget).  It must give the
same small SVD as the workspace entry point, twice in a row on the shared
static scratch, in a fresh process or after the other tests.  Collected last
(file name), so that a first-failure run has already run every other test.

Limits of the 16 MiB static scratch: l <= 512 in FP64 and l <= 720 in FP32 run;
l = 513 (FP64) and l = 721 (FP32) are rejected with RSVD_ERR_WORKSPACE.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")


def _matrix(l, seed, dtype):
    rng = np.random.default_rng(seed)
    G1, _ = np.linalg.qr(rng.standard_normal((l, l)))
    G2, _ = np.linalg.qr(rng.standard_normal((l, l)))
    M = np.linalg.qr((G1 * np.logspace(0, -3, l)) @ G2.T)[1]
    return torch.from_numpy(M).to("cuda:0", dtype)


def _noalloc_status(M):
    """(status, Uh, Sh, Vh, info) of one rsvd_small_svd_noalloc call."""
    l = M.shape[0]
    dt = rs.F64 if M.dtype == torch.float64 else rs.F32
    Uh = torch.empty(l, l, dtype=M.dtype, device=M.device)
    Vh = torch.empty(l, l, dtype=M.dtype, device=M.device)
    Sh = torch.empty(l, dtype=torch.float64, device=M.device)
    info = torch.zeros(1, dtype=torch.int32, device=M.device)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = rs.lib().rsvd_small_svd_noalloc(l, dt, ctypes.c_void_p(M.data_ptr()), l,
                                         ctypes.c_void_p(Uh.data_ptr()), l,
                                         ctypes.c_void_p(Sh.data_ptr()),
                                         ctypes.c_void_p(Vh.data_ptr()), l,
                                         ctypes.c_void_p(info.data_ptr()), stream, None)
    return st, Uh, Sh, Vh, info


def _noalloc(M):
    st, Uh, Sh, Vh, info = _noalloc_status(M)
    assert st == 0, rs.STATUS.get(st, st)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    return Uh, Sh, Vh


def _agree(M, Uh, Sh, Vh, tol, what):
    Ur, Sr, Vr = rs.small_svd(M)
    s_ref = Sr.cpu().numpy()
    assert np.max(np.abs(Sh.cpu().numpy() - s_ref) / s_ref) <= tol, what
    # singular vectors agree up to sign
    cu = np.abs(np.sum(Uh.double().cpu().numpy() * Ur.double().cpu().numpy(), axis=0))
    cv = np.abs(np.sum(Vh.double().cpu().numpy() * Vr.double().cpu().numpy(), axis=0))
    assert np.min(cu) > 1 - 100 * tol and np.min(cv) > 1 - 100 * tol, what


@pytest.mark.parametrize("dtype,l", [(torch.float32, 224), (torch.float64, 60)])
def test_noalloc_matches_workspace_entry_point_twice(dtype, l):
    tol = 1e-6 if dtype == torch.float32 else 1e-12
    for call, seed in enumerate((11, 12)):          # two calls in a row, different inputs
        M = _matrix(l, seed, dtype)
        Uh, Sh, Vh = _noalloc(M)
        _agree(M, Uh, Sh, Vh, tol, call)


@pytest.mark.parametrize("dtype,l_big,l_small", [(torch.float32, 224, 96),
                                                 (torch.float64, 120, 40)])
def test_noalloc_smaller_call_after_larger(dtype, l_big, l_small):
    """A larger l first leaves its values in the shared array under the second,
    smaller call's buffers: the second call must not read them."""
    tol = 1e-6 if dtype == torch.float32 else 1e-12
    for l, seed in ((l_big, 21), (l_small, 22)):
        M = _matrix(l, seed, dtype)
        Uh, Sh, Vh = _noalloc(M)
        _agree(M, Uh, Sh, Vh, tol, l)


@pytest.mark.parametrize("dtype,l", [(torch.float64, 512), (torch.float32, 720)])
def test_noalloc_largest_sizes_run(dtype, l):
    tol = 2e-6 if dtype == torch.float32 else 1e-12
    M = _matrix(l, 31, dtype)
    Uh, Sh, Vh = _noalloc(M)
    _agree(M, Uh, Sh, Vh, tol, l)


@pytest.mark.parametrize("dtype,l", [(torch.float64, 513), (torch.float32, 721)])
def test_noalloc_rejects_first_size_beyond(dtype, l):
    M = torch.zeros(l, l, dtype=dtype, device="cuda:0")
    st = _noalloc_status(M)[0]
    assert st == 2                                   # RSVD_ERR_WORKSPACE


def test_noalloc_rejects_too_large():
    M = torch.zeros(1024, 1024, dtype=torch.float64, device="cuda:0")
    l = 1024
    out = torch.empty(l, l, dtype=torch.float64, device="cuda:0")
    Sh = torch.empty(l, dtype=torch.float64, device="cuda:0")
    st = rs.lib().rsvd_small_svd_noalloc(l, rs.F64, ctypes.c_void_p(M.data_ptr()), l,
                                         ctypes.c_void_p(out.data_ptr()), l,
                                         ctypes.c_void_p(Sh.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), l, None,
                                         ctypes.c_void_p(0), None)
    assert st == 2                                   # RSVD_ERR_WORKSPACE
