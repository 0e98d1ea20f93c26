"""Python binding of librsvd.so: randomized QB / RSVD / ID / CUR on one GB300.

Argument marshalling only.  Every step of the computation runs in the CUDA
kernels of librsvd.so (C ABI declared in include/rsvd.h); this module turns
torch CUDA tensors into pointers, sizes and the current stream, allocates the
outputs and the workspace with torch, and raises on a non-OK status.  There is
no fallback: importing works without the library, but every call fails loudly
when librsvd.so has not been built.

Functions (names follow the C ABI):
  qb, svd, id, cur, svd_id_cur       - the routines of the paper's Alg. 5 / Sec. 3.5-3.6
  svd_tol, id_tol, cur_tol           - the same to a tolerance (Sec. 2.6, Sec. 4 TOL mode)
  id_left                            - the ID from the left sketch (Sec. 3.5, Alg. 6)
  svd_vjp, svd_autograd              - the adjoint of Alg. 5 (rsvd_svd_vjp) and a
                                       torch.autograd.Function around it
  omega, omega_words                 - the Philox Gaussian test matrix (checking aid)
  sample, apply, orth, small_svd     - the individual steps of the path
  cpqr_id                            - column ID of an explicit FP64 matrix (Alg. 1)
"""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librsvd.so")

F32, F64, BF16 = 0, 1, 2
PREC_TC, PREC_SIMT, PREC_MIXED, PREC_FP8 = 0, 1, 2, 3

STATUS = {
    0: "RSVD_OK", 1: "RSVD_ERR_INVALID_ARG", 2: "RSVD_ERR_WORKSPACE", 3: "RSVD_ERR_CUDA",
    4: "RSVD_ERR_UNSUPPORTED", 5: "RSVD_ERR_NOT_SPD", 6: "RSVD_ERR_NO_CONVERGENCE",
    7: "RSVD_ERR_NUMERIC", 8: "RSVD_ERR_TIMEOUT",
}


class RsvdError(RuntimeError):
    def __init__(self, code, where):
        self.code = int(code)
        super().__init__("%s: %s" % (where, STATUS.get(self.code, str(code))))


class Opts(ctypes.Structure):
    _fields_ = [("s", ctypes.c_int), ("max_sweeps", ctypes.c_int),
                ("precision", ctypes.c_int), ("reserved", ctypes.c_int * 13)]


class BatchItem(ctypes.Structure):
    """rsvd_batch_item: one problem of rsvd_svd_batched (sizes, rank, element offsets)."""
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("k", ctypes.c_int),
                ("a_off", ctypes.c_int64), ("u_off", ctypes.c_int64), ("v_off", ctypes.c_int64),
                ("s_off", ctypes.c_int64)]


_lib = None
_c_i64 = ctypes.c_int64
_c_int = ctypes.c_int
_c_u64 = ctypes.c_uint64
_c_size = ctypes.c_size_t
_vp = ctypes.c_void_p
_OPTP = ctypes.POINTER(Opts)

_SIGS = {
    "rsvd_opts_default": (None, [_OPTP]),
    "rsvd_status_string": (ctypes.c_char_p, [_c_int]),
    "rsvd_version": (_c_int, []),
    "rsvd_qb_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int, _OPTP]),
    "rsvd_svd_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int, _OPTP]),
    "rsvd_id_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int, _OPTP]),
    "rsvd_cur_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int, _OPTP]),
    "rsvd_svd_id_cur_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int,
                                                 _OPTP]),
    "rsvd_qb": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64, _c_int, _vp, _c_i64,
                         _vp, _c_i64, _vp, _c_i64, _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_svd": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64, _c_int, _vp, _c_i64,
                          _vp, _c_i64, _vp, _vp, _c_i64, _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_id": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64, _c_int, _vp, _c_i64,
                         _vp, _vp, _c_i64, _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_cur": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64, _c_int, _vp, _c_i64,
                          _vp, _vp, _vp, _c_i64, _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_svd_id_cur": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64, _c_int, _vp,
                                 _c_i64, _vp, _c_i64, _vp, _vp, _c_i64, _vp, _vp, _c_i64, _vp,
                                 _vp, _vp, _c_i64, _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_omega": (_c_int, [_c_i64, _c_int, _c_u64, _c_int, _vp, _c_i64, _vp]),
    "rsvd_omega_words": (_c_int, [_c_i64, _c_int, _c_u64, _vp, _vp]),
    "rsvd_omega_fp8": (_c_int, [_c_i64, _c_int, _c_u64, _vp, _c_i64, _vp]),
    "rsvd_sample_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _OPTP]),
    "rsvd_sample": (_c_int, [_c_i64, _c_i64, _c_int, _c_u64, _c_int, _vp, _c_i64, _vp, _c_i64,
                             _vp, _c_size, _vp, _OPTP]),
    "rsvd_apply_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _OPTP]),
    "rsvd_apply": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _vp, _c_i64, _vp, _c_i64,
                            _vp, _c_i64, _vp, _c_size, _vp, _OPTP]),
    "rsvd_orth_workspace_size": (_c_size, [_c_i64, _c_int, _c_int, _OPTP]),
    "rsvd_orth": (_c_int, [_c_i64, _c_int, _c_int, _vp, _c_i64, _vp, _c_i64, _vp, _c_i64, _vp,
                           _c_size, _vp, _vp, _OPTP]),
    "rsvd_small_svd_workspace_size": (_c_size, [_c_int, _c_int, _OPTP]),
    "rsvd_small_svd": (_c_int, [_c_int, _c_int, _vp, _c_i64, _vp, _c_i64, _vp, _vp, _c_i64, _vp,
                                _c_size, _vp, _vp, _OPTP]),
    "rsvd_cpqr_workspace_size": (_c_size, [_c_int, _c_i64, _c_int]),
    "rsvd_small_svd_noalloc": (_c_int, [_c_int, _c_int, _vp, _c_i64, _vp, _c_i64, _vp, _vp,
                                        _c_i64, _vp, _vp, _OPTP]),
    "rsvd_trace_enable": (_c_int, [_c_int]),
    "rsvd_trace_read": (_c_int, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_c_i64), _c_int]),
    "rsvd_kernel_launch_count": (_c_i64, []),
    "rsvd_test_set_barrier_wait": (_c_int, [ctypes.c_longlong, _c_int]),
    "rsvd_cpqr_id": (_c_int, [_c_int, _c_i64, _c_int, _vp, _c_i64, _vp, _vp, _c_i64, _vp, _vp,
                              _c_size, _vp, _vp]),
    "rsvd_svd_id_cur_host": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64, _c_int,
                                      _vp, _vp, _c_i64, _vp, _c_i64, _vp, _vp, _c_i64, _vp, _vp,
                                      _c_i64, _vp, _vp, _vp, _c_i64, _vp, _c_size, _vp, _vp,
                                      _OPTP]),
    "rsvd_cpqr_f32_workspace_size": (_c_size, [_c_int, _c_i64, _c_int]),
    "rsvd_svd_batched_workspace_size": (_c_size, [_c_int, ctypes.POINTER(BatchItem), _c_int,
                                                  _c_int]),
    "rsvd_svd_batched": (_c_int, [_c_int, ctypes.POINTER(BatchItem), _c_int, _c_int, _c_u64, _vp,
                                  _vp, _vp, _vp, _vp, _c_size, _vp, _vp]),
    "rsvd_batched_tuning": (_c_int, [_c_int, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                                     ctypes.POINTER(_c_int), ctypes.POINTER(ctypes.c_float)]),
    "rsvd_cpqr_id_f32": (_c_int, [_c_int, _c_i64, _c_int, _vp, _c_i64, _vp, _vp, _c_i64, _vp,
                                  _vp, _c_size, _vp, _vp]),
    "rsvd_id_tol_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int,
                                             _OPTP]),
    "rsvd_cur_tol_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int,
                                              _OPTP]),
    "rsvd_id_left_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int,
                                              _OPTP]),
    "rsvd_svd_tol": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, ctypes.c_double, _c_u64,
                              _c_int, _vp, _c_i64, _vp, _c_i64, _vp, _vp, _c_i64,
                              ctypes.POINTER(_c_int), _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_id_tol": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, ctypes.c_double, _c_u64,
                             _c_int, _vp, _c_i64, _vp, _vp, _c_i64, ctypes.POINTER(_c_int), _vp,
                             _c_size, _vp, _vp, _OPTP]),
    "rsvd_cur_tol": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, ctypes.c_double, _c_u64,
                              _c_int, _vp, _c_i64, _vp, _vp, _vp, _c_i64, ctypes.POINTER(_c_int),
                              _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_id_left": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64, _c_int, _vp, _c_i64,
                              _vp, _vp, _c_i64, _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_svd_vjp_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int,
                                              _OPTP]),
    "rsvd_svd_vjp": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_u64, _c_int, _vp, _c_i64,
                              _vp, _c_i64, _vp, _vp, _c_i64, _vp, _c_i64, _vp, _c_i64, _vp, _vp,
                              _c_i64, _vp, _c_size, _vp, _vp, _OPTP]),
    "rsvd_qb_adaptive_workspace_size": (_c_size, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_int,
                                                  _OPTP]),
    "rsvd_qb_adaptive": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, ctypes.c_double, _c_int,
                                  _c_u64, _c_int, _vp, _c_i64, _vp, _c_i64, _vp, _c_i64, _vp,
                                  ctypes.POINTER(_c_int), _vp, _c_size, _vp, _vp, _OPTP]),
}


def lib():
    """The loaded librsvd.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librsvd.so is not built (run __graft_entry__.build() or "
                               "python paper_1502_05366_gb300/build.py); there is no fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return sorted(_SIGS)


TRACE_CLASSES = ["a_omega", "a_w", "at_w", "gram", "orth_apply", "reduce", "cpqr", "jacobi",
                 "chol", "solve", "simt_gemm"]


def trace_enable(on=True):
    lib().rsvd_trace_enable(1 if on else 0)


def trace_read():
    """{class: (total ms, launches)} of the traced kernels since the last read."""
    n = len(TRACE_CLASSES)
    ms = (ctypes.c_double * n)()
    cnt = (_c_i64 * n)()
    lib().rsvd_trace_read(ms, cnt, n)
    return {TRACE_CLASSES[i]: (ms[i], cnt[i]) for i in range(n)}


def kernel_launch_count():
    return int(lib().rsvd_kernel_launch_count())


def test_set_barrier_wait(cycles, withhold=False):
    """Test aid: bound the pivoted-QR grid-barrier waits to `cycles` SM clocks
    (0 restores the default) and optionally withhold CTA 0's first arrival
    (rsvd_test_set_barrier_wait)."""
    _raise(lib().rsvd_test_set_barrier_wait(int(cycles), 1 if withhold else 0),
           "rsvd_test_set_barrier_wait")


def make_opts(s=1, max_sweeps=30, precision=PREC_TC):
    o = Opts()
    lib().rsvd_opts_default(ctypes.byref(o))
    o.s, o.max_sweeps, o.precision = int(s), int(max_sweeps), int(precision)
    return o


# ---------------------------------------------------------------------------
# tensor plumbing
# ---------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _dtype_code(t):
    torch = _torch()
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError("unsupported dtype %s (float32, float64 or bfloat16)" % t.dtype)


def _out_dtype(dtype):
    """Floating output type for an A of this dtype: bf16 A gives float32."""
    torch = _torch()
    return torch.float32 if dtype == torch.bfloat16 else dtype


def _check_matrix(t, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dim() != 2 or t.stride(1) != 1 or t.stride(0) < t.shape[1]:
        raise ValueError("%s must be a row-major 2-D tensor (unit column stride)" % name)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(_torch().cuda.current_stream().cuda_stream)


def _work(nbytes, device):
    torch = _torch()
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# Largest rank of a call that forms an ID or a CUR (the triangular solve for
# T = S11^-1 S12); the library returns RSVD_ERR_UNSUPPORTED beyond it.
ID_MAX_K = 880


def _no_workspace(where, k):
    """Raise for a workspace query that returned 0: RSVD_ERR_UNSUPPORTED when
    the rank is beyond ID_MAX_K, RSVD_ERR_INVALID_ARG otherwise."""
    raise RsvdError(4 if k > ID_MAX_K else 1, where)


def _raise(st, where):
    if st != 0:
        raise RsvdError(st, where)


def _info(device):
    return _torch().zeros(1, dtype=_torch().int32, device=device)


def check_info(info, where="device"):
    """Synchronises and raises if the device-side status is not OK."""
    v = int(info.item())
    if v != 0:
        raise RsvdError(v, where)


def _opts_ptr(opts):
    return ctypes.byref(opts) if opts is not None else None


# ---------------------------------------------------------------------------
# routines
# ---------------------------------------------------------------------------
def qb(A, k, p, q, seed, opts=None, check=True):
    """(Q, Bt) with Q m x l orthonormal and Bt = A^T Q (n x l); l = k + p."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    l = k + p
    dt = _dtype_code(A)
    Q = torch.empty(m, l, dtype=_out_dtype(A.dtype), device=A.device)
    Bt = torch.empty(n, l, dtype=_out_dtype(A.dtype), device=A.device)
    ws = lib().rsvd_qb_workspace_size(m, n, k, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        raise RsvdError(1, "rsvd_qb_workspace_size")
    W = _work(ws, A.device)
    info = _info(A.device)
    st = lib().rsvd_qb(m, n, k, p, q, seed, dt, _ptr(A), A.stride(0), _ptr(Q), l, _ptr(Bt), l,
                       _ptr(W), W.numel(), _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_qb")
    if check:
        check_info(info, "rsvd_qb")
    return Q, Bt


def qb_adaptive(A, b, M, q, eps, seed, relative=True, opts=None, overwrite=False, check=True):
    """Blocked adaptive QB to a tolerance (Alg. 7): (Q, Bt, resid).

    Q (m x r) orthonormal and Bt = A^T Q (n x r) with r = b times the number of
    blocks taken; resid = [||A||_F, residual norm after each block].  The loop
    stops at the first block whose residual is below eps (times ||A||_F when
    relative) or after M blocks.  The library overwrites its A with the
    residual: a copy is passed unless overwrite=True.
    """
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    Aw = A if overwrite else A.clone()
    cols = b * M
    Q = torch.empty(m, cols, dtype=A.dtype, device=A.device)
    Bt = torch.empty(n, cols, dtype=A.dtype, device=A.device)
    resid = torch.zeros(M + 1, dtype=torch.float64, device=A.device)
    ws = lib().rsvd_qb_adaptive_workspace_size(m, n, b, M, q, dt, _opts_ptr(opts))
    if ws == 0:
        raise RsvdError(1, "rsvd_qb_adaptive_workspace_size")
    W = _work(ws, A.device)
    info = _info(A.device)
    rank = ctypes.c_int(0)
    st = lib().rsvd_qb_adaptive(m, n, b, M, q, float(eps), 1 if relative else 0, seed, dt,
                                _ptr(Aw), Aw.stride(0), _ptr(Q), cols, _ptr(Bt), cols,
                                _ptr(resid), ctypes.byref(rank), _ptr(W), W.numel(), _ptr(info),
                                _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_qb_adaptive")
    if check:
        check_info(info, "rsvd_qb_adaptive")
    r = rank.value
    return Q[:, :r], Bt[:, :r], resid[:r // b + 1]


def svd(A, k, p, q, seed, opts=None, check=True):
    """(U, S, V): A ~ U diag(S) V^T, U m x k, S k (float64), V n x k (Alg. 5)."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    U = torch.empty(m, k, dtype=_out_dtype(A.dtype), device=A.device)
    V = torch.empty(n, k, dtype=_out_dtype(A.dtype), device=A.device)
    S = torch.empty(k, dtype=torch.float64, device=A.device)
    ws = lib().rsvd_svd_workspace_size(m, n, k, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        raise RsvdError(1, "rsvd_svd_workspace_size")
    W = _work(ws, A.device)
    info = _info(A.device)
    st = lib().rsvd_svd(m, n, k, p, q, seed, dt, _ptr(A), A.stride(0), _ptr(U), k, _ptr(S),
                        _ptr(V), k, _ptr(W), W.numel(), _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_svd")
    if check:
        check_info(info, "rsvd_svd")
    return U, S, V


def id(A, k, p, q, seed, opts=None, check=True):  # noqa: A001 - the paper's name
    """(J, T): J n int32 permutation (J[:k] skeleton), T k x (n-k)."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    J = torch.empty(n, dtype=torch.int32, device=A.device)
    T = torch.empty(k, max(n - k, 1), dtype=_out_dtype(A.dtype), device=A.device)
    ws = lib().rsvd_id_workspace_size(m, n, k, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        _no_workspace("rsvd_id_workspace_size", k)
    W = _work(ws, A.device)
    info = _info(A.device)
    st = lib().rsvd_id(m, n, k, p, q, seed, dt, _ptr(A), A.stride(0), _ptr(J), _ptr(T),
                       T.stride(0), _ptr(W), W.numel(), _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_id")
    if check:
        check_info(info, "rsvd_id")
    return J, T[:, : n - k]


def cur(A, k, p, q, seed, opts=None, check=True):
    """(Jc, Ir, U): A ~ A[:, Jc] U A[Ir, :] (Alg. 3)."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    Jc = torch.empty(k, dtype=torch.int32, device=A.device)
    Ir = torch.empty(k, dtype=torch.int32, device=A.device)
    U = torch.empty(k, k, dtype=_out_dtype(A.dtype), device=A.device)
    ws = lib().rsvd_cur_workspace_size(m, n, k, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        _no_workspace("rsvd_cur_workspace_size", k)
    W = _work(ws, A.device)
    info = _info(A.device)
    st = lib().rsvd_cur(m, n, k, p, q, seed, dt, _ptr(A), A.stride(0), _ptr(Jc), _ptr(Ir),
                        _ptr(U), k, _ptr(W), W.numel(), _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_cur")
    if check:
        check_info(info, "rsvd_cur")
    return Jc, Ir, U


def svd_tol(A, kmax, p, q, tol, seed, opts=None, check=True):
    """SVD to a tolerance (Sec. 2.6): (U, S, V) of rank r, the number of
    singular values above tol (at least 1), from a sketch of kmax + p columns."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    U = torch.empty(m, kmax, dtype=_out_dtype(A.dtype), device=A.device)
    V = torch.empty(n, kmax, dtype=_out_dtype(A.dtype), device=A.device)
    S = torch.empty(kmax, dtype=torch.float64, device=A.device)
    ws = lib().rsvd_svd_workspace_size(m, n, kmax, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        raise RsvdError(1, "rsvd_svd_workspace_size")
    W = _work(ws, A.device)
    info = _info(A.device)
    rank = ctypes.c_int(0)
    st = lib().rsvd_svd_tol(m, n, kmax, p, q, float(tol), seed, dt, _ptr(A), A.stride(0), _ptr(U),
                            kmax, _ptr(S), _ptr(V), kmax, ctypes.byref(rank), _ptr(W), W.numel(),
                            _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_svd_tol")
    if check:
        check_info(info, "rsvd_svd_tol")
    r = rank.value
    return U[:, :r], S[:r], V[:, :r]


def id_tol(A, kmax, p, q, tol, seed, opts=None, check=True):
    """Column ID to a tolerance (Sec. 2.6): (J, T, k) with ||S22||_F < tol after
    k <= kmax pivoted-QR steps of the sketch B (l = kmax + p)."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    J = torch.empty(n, dtype=torch.int32, device=A.device)
    T = torch.empty(kmax, n - 1, dtype=_out_dtype(A.dtype), device=A.device)
    ws = lib().rsvd_id_tol_workspace_size(m, n, kmax, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        _no_workspace("rsvd_id_tol_workspace_size", kmax)
    W = _work(ws, A.device)
    info = _info(A.device)
    rank = ctypes.c_int(0)
    st = lib().rsvd_id_tol(m, n, kmax, p, q, float(tol), seed, dt, _ptr(A), A.stride(0), _ptr(J),
                           _ptr(T), T.stride(0), ctypes.byref(rank), _ptr(W), W.numel(),
                           _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_id_tol")
    if check:
        check_info(info, "rsvd_id_tol")
    k = rank.value
    return J, T[:k, : n - k], k


def cur_tol(A, kmax, p, q, tol, seed, opts=None, check=True):
    """CUR to a tolerance: (Jc, Ir, U, k) on the column ID of id_tol."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    Jc = torch.empty(kmax, dtype=torch.int32, device=A.device)
    Ir = torch.empty(kmax, dtype=torch.int32, device=A.device)
    U = torch.empty(kmax, kmax, dtype=_out_dtype(A.dtype), device=A.device)
    ws = lib().rsvd_cur_tol_workspace_size(m, n, kmax, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        _no_workspace("rsvd_cur_tol_workspace_size", kmax)
    W = _work(ws, A.device)
    info = _info(A.device)
    rank = ctypes.c_int(0)
    st = lib().rsvd_cur_tol(m, n, kmax, p, q, float(tol), seed, dt, _ptr(A), A.stride(0),
                            _ptr(Jc), _ptr(Ir), _ptr(U), kmax, ctypes.byref(rank), _ptr(W),
                            W.numel(), _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_cur_tol")
    if check:
        check_info(info, "rsvd_cur_tol")
    k = rank.value
    return Jc[:k], Ir[:k], U[:k, :k], k


def id_left(A, k, p, q, seed, opts=None, check=True):
    """Column ID from the left sketch Omega~ A (A^T A)^q (Sec. 3.5, Alg. 6): (J, T)."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    J = torch.empty(n, dtype=torch.int32, device=A.device)
    T = torch.empty(k, max(n - k, 1), dtype=_out_dtype(A.dtype), device=A.device)
    ws = lib().rsvd_id_left_workspace_size(m, n, k, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        _no_workspace("rsvd_id_left_workspace_size", k)
    W = _work(ws, A.device)
    info = _info(A.device)
    st = lib().rsvd_id_left(m, n, k, p, q, seed, dt, _ptr(A), A.stride(0), _ptr(J), _ptr(T),
                            T.stride(0), _ptr(W), W.numel(), _ptr(info), _stream(),
                            _opts_ptr(opts))
    _raise(st, "rsvd_id_left")
    if check:
        check_info(info, "rsvd_id_left")
    return J, T[:, : n - k]


def svd_vjp(A, k, p, q, seed, gU, gS, gV, opts=None, check=True, with_outputs=False):
    """Cotangent of A for (U, S, V) = svd(A, k, p, q, seed) given the cotangents
    of U, S and V (rsvd_svd_vjp; Omega fixed, the forward replayed from A and
    the seed).  gU, gS, gV may be None (zero).  Returns gA, or (gA, U, S, V)."""
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    dev = A.device
    gU = torch.zeros(m, k, dtype=A.dtype, device=dev) if gU is None else \
        gU.to(A.dtype).contiguous()
    gV = torch.zeros(n, k, dtype=A.dtype, device=dev) if gV is None else \
        gV.to(A.dtype).contiguous()
    gS = torch.zeros(k, dtype=torch.float64, device=dev) if gS is None else \
        gS.to(torch.float64).contiguous()
    gA = torch.empty(m, n, dtype=A.dtype, device=dev)
    U = V = S = None
    if with_outputs:
        U = torch.empty(m, k, dtype=A.dtype, device=dev)
        V = torch.empty(n, k, dtype=A.dtype, device=dev)
        S = torch.empty(k, dtype=torch.float64, device=dev)
    ws = lib().rsvd_svd_vjp_workspace_size(m, n, k, p, q, dt, _opts_ptr(opts))
    if ws == 0:
        raise RsvdError(1, "rsvd_svd_vjp_workspace_size")
    W = _work(ws, dev)
    info = _info(dev)
    st = lib().rsvd_svd_vjp(m, n, k, p, q, seed, dt, _ptr(A), A.stride(0), _ptr(gU), k, _ptr(gS),
                            _ptr(gV), k, _ptr(gA), n, _ptr(U), k, _ptr(S), _ptr(V), k, _ptr(W),
                            W.numel(), _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_svd_vjp")
    if check:
        check_info(info, "rsvd_svd_vjp")
    return (gA, U, S, V) if with_outputs else gA


def _make_autograd():
    torch = _torch()

    class RSVD(torch.autograd.Function):
        """(U, S, V) = rsvd_svd(A) as a differentiable function of A (Omega fixed).

        The forward runs rsvd_svd and keeps only A; the backward calls
        rsvd_svd_vjp, which replays the forward from A and the seed instead of
        storing the power iteration's intermediates."""

        @staticmethod
        def forward(ctx, A, k, p, q, seed, opts):
            U, S, V = svd(A, k, p, q, seed, opts)
            ctx.save_for_backward(A)
            ctx.args = (k, p, q, seed, opts)
            return U, S, V

        @staticmethod
        def backward(ctx, gU, gS, gV):
            (A,) = ctx.saved_tensors
            k, p, q, seed, opts = ctx.args
            gA = svd_vjp(A.detach().contiguous(), k, p, q, seed, gU, gS, gV, opts)
            return gA, None, None, None, None, None

    return RSVD


_RSVD = None


def svd_autograd(A, k, p, q, seed, opts=None):
    """Differentiable randomized SVD: (U, S, V) whose backward is the library's
    adjoint of Alg. 5 (rsvd_svd_vjp)."""
    global _RSVD
    if _RSVD is None:
        _RSVD = _make_autograd()
    return _RSVD.apply(A, k, p, q, seed, opts)


class Plan:
    """Pre-allocated outputs and workspace for repeated rsvd_svd_id_cur calls."""

    def __init__(self, m, n, k, p, q, dtype, device, opts=None, with_svd=True, with_id=True,
                 with_cur=True):
        torch = _torch()
        self.m, self.n, self.k, self.p, self.q = m, n, k, p, q
        self.dt = {torch.float32: F32, torch.float64: F64, torch.bfloat16: BF16}[dtype]
        self.opts = opts
        dev = torch.device(device)
        dtype = _out_dtype(dtype)
        self.U = torch.empty(m, k, dtype=dtype, device=dev) if with_svd else None
        self.S = torch.empty(k, dtype=torch.float64, device=dev) if with_svd else None
        self.V = torch.empty(n, k, dtype=dtype, device=dev) if with_svd else None
        self.J = torch.empty(n, dtype=torch.int32, device=dev) if with_id else None
        self.T = torch.empty(k, n - k, dtype=dtype, device=dev) if with_id else None
        self.Jc = torch.empty(k, dtype=torch.int32, device=dev) if with_cur else None
        self.Ir = torch.empty(k, dtype=torch.int32, device=dev) if with_cur else None
        self.Ucur = torch.empty(k, k, dtype=dtype, device=dev) if with_cur else None
        ws = lib().rsvd_svd_id_cur_workspace_size(m, n, k, p, q, self.dt, _opts_ptr(opts))
        if ws == 0:
            _no_workspace("rsvd_svd_id_cur_workspace_size", k)
        self.work = _work(ws, dev)
        self.info = _info(dev)

    def run_host(self, A_host, A, seed):
        """As run() with A in (page-locked) host memory: A_host is copied into
        the device buffer A while the sketch consumes it (rsvd_svd_id_cur_host)."""
        _check_matrix(A, "A")
        if A_host.is_cuda or A_host.shape != A.shape or A_host.stride() != A.stride():
            raise ValueError("A_host: a host tensor with the layout of A")
        k = self.k
        st = lib().rsvd_svd_id_cur_host(
            self.m, self.n, k, self.p, self.q, seed, self.dt, A_host.data_ptr(), _ptr(A),
            A.stride(0), _ptr(self.U), k, _ptr(self.S), _ptr(self.V), k, _ptr(self.J),
            _ptr(self.T), self.n - k, _ptr(self.Jc), _ptr(self.Ir), _ptr(self.Ucur), k,
            _ptr(self.work), self.work.numel(), _ptr(self.info), _stream(),
            _opts_ptr(self.opts))
        _raise(st, "rsvd_svd_id_cur_host")

    def run(self, A, seed):
        _check_matrix(A, "A")
        k = self.k
        st = lib().rsvd_svd_id_cur(
            self.m, self.n, k, self.p, self.q, seed, self.dt, _ptr(A), A.stride(0),
            _ptr(self.U), k, _ptr(self.S), _ptr(self.V), k, _ptr(self.J), _ptr(self.T),
            self.n - k, _ptr(self.Jc), _ptr(self.Ir), _ptr(self.Ucur), k, _ptr(self.work),
            self.work.numel(), _ptr(self.info), _stream(), _opts_ptr(self.opts))
        _raise(st, "rsvd_svd_id_cur")


class QbPlan:
    """Pre-allocated Q, Bt and workspace for repeated rsvd_qb calls (the range
    finder with the power scheme and Bt = A^T Q, Alg. 5 up to the QB step)."""

    def __init__(self, m, n, k, p, q, dtype, device, opts=None):
        torch = _torch()
        self.m, self.n, self.k, self.p, self.q = m, n, k, p, q
        self.dt = {torch.float32: F32, torch.float64: F64, torch.bfloat16: BF16}[dtype]
        self.opts = opts
        dev = torch.device(device)
        l = k + p
        self.Q = torch.empty(m, l, dtype=_out_dtype(dtype), device=dev)
        self.Bt = torch.empty(n, l, dtype=_out_dtype(dtype), device=dev)
        ws = lib().rsvd_qb_workspace_size(m, n, k, p, q, self.dt, _opts_ptr(opts))
        if ws == 0:
            raise RsvdError(1, "rsvd_qb_workspace_size")
        self.work = _work(ws, dev)
        self.info = _info(dev)

    def run(self, A, seed):
        _check_matrix(A, "A")
        l = self.k + self.p
        st = lib().rsvd_qb(self.m, self.n, self.k, self.p, self.q, seed, self.dt, _ptr(A),
                           A.stride(0), _ptr(self.Q), l, _ptr(self.Bt), l, _ptr(self.work),
                           self.work.numel(), _ptr(self.info), _stream(), _opts_ptr(self.opts))
        _raise(st, "rsvd_qb")


def svd_id_cur(A, k, p, q, seed, opts=None, check=True):
    """RSVD, ID and CUR from one sketch: dict of U, S, V, J, T, Jc, Ir, Ucur."""
    _check_matrix(A, "A")
    m, n = A.shape
    plan = Plan(m, n, k, p, q, A.dtype, A.device, opts)
    plan.run(A, seed)
    if check:
        check_info(plan.info, "rsvd_svd_id_cur")
    return dict(U=plan.U, S=plan.S, V=plan.V, J=plan.J, T=plan.T, Jc=plan.Jc, Ir=plan.Ir,
                Ucur=plan.Ucur)


# ---------------------------------------------------------------------------
# step-level calls
# ---------------------------------------------------------------------------
def omega(n, l, seed, dtype, device="cuda"):
    torch = _torch()
    Om = torch.empty(n, l, dtype=dtype, device=device)
    dt = {torch.float32: F32, torch.float64: F64}[dtype]
    _raise(lib().rsvd_omega(n, l, seed, dt, _ptr(Om), l, _stream()), "rsvd_omega")
    return Om


def omega_fp8(n, l, seed, device="cuda"):
    """Omega of the FP8 sketch (rsvd_omega_fp8): n x l float32, the bf16 Omega
    quantised to E4M3 with a power-of-two scale per 32-row block of each column."""
    torch = _torch()
    Om = torch.empty(n, l, dtype=torch.float32, device=device)
    _raise(lib().rsvd_omega_fp8(n, l, seed, _ptr(Om), l, _stream()), "rsvd_omega_fp8")
    return Om


def omega_words(n, l, seed, device="cuda"):
    torch = _torch()
    nq = (l + 3) // 4
    out = torch.empty(n, nq, 4, dtype=torch.int32, device=device)
    _raise(lib().rsvd_omega_words(n, l, seed, _ptr(out), _stream()), "rsvd_omega_words")
    return out


def sample(A, l, seed, opts=None):
    torch = _torch()
    _check_matrix(A, "A")
    m, n = A.shape
    dt = _dtype_code(A)
    Y = torch.empty(m, l, dtype=_out_dtype(A.dtype), device=A.device)
    ws = lib().rsvd_sample_workspace_size(m, n, l, dt, _opts_ptr(opts))
    W = _work(ws, A.device)
    st = lib().rsvd_sample(m, n, l, seed, dt, _ptr(A), A.stride(0), _ptr(Y), l, _ptr(W),
                           W.numel(), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_sample")
    return Y


def apply(A, X, trans, opts=None):
    torch = _torch()
    _check_matrix(A, "A")
    _check_matrix(X, "X")
    m, n = A.shape
    l = X.shape[1]
    dt = _dtype_code(A)
    rows = n if trans else m
    Y = torch.empty(rows, l, dtype=_out_dtype(A.dtype), device=A.device)
    ws = lib().rsvd_apply_workspace_size(m, n, l, dt, _opts_ptr(opts))
    W = _work(ws, A.device)
    st = lib().rsvd_apply(m, n, l, int(trans), dt, _ptr(A), A.stride(0), _ptr(X), X.stride(0),
                          _ptr(Y), l, _ptr(W), W.numel(), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_apply")
    return Y


def orth(X, opts=None, check=True):
    torch = _torch()
    _check_matrix(X, "X")
    rows, l = X.shape
    dt = _dtype_code(X)
    Q = torch.empty(rows, l, dtype=X.dtype, device=X.device)
    R = torch.empty(l, l, dtype=X.dtype, device=X.device)
    ws = lib().rsvd_orth_workspace_size(rows, l, dt, _opts_ptr(opts))
    if ws == 0:
        raise RsvdError(1, "rsvd_orth_workspace_size")
    W = _work(ws, X.device)
    info = _info(X.device)
    st = lib().rsvd_orth(rows, l, dt, _ptr(X), X.stride(0), _ptr(Q), l, _ptr(R), l, _ptr(W),
                         W.numel(), _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_orth")
    if check:
        check_info(info, "rsvd_orth")
    return Q, R


def small_svd(M, opts=None, check=True):
    torch = _torch()
    _check_matrix(M, "M")
    l = M.shape[0]
    dt = _dtype_code(M)
    Uh = torch.empty(l, l, dtype=M.dtype, device=M.device)
    Vh = torch.empty(l, l, dtype=M.dtype, device=M.device)
    Sh = torch.empty(l, dtype=torch.float64, device=M.device)
    ws = lib().rsvd_small_svd_workspace_size(l, dt, _opts_ptr(opts))
    W = _work(ws, M.device)
    info = _info(M.device)
    st = lib().rsvd_small_svd(l, dt, _ptr(M), M.stride(0), _ptr(Uh), l, _ptr(Sh), _ptr(Vh), l,
                              _ptr(W), W.numel(), _ptr(info), _stream(), _opts_ptr(opts))
    _raise(st, "rsvd_small_svd")
    if check:
        check_info(info, "rsvd_small_svd")
    return Uh, Sh, Vh


def cpqr_id(M, k, check=True):
    """Column ID of an explicit CUDA matrix M (r x n): (J, T, gaps).

    float64 M: FP64 arithmetic (rsvd_cpqr_id); float32 M: the double-float
    arithmetic of the FP32 path (rsvd_cpqr_id_f32), T in float32."""
    torch = _torch()
    _check_matrix(M, "M")
    if M.dtype == torch.float64:
        size_fn, fn, name = lib().rsvd_cpqr_workspace_size, lib().rsvd_cpqr_id, "rsvd_cpqr_id"
    elif M.dtype == torch.float32:
        size_fn, fn, name = (lib().rsvd_cpqr_f32_workspace_size, lib().rsvd_cpqr_id_f32,
                             "rsvd_cpqr_id_f32")
    else:
        raise TypeError("cpqr_id takes float64 or float32")
    r, n = M.shape
    J = torch.empty(n, dtype=torch.int32, device=M.device)
    T = torch.empty(k, max(n - k, 1), dtype=M.dtype, device=M.device)
    gaps = torch.empty(k, dtype=torch.float64, device=M.device)
    ws = size_fn(r, n, k)
    if ws == 0:
        _no_workspace(name.replace("_id", "") + "_workspace_size", k)
    W = _work(ws, M.device)
    info = _info(M.device)
    st = fn(r, n, k, _ptr(M), M.stride(0), _ptr(J), _ptr(T), T.stride(0), _ptr(gaps), _ptr(W),
            W.numel(), _ptr(info), _stream())
    _raise(st, name)
    if check:
        check_info(info, name)
    return J, T[:, : n - k], gaps


# ---------------------------------------------------------------------------
# batched problems
# ---------------------------------------------------------------------------
class BatchPlan:
    """Packed outputs and workspace for rsvd_svd_batched over fixed problem sizes.

    Problem i is A_i (ms[i] x ns[i], row-major) at element a_off[i] of one packed
    float32 buffer; U_i (m x k), V_i (n x k) and S_i (k, float64) live in packed
    outputs at their offsets."""

    def __init__(self, ms, ns, ks, p, q, device):
        torch = _torch()
        self.batch = len(ms)
        self.ms, self.ns, self.ks = [int(x) for x in ms], [int(x) for x in ns], [int(x) for x in ks]
        self.p, self.q = int(p), int(q)
        dev = torch.device(device)
        items = (BatchItem * self.batch)()
        a = u = v = sk = 0
        self.a_off, self.u_off, self.v_off, self.s_off = [], [], [], []
        for i, (m, n, k) in enumerate(zip(self.ms, self.ns, self.ks)):
            items[i].m, items[i].n, items[i].k = m, n, k
            items[i].a_off, items[i].u_off, items[i].v_off, items[i].s_off = a, u, v, sk
            self.a_off.append(a)
            self.u_off.append(u)
            self.v_off.append(v)
            self.s_off.append(sk)
            a += m * n
            u += m * k
            v += n * k
            sk += k
        self.items = items
        self.a_elems = a
        self.U = torch.empty(max(u, 1), dtype=torch.float32, device=dev)
        self.V = torch.empty(max(v, 1), dtype=torch.float32, device=dev)
        self.S = torch.empty(max(sk, 1), dtype=torch.float64, device=dev)
        ws = lib().rsvd_svd_batched_workspace_size(self.batch, items, self.p, self.q)
        if ws == 0:
            raise RsvdError(1, "rsvd_svd_batched_workspace_size")
        self.work = _work(ws, dev)
        self.info = _info(dev)

    def pack(self, mats):
        """One packed float32 buffer holding the matrices at their offsets."""
        torch = _torch()
        return torch.cat([m.reshape(-1).to(torch.float32) for m in mats])

    def run(self, A_packed, seed):
        torch = _torch()
        if (not A_packed.is_cuda or A_packed.dtype != torch.float32 or A_packed.dim() != 1 or
                A_packed.numel() < self.a_elems):
            raise ValueError("A_packed: a 1-D float32 CUDA tensor of the packed matrices")
        st = lib().rsvd_svd_batched(self.batch, self.items, self.p, self.q, seed, _ptr(A_packed),
                                    _ptr(self.U), _ptr(self.S), _ptr(self.V), _ptr(self.work),
                                    self.work.numel(), _ptr(self.info), _stream())
        _raise(st, "rsvd_svd_batched")

    def result(self, i):
        m, n, k = self.ms[i], self.ns[i], self.ks[i]
        U = self.U[self.u_off[i]:self.u_off[i] + m * k].view(m, k)
        V = self.V[self.v_off[i]:self.v_off[i] + n * k].view(n, k)
        S = self.S[self.s_off[i]:self.s_off[i] + k]
        return U, S, V


TUNE_KINDS = {0: "pass over A", 1: "Gram slice", 2: "apply R^-1", 3: "lift", 4: "sketch"}


def batched_tuning():
    """The batched path's tile autotuner choices so far (rsvd_batched_tuning):
    one dict per GEMM class with the kind, the width N, the chosen block height
    and the measured ms of heights 64, 128, 256 (None where not valid)."""
    n = lib().rsvd_batched_tuning(0, None, None, None, None)
    if n <= 0:
        return []
    kind = (_c_int * n)()
    width = (_c_int * n)()
    rows = (_c_int * n)()
    ms = (ctypes.c_float * (3 * n))()
    lib().rsvd_batched_tuning(n, kind, width, rows, ms)
    return [{"kind": TUNE_KINDS.get(kind[i], kind[i]), "width": width[i], "rows": rows[i],
             "ms": [ms[3 * i + h] if ms[3 * i + h] >= 0 else None for h in range(3)]}
            for i in range(n)]


def svd_batched(mats, ks, p, q, seed, check=True):
    """[(U_i, S_i, V_i)]: the RSVD of every float32 CUDA matrix in `mats`
    (ranks ks, common p and q) in one batched call (rsvd_svd_batched)."""
    for t in mats:
        _check_matrix(t, "A_i")
    plan = BatchPlan([t.shape[0] for t in mats], [t.shape[1] for t in mats], ks, p, q,
                     mats[0].device)
    Ap = plan.pack(mats)
    plan.run(Ap, seed)
    if check:
        check_info(plan.info, "rsvd_svd_batched")
    return [plan.result(i) for i in range(plan.batch)]
