"""The FP8 sketch (RSVD_PREC_FP8) against the oracle's E4M3 quantiser.

The oracle (oracle/quant.py, pinned to the format's facts and to torch's
float8_e4m3fn cast) defines Y = deq(q(A)) deq(q(Omega)) with one power-of-two
scale per block of 32 entries along the contraction.  The GPU quantises A in
the tensor-core GEMM's converters and Omega (its bf16 Gaussians, as on the
FP32 path) once per call; the products of the dequantised values are exact in
bf16, so the GPU's Y differs from the oracle's by the fp32 accumulation only.

The kernels' fp32 Box-Muller differs from the FP64 oracle by a few fp32 ulps,
which flips the bf16 rounding of a few Omega entries in ten thousand (bounded
in test_gpu_steps); about one flip in sixteen also moves the entry's E4M3
value by one step.  The checks below compare exactly wherever the bf16
Gaussians of a block agree with the oracle's, and bound the rest by one
E4M3 step of one term.
"""
import numpy as np
import pytest

from oracle import philox, quant
from synth import make_matrix_np, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"


def _fp8_opts():
    return rs.make_opts(precision=rs.PREC_FP8)


@pytest.mark.parametrize("n,l,seed", [(2000, 60, 0xF8), (1000, 13, 7), (4099, 220, 0x5EED)])
def test_omega_fp8_quantised_like_the_oracle(n, l, seed):
    g = rs.omega_fp8(n, l, seed, DEV).double().cpu().numpy()
    gb = rs.omega(n, l, seed, torch.float32, DEV).double().cpu().numpy()
    ob = philox.omega(n, l, seed, "bf16")
    qo, so = quant.quantize(ob, 0)
    ref = qo * so
    # blocks of 32 rows of a column whose bf16 Gaussians all agree: identical
    nb = (n + 31) // 32
    same = np.ones((nb, l), dtype=bool)
    for b in range(nb):
        same[b] = np.all(gb[32 * b:32 * b + 32] == ob[32 * b:32 * b + 32], axis=0)
    assert same.mean() > 0.97
    rows_same = np.repeat(same, 32, axis=0)[:n]
    assert np.array_equal(g[rows_same], ref[rows_same])
    # the others: within one E4M3 step (2^-3 of the entry, or the subnormal step)
    d = np.abs(g - ref)[~rows_same]
    assert np.all(d <= 2.0 ** -3 * np.abs(ref[~rows_same]) + 2.0 ** -9 * so[~rows_same])


# the second case: n = 4099 (a ragged last K-chunk and quantisation block) as a
# view of rows at a 4100-float pitch (the tensor-core path's 16-byte rows)
@pytest.mark.parametrize("m,n,l,dtype", [(3000, 2000, 64, torch.float32), (1500, 4099, 220, torch.float32),
                                         (2048, 1000, 40, torch.bfloat16)])
def test_fp8_sketch_matches_oracle(m, n, l, dtype):
    seed = 0x5EED + l
    A = make_matrix_np(m, n, spectrum("logspace3", min(m, n)), noise=1e-4, seed=n + l,
                       dtype="float32")
    if dtype == torch.bfloat16:
        A = torch.from_numpy(A).to(torch.bfloat16).float().numpy()   # the stored values
    pitch = (n + 3) // 4 * 4 if dtype == torch.float32 else (n + 7) // 8 * 8
    buf = torch.zeros(m, pitch, dtype=dtype, device=DEV)
    buf[:, :n] = torch.from_numpy(A).to(DEV, dtype)
    At = buf[:, :n]
    Y = rs.sample(At, l, seed, opts=_fp8_opts()).double().cpu().numpy()
    A64 = A.astype(np.float64)
    ob = philox.omega(n, l, seed, "bf16")
    ref = quant.sketch_fp8(A64, ob)
    qa, sa = quant.quantize(A64, 1)
    qo, so = quant.quantize(ob, 0)
    S = np.abs(qa * sa) @ np.abs(qo * so)                 # sum of |term| per entry
    # columns whose quantised Omega equals the oracle's everywhere: fp32 sums only
    g = rs.omega_fp8(n, l, seed, DEV).double().cpu().numpy()
    exact_cols = np.all(g == qo * so, axis=0)
    assert exact_cols.mean() > 0.8
    d = np.abs(Y - ref)
    assert np.all(d[:, exact_cols] <= 2e-5 * S[:, exact_cols])
    if (~exact_cols).any():
        # one term moved by one E4M3 step: at most 2^-3 of the largest term of the row
        tmax = np.max(np.abs(qa * sa), axis=1, keepdims=True) * np.max(np.abs(qo * so), axis=0, keepdims=True)
        loose = 2e-5 * S + 2.0 ** -3 * tmax * np.sum(g != qo * so, axis=0, keepdims=True)
        assert np.all(d[:, ~exact_cols] <= loose[:, ~exact_cols])


def test_fp8_sketch_rsvd_against_fp32():
    """The RSVD with the FP8 sketch against the FP32 path on the same input, both
    judged by their distance to the exact SVD: an FP8-quantised sketch is
    another random sketch of the same range, so the singular values it finds
    are as close to the true ones as the FP32 path's and the reconstruction
    error is the same to within 1 %% (the bar of the mixed-precision forms:
    equal relative error).  Spectrum sigma_j = 1/j: its gap after k makes the
    power steps contract the sketch's error."""
    m, n, k, p, q, seed = 3000, 2000, 40, 10, 2, 0xF8F8
    A = make_matrix_np(m, n, spectrum("inv", n), noise=1e-5, seed=11, dtype="float32")
    At = torch.from_numpy(A).to(DEV)
    U8, S8, V8 = rs.svd(At, k, p, q, seed, opts=_fp8_opts())
    U, S, V = rs.svd(At, k, p, q, seed)
    S8, S = S8.cpu().numpy(), S.cpu().numpy()
    st = np.linalg.svd(A.astype(np.float64), compute_uv=False)[:k]
    err8 = np.max(np.abs(S8 - st) / st)
    err = np.max(np.abs(S - st) / st)
    assert err8 <= 2 * err + 1e-5, (err8, err)
    from oracle import rsvd as orc
    e8 = orc.rel_err_svd(A.astype(np.float64), U8.double().cpu().numpy(), S8,
                         V8.double().cpu().numpy())
    e = orc.rel_err_svd(A.astype(np.float64), U.double().cpu().numpy(), S, V.double().cpu().numpy())
    assert e8 <= 1.01 * e, (e8, e)


def test_fp8_rejected_off_the_tensor_cores():
    A = torch.zeros(300, 200, dtype=torch.float64, device=DEV)
    with pytest.raises(rs.RsvdError):
        rs.sample(A, 16, 1, opts=_fp8_opts())
