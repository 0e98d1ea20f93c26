"""Pins of the oracle's E4M3 quantiser and FP8 sketch (oracle/quant.py) to the
format's published facts and to torch's float8_e4m3fn cast (a library routine
that rounds to nearest even within range; it gives NaN beyond 448, where the
satfinite conversion saturates):

* 127 non-negative finite values, largest 448, smallest subnormal 2^-9,
  smallest normal 2^-6, codes in increasing order;
* rounding identical to torch's cast on random values, on every midpoint
  between neighbouring values (ties to the even code) and on subnormals;
* relative error at most 2^-4 in the normal range, absolute error at most
  2^-10 below it;
* block scales are powers of two that keep every scaled entry within 448 and
  use at least half of the range;
* the FP8 sketch errs by no more than the elementwise bound of its two
  quantisations.
"""
import numpy as np
import pytest

from oracle import quant

torch = pytest.importorskip("torch")


def _torch_e4m3(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.float8_e4m3fn).double().numpy()


def test_format_facts():
    v = quant.e4m3_values()
    assert v.size == 127 and v[0] == 0.0
    assert v[-1] == 448.0 and v[1] == 2.0 ** -9 and v[8] == 2.0 ** -6
    assert np.all(np.diff(v) > 0)
    # every value is its own rounding, and torch's cast agrees
    assert np.array_equal(quant.round_e4m3(v), v)
    assert np.array_equal(_torch_e4m3(v), v)


def test_rounding_matches_torch_cast():
    rng = np.random.default_rng(1)
    v = quant.e4m3_values()
    mids = (v[:-1] + v[1:]) / 2                                # exact in fp32
    x = np.concatenate([rng.standard_normal(20000) * 30, rng.uniform(0, 2 ** -5, 5000),
                        mids, -mids, rng.uniform(-448, 448, 5000)]).astype(np.float32)
    assert np.array_equal(quant.round_e4m3(x.astype(np.float64)), _torch_e4m3(x))


def test_saturation_and_error_bounds():
    assert quant.round_e4m3(np.array([449.0, 1e6, -500.0])).tolist() == [448.0, 448.0, -448.0]
    rng = np.random.default_rng(2)
    x = np.exp(rng.uniform(np.log(2 ** -6), np.log(448), 50000)) * rng.choice([-1, 1], 50000)
    assert np.all(np.abs(quant.round_e4m3(x) - x) <= 2.0 ** -4 * np.abs(x))
    s = rng.uniform(-2 ** -6, 2 ** -6, 50000)
    assert np.all(np.abs(quant.round_e4m3(s) - s) <= 2.0 ** -10)


def test_block_scales():
    rng = np.random.default_rng(3)
    M = rng.standard_normal((40, 100)) * np.exp(rng.uniform(-20, 20, (40, 1)))
    M[3, :] = 0.0
    S = quant.block_scales(M, 1)
    e = np.log2(S)
    assert np.array_equal(e, np.round(e))                      # powers of two
    for k0 in range(0, 100, 32):
        blk, sc = M[:, k0:k0 + 32], S[:, k0:k0 + 32]
        assert np.all(sc == sc[:, :1])                         # one scale per block
        amax = np.max(np.abs(blk / sc), axis=1)
        assert np.all(amax <= 448.0)
        nz = np.max(np.abs(blk), axis=1) > 0
        assert np.all(amax[nz] > 224.0)
    assert np.all(S[3] == 1.0)


def test_fp8_sketch_error_bound():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((64, 300)) * np.logspace(0, -3, 300)[None, :]
    Om = rng.standard_normal((300, 24))
    Y = quant.sketch_fp8(A, Om)
    qa, sa = quant.quantize(A, 1)
    qo, so = quant.quantize(Om, 0)
    dA = np.abs(qa * sa - A)
    dO = np.abs(qo * so - Om)
    # |A^ O^ - A O| <= |dA| |O^| + |A| |dO|, entrywise
    bound = dA @ np.abs(qo * so) + np.abs(A) @ dO
    assert np.all(np.abs(Y - A @ Om) <= bound * (1 + 1e-12) + 1e-15)
    # and each quantisation is within its format bound
    assert np.all(dA <= 2.0 ** -4 * np.abs(A) + sa * 2.0 ** -10)
    assert np.all(dO <= 2.0 ** -4 * np.abs(Om) + so * 2.0 ** -10)
