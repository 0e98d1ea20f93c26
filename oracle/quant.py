"""FP8 (E4M3) quantisation with block scales for the FP8 sketch (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper fixes no reduced precision for the sketch; it only notes (Sec. 3.2,
Sec. 3.5) that the power scheme without re-orthonormalisation is limited by
the machine precision.  The FP8 sketch is therefore a reading: Y = A Omega
with both operands in FP8 E4M3 and one power-of-two scale per block of 32
consecutive entries along the contraction (the form Blackwell's block-scaled
tensor-core products take).  This module holds the plain definitions:

* the E4M3 format (the "FN" variant of the OCP 8-bit floating-point
  specification): 1 sign bit, 4 exponent bits with bias 7, 3 mantissa bits; no
  infinities; the all-ones code is NaN; largest finite value 448 = 1.75 * 2^8;
  subnormals m * 2^-9, m = 1..7;
* round to nearest, ties to the even code, saturating to +-448 (the
  "satfinite" conversion);
* block scales X = 2^ceil(log2(amax / 448)) (1 for an all-zero block), so that
  no scaled entry exceeds 448;
* the sketch of the dequantised operands, in FP64.
"""
import numpy as np

E4M3_MAX = 448.0
BLOCK = 32


def e4m3_values():
    """The 127 non-negative finite E4M3 values in code order (code = index)."""
    vals = [m * 2.0 ** -9 for m in range(8)]                      # exponent field 0
    for e in range(1, 16):
        for m in range(8):
            if e == 15 and m == 7:                                # NaN code
                continue
            vals.append((1.0 + m / 8.0) * 2.0 ** (e - 7))
    return np.array(vals)


_GRID = e4m3_values()


def round_e4m3(x):
    """x rounded to E4M3: nearest value, ties to the even code, |x| > 448 -> 448."""
    x = np.asarray(x, dtype=np.float64)
    a = np.minimum(np.abs(x), E4M3_MAX)
    hi = np.searchsorted(_GRID, a, side="left")                   # first grid value >= a
    hi = np.minimum(hi, _GRID.size - 1)
    lo = np.maximum(hi - 1, 0)
    exact = _GRID[hi] == a
    dlo = a - _GRID[lo]
    dhi = _GRID[hi] - a
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (hi % 2 == 0))
    code = np.where(exact, hi, np.where(pick_hi, hi, lo))
    return np.sign(x) * _GRID[code]


def block_scales(M, axis):
    """Power-of-two scale of every block of BLOCK entries of M along `axis`
    (the contraction axis); the last block may be short.  Returns the scales
    broadcast back to M's shape."""
    M = np.asarray(M, dtype=np.float64)
    Mt = np.moveaxis(M, axis, -1)
    K = Mt.shape[-1]
    S = np.empty_like(Mt)
    for k0 in range(0, K, BLOCK):
        amax = np.max(np.abs(Mt[..., k0:k0 + BLOCK]), axis=-1, keepdims=True)
        with np.errstate(divide="ignore"):
            e = np.ceil(np.log2(amax / E4M3_MAX))
        S[..., k0:k0 + BLOCK] = np.where(amax > 0, 2.0 ** e, 1.0)
    return np.moveaxis(S, -1, axis)


def quantize(M, axis):
    """(codes as E4M3 values, scales): M ~ values * scales, blocks along `axis`."""
    S = block_scales(M, axis)
    return round_e4m3(np.asarray(M, dtype=np.float64) / S), S


def sketch_fp8(A, Omega):
    """Y = deq(q(A)) deq(q(Omega)) in FP64: A (m x n) with blocks along its rows'
    contraction index (axis 1), Omega (n x l) with blocks along axis 0."""
    qa, sa = quantize(A, 1)
    qo, so = quantize(Omega, 0)
    return (qa * sa) @ (qo * so)
