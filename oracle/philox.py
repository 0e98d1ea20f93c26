"""Philox4x32-10 counter stream and the Gaussian test matrix Omega (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper draws Omega as a GIID matrix with Matlab's ``randn`` (Fig. 1 step 1,
Sec. 2.1 "GIID matrix", Alg. 5 first step) and fixes no generator.  The reading
taken here, identical on the CUDA side and written independently there, is:

* Philox4x32 with 10 rounds (Salmon, Moraes, Dror & Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC'11).  One round maps the counter
  (c0, c1, c2, c3) with key (k0, k1) to
      (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
  with multipliers M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is
  bumped by the Weyl constants (0x9E3779B9, 0xBB67AE85).
* Key = (seed mod 2^32, seed div 2^32).
* Omega[i, j] (i < n rows, j < l columns) takes its four words from the counter
  (i, j // 4, tag, batch); tag 0 is the range-finder Omega.
* Uniform from a word x: u = (2*(x >> 9) + 1) * 2^-24, which lies in (0, 1) and
  is exact in both fp32 and fp64.
* Box-Muller (Box & Muller 1958): words (x0, x1) give columns 4*(j//4)+0/1 as
  r*cos(2*pi*u1), r*sin(2*pi*u1) with r = sqrt(-2 ln u0); words (x2, x3) give
  columns +2/+3 the same way.
* Rounding of Omega follows the arithmetic that consumes it: FP64 inputs use the
  FP64 value; FP32 inputs use the value rounded to fp32 and then to bf16
  (round to nearest even), because the tensor-core path multiplies bf16-exact
  Omega entries.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

TAG_OMEGA = 0
TAG_OMEGA_LEFT = 1      # the left test matrix Omega~ of the sketch Omega~ A (Sec. 3.5)


def philox4x32_10(ctr, key):
    """Apply Philox4x32-10 to an (N, 4) uint32 counter array with key (k0, k1).

    Returns an (N, 4) uint32 array of output words.
    """
    c = [np.asarray(ctr[:, t], dtype=np.uint64) for t in range(4)]
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c[0]                       # < 2^64, exact in uint64
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack([x.astype(np.uint32) for x in c], axis=1)


def seed_key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & 0xFFFFFFFF, seed >> 32)


def omega_words(n, l, seed, tag=TAG_OMEGA, batch=0):
    """uint32 words for Omega: array (n, ceil(l/4), 4); [i, q, t] feeds column 4q+t."""
    nq = (l + 3) // 4
    i = np.repeat(np.arange(n, dtype=np.uint64), nq)
    q = np.tile(np.arange(nq, dtype=np.uint64), n)
    ctr = np.stack([i, q, np.full_like(i, tag), np.full_like(i, batch)], axis=1)
    w = philox4x32_10(ctr.astype(np.uint32), seed_key(seed))
    return w.reshape(n, nq, 4)


def uniform_from_word(x):
    """u = (2*(x >> 9) + 1) * 2^-24, in (0, 1), exact in fp32 and fp64."""
    x = np.asarray(x, dtype=np.uint32)
    return (2.0 * (x >> np.uint32(9)).astype(np.float64) + 1.0) * 2.0 ** -24


def round_f32_to_bf16(x32):
    """Round fp32 values to bf16 (nearest, ties to even); returned as float64."""
    b = np.asarray(x32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))
    r = ((b + bias) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def omega(n, l, seed, rounding="f64", tag=TAG_OMEGA, batch=0):
    """The n x l Gaussian test matrix Omega in float64 holding the rounded values.

    rounding: "f64" (no rounding), "f32" (fp32) or "bf16" (fp32 then bf16).
    """
    w = omega_words(n, l, seed, tag, batch)
    u = uniform_from_word(w)                       # (n, nq, 4)
    r01 = np.sqrt(-2.0 * np.log(u[:, :, 0]))
    r23 = np.sqrt(-2.0 * np.log(u[:, :, 2]))
    t01 = 2.0 * np.pi * u[:, :, 1]
    t23 = 2.0 * np.pi * u[:, :, 3]
    z = np.stack([r01 * np.cos(t01), r01 * np.sin(t01),
                  r23 * np.cos(t23), r23 * np.sin(t23)], axis=2)
    z = z.reshape(n, -1)[:, :l]
    if rounding == "f64":
        return np.ascontiguousarray(z)
    z32 = z.astype(np.float32)
    if rounding == "f32":
        return z32.astype(np.float64)
    if rounding == "bf16":
        return round_f32_to_bf16(z32)
    raise ValueError(rounding)


def omega_rounding_for(dtype):
    """Rounding of Omega used for an input matrix of the given numpy dtype name."""
    name = np.dtype(dtype).name if not isinstance(dtype, str) else dtype
    if name in ("float64", "f64"):
        return "f64"
    if name in ("float32", "f32", "bfloat16", "bf16"):
        return "bf16"
    raise ValueError(dtype)
