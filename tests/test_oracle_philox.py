"""Pins for the oracle's Philox stream and Gaussian Omega (CPU only).

What pins it: the round structure is checked by inverting ten rounds back to
the counter (each round is a bijection by the SC'11 construction); the words by
bit balance and a chi-square test; the Gaussians by their moments, a
Kolmogorov-Smirnov test, and the column-norm lemma of Sec. 3.1
(E ||Omega~ a||^2 / ||a||^2 = l, Var = 2l).  bf16 rounding is checked against
torch's own float -> bfloat16 conversion (a different implementation).
"""
import numpy as np
import pytest
import scipy.stats as st

from oracle import philox

MOD = 1 << 32


def _inv_round(y, k0, k1):
    """Invert one Philox4x32 round with plain Python integers."""
    y0, y1, y2, y3 = (int(v) for v in y)
    m0inv = pow(0xD2511F53, -1, MOD)
    m1inv = pow(0xCD9E8D57, -1, MOD)
    c0 = (y3 * m0inv) % MOD
    c2 = (y1 * m1inv) % MOD
    hi0 = (0xD2511F53 * c0) >> 32
    hi1 = (0xCD9E8D57 * c2) >> 32
    c1 = y0 ^ hi1 ^ k0
    c3 = y2 ^ hi0 ^ k1
    return (c0, c1, c2, c3)


def test_rounds_invert_to_counter():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, MOD, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    key = (0x12345678, 0x9ABCDEF0)
    out = philox.philox4x32_10(ctr, key)
    keys = []
    k0, k1 = key
    for r in range(10):
        if r:
            k0 = (k0 + 0x9E3779B9) % MOD
            k1 = (k1 + 0xBB67AE85) % MOD
        keys.append((k0, k1))
    for row in range(ctr.shape[0]):
        y = tuple(int(v) for v in out[row])
        for kk in reversed(keys):
            y = _inv_round(y, *kk)
        assert y == tuple(int(v) for v in ctr[row])


def test_words_depend_on_every_counter_word_and_key():
    base = np.zeros((1, 4), dtype=np.uint32)
    ref = philox.philox4x32_10(base, (7, 9))
    for t in range(4):
        c = base.copy()
        c[0, t] = 1
        assert not np.array_equal(philox.philox4x32_10(c, (7, 9)), ref)
    assert not np.array_equal(philox.philox4x32_10(base, (8, 9)), ref)
    assert not np.array_equal(philox.philox4x32_10(base, (7, 10)), ref)


def test_word_bits_balanced_and_uniform():
    w = philox.omega_words(4096, 64, seed=0x5EED).reshape(-1)      # 262144 words
    n = w.size
    for b in range(32):
        frac = np.mean((w >> np.uint32(b)) & np.uint32(1))
        assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(n)
    counts = np.bincount((w >> np.uint32(24)).astype(np.int64), minlength=256)
    chi2 = np.sum((counts - n / 256) ** 2 / (n / 256))
    assert st.chi2.sf(chi2, 255) > 1e-4


def test_uniforms_exact_and_open_interval():
    x = np.array([0, 1, 511, 512, 0xFFFFFFFF, 0x80000000], dtype=np.uint32)
    u = philox.uniform_from_word(x)
    assert u.min() > 0 and u.max() < 1
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    assert u[0] == 2.0 ** -24 and u[4] == 1 - 2.0 ** -24
    assert u[2] == u[0] and u[3] == 3 * 2.0 ** -24


def test_gaussian_moments_and_ks():
    z = philox.omega(20000, 200, seed=123).reshape(-1)              # 4e6 draws
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1) < 5 * np.sqrt(2 / n)
    assert abs(np.mean(z ** 4) - 3) < 5 * np.sqrt(96 / n)
    assert st.kstest(z[:200000], "norm").pvalue > 1e-4


def test_columns_and_rows_uncorrelated():
    z = philox.omega(50000, 8, seed=5)
    C = np.corrcoef(z.T)
    off = C[~np.eye(8, dtype=bool)]
    assert np.max(np.abs(off)) < 5 / np.sqrt(50000)


def test_column_norm_lemma():
    """Sec. 3.1: for fixed a, ||Omega~ a||^2 / ||a||^2 ~ chi^2_l (E = l, Var = 2l)."""
    l, m, trials = 8, 64, 3000
    a = np.linspace(-1.0, 2.0, m)
    vals = np.empty(trials)
    for t in range(trials):
        Om = philox.omega(m, l, seed=1000 + t)       # Omega~ = Om^T is l x m
        y = Om.T @ a
        vals[t] = y @ y / (a @ a)
    assert abs(vals.mean() - l) < 5 * np.sqrt(2 * l / trials)
    assert abs(vals.var() / (2 * l) - 1) < 0.15
    assert st.kstest(vals, st.chi2(l).cdf).pvalue > 1e-4


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    x = rng.standard_normal(100000).astype(np.float32)
    ties = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8)], dtype=np.float32)
    x = np.concatenate([x, ties])
    ours = philox.round_f32_to_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)
    assert ours[-3] == 1.0 and ours[-2] == 1 + 4 * 2 ** -8


def test_omega_layout_and_rounding_modes():
    n, l = 9, 11
    z = philox.omega(n, l, seed=77)
    w = philox.omega_words(n, l, seed=77)
    u = philox.uniform_from_word(w)
    i, j = 4, 6                                    # j = 4*1 + 2 -> words x2, x3
    r = np.sqrt(-2 * np.log(u[i, 1, 2]))
    assert z[i, j] == pytest.approx(r * np.cos(2 * np.pi * u[i, 1, 3]), rel=1e-15)
    assert z[i, j + 1] == pytest.approx(r * np.sin(2 * np.pi * u[i, 1, 3]), rel=1e-15)
    zb = philox.omega(n, l, seed=77, rounding="bf16")
    bits = zb.astype(np.float32).view(np.uint32)
    assert np.all(bits & np.uint32(0xFFFF) == 0)
    assert np.max(np.abs(zb - z) / np.abs(z)) <= 2.0 ** -8
    # a different tag or batch gives an independent stream
    assert not np.allclose(philox.omega(n, l, 77, tag=1), z)
    assert not np.allclose(philox.omega(n, l, 77, batch=1), z)
