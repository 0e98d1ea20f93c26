"""The stored oracle results for the reduced mixed-precision recipe
(tests/golden/c3_reduced_oracle.txt) against what the construction fixes.

A = U diag(sigma) V^T + E with orthonormal U, V, sigma_j = exp(-j/100) + 1e-3
and E of i.i.d. N(0, 1e-8) entries.  Weyl's inequality bounds every singular
value of A within ||E||_2 of sigma_j, and ||E||_2 <= 1e-4 (sqrt(m) + sqrt(n))
up to a small-deviation factor (Gordon's bound on the expected norm; 1.1 leaves
room for the fluctuation, which is O(1e-4) absolute).  The randomized estimates
never exceed the true values (sigma_i(Q^T A) <= sigma_i(A)), and with q = 2 and
l = 550 the top 100 are resolved far below that band.
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_c3_reduced as golden   # noqa: E402


def test_c3_golden_against_construction():
    g = golden.load()
    m, n, k = golden.M, golden.N, 500
    enorm = 1.1 * 1e-4 * (np.sqrt(m) + np.sqrt(n))
    j = np.arange(1, k + 1, dtype=np.float64)
    sig = np.exp(-j / 100.0) + 1e-3
    for name in ("f32", "bf16"):
        S = g["sigma_" + name]
        assert S.shape == (k,)
        assert np.all(np.diff(S) <= 0) and S[-1] > 0
        assert np.all(S <= sig + enorm + 1e-3 * 2 ** -8), name   # + bf16 rounding of A
        assert np.all(np.abs(S[:100] - sig[:100]) <= enorm), name
        # the relative error is at least the optimal rank-k tail of A's spectrum
        # (sigma_j beyond k plus the noise's mass), and the tail of the
        # construction alone already sets its scale
        tail = np.sqrt(np.sum((np.exp(-np.arange(k + 1, 2001) / 100.0) + 1e-3) ** 2))
        total = np.sqrt(np.sum((np.exp(-np.arange(1, 2001) / 100.0) + 1e-3) ** 2)
                        + 1e-8 * m * n)
        assert g["rel_err_" + name] >= 0.9 * tail / total
        assert g["rel_err_" + name] <= 1.1 * np.sqrt(tail ** 2 + 1e-8 * m * n) / total
    # the bf16 rounding of A moves sigma_1 by about 2^-9 ||A||_F / sqrt(mn) at most
    assert abs(g["sigma_f32"][0] - g["sigma_bf16"][0]) <= 1e-4
