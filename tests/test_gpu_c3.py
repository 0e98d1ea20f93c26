"""The mixed-precision workload's recipe (sigma_j = exp(-j/100) + 1e-3 on
r = 2000 directions, 1e-4 noise, k = 500, p = 50, q = 2, so l = 550: three
column chunks per pass, the 16-CTA Jacobi) at m = 10000, n = 5000 against the
FP64 oracle's results stored in tests/golden/c3_reduced_oracle.txt (written by
make_c3_reduced.py beside it from oracle.rsvd alone).

Bars:
* FP32 A and bf16 A (the oracle ran on the same bf16 values): every one of the
  k singular values within relative 1e-5 of the oracle's, and the relative
  error ||A - U S V^T||_F / ||A||_F (against the FP32 A) within 1 % of the
  oracle's;
* the single-term power scheme (RSVD_PREC_MIXED) and the FP8 sketch
  (RSVD_PREC_FP8) change the arithmetic of the sketch or the power passes, not
  only its rounding: their relative error within 1 % of the oracle's (the
  equal-error comparison) and sigma_i within relative 1e-3 above the noise
  edge 2 * 1e-4 (sqrt(m) + sqrt(n)).  Inside the noise bulk a Ritz value
  depends on the particular test matrix, and the quantised Omega is another
  test matrix (measured: 4.5e-3 at i = 430 with the FP8 sketch, 3.7e-6 at the
  top).
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))
import make_c3_reduced as golden   # noqa: E402


@pytest.fixture(scope="module")
def c3():
    cfg, A32, Ab = golden.reduced_inputs()
    return cfg, A32, Ab, golden.load()


def _rel_err(A64, U, S, V):
    R = A64 - (U * S[None, :]) @ V.T
    return np.linalg.norm(R) / np.linalg.norm(A64)


@pytest.mark.parametrize("form", ["f32", "bf16", "bf16_mixed", "f32_fp8", "bf16_fp8"])
def test_c3_recipe_against_oracle(c3, form):
    cfg, A32, Ab, gold = c3
    k, p, q, seed = cfg["k"], cfg["p"], cfg["q"], cfg["omega_seed"]
    storage = "bf16" if form.startswith("bf16") else "f32"
    prec = {"bf16_mixed": rs.PREC_MIXED, "f32_fp8": rs.PREC_FP8,
            "bf16_fp8": rs.PREC_FP8}.get(form, rs.PREC_TC)
    Ad = torch.from_numpy(Ab if storage == "bf16" else A32).to(DEV)
    if storage == "bf16":
        Ad = Ad.to(torch.bfloat16)          # exact: Ab holds bf16 values
    out = rs.svd_id_cur(Ad, k, p, q, seed, rs.make_opts(precision=prec))
    S = out["S"].cpu().numpy()
    U = out["U"].double().cpu().numpy()
    V = out["V"].double().cpu().numpy()
    So = gold["sigma_" + storage]
    rel = np.abs(S - So) / So
    e = _rel_err(A32.astype(np.float64), U, S, V)
    eo = gold["rel_err_" + storage]
    if form in ("f32", "bf16"):
        assert rel.max() <= 1e-5, (form, rel.max(), int(np.argmax(rel)))
    else:
        m, n = A32.shape
        edge = So > 2 * 1e-4 * (np.sqrt(m) + np.sqrt(n))
        assert edge.sum() >= 100
        assert rel[edge].max() <= 1e-3, (form, rel[edge].max(), int(np.argmax(rel[edge])))
    assert abs(e - eo) <= 0.01 * eo, (form, e, eo)
    J = out["J"].cpu().numpy()
    assert sorted(J.tolist()) == list(range(A32.shape[1]))
