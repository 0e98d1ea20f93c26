"""Writes c3_reduced_oracle.txt: the FP64 oracle's RSVD (Alg. 5) on a reduced
matrix of the mixed-precision workload's recipe.

The workload is m = 100000, n = 50000, k = 500, p = 50, q = 2 with
sigma_j = exp(-j/100) + 1e-3 (r = 2000) and 1e-4 Gaussian noise, A stored as
bf16.  The oracle cannot run at that size within a test, so the file holds its
results at m = 10000, n = 5000 with the same k, p, q, spectrum, noise and
seeds: the k singular values and the relative error ||A - U S V^T||_F / ||A||_F
(against the FP32 A), once on the FP32 matrix and once on its bf16 rounding.
The matrix comes from synth.make_matrix_np (seeded numpy); the Omega stream is
the library's Philox stream with bf16-rounded Gaussians.

Run from the repository root:  python tests/golden/make_c3_reduced.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import rsvd as orc          # noqa: E402
from synth import config, make_matrix_np, spectrum   # noqa: E402

M, N = 10000, 5000
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_reduced_oracle.txt")


def reduced_inputs():
    """(cfg, A32, Ab): the reduced matrix in FP32 and its bf16 rounding (as fp32)."""
    cfg = config("c3_bf16_100000x50000")
    sig = spectrum(cfg["spectrum"], cfg["r"])
    A32 = make_matrix_np(M, N, sig, noise=cfg["noise"], seed=cfg["a_seed"], dtype="float32")
    Ab = make_matrix_np(M, N, sig, noise=cfg["noise"], seed=cfg["a_seed"], dtype="bfloat16")
    return cfg, A32, Ab


def main():
    cfg, A32, Ab = reduced_inputs()
    k, p, q, seed = cfg["k"], cfg["p"], cfg["q"], cfg["omega_seed"]
    A64 = A32.astype(np.float64)
    rows = []
    for name, X in (("f32", A64), ("bf16", Ab.astype(np.float64))):
        U, S, V, _ = orc.rsvd(X, k, p, q, seed, rounding="bf16")
        e = orc.rel_err_svd(A64, U, S, V)
        rows.append((name, e, S))
        print(name, "rel_err", e, "sigma_1", S[0], "sigma_k", S[-1])
    with open(OUT, "w") as f:
        f.write("# FP64 oracle RSVD (Alg. 5) of the mixed-precision workload's recipe at reduced size\n")
        f.write("# written by tests/golden/make_c3_reduced.py (calls oracle.rsvd only)\n")
        f.write("# m %d n %d k %d p %d q %d a_seed %d omega_seed %d spectrum %s r %d noise %g\n"
                % (M, N, k, p, q, cfg["a_seed"], seed, cfg["spectrum"], cfg["r"], cfg["noise"]))
        f.write("# rel_err_<A>: ||A32 - U S V^T||_F / ||A32||_F of the oracle run on <A>\n")
        f.write("# sigma_<A>: the oracle's k singular values on <A> (f32: the FP32 matrix; "
                "bf16: its bf16 rounding)\n")
        for name, e, S in rows:
            f.write("rel_err_%s %.17g\n" % (name, e))
        for name, e, S in rows:
            f.write("sigma_%s %s\n" % (name, " ".join("%.17g" % s for s in S)))


def load(path=OUT):
    """{'rel_err_f32': float, ..., 'sigma_f32': ndarray, ...} from the file."""
    out = {}
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            v = np.array([float(x) for x in vals])
            out[key] = v if key.startswith("sigma_") else float(v[0])
    return out


if __name__ == "__main__":
    main()
