"""GPU parity of the batched RSVD (rsvd_svd_batched) against the oracle, problem by problem.

Each problem's Omega is the Philox stream of the call's seed with the problem
index as the counter's batch word; the oracle draws the same Omega and runs
Alg. 5 on the problem's fp32 values in FP64.  The batched products are plain
fp32, the bars those of the FP32 path: sigma relative 1e-5, reconstruction
error within 1 % of the oracle's, orthonormal U and V, the sign rule.
"""
import numpy as np
import pytest

from oracle import philox, rsvd as orc
from synth import make_matrix_np, spectrum

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
rs = pytest.importorskip("paper_1502_05366_gb300")
DEV = "cuda:0"

# (m, n, k): the workload's ranges, ragged sizes, k = 64 (l = 72) and tiny cases
SIZES = [(300, 150, 8), (1000, 700, 16), (257, 129, 32), (2048, 1024, 64), (513, 200, 64),
         (96, 80, 8), (4096, 2048, 32), (1500, 1499, 16), (72, 72, 64), (4000, 130, 8)]


def test_svd_batched_parity():
    p, q, seed = 8, 1, 0xBA7C
    mats, mats64 = [], []
    for i, (m, n, k) in enumerate(SIZES):
        r = min(n, 6 * k)
        A = make_matrix_np(m, n, spectrum("expk", r, k), seed=0xD000 + i, dtype="float32")
        mats.append(torch.from_numpy(A).to(DEV))
        mats64.append(A.astype(np.float64))
    out = rs.svd_batched(mats, [s[2] for s in SIZES], p, q, seed)
    for i, ((m, n, k), (U, S, V)) in enumerate(zip(SIZES, out)):
        l = k + p
        Om = philox.omega(n, l, seed, "bf16", batch=i)
        Uo, So, Vo, _ = orc.rsvd(mats64[i], k, p, q, seed, rounding="bf16", Omega=Om)
        S = S.cpu().numpy()
        U = U.double().cpu().numpy()
        V = V.double().cpu().numpy()
        rel = np.abs(S - So) / So
        assert rel.max() <= 1e-5, (i, rel.max(), np.argmax(rel))
        e = orc.rel_err_svd(mats64[i], U, S, V)
        eo = orc.rel_err_svd(mats64[i], Uo, So, Vo)
        assert abs(e - eo) <= 0.01 * eo + 1e-7, (i, e, eo)
        assert np.linalg.norm(U.T @ U - np.eye(k)) <= 5e-5, i
        assert np.linalg.norm(V.T @ V - np.eye(k)) <= 5e-5, i
        idx = np.argmax(np.abs(V), axis=0)
        assert np.all(V[idx, np.arange(k)] > 0), i
        gap = np.minimum(np.abs(np.diff(np.r_[np.inf, So])), np.abs(np.diff(np.r_[So, 0.0])))
        well = gap / So > 1e-2
        assert np.all(np.abs(np.sum(U * Uo, axis=0))[well] > 1 - 1e-4), i


def test_svd_batched_one_problem_matches_batch_slot():
    """A problem's result does not depend on the other problems of the batch."""
    p, q, seed = 8, 1, 77
    sizes = [(600, 300, 16), (800, 400, 32), (300, 300, 8)]
    mats = [torch.from_numpy(make_matrix_np(m, n, spectrum("expk", min(n, 6 * k), k),
                                            seed=40 + i, dtype="float32")).to(DEV)
            for i, (m, n, k) in enumerate(sizes)]
    full = rs.svd_batched(mats, [s[2] for s in sizes], p, q, seed)
    # the same problem in slot 0 of a batch of one gives problem 0's result
    one = rs.svd_batched(mats[:1], [sizes[0][2]], p, q, seed)
    for a, b in zip(full[0], one[0]):
        assert torch.equal(a, b)


def test_svd_batched_rejects_bad_items():
    A = torch.zeros(100, 50, device=DEV)
    with pytest.raises(rs.RsvdError):
        rs.svd_batched([A], [50], 8, 1, 1)          # l = 58 > n
    with pytest.raises(rs.RsvdError):
        rs.svd_batched([torch.zeros(300, 200, device=DEV)], [125], 8, 1, 1)   # l > 128


def test_batched_autotuner_choices_and_repeatability():
    """The tile autotuner keeps, per GEMM class, the fastest valid block height
    it measured; a later call with the tuned heights in place gives the same
    bits (every height computes each entry by the same multiply-adds)."""
    p, q, seed = 8, 1, 0x70E
    sizes = [(700, 300, 8), (900, 500, 16), (400, 300, 32), (1200, 640, 64)]
    mats = [torch.from_numpy(make_matrix_np(m, n, spectrum("expk", min(n, 6 * k), k),
                                            seed=90 + i, dtype="float32")).to(DEV)
            for i, (m, n, k) in enumerate(sizes)]
    first = rs.svd_batched(mats, [s[2] for s in sizes], p, q, seed)
    tune = rs.batched_tuning()
    assert tune, "no tuned class"
    for t in tune:
        assert t["rows"] in (64, 128, 256)
        valid = [(ms, 64 << h) for h, ms in enumerate(t["ms"]) if ms is not None]
        assert valid, t
        assert min(valid)[1] == t["rows"] or min(valid)[0] == t["ms"][t["rows"].bit_length() - 7], t
        # a block is 8192 / rows columns wide: only heights whose block covers N
        for h, ms in enumerate(t["ms"]):
            assert (ms is not None) == (t["width"] <= 8192 // (64 << h)), t
    second = rs.svd_batched(mats, [s[2] for s in sizes], p, q, seed)
    for a, b in zip(first, second):
        for x, y in zip(a, b):
            assert torch.equal(x, y)
