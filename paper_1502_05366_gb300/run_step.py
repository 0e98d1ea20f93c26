"""Run one step of the randomized-SVD path on seeded synthetic inputs.

Used to time or profile a single kernel at the sizes it sees inside the full
path without holding the full matrix A on the device:

  sample     Y = A Omega (Sec. 3.1, Omega generated in the kernel), A m x n
             (--dtype bfloat16 for A stored as bf16 in sample / apply_n / apply_t)
  apply_n    Y = A X,  X n x l stored                          (power step)
  apply_t    Z = A^T X, X m x l stored                         (power step / QB)
  orth       CholeskyQR of an m x l sample                     (re-orthonormalisation)
  small_svd  SVD of an l x l upper-triangular factor           (Alg. 5)
  cpqr       k-step column-pivoted QR + T = S11^-1 S12 of r x n (Sec. 4, ID);
             float32: the double-float kernel of the FP32 path, float64: FP64
  batched    one rsvd_svd_batched call on the 512-problem workload (uneven FP32
             problems, sigma_j = exp(-j/k)); --batch limits the problem count
  adaptive   one rsvd_qb_adaptive call (Alg. 7) on a Gaussian m x n A with
             eps = 0, so exactly --blocks blocks of --l columns with --q power
             iterations each; A is overwritten (the residual), not copied

Example:  python -m paper_1502_05366_gb300.run_step --step cpqr --r 220 --n 20000 --k 200

Prints one line per repetition with the step's device time (CUDA events on
the launching stream).
"""
import argparse
import sys

import torch

import paper_1502_05366_gb300 as rs


def _inputs(args, dev):
    g = torch.Generator(device="cpu").manual_seed(args.seed)
    dt = {"float32": torch.float32, "float64": torch.float64,
          "bfloat16": torch.bfloat16}[args.dtype]
    if args.step in ("sample", "apply_n", "apply_t"):
        A = torch.randn(args.m, args.n, generator=g, dtype=torch.float32).to(dev, dt)
        rows = args.n if args.step == "apply_n" else args.m
        xdt = torch.float32 if dt == torch.bfloat16 else dt   # bf16 A takes an fp32 X
        X = torch.randn(rows, args.l, generator=g, dtype=torch.float32).to(dev, xdt)
        return A, X
    if args.step == "orth":
        return torch.randn(args.m, args.l, generator=g, dtype=torch.float64).to(dev, dt), None
    if args.step == "small_svd":
        # an upper-triangular factor with the graded columns of a sketch of a
        # matrix whose singular values decay like 1/j
        M = torch.randn(args.l, args.l, generator=g, dtype=torch.float64)
        M = torch.triu(M) * (1.0 / torch.arange(1, args.l + 1, dtype=torch.float64))
        return M.to(dev, dt), None
    if args.step == "batched":
        from synth import BATCH_CONFIGS, batch_sizes, make_batch_torch
        c = BATCH_CONFIGS["c4_f32_batched512"]
        ms, ns, ks = batch_sizes("c4_f32_batched512", args.batch)
        mats = make_batch_torch(ms, ns, ks, 0xA000 + c["index"], device=dev)
        plan = rs.BatchPlan(ms, ns, ks, c["p"], c["q"], dev)
        return plan, plan.pack(mats)
    if args.step == "adaptive":
        gd = torch.Generator(device=dev).manual_seed(args.seed)
        return torch.randn(args.m, args.n, generator=gd, device=dev, dtype=dt), None
    if args.step == "cpqr":
        # rows scaled by 1/i like B = Q^T A of the same spectrum
        M = torch.randn(args.r, args.n, generator=g, dtype=torch.float64)
        M = M * (1.0 / torch.arange(1, args.r + 1, dtype=torch.float64))[:, None]
        return M.to(dev, dt), None
    raise ValueError(args.step)


def _call(args, X0, X1):
    s = args.step
    if s == "sample":
        return rs.sample(X0, args.l, args.seed)
    if s == "apply_n":
        return rs.apply(X0, X1, trans=False)
    if s == "apply_t":
        return rs.apply(X0, X1, trans=True)
    if s == "orth":
        return rs.orth(X0, check=False)
    if s == "small_svd":
        return rs.small_svd(X0, check=False)
    if s == "cpqr":
        return rs.cpqr_id(X0, args.k, check=False)
    if s == "batched":
        return X0.run(X1, args.seed)
    if s == "adaptive":
        return rs.qb_adaptive(X0, args.l, args.blocks, args.q, 0.0, args.seed, relative=False,
                              overwrite=True, check=False)
    raise ValueError(s)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--step", required=True,
                    choices=["sample", "apply_n", "apply_t", "orth", "small_svd", "cpqr",
                             "batched", "adaptive"])
    ap.add_argument("--m", type=int, default=50000)
    ap.add_argument("--n", type=int, default=20000)
    ap.add_argument("--l", type=int, default=220)
    ap.add_argument("--r", type=int, default=220)
    ap.add_argument("--k", type=int, default=200)
    ap.add_argument("--dtype", default="float32", choices=["float32", "float64", "bfloat16"],
                    help="element type of A (bfloat16: the passes over A only)")
    ap.add_argument("--seed", type=int, default=0x5EED)
    ap.add_argument("--batch", type=int, default=None, help="problems of --step batched")
    ap.add_argument("--blocks", type=int, default=4, help="blocks of --step adaptive")
    ap.add_argument("--q", type=int, default=1, help="power iterations of --step adaptive")
    ap.add_argument("--reps", type=int, default=3)
    args = ap.parse_args(argv)
    if not torch.cuda.is_available():
        print("run_step needs a CUDA device", file=sys.stderr)
        return 1
    dev = torch.device("cuda", 0)
    X0, X1 = _inputs(args, dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    for rep in range(args.reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _call(args, X0, X1)
        e1.record(stream)
        torch.cuda.synchronize()
        print("%s rep %d: %.3f ms" % (args.step, rep, e0.elapsed_time(e1)))
    return 0


if __name__ == "__main__":
    sys.exit(main())
