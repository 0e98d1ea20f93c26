"""Benchmark: randomized SVD + ID + CUR from one QB sketch on GB300.

One step = the whole path on one synthetic matrix: range finder with q power
iterations (A Omega with Omega generated in-kernel, CholeskyQR re-
orthonormalisation, A^T Y, A Z), the QB step Bt = A^T Q, the small SVD of B
(Alg. 5), the k-step pivoted QR of B for the ID and the CUR (Alg. 3).

Workload (default): FP32 A = G1 diag(1/j) G2^T + 1e-4 N(0,1), m = 50000,
n = 20000, r = 2000, k = 200, p = 20, q = 2 (4 GB row-major, larger than L2).

JSON line fields: value = algorithmic TFLOP/s of the step (flop count of every
step of the path, dominated by the 2q+2 passes over A at 2 m n l flops each)
divided by the measured step time; roofline = the dominant kernel class (CUDA
events recorded by the library on its own stream) against its hardware bound
(HBM copy bandwidth for the passes over A, the FP64 pipe for the pivoted QR);
qb_sketch = rsvd_qb (Y = A Omega through Bt = A^T Q) timed as one unit against
2q + 2 reads of A at the HBM bandwidth; e2e = the same metric through the host-input
entry point (A in pinned host memory, copied by the library in row chunks that
the sketch consumes as they land) with the outputs copied back, all inside the
timed region;
cpu_baseline = the FP64 oracle, one step on the GPU step's own matrix.
With --impl reference the oracle itself is the timed arm (host cores).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QB-sketch TFLOP/s & % roofline; mixed-prec/batched vs FP32 at equal rel. error"
UNIT = "TFLOP/s"


def step_flops(m, n, k, p, q, with_id=True, with_cur=True):
    """Algorithmic flops of one step (plain definitions, no split products)."""
    l = k + p
    f = 2.0 * m * n * l * (2 * q + 2)                       # A Omega, power steps, Bt
    n_orth_m = q + 1                                        # orth of m x l samples
    n_orth_n = q + 1                                        # orth of n x l (power + Bt)
    f += n_orth_m * 2 * 2.0 * m * l * l + n_orth_n * 2 * 2.0 * n * l * l   # CholQR2
    f += 2.0 * (m + n) * l * k                              # lift U = Q Vh, V = Qh Uh
    f += 3.0 * l ** 3 * 8                                   # Jacobi sweeps (~8)
    if with_id:
        f += 4.0 * k * l * n + k * k * (n - k)              # CPQR(B), T = S11^-1 S12
    if with_cur:
        f += 4.0 * k * k * m + 4.0 * n * k * k + 2.0 * k * k * (n - k)
    return f


def a_pass_bytes(m, n, elem=4):
    return float(m) * n * elem


ELEM = {"float32": 4, "float64": 8, "bfloat16": 2}   # bytes per entry of A


# Algorithmic work of one launch of each kernel class at the bench workload:
# HBM bytes for the passes over A (one read of the m x n fp32 matrix),
# FP64-equivalent flops for the pivoted QR and the triangular solves.
SM_COUNT = 152
FP64_FLOP_PER_CLK_SM = 4   # 2 DFMA per clock per SM (1.25 TFLOP/s at 2070 MHz, 152 SMs)
FP32_LANES_PER_SM = 128    # FP32 instructions issued per clock per SM (4 x 32)


def cpqr_flops(r, n, k):
    """Householder k-step CPQR of an r x n matrix: per step j the dot products and
    the rank-1 update of the (r - j) x (n - j - 1) trailing block, 2 flops each."""
    return float(sum(4.0 * (r - j) * (n - j - 1) for j in range(k)))


def solve_flops(k, ncols):
    """Upper-triangular solve with k x k factor for ncols right-hand sides."""
    return float(k) * k * ncols


def load_traffic():
    """dram bytes per launch measured by ncu, from profiles/traffic.txt
    (lines: class workload bytes_per_launch)."""
    out = {}
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if os.path.exists(p):
        with open(p) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 3 and not line.startswith("#"):
                    out[(parts[0], parts[1])] = float(parts[2])
    return out


def class_roofline(cls, trace, cfg, peaks, peak_kind, sm_mhz):
    ms_total, launches = trace[cls]
    if launches <= 0 or ms_total <= 0:
        return None
    avg_ms = ms_total / launches
    m, n, k, p = cfg["m"], cfg["n"], cfg["k"], cfg["p"]
    l = k + p
    traffic = load_traffic().get((cls, cfg["name"]))
    base = {"kernel_class": cls, "avg_launch_ms": avg_ms, "launches": launches,
            "traffic": traffic}
    if cls in ("a_omega", "a_w", "at_w"):
        achieved = a_pass_bytes(m, n, ELEM[cfg["dtype"]]) / (avg_ms * 1e-3) / 1e9
        base.update({"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"],
                     "unit": "GB/s", "frac": achieved / peaks["hbm_gbs"],
                     "peak_source": peak_kind + " STREAM-style copy",
                     "work_per_launch": "m n 4 bytes (one read of A)"})
        return base
    mhz = sm_mhz or peaks.get("sm_max_mhz", 2070.0)
    # The pivoted QR and the solves compute FP64-accurate results (double-float
    # pairs on the FP32 pipe); their roofline is the hardware FP64 rate they
    # stand in for: 152 SMs x 4 FP64 flops per clock (2 DFMA) x the SM clock
    # sampled during the timed region.  Two launches per step in both classes;
    # flops averaged over the pair.
    fp64_peak = SM_COUNT * FP64_FLOP_PER_CLK_SM * mhz * 1e6 / 1e12
    fp32_peak = SM_COUNT * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    if cls == "cpqr":
        flops = cpqr_flops(l, n, k) + cpqr_flops(k, m, k)    # ID of B, row ID of C^T
    elif cls == "solve":
        flops = solve_flops(k, n - k) + solve_flops(k, k)      # T = S11^-1 S12, U_cur
    else:
        return dict(base, bound=None, note="no work model for this class")
    achieved = (flops / 2.0) / (avg_ms * 1e-3) / 1e12
    base.update({"bound": "alu", "achieved": achieved, "peak": fp64_peak,
                 "unit": "TFLOP/s (FP64 flops of the algorithm)",
                 "frac": achieved / fp64_peak,
                 "peak_source": "hardware FP64 pipe: 152 SMs x 4 flops/clk x %.0f MHz "
                                "(clock sampled under load)" % mhz,
                 "fp32_pipe_peak": fp32_peak,
                 "arithmetic": "double-float (hi + lo fp32 pairs) on the FP32 pipe, ~48-bit",
                 "work_per_launch": "FP64 flops of the launch (both launches averaged)"})
    return base


# bf16 tensor-core products issued per K-step and output tile by each pass
# over A on the default path (RSVD_PREC_TC): fp32 A is split a = a0 + a1;
# Omega is one bf16 term, a stored operand two (w0, w1).
#   A Omega:      a0 w0 + a1 w0            (bf16 A: a0 w0)
#   A W, A^T W:   a0 w0 + a1 w0 + a0 w1    (bf16 A: a0 w0 + a0 w1)
PASS_PRODUCTS = {("a_omega", 4): 2, ("a_w", 4): 3, ("at_w", 4): 3,
                 ("a_omega", 2): 1, ("a_w", 2): 2, ("at_w", 2): 2}


def pass_bounds(cfg, peaks):
    """Per pass class: the time of its bytes at the measured HBM bandwidth and
    of its issued bf16 products at the measured sustained bf16 rate (the
    passes run inside a long step), MMA width N = l rounded up to 16."""
    m, n, l = cfg["m"], cfg["n"], cfg["k"] + cfg["p"]
    elem = ELEM[cfg["dtype"]]
    lpad = (l + 15) // 16 * 16
    out = {}
    for c in ("a_omega", "a_w", "at_w"):
        hbm_ms = a_pass_bytes(m, n, elem) / (peaks["hbm_gbs"] * 1e9) * 1e3
        # the recipe's sustained fallback when the file gives no tensor rate
        tflops = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops") or 1700.0
        tensor_ms = PASS_PRODUCTS[(c, elem)] * 2.0 * m * n * lpad / (tflops * 1e12) * 1e3
        out[c] = {"hbm_ms": hbm_ms, "tensor_ms": tensor_ms,
                  "bound": "hbm" if hbm_ms >= tensor_ms else "tensor",
                  "bound_ms": max(hbm_ms, tensor_ms)}
    return out


def sketch_roofline(trace, cfg, peaks, peak_kind):
    """The 2q+2 passes over A (a1-a7) against HBM: one read of A per pass;
    beside it each class against the slower of its two bounds (pass_bounds)."""
    m, n, q = cfg["m"], cfg["n"], cfg["q"]
    cls = [c for c in ("a_omega", "a_w", "at_w") if c in trace]
    ms = sum(trace[c][0] for c in cls)
    nl = sum(trace[c][1] for c in cls)
    if nl <= 0 or ms <= 0:
        return None
    achieved = nl * a_pass_bytes(m, n, ELEM[cfg["dtype"]]) / (ms * 1e-3) / 1e9
    t = load_traffic()
    pb = pass_bounds(cfg, peaks)
    per = {}
    for c in cls:
        avg = trace[c][0] / trace[c][1]
        per[c] = dict(pb[c], measured_ms=avg, frac=pb[c]["bound_ms"] / avg)
    bound_total = sum(pb[c]["bound_ms"] * trace[c][1] for c in cls)
    return {"kernels": "tc_omega2_kernel (A Omega), tc_unit_kernel (A W, A^T W)",
            "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "passes_timed": nl,
            "per_class_ms": {c: trace[c][0] / trace[c][1] for c in cls},
            "traffic": {c: t.get((c, cfg["name"])) for c in cls},
            "peak_source": peak_kind + " STREAM-style copy",
            "slower_bound": {
                "what": "each class against the slower of its bytes at the measured HBM "
                        "bandwidth and its issued bf16 products (split arithmetic, "
                        "PASS_PRODUCTS) at the measured sustained bf16 rate",
                "per_class": per, "frac": bound_total / ms,
                "tensor_peak_tflops": peaks.get("bf16_tflops_sustained")}}


def qb_sketch_unit(rs, A, cfg, args, seed, world, dev, peaks, peak_kind):
    """The QB sketch (Y = A Omega through Bt = A^T Q: the range finder, its q
    power iterations with their CholeskyQR orthonormalisations, the final orth
    and the QB step) timed as one stream-ordered unit: rsvd_qb, W untimed then K
    timed calls bracketed by CUDA events on the library's stream.  Roofline:
    its algorithmic bytes, 2q + 2 reads of A, against the measured HBM copy
    bandwidth; flops 2 m n l (2q + 2) plus the CholeskyQR Grams and applies."""
    import torch
    m, n, k, p, q = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["q"]
    l = k + p
    plan = rs.QbPlan(m, n, k, p, q, A.dtype, dev)
    for _ in range(args.warmup):
        plan.run(A, seed)
    torch.cuda.synchronize()
    rs.check_info(plan.info, "qb warmup")
    stream = torch.cuda.current_stream()
    rs.trace_enable(True)
    rs.trace_read()
    launches0 = rs.kernel_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.run(A, seed)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = (rs.kernel_launch_count() - launches0) / args.steps
    trace = rs.trace_read()
    rs.trace_enable(False)
    rs.check_info(plan.info, "qb steps")
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    bytes_ = (2 * q + 2) * a_pass_bytes(m, n, ELEM[cfg["dtype"]])
    flops = 2.0 * m * n * l * (2 * q + 2) + (q + 1) * 4.0 * (m + n) * l * l
    gbs = bytes_ / (ms * 1e-3) / 1e9
    del plan
    return {"what": "rsvd_qb: Y = A Omega, q power iterations with CholeskyQR, Q = orth(Y), "
                    "Bt = A^T Q (one stream-ordered unit)",
            "ms": ms, "tflops": world * flops / (ms * 1e-3) / 1e12,
            "bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peaks["hbm_gbs"],
            "peak_source": peak_kind + " STREAM-style copy",
            "work": "%d reads of A (%.1f GB each) per call" % (2 * q + 2, bytes_ / (2 * q + 2) / 1e9),
            "launches_per_call": launches,
            "kernels": {c: {"ms_per_call": v[0] / args.steps, "launches_per_call": v[1] / args.steps}
                        for c, v in trace.items() if v[1] > 0}}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        med = float(np.median(sm)) if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job(flops_per_step, ms_local, world, device):
    """(slowest rank's ms per step, whole-job TFLOP/s).  Every rank runs its
    own replica of the step, so the job processes world x flops_per_step per
    step in the time of its slowest rank."""
    ms = max_over_ranks(ms_local, world, device)
    return ms, world * flops_per_step / (ms * 1e-3) / 1e12


def _oracle_sample_setup(cfg, frac_rows=25, frac_cols=5):
    """A bounded sample of the same recipe (m/frac_rows x n/frac_cols) for the oracle."""
    from synth import make_matrix_np, spectrum
    m = max(cfg["m"] // frac_rows, cfg["k"] + cfg["p"] + 8)
    n = max(cfg["n"] // frac_cols, cfg["k"] + cfg["p"] + 8)
    r = min(cfg["r"], m, n)
    A = make_matrix_np(m, n, spectrum(cfg["spectrum"], r), noise=cfg["noise"],
                       seed=cfg["a_seed"], dtype=cfg["dtype"]).astype(np.float64)
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    desc = ("FP64 numpy oracle (OpenBLAS threads on all affinity cores), RSVD + ID + CUR of the "
            "same recipe at m=%d n=%d k=%d p=%d q=%d (1/%d of the rows, 1/%d of the columns)"
            % (m, n, cfg["k"], cfg["p"], cfg["q"], frac_rows, frac_cols))
    return A, m, n, cores, desc


def _oracle_step(A, cfg):
    from oracle import rsvd as orc
    k, p, q = cfg["k"], cfg["p"], cfg["q"]
    t0 = time.perf_counter()
    orc.rsvd(A, k, p, q, cfg["omega_seed"], rounding="bf16")
    orc.rcur(A, k, p, q, cfg["omega_seed"], rounding="bf16")
    return time.perf_counter() - t0


def cpu_oracle_sample(cfg, reps=3):
    """The FP64 oracle timed on a bounded sample of the same recipe."""
    A, m, n, cores, desc = _oracle_sample_setup(cfg)
    dt = float(np.median([_oracle_step(A, cfg) for _ in range(reps)]))
    fl = step_flops(m, n, cfg["k"], cfg["p"], cfg["q"])
    return {"value": fl / dt / 1e12, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": desc + ", %.2f s per step (median of %d)" % (dt, reps)}


def cpu_oracle_full(A_host, cfg):
    """The FP64 oracle, as it stands, timed for one step (RSVD, then ID + CUR) on
    the very matrix the GPU step used (copied to the host and promoted to
    float64), with OpenBLAS threads on every affinity core."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count()
    A64 = A_host.numpy().astype(np.float64)
    dt = _oracle_step(A64, cfg)
    del A64
    m, n = cfg["m"], cfg["n"]
    fl = step_flops(m, n, cfg["k"], cfg["p"], cfg["q"])
    return {"value": fl / dt / 1e12, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "the full workload (m=%d n=%d k=%d p=%d q=%d, the GPU step's own A in "
                      "FP64): one step of oracle.rsvd + oracle.rcur, %.1f s"
                      % (m, n, cfg["k"], cfg["p"], cfg["q"], dt),
            "one_thread": cpu_oracle_one_thread()}


def oracle_one_thread_child():
    """--oracle-one-thread: read (config name, A as .npy) from stdin, time the
    oracle's QB (a1-a7) and one step of oracle.rsvd + oracle.rcur on it, print
    one JSON line.  The parent starts this process with one BLAS thread."""
    import io
    name = sys.stdin.buffer.readline().decode().strip()
    A = np.load(io.BytesIO(sys.stdin.buffer.read()))
    from synth import config as get_config
    from oracle import rsvd as orc
    cfg = get_config(name)
    k, p, q, seed = cfg["k"], cfg["p"], cfg["q"], cfg["omega_seed"]
    rounding = "f64" if cfg["dtype"] == "float64" else "bf16"
    t0 = time.perf_counter()
    orc.qb(A, k, p, q, seed, rounding=rounding)
    t_qb = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc.rsvd(A, k, p, q, seed, rounding=rounding)
    orc.rcur(A, k, p, q, seed, rounding=rounding)
    t_step = time.perf_counter() - t0
    m, n = A.shape
    print(json.dumps({"workload": name, "qb_s": t_qb, "step_s": t_step,
                      "step_tflops": step_flops(m, n, k, p, q) / t_step / 1e12}))
    return 0


def cpu_oracle_one_thread(names=("c1_f64_2000x1000", "c5_f32_8192x4096")):
    """The oracle with one BLAS thread on the small workloads (their matrices
    built here with every core and handed over through a pipe)."""
    import io
    import subprocess
    from synth import config as get_config, make_matrix_np, spectrum
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    out = {}
    for name in names:
        c = get_config(name)
        A = make_matrix_np(c["m"], c["n"], spectrum(c["spectrum"], c["r"]), noise=c["noise"],
                           seed=c["a_seed"], dtype=c["dtype"]).astype(np.float64)
        buf = io.BytesIO()
        np.save(buf, A)
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-one-thread"],
                           input=name.encode() + b"\n" + buf.getvalue(), env=env,
                           capture_output=True, timeout=600)
        lines = [ln for ln in r.stdout.decode().splitlines() if ln.startswith("{")]
        out[name] = json.loads(lines[0]) if r.returncode == 0 and lines else \
            {"error": r.stderr.decode()[-300:]}
    return out


def run_reference(args, cfg, rank):
    """--impl reference: the oracle on the host cores (rank 0 only), W untimed
    warm-up steps then K timed steps of the bounded sample."""
    if rank != 0:
        return 0
    A, m, n, cores, desc = _oracle_sample_setup(cfg)
    for _ in range(args.warmup):
        _oracle_step(A, cfg)
    times = [_oracle_step(A, cfg) for _ in range(args.steps)]
    tot = float(sum(times))
    fl = step_flops(m, n, cfg["k"], cfg["p"], cfg["q"])
    v = fl * len(times) / tot / 1e12
    ms = 1e3 * tot / len(times)
    sample = desc + ", %.2f s per step" % (tot / len(times))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": len(times), "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": cfg["name"], "sample": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def rel_err_device(rs, A, U, S, V):
    """||A - U diag(S) V^T||_F / ||A||_F for orthonormal U, V:
    ||A||^2 - 2 sum_i S_i u_i^T A v_i + sum_i S_i^2, with A V from the library's
    own FP32-accurate apply kernel and the sums in float64."""
    import torch
    AV = rs.apply(A, V.contiguous(), trans=False)
    t = (U.double() * AV.double()).sum(dim=0)
    s = S.double()
    a2 = sum(float(blk.double().pow(2).sum()) for blk in torch.split(A, 4096, dim=0))
    e2 = a2 - 2.0 * float((s * t).sum()) + float((s * s).sum())
    return (max(e2, 0.0) / a2) ** 0.5


def _time_variant(rs, Ad, opts, cfg, args, seed, world, dev):
    """(ms per step, per-class trace, plan) of the whole step on A as given."""
    import torch
    m, n, k, p, q = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["q"]
    plan = rs.Plan(m, n, k, p, q, Ad.dtype, dev, opts)
    for _ in range(args.warmup):
        plan.run(Ad, seed)
    torch.cuda.synchronize()
    rs.check_info(plan.info, "mixed warmup")
    stream = torch.cuda.current_stream()
    rs.trace_enable(True)
    rs.trace_read()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.run(Ad, seed)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    trace = rs.trace_read()
    rs.trace_enable(False)
    rs.check_info(plan.info, "mixed steps")
    return max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev), trace, plan


def mixed_precision_line(rs, A, plan32, cfg, args, seed, world, dev, ms32, peaks, peak_kind):
    """The same step in the mixed-precision forms, each timed like the main
    line and judged by its relative error against the FP32 A next to the FP32
    path's (equal-error comparison):
      bf16_storage        A held as bf16 (RSVD_BF16), RSVD_PREC_TC arithmetic;
      bf16_storage_mixed  A as bf16 and single-term bf16 power scheme (RSVD_PREC_MIXED);
      f32_mixed           fp32 A, single-term bf16 power scheme (RSVD_PREC_MIXED);
      f32_fp8_sketch      fp32 A, the sketch Y = A Omega on E4M3-quantised A and Omega
                          with 32-entry block scales (RSVD_PREC_FP8);
      bf16_fp8_sketch     the same with A held as bf16."""
    import torch
    m, n, k, p, q = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["q"]
    flops = step_flops(m, n, k, p, q)
    e32 = rel_err_device(rs, A, plan32.U, plan32.S, plan32.V)
    Ab = A.to(torch.bfloat16)
    mixed_opts = rs.make_opts(precision=rs.PREC_MIXED)
    fp8_opts = rs.make_opts(precision=rs.PREC_FP8)
    out = {"rel_err_fp32": e32,
           "rel_err_definition": "||A - U S V^T||_F / ||A||_F against the FP32 A",
           "fp32_ms_per_step": ms32}
    for name, Ad, opts, elem, what in (
            ("bf16_storage", Ab, None, 2,
             "A in bf16 (RSVD_BF16): sketch, power and QB passes on exact bf16 A, one "
             "tensor-core product per stored-operand term; the rest as the FP32 path"),
            ("bf16_storage_mixed", Ab, mixed_opts, 2,
             "A in bf16 and RSVD_PREC_MIXED: the power scheme's passes take one bf16 term "
             "of the stored operand (one product per K-step); Bt = A^T Q split"),
            ("f32_mixed", A, mixed_opts, 4,
             "fp32 A and RSVD_PREC_MIXED: the power scheme's passes take a0 w0 only"),
            ("f32_fp8_sketch", A, fp8_opts, 4,
             "fp32 A and RSVD_PREC_FP8: the sketch on E4M3-quantised A and Omega (one "
             "power-of-two scale per 32 entries along the contraction), products of the exact "
             "dequantised values on the bf16 tensor cores; the rest as the FP32 path"),
            ("bf16_fp8_sketch", Ab, fp8_opts, 2,
             "A in bf16 and RSVD_PREC_FP8: the FP8 sketch of the bf16 values")):
        ms, trace, plan = _time_variant(rs, Ad, opts, cfg, args, seed, world, dev)
        e = rel_err_device(rs, A, plan.U, plan.S, plan.V)
        pass_ms = sum(v[0] for c, v in trace.items()
                      if c in ("a_omega", "a_w", "at_w")) / args.steps
        gbs = (2 * q + 2) * a_pass_bytes(m, n, elem) / (pass_ms * 1e-3) / 1e9 if pass_ms else None
        out[name] = {
            "what": what,
            "value": world * flops / (ms * 1e-3) / 1e12, "unit": UNIT, "ms_per_step": ms,
            "speedup_vs_fp32": ms32 / ms, "rel_err": e, "rel_err_ratio_vs_fp32": e / e32,
            "a_pass_ms_per_step": pass_ms,
            "a_pass_hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                           "frac": gbs / peaks["hbm_gbs"] if gbs else None,
                           "peak_source": peak_kind + " STREAM-style copy",
                           "work": "m n %d bytes per pass" % elem},
            "kernels": {c: {"ms_per_step": v[0] / args.steps,
                            "launches_per_step": v[1] / args.steps}
                        for c, v in trace.items()},
        }
        del plan
    del Ab
    return out


C3_NAME = "c3_bf16_100000x50000"
C3_GOLDEN = os.path.join(ROOT, "tests", "golden", "c3_reduced_oracle.txt")
C3_RANKS = (1, 10, 50, 100, 200, 300, 400, 500)


def load_c3_golden(path=C3_GOLDEN):
    """(sizes, values) of the stored FP64-oracle results for the reduced matrix of
    the mixed-precision recipe: sizes from the '# m .. n ..' header line, values
    rel_err_<A> (float) and sigma_<A> (array) for A = f32 and bf16."""
    meta, vals = {}, {}
    with open(path) as f:
        for line in f:
            if line.startswith("# m "):
                t = line[2:].split()
                meta = {t[i]: t[i + 1] for i in range(0, len(t) - 1, 2)}
            elif line.startswith("#") or not line.strip():
                continue
            else:
                key, *v = line.split()
                vals[key] = (np.array([float(x) for x in v]) if key.startswith("sigma_")
                             else float(v[0]))
    return meta, vals


def c3_variants(rs):
    """(name, storage, opts, description) of the mixed-precision workload's forms."""
    import torch
    mixed = rs.make_opts(precision=rs.PREC_MIXED)
    fp8 = rs.make_opts(precision=rs.PREC_FP8)
    return (
        ("f32", torch.float32, None,
         "fp32 A; split-bf16 tensor-core products, fp32 accumulation (the plain FP32 path)"),
        ("bf16", torch.bfloat16, None,
         "A stored as bf16; exact bf16 products, fp32 accumulation; Bt = A^T Q with Q split "
         "into bf16 terms"),
        ("bf16_mixed", torch.bfloat16, mixed,
         "A as bf16; the power scheme's passes take one bf16 term of the stored operand"),
        ("bf16_fp8_sketch", torch.bfloat16, fp8,
         "A as bf16; the sketch Y = A Omega on E4M3-quantised A and Omega with one power-of-two "
         "scale per 32 entries along the contraction"),
        ("f32_fp8_sketch", torch.float32, fp8,
         "fp32 A; the same FP8 sketch"),
    )


def c3_line(rs, args, world, dev, peaks, peak_kind):
    """The mixed-precision workload (m = 100000, n = 50000, k = 500, p = 50, q = 2,
    sigma_j = exp(-j/100) + 1e-3 on r = 2000 directions, 1e-4 noise) in each form
    of c3_variants: the whole step (QB + SVD + ID + CUR) timed like the main line
    at full size and judged by ||A - U S V^T||_F / ||A||_F against the FP32 A
    (equal-error comparison).  The error against the FP64 oracle at every rank
    i <= k is taken on the reduced matrix of the same recipe whose oracle results
    are stored (tests/golden/c3_reduced_oracle.txt): each form's sigma_i against
    the oracle's on the same storage, and its relative error against the oracle's."""
    import torch
    from types import SimpleNamespace
    from synth import config as get_config, make_matrix_np, make_matrix_torch, spectrum
    cfg = get_config(C3_NAME)
    m, n, k, p, q = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["q"]
    seed = cfg["omega_seed"]
    sig = spectrum(cfg["spectrum"], cfg["r"])
    sub = SimpleNamespace(steps=min(args.steps, 2), warmup=max(args.warmup, 3))
    out = {"workload": C3_NAME, "m": m, "n": n, "k": k, "p": p, "q": q,
           "spectrum": "sigma_j = exp(-j/100) + 1e-3, r = %d, noise %g" % (cfg["r"], cfg["noise"]),
           "steps": sub.steps, "warmup": sub.warmup,
           "rel_err_definition": "||A - U S V^T||_F / ||A||_F against the FP32 A"}

    # ---- error against the FP64 oracle at every rank (reduced matrix) ----
    meta, gold = load_c3_golden()
    mr, nr = int(meta["m"]), int(meta["n"])
    A32r = torch.from_numpy(make_matrix_np(mr, nr, sig, noise=cfg["noise"], seed=cfg["a_seed"],
                                           dtype="float32")).to(dev)
    Abr = A32r.to(torch.bfloat16)          # round to nearest even, as the stored oracle input
    vs_oracle = {"sizes": "m=%d n=%d k=%d p=%d q=%d, same spectrum, noise and seeds" % (mr, nr, k, p, q),
                 "oracle_rel_err": {"f32": gold["rel_err_f32"], "bf16": gold["rel_err_bf16"]},
                 "ranks_reported": list(C3_RANKS)}
    for name, dt, opts, _ in c3_variants(rs):
        Ar = Abr if dt == torch.bfloat16 else A32r
        ref = gold["sigma_bf16" if dt == torch.bfloat16 else "sigma_f32"]
        plan = rs.Plan(mr, nr, k, p, q, dt, dev, opts)
        plan.run(Ar, seed)
        torch.cuda.synchronize()
        rs.check_info(plan.info, "c3 reduced " + name)
        S = plan.S.double().cpu().numpy()
        rel = np.abs(S - ref) / ref
        e = rel_err_device(rs, A32r, plan.U, plan.S, plan.V)
        oe = gold["rel_err_bf16" if dt == torch.bfloat16 else "rel_err_f32"]
        vs_oracle[name] = {
            "sigma_rel_err_max": float(rel.max()),
            "sigma_rel_err_median": float(np.median(rel)),
            "sigma_rel_err_at_rank": [float(rel[i - 1]) for i in C3_RANKS],
            "rel_err": e, "rel_err_vs_oracle": e / oe}
        del plan
    del A32r, Abr
    torch.cuda.empty_cache()
    out["vs_fp64_oracle"] = vs_oracle

    # ---- full size: timing and the equal-error comparison ----
    A32 = make_matrix_torch(m, n, sig, noise=cfg["noise"], seed=cfg["a_seed"], dtype="float32",
                            device=dev)
    Ab = A32.to(torch.bfloat16)
    torch.cuda.synchronize()
    flops = step_flops(m, n, k, p, q)
    ms32 = None
    for name, dt, opts, what in c3_variants(rs):
        Ad = Ab if dt == torch.bfloat16 else A32
        ms, trace, plan = _time_variant(rs, Ad, opts, cfg, sub, seed, world, dev)
        e = rel_err_device(rs, A32, plan.U, plan.S, plan.V)
        del plan
        ms, value = whole_job(flops, ms, world, dev)
        if ms32 is None:
            ms32 = ms
        pass_ms = sum(v[0] for c, v in trace.items()
                      if c in ("a_omega", "a_w", "at_w")) / sub.steps
        elem = 2 if dt == torch.bfloat16 else 4
        out[name] = {
            "what": what, "value": value, "unit": UNIT, "ms_per_step": ms,
            "speedup_vs_fp32": ms32 / ms, "rel_err": e,
            "a_pass_ms_per_step": pass_ms,
            "a_pass_gbs": ((2 * q + 2) * a_pass_bytes(m, n, elem) / (pass_ms * 1e-3) / 1e9
                           if pass_ms else None),
            "kernels": {c: round(v[0] / sub.steps, 3) for c, v in trace.items()}}
    out["rel_err_fp32"] = out["f32"]["rel_err"]
    del A32, Ab
    torch.cuda.empty_cache()
    return out


def batched_line(rs, args, world, dev, peaks, peak_kind, name="c4_f32_batched512"):
    """The batched workload (512 FP32 problems of uneven sizes): the batched
    call timed like the main line, against the same problems run one by one
    through the FP32 path (rsvd_svd), both judged by their relative errors."""
    import torch
    from synth import BATCH_CONFIGS, batch_sizes, make_batch_torch
    c = BATCH_CONFIGS[name]
    p, q = c["p"], c["q"]
    ms, ns, ks = batch_sizes(name)
    seed = 0x5EED + c["index"]
    mats = make_batch_torch(ms, ns, ks, 0xA000 + c["index"], device=dev)
    plan = rs.BatchPlan(ms, ns, ks, p, q, dev)
    Ap = plan.pack(mats)
    for _ in range(args.warmup):
        plan.run(Ap, seed)
    torch.cuda.synchronize()
    rs.check_info(plan.info, "batched warmup")
    stream = torch.cuda.current_stream()
    rs.trace_enable(True)
    rs.trace_read()
    launches0 = rs.kernel_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.run(Ap, seed)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = (rs.kernel_launch_count() - launches0) / args.steps
    trace = rs.trace_read()
    rs.trace_enable(False)
    rs.check_info(plan.info, "batched steps")
    ms_b = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world, dev)
    # the same problems through the single-problem FP32 path, one call each
    for i in range(min(4, len(mats))):
        rs.svd(mats[i], ks[i], p, q, seed)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    single = [rs.svd(mats[i], ks[i], p, q, seed, check=False) for i in range(len(mats))]
    e1.record(stream)
    torch.cuda.synchronize()
    ms_s = e0.elapsed_time(e1)
    errs_b, errs_s = [], []
    for i, A in enumerate(mats):
        U, S, V = plan.result(i)
        errs_b.append(rel_err_device(rs, A, U, S, V))
        errs_s.append(rel_err_device(rs, A, *single[i]))
    flops = sum(2.0 * m * n * (k + p) * (2 * q + 2) for m, n, k in zip(ms, ns, ks))
    a_bytes = sum(4.0 * m * n for m, n in zip(ms, ns))
    gbs = (2 * q + 2) * a_bytes / (ms_b * 1e-3) / 1e9
    eb, es = float(np.mean(errs_b)), float(np.mean(errs_s))
    # the grouped tensor-core passes over A (trace classes of the library's stream)
    tc_cls = [c for c in ("a_omega", "a_w", "at_w") if c in trace]
    tc_ms = sum(trace[c][0] for c in tc_cls) / args.steps
    tc_n = sum(trace[c][1] for c in tc_cls) / args.steps
    tc_pass = None
    if tc_n > 0 and tc_ms > 0:
        g = tc_n * a_bytes / (tc_ms * 1e-3) / 1e9
        tc_pass = {"kernel": "tc_group_kernel (grouped tcgen05, one launch per pass over all A_i)",
                   "passes": tc_n, "ms_per_pass": tc_ms / tc_n, "achieved": g,
                   "peak": peaks["hbm_gbs"], "unit": "GB/s", "frac": g / peaks["hbm_gbs"],
                   "peak_source": peak_kind + " STREAM-style copy",
                   "work": "one read of every A_i (4 B per entry) per pass"}
    classes = {c: {"ms_per_step": trace[c][0] / args.steps,
                   "launches_per_step": trace[c][1] / args.steps} for c in trace}
    return {
        "workload": "%s: %d FP32 problems, m in [%d, %d], n in [%d, %d], k in %s, p = %d, q = %d, "
                    "sigma_j = exp(-j/k)" % (name, len(ms), min(ms), max(ms), min(ns), max(ns),
                                             sorted(set(ks)), p, q),
        "ms_per_step": ms_b, "unit": UNIT,
        "value": world * flops / (ms_b * 1e-3) / 1e12,
        "flops_definition": "sum over problems of 2 m n l (2q + 2) (the passes over A)",
        "launches_per_step": launches,
        "fp32_one_by_one_ms": ms_s,
        "speedup_vs_fp32_one_by_one": ms_s / ms_b,
        "rel_err_mean": eb, "rel_err_fp32_mean": es, "rel_err_ratio": eb / es,
        "rel_err_max_ratio": float(np.max(np.array(errs_b) / np.array(errs_s))),
        "rel_err_definition": "||A_i - U_i S_i V_i^T||_F / ||A_i||_F, mean over problems",
        "a_pass_hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                       "frac": gbs / peaks["hbm_gbs"], "peak_source": peak_kind + " STREAM-style copy",
                       "work": "(2q + 2) reads of every A_i per step (4 B per entry), whole-step time"},
        "tc_pass_hbm": tc_pass,
        "kernels": classes,
        "autotuner": rs.batched_tuning(),
    }


def adaptive_line(rs, A, cfg, args, world, dev, peaks, peak_kind, b=64, M=4, q=1):
    """The blocked adaptive QB (Alg. 7) on the workload's matrix: M blocks of b
    columns (tolerance 0, so all M blocks run), q power steps per block.  Each
    call gets a fresh copy of A (the algorithm overwrites A with its residual),
    made outside the timed region; CUDA events around the call, which
    synchronises with the host once per block to test the tolerance."""
    import torch
    m, n = cfg["m"], cfg["n"]
    seed = cfg["omega_seed"]
    reps = max(1, min(args.steps, 3))
    times = []
    for r in range(reps + 1):
        Aw = A.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        Q, Bt, resid = rs.qb_adaptive(Aw, b, M, q, 0.0, seed, relative=False, overwrite=True)
        e1.record()
        torch.cuda.synchronize()
        if r > 0:                      # the first call is an untimed warm-up
            times.append(e0.elapsed_time(e1))
        del Aw
    ms = max_over_ranks(float(np.median(times)), world, dev)
    es = ELEM[cfg["dtype"]]
    # per block: sketch, q power steps (2 passes each), Bt: 2q + 2 reads of A;
    # the update reads and writes A; plus the norm of A_in
    bytes_ = M * ((2 * q + 2) + 2) * a_pass_bytes(m, n, es) + a_pass_bytes(m, n, es)
    flops = M * (2.0 * m * n * b * (2 * q + 2) + 2.0 * m * n * b)
    gbs = bytes_ / (ms * 1e-3) / 1e9
    r = resid.cpu().numpy()
    return {"what": "rsvd_qb_adaptive (Alg. 7): %d blocks of b = %d, q = %d, tolerance 0" % (M, b, q),
            "ms_per_call": ms, "calls_timed": len(times),
            "tflops": world * flops / (ms * 1e-3) / 1e12,
            "hbm": {"achieved": gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": gbs / peaks["hbm_gbs"], "peak_source": peak_kind + " STREAM-style copy",
                    "work": "per block 2q + 2 reads of A and the update's read + write, plus "
                            "the first norm read"},
            "residual_norms": [float(x) for x in r]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="c2_f32_50000x20000")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-baseline-sample", action="store_true",
                    help="time the oracle on a bounded sample instead of the full workload")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the BF16-storage (mixed precision) measurement")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-workload (512 small problems) measurement")
    ap.add_argument("--no-c3", action="store_true",
                    help="skip the mixed-precision workload (100000 x 50000, l = 550)")
    ap.add_argument("--no-adaptive", action="store_true",
                    help="skip the blocked adaptive QB (Alg. 7) measurement")
    ap.add_argument("--oracle-one-thread", action="store_true", help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.oracle_one_thread:
        return oracle_one_thread_child()

    from synth import config as get_config
    cfg = get_config(args.config)
    cfg["name"] = args.config
    if args.impl == "reference":
        # host cores only, no exchange between ranks: rank 0 runs, the others
        # exit without work (and without joining a process group)
        return run_reference(args, cfg, int(os.environ.get("RANK", "0")))
    world, rank, local = dist_setup()

    import torch
    import paper_1502_05366_gb300 as rs
    from synth import make_matrix_torch, spectrum

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    m, n, k, p, q = cfg["m"], cfg["n"], cfg["k"], cfg["p"], cfg["q"]
    tdt = {"float32": torch.float32, "float64": torch.float64,
           "bfloat16": torch.bfloat16}[cfg["dtype"]]
    A = make_matrix_torch(m, n, spectrum(cfg["spectrum"], cfg["r"]), noise=cfg["noise"],
                          seed=cfg["a_seed"] + rank, dtype=cfg["dtype"], device=dev)
    torch.cuda.synchronize()
    plan = rs.Plan(m, n, k, p, q, tdt, dev)
    seed = cfg["omega_seed"]
    stream = torch.cuda.current_stream()

    for _ in range(args.warmup):
        plan.run(A, seed)
    torch.cuda.synchronize()
    rs.check_info(plan.info, "warmup")

    # ---------------- timed region (device-resident inputs) ----------------
    rs.trace_enable(True)
    rs.trace_read()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = rs.kernel_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        plan.run(A, seed)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = rs.kernel_launch_count() - launches0
    clk = clocks.stop()
    trace = rs.trace_read()
    rs.trace_enable(False)
    rs.check_info(plan.info, "timed steps")
    flops = step_flops(m, n, k, p, q)
    ms, value = whole_job(flops, ev0.elapsed_time(ev1) / args.steps, world, dev)

    # ---------------- roofline of the dominant kernel class ----------------
    peaks, peak_kind = load_peaks()
    sm_mhz = None
    if clk and clk.get("sm_mhz"):
        sm_mhz = float(clk["sm_mhz"])
    dom = max(trace, key=lambda c: trace[c][0])
    roof = class_roofline(dom, trace, cfg, peaks, peak_kind, sm_mhz)
    roof_sketch = sketch_roofline(trace, cfg, peaks, peak_kind)
    breakdown = {c: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps}
                 for c, v in trace.items()}
    pass_ms = sum(v[0] for c, v in trace.items() if c in ("a_omega", "a_w", "at_w")) / args.steps
    qb_flops = 2.0 * m * n * (k + p) * (2 * q + 2)

    # ---------------- end to end: host A in, host outputs out ----------------
    A_host = A.cpu().pin_memory()
    outs = [t for t in (plan.U, plan.S, plan.V, plan.J, plan.T, plan.Jc, plan.Ir, plan.Ucur)
            if t is not None]
    outs_host = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in outs]
    h2d = A_host.numel() * A_host.element_size()
    d2h = sum(t.numel() * t.element_size() for t in outs)
    plan.run_host(A_host, A, seed)          # untimed: first use of the host buffers
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.e2e_steps + 1)]
    evs[0].record(stream)
    for i in range(args.e2e_steps):
        # the library call with A in host memory: it copies A into the device
        # buffer in row chunks while the sketch consumes them
        plan.run_host(A_host, A, seed)
        for h, d in zip(outs_host, outs):
            h.copy_(d, non_blocking=True)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    rs.check_info(plan.info, "end-to-end steps")
    steps_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.e2e_steps)]
    e2e_ms, e2e_value = whole_job(flops, float(np.median(steps_ms)), world, dev)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
           "ms_steps": steps_ms, "statistic": "median of the steps"}

    qb_unit = qb_sketch_unit(rs, A, cfg, args, seed, world, dev, peaks, peak_kind)

    mixed = None
    if not args.no_mixed and tdt == torch.float32:
        mixed = mixed_precision_line(rs, A, plan, cfg, args, seed, world, dev, ms, peaks,
                                     peak_kind)

    batched = None
    if not args.no_batched:
        batched = batched_line(rs, args, world, dev, peaks, peak_kind)

    adaptive = None
    if not args.no_adaptive and tdt == torch.float32:
        adaptive = adaptive_line(rs, A, cfg, args, world, dev, peaks, peak_kind)

    c3 = None
    if not args.no_c3 and cfg["name"] != C3_NAME:
        # the main workload's buffers are released first (A32 + its bf16 copy
        # of the mixed-precision workload hold 30 GB)
        del plan
        torch.cuda.empty_cache()
        c3 = c3_line(rs, args, world, dev, peaks, peak_kind)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            cpu = (cpu_oracle_sample(cfg) if args.cpu_baseline_sample
                   else cpu_oracle_full(A_host, cfg))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"float32": "f32", "float64": "f64", "bfloat16": "bf16 A, f32"}[cfg["dtype"]],
            "data": "synthetic",
            "config": {"workload": cfg["name"], "m": m, "n": n, "k": k, "p": p, "q": q,
                       "spectrum": "sigma_j = 1/j, r = %d, noise %g" % (cfg["r"], cfg["noise"]),
                       "precision": {"float32": "fp32 storage; split-bf16 tcgen05 products, "
                                                 "fp32 accumulate",
                                     "bfloat16": "bf16 storage; exact bf16 tcgen05 products, "
                                                 "fp32 accumulate",
                                     "float64": "fp64 storage; FP64 SIMT"}[cfg["dtype"]],
                       "step": "QB sketch + SVD + ID + CUR from one sketch",
                       "l2": "A (%.1f GB) larger than L2 on every pass"
                             % (ELEM[cfg["dtype"]] * m * n / 1e9),
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "qb_sketch": dict(qb_unit, a_pass_ms_per_step=pass_ms,
                              a_pass_tflops=qb_flops / (pass_ms * 1e-3) / 1e12 if pass_ms else None,
                              a_passes_per_step=2 * q + 2),
            "roofline": roof,
            "roofline_sketch": roof_sketch,
            "kernels": breakdown,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": launches,
            "cpu_baseline": cpu,
            "mixed": mixed,
            "batched": batched,
            "adaptive_qb": adaptive,
            "mixed_c3": c3,
        }
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
