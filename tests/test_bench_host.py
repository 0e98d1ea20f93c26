"""Host logic of bench.py on CPU: the work model behind the roofline object, the
files it reads, and the JSON line of the reference arm (the oracle timed on the
host cores) at N = 1."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

CFG = {"name": "c2_f32_50000x20000", "m": 50000, "n": 20000, "k": 200, "p": 20, "q": 2,
       "dtype": "float32"}
PEAKS = {"hbm_gbs": 6784.8, "sm_max_mhz": 2070.0}


def test_pass_roofline_is_bytes_of_a_over_the_average_launch():
    # 6 launches of the A-pass class in 3.6 ms: 0.6 ms each, 4 GB read each
    trace = {"a_w": (3.6, 6)}
    r = bench.class_roofline("a_w", trace, CFG, PEAKS, "measured", None)
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(50000 * 20000 * 4 / 0.6e-3 / 1e9, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / 6784.8, rel=1e-12)
    assert r["peak"] == 6784.8
    assert r["traffic"] == bench.load_traffic()[("a_w", "c2_f32_50000x20000")]   # per launch
    # bf16 storage halves the algorithmic bytes of a pass
    r16 = bench.class_roofline("a_w", trace, dict(CFG, dtype="bfloat16"), PEAKS, "measured",
                               None)
    assert r16["achieved"] == pytest.approx(r["achieved"] / 2, rel=1e-12)


def test_alu_roofline_of_the_pivoted_qr():
    trace = {"cpqr": (8.0, 2)}
    r = bench.class_roofline("cpqr", trace, CFG, PEAKS, "measured", 1500.0)
    assert r["bound"] == "alu"
    # peak = the hardware FP64 pipe: SMs x 4 flops per clock x the sampled clock
    assert r["peak"] == pytest.approx(152 * 4 * 1500e6 / 1e12, rel=1e-12)
    # the two launches of a step (ID of B: l x n; row ID of C^T: k x m), averaged
    l, k, m, n = 220, 200, 50000, 20000
    work = sum(4.0 * (l - j) * (n - j - 1) for j in range(k)) + \
        sum(4.0 * (k - j) * (m - j - 1) for j in range(k))
    assert r["achieved"] == pytest.approx(work / 2 / 4e-3 / 1e12, rel=1e-12)
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"], rel=1e-12)


def test_cpqr_flops_closed_form():
    # sum_{j<k} 4 (r - j)(n - j - 1) against its closed form
    r, n, k = 220, 20000, 200
    j = k * (k - 1) / 2.0
    j2 = (k - 1) * k * (2 * k - 1) / 6.0
    closed = 4.0 * (k * r * (n - 1) - (r + n - 1) * j + j2)
    assert bench.cpqr_flops(r, n, k) == pytest.approx(closed, rel=1e-14)


def test_sketch_roofline_covers_every_pass():
    # q = 2: one A Omega, q A^T W and q A W passes for the power scheme, plus Bt
    trace = {"a_omega": (0.6, 1), "at_w": (2.0, 3), "a_w": (1.2, 2), "cpqr": (9.0, 2)}
    r = bench.sketch_roofline(trace, CFG, PEAKS, "measured")
    assert r["passes_timed"] == 6 == 2 * CFG["q"] + 2
    assert r["achieved"] == pytest.approx(6 * 50000 * 20000 * 4 / 3.8e-3 / 1e9, rel=1e-12)
    assert set(r["per_class_ms"]) == {"a_omega", "at_w", "a_w"}


def test_step_flops_is_dominated_by_the_passes_over_a():
    m, n, k, p, q = 50000, 20000, 200, 20, 2
    passes = 2.0 * m * n * (k + p) * (2 * q + 2)
    f = bench.step_flops(m, n, k, p, q)
    assert passes < f < 1.1 * passes
    assert bench.step_flops(m, n, k, p, q, False, False) < f


def test_measured_peaks_and_traffic_files():
    peaks, kind = bench.load_peaks()
    assert kind == "measured" and peaks["hbm_gbs"] > 1000
    t = bench.load_traffic()
    for cls in ("a_omega", "at_w", "a_w", "cpqr"):
        assert t[(cls, "c2_f32_50000x20000")] > 1e9


def test_reference_arm_json_line_single_rank():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="", OMP_NUM_THREADS="2")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--config", "c1_f64_2000x1000"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1
    d = lines[0]
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2
    assert d["warmup"] == 1 and d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["cpu_baseline"]["cores"] >= 1 and "sample" in d["cpu_baseline"]


def test_pass_bounds_slower_of_hbm_and_issued_products():
    peaks = {"hbm_gbs": 6000.0, "bf16_tflops": 2000.0, "bf16_tflops_sustained": 1500.0}
    pb = bench.pass_bounds(CFG, peaks)
    m, n, lpad = 50000, 20000, 224                    # l = 220 rounded up to 16
    assert pb["a_w"]["hbm_ms"] == pytest.approx(m * n * 4 / 6000e9 * 1e3, rel=1e-12)
    # fp32 A, stored operand: a0 w0 + a1 w0 + a0 w1 at the sustained rate
    assert pb["a_w"]["tensor_ms"] == pytest.approx(3 * 2.0 * m * n * lpad / 1500e12 * 1e3,
                                                   rel=1e-12)
    assert pb["a_omega"]["tensor_ms"] == pytest.approx(pb["a_w"]["tensor_ms"] * 2 / 3, rel=1e-12)
    for c in ("a_omega", "a_w", "at_w"):
        b = pb[c]
        assert b["bound_ms"] == max(b["hbm_ms"], b["tensor_ms"])
        assert b["bound"] == ("hbm" if b["hbm_ms"] >= b["tensor_ms"] else "tensor")
    # bf16 storage halves the bytes and drops the a1 products
    pb16 = bench.pass_bounds(dict(CFG, dtype="bfloat16"), peaks)
    assert pb16["a_w"]["hbm_ms"] == pytest.approx(pb["a_w"]["hbm_ms"] / 2, rel=1e-12)
    assert pb16["a_w"]["tensor_ms"] == pytest.approx(pb["a_w"]["tensor_ms"] * 2 / 3, rel=1e-12)
    r = bench.sketch_roofline({"a_omega": (1.6, 1), "a_w": (1.7, 2), "at_w": (2.8, 3)}, CFG,
                              peaks, "measured")
    sb = r["slower_bound"]
    assert sb["frac"] == pytest.approx(
        (pb["a_omega"]["bound_ms"] + 2 * pb["a_w"]["bound_ms"] + 3 * pb["at_w"]["bound_ms"]) / 6.1,
        rel=1e-12)


def test_one_thread_oracle_timing_of_a_small_workload():
    r = bench.cpu_oracle_one_thread(("c1_f64_2000x1000",))["c1_f64_2000x1000"]
    assert "error" not in r, r
    assert r["workload"] == "c1_f64_2000x1000"
    assert 0 < r["qb_s"] < r["step_s"] and r["step_tflops"] > 0
