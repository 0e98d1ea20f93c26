"""The multi-rank (N > 1) host logic of bench.py on CPU, as world_size-2 gloo ranks.

The path does not shard: every rank runs an independent replica of the step
on its own GPU, and the only exchanges are the barrier around the timed region
and the max over ranks of the step time.  These tests launch two ranks with
torch.distributed.run on 127.0.0.1, as the multi-GPU launch does, and check
those exchanges and the whole-job aggregation; no GPU is touched.
"""
import json
import os
import socket
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
if not dist.is_available() or not dist.is_gloo_available():
    pytest.skip("torch.distributed without gloo", allow_module_level=True)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _torchrun(args, timeout=240):
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    env["OMP_NUM_THREADS"] = "2"
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port())] + args
    return subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True,
                          timeout=timeout)


WORKER = textwrap.dedent("""
    import json, os, sys
    sys.path.insert(0, %r)
    import bench
    world, rank, local = bench.dist_setup()
    bench.barrier(world)
    # rank r took (3 + 2 r) ms per step on its replica of a 6e9-flop step
    ms, value = bench.whole_job(6e9, 3.0 + 2.0 * rank, world, "cpu")
    mx = bench.max_over_ranks(float(10 - rank), world, "cpu")
    bench.barrier(world)
    with open(os.path.join(%r, "rank%%d.json" %% rank), "w") as f:
        json.dump({"rank": rank, "world": world, "local": local, "ms": ms, "value": value,
                   "mx": mx}, f)
    import torch.distributed as dist
    dist.destroy_process_group()
""")


def test_barrier_max_and_whole_job_value_two_ranks(tmp_path):
    script = tmp_path / "worker.py"
    script.write_text(WORKER % (ROOT, str(tmp_path)))
    r = _torchrun([str(script)])
    assert r.returncode == 0, r.stderr[-2000:]
    res = [json.loads((tmp_path / ("rank%d.json" % i)).read_text()) for i in range(2)]
    assert sorted(x["rank"] for x in res) == [0, 1]
    for x in res:
        assert x["world"] == 2 and x["local"] == x["rank"]
        # both ranks see the slowest rank's time ...
        assert x["ms"] == 5.0 and x["mx"] == 10.0
        # ... and the whole job's throughput: 2 replicas x 6e9 flop in 5 ms
        assert x["value"] == pytest.approx(2 * 6e9 / 5e-3 / 1e12, rel=1e-12)


def test_whole_job_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    ms, value = bench.whole_job(4e9, 2.0, 1, "cpu")
    assert ms == 2.0 and value == pytest.approx(4e9 / 2e-3 / 1e12, rel=1e-12)
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5


def test_reference_arm_two_ranks_rank0_alone_prints():
    """bench.py --impl reference under a 2-rank launch: rank 0 times the oracle
    on a bounded sample and prints one JSON line; rank 1 exits 0 without work."""
    r = _torchrun(["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                   "--warmup", "0", "--config", "c1_f64_2000x1000"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(s) for s in r.stdout.splitlines() if s.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["steps"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["workload"] == "c1_f64_2000x1000"
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
