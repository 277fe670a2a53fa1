"""Host logic of the benchmark's multi-rank launch (one process per GPU, replicas of the solve),
run here as two gloo ranks on the CPU: the rank environment, the max-over-ranks timing, and the
reference arm doing its work on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["REPO_ROOT"])
import torch.distributed as dist
import bench
ws, rank, local = bench.dist_env()
dist.init_process_group("gloo", rank=rank, world_size=ws)
t = bench.max_over_ranks(10.0 + 5.0 * rank, ws)
dist.barrier()
print(json.dumps({"rank": rank, "ws": ws, "local": local, "max": t}))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, ws, port):
    env = dict(os.environ)
    env.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
               LOCAL_RANK=str(rank), REPO_ROOT=ROOT)
    return env


def test_max_over_ranks_with_two_gloo_ranks():
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", WORKER], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["ws"] == 2 and o["local"] == o["rank"]
        assert o["max"] == 15.0  # every rank reports the slowest replica


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_reference_arm_runs_on_rank_zero_only():
    # a non-zero rank of the reference arm exits 0 at once and prints nothing
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=_env(1, 2, _free_port()), capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line():
    """Rank 0 of a one-process launch prints one JSON line with the contract's keys; its value, the
    CPU baseline's and the end-to-end figure are the same estimated oracle time per solve, the step
    time is the sample's own time, the config is the GPU arm's, and the sample is extrapolated to
    the workload's own iteration count (small workload)."""
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "0", "--workload", "grid10x10x5_k4"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 0
    assert d["higher_is_better"] is False and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"] == "grid10x10x5_k4"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["estimated"] is True
    assert d["iterations_assumed"] == 26
    sys.path.insert(0, ROOT)
    import bench
    from paper_1401_7227_gb300 import synth
    w = synth.WORKLOADS["grid10x10x5_k4"]
    assert d["config"] == json.loads(json.dumps(bench.workload_config(w, synth.make(w), "fp32")))
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["unit"] == d["unit"] and cb["cores"] >= 1
    assert cb["sample"]
    e = d["e2e"]
    assert e == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
