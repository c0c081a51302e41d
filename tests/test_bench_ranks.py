"""Host logic of bench.py's multi-GPU launch, on CPU with gloo (world size 2).

The path does not shard: every rank solves its own problem (replicas, seed
1002 + rank) and the job's time is the maximum over ranks.  No GPU is used.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["BENCH_ROOT"])
import torch.distributed as dist
import bench
rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
try:
    out = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 5.0], "cpu")
    print(json.dumps({"rank": rank, "out": out, "seed": bench.replica_seed(rank)}), flush=True)
finally:
    dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    env = dict(os.environ)
    env.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
               WORLD_SIZE=str(world), BENCH_ROOT=ROOT, CUDA_VISIBLE_DEVICES="")
    return env


def test_max_over_ranks_gloo_two_ranks():
    pytest.importorskip("torch")
    port = _free_port()
    procs = [subprocess.Popen([sys.executable, "-c", WORKER], env=_env(r, 2, port), stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = []
    for p in procs:
        try:
            o, e = p.communicate(timeout=180)
        except subprocess.TimeoutExpired:
            for q in procs:
                q.kill()
            raise
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    assert sorted(r["rank"] for r in outs) == [0, 1]
    for r in outs:
        assert r["out"] == [2.0, 10.0, 5.0]          # the slowest rank's value, element-wise
        assert r["seed"] == 1002 + r["rank"]          # independent problems


def test_max_over_ranks_without_group_is_identity():
    pytest.importorskip("torch")
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 1.5], "cpu") == [3.0, 1.5]


def test_reference_arm_runs_on_rank_zero_only():
    """Under a multi-rank launch the reference arm's other ranks exit 0 at once,
    without output and without running the oracle."""
    env = _env(1, 2, _free_port())
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_reference_arm_prints_one_contract_line_on_rank_zero():
    """Rank 0 times the CPU oracle on a bounded sample and prints one JSON line
    with the contract's keys, its cpu_baseline and a zero-copy e2e."""
    env = _env(0, 1, _free_port())
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1", "--cpu-sample-n", "256", "--cpu-sample-m", "64"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr
    lines = [l for l in p.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    r = json.loads(lines[0])
    assert r["impl"] == "reference" and r["unit"] == "ms" and r["higher_is_better"] is False
    assert r["n_gpus"] == 1 and r["steps"] == 2 and r["warmup"] == 1
    assert r["value"] > 0 and r["ms_per_step"] == r["value"]
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"] and "N=256" in cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert r["config"]["n_train"] == 32768 and r["config"]["n_test"] == 8192
