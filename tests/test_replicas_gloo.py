"""The N > 1 path of the bench on CPU: two gloo ranks (no GPU).

With N ranks each GPU runs an independent replica (its own seeded matrix); the
only collectives are a barrier and the max over ranks of the timed region.
Whole-job throughput is all ranks' solves divided by the slowest rank's time.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    ms = 1000.0 * (rank + 1)             # rank 1 is the slow one
    ms_max = bench.max_over_ranks(ms, torch.device("cpu"), world)
    rate = bench.whole_job_rate(3, ms_max, world)
    A, d = bench.workload(64, rank, 0.1)
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump({"ms_max": ms_max, "rate": rate, "a00": float(A[0, 0]),
                   "d": sorted(map(float, d))[:3]}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r0 = json.load(open(tmp_path / "r0.json"))
    r1 = json.load(open(tmp_path / "r1.json"))
    # every rank sees the slowest rank's time, and 2 x 3 solves in 2 s
    assert r0["ms_max"] == r1["ms_max"] == 2000.0
    assert r0["rate"] == r1["rate"] == pytest.approx(3.0)
    # replicas solve different matrices (rank-seeded inputs)
    assert r0["a00"] != r1["a00"] and r0["d"] != r1["d"]


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1234.5, None, 1) == 1234.5
    assert bench.whole_job_rate(3, 1500.0, 1) == pytest.approx(2.0)


def test_reference_arm_prints_on_rank_0_only():
    """Under torchrun only rank 0 runs the oracle and prints the JSON line."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", PYTHONPATH=ROOT)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert p.returncode == 0 and p.stdout.strip() == ""


def test_reference_arm_json_line():
    """Rank 0 of the reference arm times the oracle on a bounded sample and
    prints one JSON line with the contract's keys (about 10-20 s of CPU)."""
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", PYTHONPATH=ROOT)
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    line = json.loads(p.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
