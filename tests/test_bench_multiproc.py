"""The N > 1 path of bench.py on CPU (gloo, world size 2).

Ranks run independent replicas of the workload (different seeds, no data-path
collective); the job's time is the slowest rank's (all-reduce MAX); under
torchrun only rank 0 of the reference arm prints its line.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    slowest = bench.job_max_ms(10.0 + 5.0 * rank, dist, "cpu")
    u, v, t = bench.make_events(bench.WORKLOADS["uniform-small"], rank)
    np.save(os.path.join(out_dir, f"u{rank}.npy"), u)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "seed": bench.replica_seed(bench.WORKLOADS["uniform-small"], rank)}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_distinct_replicas(tmp_path):
    import torch.multiprocessing as mp

    port = free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    r0 = json.load(open(tmp_path / "r0.json"))
    r1 = json.load(open(tmp_path / "r1.json"))
    assert r0["slowest"] == r1["slowest"] == 15.0
    assert r0["seed"] != r1["seed"]
    u0, u1 = np.load(tmp_path / "u0.npy"), np.load(tmp_path / "u1.npy")
    assert len(u0) == len(u1) and not np.array_equal(u0, u1)  # weak scaling: same size, own data


def test_reference_arm_prints_once_under_torchrun():
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "uniform-small", "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.5", "--gpus", "2"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_of_the_online_workload():
    """The online workload's reference arm times the oracle on a prefix and
    reports events/s, the unit of the online line."""
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "online", "--steps", "1",
           "--warmup", "0", "--cpu-seconds", "0.5"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    rec = json.loads([ln for ln in res.stdout.splitlines() if ln.startswith("{")][-1])
    assert rec["impl"] == "reference" and rec["unit"] == "events/s" and rec["value"] > 0
    assert rec["metric"].startswith("events/s through the online state")
    assert rec["cpu_baseline"]["kind"] == "oracle" and rec["e2e"]["unit"] == "events/s"
