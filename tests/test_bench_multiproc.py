"""The N > 1 paths of bench.py on CPU (gloo, world size 2).

The exact workloads split the source columns over the ranks (columns never
interact, Section 3.1): every rank streams all events over its own block of
columns and the out-sizes are all-gathered, with the largest out-component
taken over the gathered sizes.  The hashed workload deals its R replicas over
the ranks, broadcasts every proxy matrix to every rank (the fusion intersects
all replicas, Section 4.2) and splits the sampled sources; estimates and exact
sizes are all-gathered.  Here each rank computes its share with the oracle and
runs bench.py's exchange steps.  The online workload runs independent
replicas (different seeds); the job's time is the slowest rank's (all-reduce
MAX); under torchrun only rank 0 of the reference arm prints its line.
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


def _split_rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    w = bench.WORKLOADS["uniform-small"]
    u, v, t = bench.make_events(w)  # the same events on every rank
    n = w["n"]
    c0, c1 = bench.column_range(n, rank, world)
    S = oracle.component_matrix(u, v, t, n, src=np.arange(c0, c1, dtype=np.uint32))
    counts = oracle.column_counts(S, c1 - c0)
    local = torch.from_numpy(counts.astype(np.int32))
    full, am = bench.gather_sizes(local, oracle.argmax(counts), n, rank, world, dist)
    np.save(os.path.join(out_dir, f"sizes{rank}.npy"), full.numpy())
    with open(os.path.join(out_dir, f"split{rank}.json"), "w") as f:
        json.dump({"argmax": am, "c0": c0, "c1": c1}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_column_split_gathers_the_whole_matrix_sizes(tmp_path, world):
    """n = 1,000, m = 20,000 (the uniform small workload): the gathered sizes
    and the argmax equal the oracle's on the whole matrix, on every rank."""
    import torch.multiprocessing as mp
    import oracle

    port = free_port()
    mp.start_processes(_split_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    sys.path.insert(0, ROOT)
    import bench
    w = bench.WORKLOADS["uniform-small"]
    u, v, t = bench.make_events(w)
    want = oracle.column_counts(oracle.component_matrix(u, v, t, w["n"]), w["n"])
    blocks = []
    for r in range(world):
        rec = json.load(open(tmp_path / f"split{r}.json"))
        assert np.array_equal(np.load(tmp_path / f"sizes{r}.npy").view(np.uint32), want)
        assert rec["argmax"] == oracle.argmax(want)
        blocks.append((rec["c0"], rec["c1"]))
    assert blocks[0][0] == 0 and blocks[-1][1] == w["n"]
    assert all(a[1] == b[0] and a[0] < a[1] for a, b in zip(blocks, blocks[1:]))


def _tie_rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    # n = 6 over 2 ranks: sizes [2, 7, 7 | 7, 1, 7]; every rank's own largest is
    # its first 7, the whole matrix's is node 1
    local = torch.tensor([[2, 7, 7], [7, 1, 7]][rank], dtype=torch.int32)
    full, am = bench.gather_sizes(local, [1, 0][rank], 6, rank, world, dist)
    with open(os.path.join(out_dir, f"tie{rank}.json"), "w") as f:
        json.dump({"argmax": am, "sizes": full.tolist()}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_gather_breaks_size_ties_by_lowest_id(tmp_path):
    import torch.multiprocessing as mp

    port = free_port()
    mp.start_processes(_tie_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        rec = json.load(open(tmp_path / f"tie{r}.json"))
        assert rec["argmax"] == 1 and rec["sizes"] == [2, 7, 7, 7, 1, 7]


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


def test_reference_arm_of_the_er_small_workload():
    """The ER n = 10^4 workload (the resident-slab form's bench line) has a
    reference arm: the oracle over seeded column blocks of the same events."""
    cmd = [sys.executable, "bench.py", "--impl", "reference", "--workload", "er-small", "--steps", "1",
           "--warmup", "0", "--cpu-seconds", "0.5"]
    res = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stderr[-2000:]
    rec = json.loads([ln for ln in res.stdout.splitlines() if ln.startswith("{")][-1])
    assert rec["impl"] == "reference" and rec["unit"] == "bit-updates/s" and rec["value"] > 0
    assert rec["config"]["n"] == 10_000 and rec["config"]["m"] == 10_000_000
    assert rec["cpu_baseline"]["kind"] == "oracle"


def _hashed_rank_main(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    import oracle
    from paper_2307_04890_gb300 import synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    n, m, k, R, seed, nsrc = 2000, 20_000, 97, 5, 3, 301
    u, v, t = synth.uniform_events(n, m, t_range=8000, seed=21)  # the same events on every rank
    src = np.sort(np.random.default_rng(4).choice(n, nsrc, replace=False)).astype(np.uint32)
    H = oracle.hash_nodes(seed, R, k, n)  # every rank hashes with all R replicas
    W = (k + 63) // 64
    P = torch.zeros((R, k, W), dtype=torch.int64)
    for j in range(R):  # this rank builds the replicas it owns
        if bench.replica_owner(j, world) == rank:
            P[j] = torch.from_numpy(oracle.proxy_matrices(u, v, t, H[j:j + 1], k)[0].view(np.int64))
    bench.share_proxies(P, R, world, dist)
    s0, s1 = bench.column_range(nsrc, rank, world)
    Pn = P.numpy().view(np.uint64)
    est = torch.from_numpy(oracle.hash_estimate(Pn, H, n, src[s0:s1]).view(np.int32))
    exact = torch.from_numpy(oracle.column_counts(oracle.component_matrix(u, v, t, n, src[s0:s1]),
                                                  s1 - s0).view(np.int32))
    est = bench.gather_blocks(est, nsrc, rank, world, dist)
    exact = bench.gather_blocks(exact, nsrc, rank, world, dist)
    np.save(os.path.join(out_dir, f"P{rank}.npy"), Pn)
    np.save(os.path.join(out_dir, f"est{rank}.npy"), est.numpy().view(np.uint32))
    np.save(os.path.join(out_dir, f"exact{rank}.npy"), exact.numpy().view(np.uint32))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_hashed_split_equals_the_whole_job(tmp_path, world):
    """R = 5 replicas dealt over 2 or 3 ranks (uneven), 301 sampled sources
    split: after the broadcasts every rank holds all R proxy matrices, and the
    gathered estimates and exact sizes equal the single-process oracle's."""
    import torch.multiprocessing as mp
    import oracle
    from paper_2307_04890_gb300 import synth

    port = free_port()
    mp.start_processes(_hashed_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    n, m, k, R, seed, nsrc = 2000, 20_000, 97, 5, 3, 301
    u, v, t = synth.uniform_events(n, m, t_range=8000, seed=21)
    src = np.sort(np.random.default_rng(4).choice(n, nsrc, replace=False)).astype(np.uint32)
    H = oracle.hash_nodes(seed, R, k, n)
    Pref = oracle.proxy_matrices(u, v, t, H, k)
    want_est = oracle.hash_estimate(Pref, H, n, src)
    want_exact = oracle.column_counts(oracle.component_matrix(u, v, t, n, src), nsrc)
    assert (want_est >= want_exact).all() and (want_est > want_exact).any()  # a non-trivial estimate
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"P{r}.npy"), Pref)
        assert np.array_equal(np.load(tmp_path / f"est{r}.npy"), want_est)
        assert np.array_equal(np.load(tmp_path / f"exact{r}.npy"), want_exact)
