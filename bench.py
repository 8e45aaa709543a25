#!/usr/bin/env python
"""Throughput of the exact component-matrix path on one GB300.

Workload (default): activity-driven temporal network, n = 100,000 nodes,
m = 10^7 events (power-law activity, exponent 2.1, a_min = 1e-3; uniform
partners; exponential gaps; microsecond ticks), seeded and synthetic.  One step
is one pass of the whole exact path over that batch, inputs resident in HBM:
validation + schedule (tn_plan_create), S <- I (tn_init_matrix), the
column-slab event stream (tn_plan_apply), out-sizes + largest out-component
(tn_out_sizes).  The metric is bit-updates/s = n * m / step time (also
reported as events/s).

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle (the
only reference this project has) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "events/s and bit-updates/s (n·m/time) at 1 GB300; achieved HBM GB/s vs peak"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "stream_kernel_activity_n1e5_m1e7.txt")
KERNEL_SOURCES = ["paper_2307_04890_gb300/csrc/tn_apply.cu", "paper_2307_04890_gb300/csrc/tn_internal.cuh"]

WORKLOADS = {
    "activity": dict(desc="activity-driven n=100000 m=10000000 (power-law activity 2.1, a_min 1e-3, us ticks)",
                     kind="activity", n=100_000, m=10_000_000, seed=2),
    "uniform-small": dict(desc="uniform pairs n=1000 m=20000, t uniform in [0,1e4)", kind="uniform",
                          n=1000, m=20_000, seed=1, t_range=10_000),
    "serving": dict(desc="serving: Poisson arrivals 200 req/s, n log-uniform [1e3,1e5], m log-uniform [1e4,1e7], "
                         "uniform endpoints, 4 incremental batches per job", kind="serving", n=0, m=0, seed=5),
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="activity")
    ap.add_argument("--window", type=int, default=0, help="events per scheduling window (0 = library default)")
    ap.add_argument("--slab", type=int, default=0, help="row words per CTA (0 = library default)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--jobs", type=int, default=200, help="serving: number of jobs")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean arrivals per second")
    ap.add_argument("--max-active", type=int, default=16, help="serving: jobs resident at once")
    return ap.parse_args()


def make_events(w, rank=0):
    from paper_2307_04890_gb300 import synth
    if w["kind"] == "activity":
        return synth.activity_driven(w["n"], w["m"], seed=w["seed"] + 1000 * rank)
    return synth.uniform_events(w["n"], w["m"], t_range=w["t_range"], seed=w["seed"] + 1000 * rank)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(workload_key):
    """DRAM bytes per launch of the stream kernel from the committed ncu summary,
    if it was taken on the current kernel source and this workload."""
    try:
        fields = {}
        with open(PROFILE_SUMMARY) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    fields[k.strip()] = v.strip()
        if fields.get("kernel_source_sha256_16") != kernel_source_sha():
            return None
        if fields.get("workload") != workload_key:
            return None
        return float(fields["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")
        self.gpu = gpu_index

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.gpu), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_sample(u, v, t, n, target_s):
    """Time the CPU oracle on a prefix of the workload (all n columns)."""
    import oracle
    oracle.build_oracle()
    probe = min(len(u), 20_000)
    t0 = time.perf_counter()
    oracle.component_matrix(u[:probe], v[:probe], t[:probe], n)
    dt = time.perf_counter() - t0
    ms = int(min(len(u), max(probe, probe * target_s / max(dt, 1e-6))))
    # end the sample at a timestamp-group boundary
    ms = int(np.searchsorted(t, t[ms - 1], side="right")) if ms < len(u) else ms
    t0 = time.perf_counter()
    oracle.component_matrix(u[:ms], v[:ms], t[:ms], n)
    dt = time.perf_counter() - t0
    return ms, dt


def run_reference_serving(args, w, world):
    """The oracle on whole jobs of the serving stream, in arrival order, until
    about --cpu-seconds of CPU time: events/s of the sample."""
    import oracle
    from paper_2307_04890_gb300 import synth
    oracle.build_oracle()
    specs = synth.serving_jobs(args.jobs, rate=args.rate, seed=w["seed"])
    done_events, spent, jobs_done = 0, 0.0, 0
    for spec in specs:
        if spent >= args.cpu_seconds:
            break
        if spec["n"] * spec["m"] > 2e11:  # one job alone would exceed the sample budget
            continue
        u, v, t = synth.job_events(spec)
        t0 = time.perf_counter()
        oracle.column_counts(oracle.component_matrix(u, v, t, spec["n"]), spec["n"])
        spent += time.perf_counter() - t0
        done_events += len(u)
        jobs_done += 1
    value = done_events / max(spent, 1e-9)
    sample = f"{jobs_done} whole jobs of the stream (n*m <= 2e11), one thread, {spent:.1f} s"
    line = {"impl": "reference", "metric": METRIC + " (serving)", "value": value, "unit": "events/s",
            "n_gpus": world, "steps": jobs_done, "warmup": 0, "ms_per_step": spent * 1e3 / max(jobs_done, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": w["desc"], "jobs": jobs_done},
            "cpu_baseline": {"value": value, "unit": "events/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args, w, rank, world):
    if rank != 0:
        return
    if w["kind"] == "serving":
        run_reference_serving(args, w, world)
        return
    u, v, t = make_events(w)
    n = w["n"]
    times, ms = [], 0
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup) * 2)
    for i in range(args.warmup + args.steps):
        ms, dt = cpu_oracle_sample(u, v, t, n, per_step)
        if i >= args.warmup:
            times.append(dt)
    mean = sum(times) / len(times)
    value = n * ms / mean
    sample = f"first {ms} of {w['m']} events (group boundary), all {n} columns, one thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "bit-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": w["desc"], "n": n, "m": w["m"]},
            "events_per_s": ms / mean,
            "cpu_baseline": {"value": value, "unit": "bit-updates/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "bit-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_serving(args, w, rank, world, local_rank):
    """Continuous admission of a Poisson stream of jobs through tn_server_*.
    Latency = submit -> out-sizes on the host; throughput = all events (and
    n * m bit-updates) of all jobs / wall time from the first submit to the
    last result."""
    import torch
    import paper_2307_04890_gb300 as tn
    from paper_2307_04890_gb300 import synth
    from paper_2307_04890_gb300.build import build_library

    build_library()
    tn.load_library()
    torch.cuda.set_device(local_rank)
    specs = synth.serving_jobs(args.jobs, rate=args.rate, seed=w["seed"] + 1000 * rank)
    jobs = []
    for spec in specs:
        u, v, t = synth.job_events(spec)
        offs = np.array([0] + [b for _, b in synth.split_batches(t, 4)], dtype=np.uint64)
        jobs.append((spec, u, v, t, offs))
    # warm-up: the first jobs once, unmeasured
    with tn.Server(max_active=args.max_active) as srv:
        for spec, u, v, t, offs in jobs[: max(3, args.warmup)]:
            srv.submit(spec["job"], spec["n"], u, v, t, offs)
        got = 0
        while got < min(len(jobs), max(3, args.warmup)):
            got += len(srv.poll(wait_ms=100))
    srv = tn.Server(max_active=args.max_active)
    recs = []
    with ClockSampler(torch.cuda.current_device()) as clocks:
        t0 = time.perf_counter()
        for spec, u, v, t, offs in jobs:
            delay = t0 + spec["arrival"] - time.perf_counter()
            if delay > 0:
                recs += srv.poll(wait_ms=0)
                time.sleep(max(0.0, t0 + spec["arrival"] - time.perf_counter()))
            srv.submit(spec["job"], spec["n"], u, v, t, offs)
        while len(recs) < len(jobs):
            recs += srv.poll(wait_ms=100)
        wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    bad = [r for r in recs if r["status"] != 0]
    lat = np.array([(r["t_done_ns"] - r["t_submit_ns"]) / 1e6 for r in recs])
    queue = np.array([(r["t_admit_ns"] - r["t_submit_ns"]) / 1e6 for r in sorted(recs, key=lambda r: r["t_submit_ns"])])
    q = max(1, len(queue) // 4)
    events = sum(len(j[1]) for j in jobs)
    bit_updates = sum(j[0]["n"] * len(j[1]) for j in jobs)
    result = {"metric": METRIC + " (serving)", "value": events / wall, "unit": "events/s", "n_gpus": world,
              "steps": len(jobs), "warmup": max(3, args.warmup), "ms_per_step": wall * 1e3 / len(jobs),
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
              "config": {"workload": w["desc"], "jobs": len(jobs), "rate_per_s": args.rate,
                         "max_active": args.max_active, "l2": "per-job matrices up to 1.25 GB; jobs overlap"},
              "bit_updates_per_s": bit_updates / wall,
              "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                             "mean": float(lat.mean()), "max": float(lat.max())},
              "queue_delay_ms": {"first_quarter_median": float(np.median(queue[:q])),
                                 "last_quarter_median": float(np.median(queue[-q:]))},
              "offered_events_per_s": events / max(specs[-1]["arrival"], 1e-9),
              "server": st, "failed_jobs": len(bad), "clocks": clocks.summary(),
              "e2e": {"value": events / wall, "unit": "events/s",
                      "h2d_bytes_per_step": events * 16 / len(jobs),
                      "d2h_bytes_per_step": sum(j[0]["n"] * 4 + 4 for j in jobs) / len(jobs)}}
    if rank == 0:
        print(json.dumps(result), flush=True)


def main():
    args = parse_args()
    w = WORKLOADS[args.workload]
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if w["kind"] == "serving" and args.impl == "ours":
        run_serving(args, w, rank, world, local_rank)
        return
    if args.impl == "reference":
        run_reference(args, w, rank, world)
        return

    import torch
    import paper_2307_04890_gb300 as tn
    from paper_2307_04890_gb300.build import build_library

    build_library()
    tn.load_library()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    n, m = w["n"], w["m"]
    u, v, t = make_events(w, rank)
    du = torch.from_numpy(u.view(np.int32)).to(dev)
    dv = torch.from_numpy(v.view(np.int32)).to(dev)
    dt = torch.from_numpy(t).to(dev)
    W = tn.tn_row_words(n)
    S = torch.empty((n, W), dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    k1_events = []

    def step(record):
        plan = tn.Plan(du, dv, dt, n, window_events=args.window, slab_words=args.slab)  # a1
        tn.tn_init_matrix(S, n)                                                          # a2
        if record:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        plan.apply(S)                                                                    # a3
        if record:
            e1.record(stream)
            k1_events.append((e0, e1))
        out, _, am = tn.tn_out_sizes(S, n, n, argmax=True)                               # a4
        stats = plan.stats()
        plan.destroy()
        return out, am, stats

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches0 = tn.tn_kernel_launches()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clocks:
        torch.cuda.synchronize()
        start.record(stream)
        for _ in range(args.steps):
            out, am, stats = step(True)
        end.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = tn.tn_kernel_launches() - launches0
    ms_total = start.elapsed_time(end)
    if dist:
        tt = torch.tensor([ms_total], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_total = float(tt.item())
    ms_step = ms_total / args.steps
    k1_ms = sum(a.elapsed_time(b) for a, b in k1_events) / len(k1_events)
    value = world * n * m / (ms_step * 1e-3)

    # roofline of the dominant kernel (the column-slab stream)
    words = (n + 63) // 64
    alg_bytes = m * 4 * words * 8
    achieved = alg_bytes / (k1_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()
    traffic = profiled_traffic(args.workload)
    roofline = {"bound": "hbm", "kernel": "stream_kernel", "achieved": achieved, "peak": peak,
                "peak_source": f"{peak_kind} MEASURED_PEAKS hbm_gbs" if peak_kind == "measured" else "fallback",
                "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": k1_ms}

    result = {"metric": METRIC, "value": value, "unit": "bit-updates/s", "n_gpus": world, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "u64", "data": "synthetic",
              "config": {"workload": w["desc"], "n": n, "m": m, "global_batch": m * world,
                         "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                         "l2": "inputs larger than L2 (S %.2f GB, events %.0f MB)" % (n * W * 8 / 1e9, m * 16 / 1e6),
                         "window_events": args.window or 640, "slab_words": args.slab or 16,
                         "levels": stats["levels"], "ops": stats["ops"]},
              "events_per_s": world * m / (ms_step * 1e-3),
              "roofline": roofline, "gpu_launches": launches, "clocks": clocks.summary(),
              "largest_out_component": {"node": int(am.item()), "size": int(out.max().item())}}

    if rank == 0 and not args.no_e2e:
        # end to end through the host-buffer C-ABI call, pinned inputs
        hu = torch.from_numpy(u.view(np.int32)).pin_memory()
        hv = torch.from_numpy(v.view(np.int32)).pin_memory()
        ht = torch.from_numpy(t).pin_memory()
        hout = torch.empty(n, dtype=torch.int32).pin_memory()
        ham = torch.empty(1, dtype=torch.int32).pin_memory()
        for i in range(args.warmup + args.steps):
            if i == args.warmup:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            tn.tn_out_component_sizes_host_ptrs(hu.data_ptr(), hv.data_ptr(), ht.data_ptr(), m, n,
                                                hout.data_ptr(), ham.data_ptr())
        e2e_s = (time.perf_counter() - t0) / args.steps
        assert np.array_equal(hout.numpy(), out.cpu().numpy()), "host entry point disagrees with device path"
        result["e2e"] = {"value": n * m / e2e_s, "unit": "bit-updates/s", "h2d_bytes_per_step": m * 16,
                         "d2h_bytes_per_step": n * 4 + 4, "ms_per_step": e2e_s * 1e3}

    if rank == 0 and not args.no_cpu_baseline:
        ms, sec = cpu_oracle_sample(u, v, t, n, args.cpu_seconds)
        result["cpu_baseline"] = {"value": n * ms / sec, "unit": "bit-updates/s", "cores": 1, "kind": "oracle",
                                  "sample": f"first {ms} of {m} events (group boundary), all {n} columns, "
                                            f"one thread, {sec:.1f} s"}
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
