"""Serving engine (tn_server_*, needs a GPU: -m gpu).

Each job's out-sizes must be bit-identical whether it runs alone or in a mix
of concurrently admitted jobs, whether its batches come all at once (submit)
or one at a time while other jobs run (open + push), and identical to the
one-shot host entry point and (for the small jobs) to the CPU oracle.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2307_04890_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2307_04890_gb300 as tn
    from paper_2307_04890_gb300.build import build_library

    build_library()
    oracle.build_oracle()


def make_jobs(count, seed, n_range=(200, 6000), m_range=(1000, 80_000)):
    specs = synth.serving_jobs(count, rate=1000.0, n_range=n_range, m_range=m_range, seed=seed)
    jobs = []
    for spec in specs:
        u, v, t = synth.job_events(spec)
        parts = synth.split_batches(t, 4)
        offs = np.array([0] + [b for _, b in parts], dtype=np.uint64)
        jobs.append((spec["job"], spec["n"], u, v, t, offs))
    return jobs


def run(server, jobs, timeout=120.0):
    for jid, n, u, v, t, offs in jobs:
        server.submit(jid, n, u, v, t, offs)
    recs, deadline = [], time.time() + timeout
    while len(recs) < len(jobs) and time.time() < deadline:
        recs += server.poll(wait_ms=50)
    assert len(recs) == len(jobs), "jobs did not finish"
    return {r["job_id"]: r for r in recs}


def test_mix_equals_alone_and_one_shot():
    jobs = make_jobs(12, seed=5)
    with tn.Server(max_active=4) as srv:
        recs = run(srv, jobs)
        mix = dict(srv.results)
        st = srv.stats()
    assert all(r["status"] == 0 for r in recs.values())
    assert st["completed"] == len(jobs) and st["peak_active"] <= 4
    for jid, n, u, v, t, offs in jobs:
        alone_srv = tn.Server(max_active=1)
        run(alone_srv, [(jid, n, u, v, t, offs)])
        alone = alone_srv.results[jid]
        alone_srv.close()
        one_shot, am = tn.tn_out_component_sizes_host(u, v, t, n)
        assert np.array_equal(mix[jid][0], alone[0]), jid
        assert np.array_equal(mix[jid][0], one_shot), jid
        assert mix[jid][1] == alone[1] == am
        if n * len(u) <= 5e7:
            want = oracle.column_counts(oracle.component_matrix(u, v, t, n), n)
            assert np.array_equal(mix[jid][0], want), jid
        r = recs[jid]
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_done_ns"] and r["events"] == len(u)


def test_admission_respects_memory_budget():
    jobs = make_jobs(8, seed=9, n_range=(3000, 3000), m_range=(20_000, 20_000))
    # room for two of these jobs at a time (the charge of a job: its matrix,
    # sizes and 160 B per event of its largest batch)
    per_job = max(tn.tn_server_job_bytes(n, int(np.diff(offs).max())) for _, n, _, _, _, offs in jobs)
    n0 = 3000
    assert tn.tn_server_job_bytes(n0, 1000) == 3072 * tn.tn_row_words(n0) * 8 + n0 * 4 + 256 + 1000 * 160
    budget = int(2.5 * per_job)
    with tn.Server(memory_budget=budget, max_active=8) as srv:
        recs = run(srv, jobs)
        st = srv.stats()
        results = dict(srv.results)
    assert st["peak_bytes"] <= budget and st["peak_active"] <= 2
    for jid, n, u, v, t, offs in jobs:
        assert recs[jid]["status"] == 0
        assert np.array_equal(results[jid][0], tn.tn_out_component_sizes_host(u, v, t, n)[0])


def test_job_larger_than_budget_is_rejected():
    with tn.Server(memory_budget=1 << 20) as srv:
        n = 20_000
        u = np.zeros(10, np.uint32); v = np.ones(10, np.uint32); t = np.arange(10, dtype=np.int64)
        with pytest.raises(tn.TnError) as exc:
            srv.submit(1, n, u, v, t, [0, 10])
        assert exc.value.status == tn.TN_ENOMEM


def test_batch_order_violation_is_reported_and_isolated():
    good = make_jobs(3, seed=13)
    n = 500
    u, v, t = synth.uniform_events(n, 4000, t_range=4000, seed=2)
    # second batch starts before the first one ends: TN_EORDER for this job only
    t_bad = np.concatenate([t[:2000], t[:2000]])
    u_bad = np.concatenate([u[:2000], u[2000:]]); v_bad = np.concatenate([v[:2000], v[2000:]])
    with tn.Server(max_active=4) as srv:
        jobs = good + [(99, n, u_bad, v_bad, t_bad, np.array([0, 2000, 4000], np.uint64))]
        recs = run(srv, jobs)
        results = dict(srv.results)
    assert recs[99]["status"] == tn.TN_EORDER
    for jid, n_, uu, vv, tt, offs in good:
        assert recs[jid]["status"] == 0
        assert np.array_equal(results[jid][0], tn.tn_out_component_sizes_host(uu, vv, tt, n_)[0])


def test_out_of_range_endpoint_is_reported():
    with tn.Server() as srv:
        u = np.array([0, 5, 1], np.uint32); v = np.array([1, 2, 9], np.uint32); t = np.arange(3, dtype=np.int64)
        recs = run(srv, [(7, 6, u, v, t, np.array([0, 3], np.uint64))])
    assert recs[7]["status"] == tn.TN_ERANGE


def test_batches_that_split_timestamp_groups():
    """Batch boundaries inside timestamp groups (Section 2.1: a group is one
    snapshot): the job's online state holds a split group back until it is
    complete, so every group is applied whole: the out-sizes equal the
    one-shot call and the oracle.  One job has a single giant group spanning
    every batch."""
    jobs = []
    for jid, (n, m, t_range) in enumerate([(400, 6000, 60), (900, 12_000, 300), (300, 3000, 1)], start=50):
        u, v, t = synth.uniform_events(n, m, t_range=t_range, seed=jid)
        starts = np.flatnonzero(np.r_[True, t[1:] != t[:-1]])
        inside = np.setdiff1d(np.arange(1, m), starts)  # cut positions between equal timestamps
        cuts = np.sort(np.random.default_rng(jid).choice(inside, 5, replace=False))
        offs = np.r_[0, cuts, m].astype(np.uint64)
        jobs.append((jid, n, u, v, t, offs))
    with tn.Server(max_active=4) as srv:
        recs = run(srv, jobs)
        results = dict(srv.results)
    for jid, n, u, v, t, offs in jobs:
        assert recs[jid]["status"] == 0, jid
        assert np.array_equal(results[jid][0], tn.tn_out_component_sizes_host(u, v, t, n)[0]), jid
        want = oracle.column_counts(oracle.component_matrix(u, v, t, n), n)
        assert np.array_equal(results[jid][0], want), jid


def test_incremental_batches_while_other_jobs_run():
    """Jobs opened at staggered times receive their 4 batches one at a time,
    with pauses between them, while other jobs are resident: every job's
    out-sizes equal the one-shot call (and the oracle for small jobs), and
    the records show at least two jobs resident at the same time."""
    jobs = make_jobs(10, seed=21, n_range=(500, 8000), m_range=(20_000, 300_000))
    with tn.Server(max_active=6, workers=4) as srv:
        pending = []
        for jid, n, u, v, t, offs in jobs:
            srv.open(jid, n, int(np.diff(offs).max()))
            pending.append((jid, u, v, t, offs, 0))
        while pending:
            nxt = []
            for jid, u, v, t, offs, b in pending:
                a, e = int(offs[b]), int(offs[b + 1])
                srv.push(jid, u[a:e], v[a:e], t[a:e], last=b + 2 == len(offs))
                if b + 2 < len(offs):
                    nxt.append((jid, u, v, t, offs, b + 1))
            pending = nxt
            time.sleep(0.02)
        recs, deadline = [], time.time() + 120
        while len(recs) < len(jobs) and time.time() < deadline:
            recs += srv.poll(wait_ms=50)
        results = dict(srv.results)
        st = srv.stats()
    assert len(recs) == len(jobs)
    by_id = {r["job_id"]: r for r in recs}
    for jid, n, u, v, t, offs in jobs:
        r = by_id[jid]
        assert r["status"] == 0 and r["events"] == len(u)
        assert r["t_submit_ns"] <= r["t_admit_ns"] <= r["t_enqueued_ns"] <= r["t_done_ns"]
        assert r["t_last_push_ns"] <= r["t_enqueued_ns"]
        assert np.array_equal(results[jid][0], tn.tn_out_component_sizes_host(u, v, t, n)[0]), jid
        if n * len(u) <= 5e8:
            want = oracle.column_counts(oracle.component_matrix(u, v, t, n), n)
            assert np.array_equal(results[jid][0], want), jid
    # resident at once: admission-to-results intervals that overlap
    spans = sorted((r["t_admit_ns"], r["t_done_ns"]) for r in recs)
    most = max(sum(1 for a, b in spans if a <= s0 < b) for s0, _ in spans)
    assert most >= 2 and st["peak_active"] >= 2


def test_push_errors():
    with tn.Server(max_active=2) as srv:
        srv.open(1, 100, 10)
        u = np.zeros(11, np.uint32); v = np.ones(11, np.uint32); t = np.arange(11, dtype=np.int64)
        with pytest.raises(tn.TnError):
            srv.push(1, u, v, t)  # more events than the job's bound
        with pytest.raises(tn.TnError):
            srv.push(2, u[:3], v[:3], t[:3])  # never opened
        with pytest.raises(tn.TnError):
            srv.open(1, 100, 10)  # already open
        srv.push(1, u[:5], v[:5], t[:5])
        srv.push(1, u[5:10], v[5:10], t[5:10], last=True)
        with pytest.raises(tn.TnError):
            srv.push(1, u[:1], v[:1], t[:1] + 100)  # after the last batch
        recs, deadline = [], time.time() + 30
        while not recs and time.time() < deadline:
            recs += srv.poll(wait_ms=50)
        assert recs[0]["job_id"] == 1 and recs[0]["status"] == 0
        sizes = srv.results[1][0]
    assert np.array_equal(sizes, tn.tn_out_component_sizes_host(u[:10], v[:10], t[:10], 100)[0])
