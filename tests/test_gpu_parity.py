"""Parity of the CUDA path with the CPU oracle (needs a GPU: -m gpu).

Integer work throughout, so every comparison is bit-exact: the full component
matrix (including zero padding), out- and in-sizes, argmax, hash tables,
super-events and fused estimates.  Large configurations are checked on seeded
column samples that the oracle computes exactly (columns are independent).
"""
import numpy as np
import pytest

import oracle
from conftest import golden_names, load_golden
from paper_2307_04890_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2307_04890_gb300 as tn
    from paper_2307_04890_gb300.build import build_library

    build_library()
    oracle.build_oracle()


def dev_events(u, v, t):
    d = torch.device("cuda")
    return (torch.from_numpy(np.ascontiguousarray(u, np.uint32).view(np.int32)).to(d),
            torch.from_numpy(np.ascontiguousarray(v, np.uint32).view(np.int32)).to(d),
            torch.from_numpy(np.ascontiguousarray(t, np.int64)).to(d))


def host_matrix(S, ncols):
    """GPU matrix -> uint64 [rows, ceil(ncols/64)], asserting zero padding."""
    a = S.cpu().numpy().view(np.uint64)
    w = (ncols + 63) // 64
    assert not a[:, w:].any(), "padding words must stay zero"
    if ncols % 64:
        assert not (a[:, w - 1] >> np.uint64(ncols % 64)).any(), "padding bits must stay zero"
    return a[:, :w]


def gpu_matrix(u, v, t, n, **kw):
    du, dv, dt = dev_events(u, v, t)
    S = tn.tn_component_matrix(du, dv, dt, n, **kw)
    torch.cuda.synchronize()
    return host_matrix(S, n)


def u32(x):
    return x.cpu().numpy().view(np.uint32)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", golden_names())
def test_golden(name):
    n, events, oc, rows = load_golden(name)
    ev = np.array(events, np.int64).reshape(-1, 3)
    u, v, t = ev[:, 0].astype(np.uint32), ev[:, 1].astype(np.uint32), ev[:, 2]
    B = oracle.to_bool(gpu_matrix(u, v, t, n), n)
    for j, want in oc.items():
        assert sorted(np.flatnonzero(B[:, j]).tolist()) == want
    for i, want in rows.items():
        assert sorted(np.flatnonzero(B[i]).tolist()) == want


@pytest.mark.parametrize("seed", range(40))
def test_fuzz_dense_ties(seed):
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(1, 71))
    m = int(rng.integers(1, 301))
    u = rng.integers(0, n, m).astype(np.uint32)
    v = rng.integers(0, n, m).astype(np.uint32)
    t = np.sort(rng.integers(0, int(rng.integers(1, 12)), m))
    win = int(rng.choice([32, 64, 2048]))
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, window_events=win, slab_words=int(rng.choice([2, 4, 8, 16])),
                   smem_rows=int(rng.choice([0, 1, 64])))
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    plan.apply(S, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


def test_config1_full():
    """n=1000, m=20000, uniform pairs, t uniform in [0, 1e4) (dense ties)."""
    n = 1000
    u, v, t = synth.uniform_events(n, 20000, t_range=10**4, seed=1)
    du, dv, dt = dev_events(u, v, t)
    S = tn.tn_component_matrix(du, dv, dt, n)
    out, ins, am = tn.tn_out_sizes(S, n, n, in_sizes=True, argmax=True)
    torch.cuda.synchronize()
    ref = oracle.component_matrix(u, v, t, n)
    assert np.array_equal(host_matrix(S, n), ref)
    want = oracle.column_counts(ref, n)
    assert np.array_equal(u32(out), want)
    assert np.array_equal(u32(ins), oracle.row_counts(ref))
    assert int(am.item()) == oracle.argmax(want)
    B = oracle.to_bool(ref, n)
    for j in np.random.default_rng(0).choice(n, 25, replace=False):  # brute-force SI
        assert np.array_equal(B[:, j], oracle.si_reach(u, v, t, n, int(j)))


@pytest.mark.parametrize("slab", [2, 4, 6, 8, 10, 12, 14, 16])
@pytest.mark.parametrize("window", [40, 700, 4096])
def test_schedule_options_identical(slab, window):
    n = 1500  # several slabs, ragged last slab, several windows, ragged last window
    u, v, t = synth.uniform_events(n, 31_001, t_range=12_000, seed=3)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, window_events=window, slab_words=slab)
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    plan.apply(S, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


@pytest.mark.parametrize("slab", [16, 12])
@pytest.mark.parametrize("smem_rows", [1, 0, 600])
def test_local_and_global_windows_identical(smem_rows, slab):
    """smem_rows=1 sends every window through the global-memory path; the
    default and a large buffer apply most windows in shared memory."""
    n = 5000
    u, v, t = synth.uniform_events(n, 60_000, t_range=25_000, seed=14)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, window_events=300, slab_words=slab, smem_rows=smem_rows)
    st = plan.stats()
    if smem_rows == 1:
        assert st["local_windows"] == 0
    else:
        assert st["local_windows"] > 0
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    plan.apply(S, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


@pytest.mark.parametrize("slab", [18, 26, 40, 52, 64])
@pytest.mark.parametrize("smem_rows", [1, 0])
def test_wide_slabs_identical(slab, smem_rows):
    """Slabs wider than 16 words (up to 512-byte row segments) with the 192 KB
    row buffer: three or more CTAs per row, the last one ragged (141 row words,
    stride 144), through the direct global-memory path (smem_rows=1: a buffer
    too small for the ring) and through shared-memory records (default)."""
    n = 9000
    u, v, t = synth.uniform_events(n, 60_000, t_range=20_000, seed=21)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, window_events=200, slab_words=slab, smem_rows=smem_rows)
    st = plan.stats()
    assert (st["local_windows"] == 0) == (smem_rows == 1)
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    plan.apply(S, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


@pytest.mark.parametrize("slab", [16, 26, 52])
def test_bursty_big_windows_global_ring(slab):
    """Power-law degrees and Pareto gaps rounded to seconds (tie groups of
    about 120 events, hub nodes), in windows of 3,000 events: a window touches
    more rows than the row buffer holds, so it streams from global memory
    through the per-thread ring of copies (the buffer holds at least 16 slots
    per row group: 1,280 >= 16 * 48 at 16 words, 945 >= 16 * 29 at 26 words,
    472 >= 16 * 14 at 52 words), then applies the hub PULLs."""
    n = 20_000
    u, v, t = synth.powerlaw_bursty(n, 400_000, seed=9)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, window_events=3000, slab_words=slab)
    st = plan.stats()
    assert st["local_windows"] * 10 <= st["windows"] and st["aux"] > 0
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    plan.apply(S, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


@pytest.mark.parametrize("slab,wave", [(64, 5), (26, 7), (64, 152), (16, 3), (128, 2)])
@pytest.mark.parametrize("window,smem_rows", [(3000, 0), (200, 0)])
def test_wave_ctas_identical(slab, wave, window, smem_rows):
    """A matrix spread over a given number of CTAs of two widths (141 row
    words, stride 144): 64/5 -> 4 x 32 + 1 x 16 words, 26/7 -> 2 x 22 + 5 x 20,
    64/152 -> 72 x 2 (fewer 16-word units than CTAs), 16/3 -> 9 x 16 (raised
    to the slab count), 128/2 -> 1 x 80 + 1 x 64 -- through global windows
    (3,000 events) and shared-memory records (200)."""
    n = 9000
    u, v, t = synth.uniform_events(n, 60_000, t_range=20_000, seed=22)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, window_events=window, slab_words=slab, smem_rows=smem_rows, wave_ctas=wave)
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    plan.apply(S, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


def test_slab_width_limits():
    u, v, t = synth.uniform_events(100, 1000, t_range=500, seed=2)
    du, dv, dt = dev_events(u, v, t)
    for bad in (130, 129, 17):
        with pytest.raises(tn.TnError):
            tn.Plan(du, dv, dt, 100, slab_words=bad)
    with pytest.raises(tn.TnError):  # a row buffer above 192 KB
        tn.Plan(du, dv, dt, 100, slab_words=64, smem_rows=385)
    tn.Plan(du, dv, dt, 100, slab_words=64, smem_rows=384).destroy()


def test_carry_across_empty_window():
    """A tie group that spans a nominal window boundary leaves an empty window
    between two local records that share rows."""
    rng = np.random.default_rng(15)
    n = 40
    t = np.concatenate([np.arange(60), np.full(70, 60), 61 + np.arange(200)]).astype(np.int64)
    u = rng.integers(0, n, len(t)).astype(np.uint32)
    v = rng.integers(0, n, len(t)).astype(np.uint32)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, window_events=64, slab_words=16)
    st = plan.stats()
    assert st["local_windows"] >= 2 and st["items"] < st["windows"]  # some window is empty
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    plan.apply(S, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


def test_activity_driven_medium():
    n = 3000
    u, v, t = synth.activity_driven(n, 200_000, seed=4)
    assert np.array_equal(gpu_matrix(u, v, t, n), oracle.component_matrix(u, v, t, n))


def test_bursty_medium_big_groups():
    """Power-law + Pareto times rounded to seconds: large tie groups with hubs."""
    n = 20_000
    u, v, t = synth.powerlaw_bursty(n, 150_000, seed=5)
    ref = oracle.component_matrix(u, v, t, n, src=np.arange(0, n, 37, dtype=np.uint32))
    du, dv, dt = dev_events(u, v, t)
    src = torch.arange(0, n, 37, dtype=torch.int32, device="cuda")
    S = tn.tn_component_columns(du, dv, dt, n, src)
    torch.cuda.synchronize()
    assert np.array_equal(host_matrix(S, src.numel()), ref)


def test_single_giant_group():
    """All events share one timestamp: the window exceeds the shared-memory
    scheduler and takes the large-window path; S = I + adjacency."""
    n, m = 3000, 20_000
    rng = np.random.default_rng(6)
    u = rng.integers(0, n, m).astype(np.uint32)
    v = rng.integers(0, n, m).astype(np.uint32)
    t = np.full(m, 7, np.int64)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n)
    assert plan.stats()["big_windows"] >= 1
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    plan.apply(S, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


def test_mixed_giant_and_small_groups():
    rng = np.random.default_rng(8)
    n = 2000
    parts = []
    for g in range(30):
        size = int(rng.choice([1, 2, 5, 9000 if g in (7, 21) else 40]))
        parts.append((rng.integers(0, n, size), rng.integers(0, n, size), np.full(size, g)))
    u = np.concatenate([p[0] for p in parts]).astype(np.uint32)
    v = np.concatenate([p[1] for p in parts]).astype(np.uint32)
    t = np.concatenate([p[2] for p in parts]).astype(np.int64)
    assert np.array_equal(gpu_matrix(u, v, t, n), oracle.component_matrix(u, v, t, n))


def test_self_loops_only_and_empty():
    n = 100
    u = np.arange(50, dtype=np.uint32)
    assert np.array_equal(gpu_matrix(u, u, np.arange(50), n), oracle.init_sources(n)[:, :2])
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    tn.tn_component_matrix(e, e, torch.empty(0, dtype=torch.int64, device="cuda"), n, S=S)
    torch.cuda.synchronize()
    assert np.array_equal(host_matrix(S, n), oracle.init_sources(n))


def test_incremental_batches_with_t_last():
    n = 800
    u, v, t = synth.uniform_events(n, 24_000, t_range=9_000, seed=9)
    du, dv, dt = dev_events(u, v, t)
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    t_last = torch.full((1,), -(2**62), dtype=torch.int64, device="cuda")
    first = True
    for a, b in synth.split_batches(t, 4):
        tn.tn_component_matrix(du[a:b], dv[a:b], dt[a:b], n, S=S, t_last=t_last, init=first)
        first = False
    torch.cuda.synchronize()
    assert int(t_last.item()) == int(t[-1])
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))
    # a batch that does not start after t_last is rejected, S untouched
    before = S.clone()
    with pytest.raises(tn.TnError) as e:
        tn.tn_component_matrix(du[:10], dv[:10], dt[:10], n, S=S, t_last=t_last, init=False)
    assert e.value.status == tn.TN_EORDER
    assert torch.equal(before, S)


def test_plan_apply_order_gate():
    n = 50
    u, v, t = synth.uniform_events(n, 500, t_range=100, seed=10)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n)
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    t_last = torch.full((1,), int(t[-1]), dtype=torch.int64, device="cuda")
    plan.apply(S, t_last=t_last, init=True)
    assert plan.status() == tn.TN_EORDER
    assert plan.status() == 0  # cleared by reading


def test_validation_errors():
    n = 10
    du, dv, dt = dev_events(np.array([1, 2]), np.array([3, 10]), np.array([0, 1]))
    with pytest.raises(tn.TnError) as e:
        tn.tn_component_matrix(du, dv, dt, n)
    assert e.value.status == tn.TN_ERANGE
    du, dv, dt = dev_events(np.array([1, 2]), np.array([3, 4]), np.array([5, 1]))
    with pytest.raises(tn.TnError) as e:
        tn.tn_component_matrix(du, dv, dt, n)
    assert e.value.status == tn.TN_EORDER


def test_column_subset_repeats():
    n = 700
    u, v, t = synth.uniform_events(n, 9000, t_range=3000, seed=12)
    src = np.array([5, 5, 699, 0, 311] * 30, np.uint32)
    du, dv, dt = dev_events(u, v, t)
    S = tn.tn_component_columns(du, dv, dt, n, torch.from_numpy(src.view(np.int32)).cuda())
    out, _, _ = tn.tn_out_sizes(S, n, len(src))
    torch.cuda.synchronize()
    ref = oracle.component_matrix(u, v, t, n, src=src)
    assert np.array_equal(host_matrix(S, len(src)), ref)
    assert np.array_equal(u32(out), oracle.column_counts(ref, len(src)))


def test_batched_apply_equals_single():
    plans, mats, refs = [], [], []
    for i, (n, m) in enumerate([(300, 4000), (1200, 9000), (64, 700), (2500, 30000)]):
        u, v, t = synth.uniform_events(n, m, t_range=m // 2, seed=20 + i)
        du, dv, dt = dev_events(u, v, t)
        plans.append(tn.Plan(du, dv, dt, n, slab_words=[2, 4, 8, 4][i]))
        mats.append(torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda"))
        refs.append(oracle.component_matrix(u, v, t, n))
    tn.tn_plan_apply_batch(plans, mats)
    torch.cuda.synchronize()
    for p, S, ref in zip(plans, mats, refs):
        assert p.status() == 0
        assert np.array_equal(host_matrix(S, p.n), ref)


def test_host_entry_point():
    n = 900
    u, v, t = synth.activity_driven(n, 40_000, seed=13)
    sizes, am = tn.tn_out_component_sizes_host(u, v, t, n)
    ref = oracle.column_counts(oracle.component_matrix(u, v, t, n), n)
    assert np.array_equal(sizes, ref)
    assert am == oracle.argmax(ref)


# --------------------------------------------------------------------------
# hashing (Section 4)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,k,R,seed", [(1000, 97, 3, 1), (70_000, 4096, 2, 123456789), (5, 1, 1, 0)])
def test_hash_tables_and_super_events(n, k, R, seed):
    u, v, t = synth.uniform_events(n, 5000, t_range=1000, seed=seed % 1000, self_loops=True)
    du, dv, dt = dev_events(u, v, t)
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, seed)
    torch.cuda.synchronize()
    Href = oracle.hash_nodes(seed, R, k, n)
    assert np.array_equal(u32(H), Href)
    for j in range(R):
        a, b = oracle.proxy_events(u, v, Href[j])
        assert np.array_equal(u32(pu[j]), a) and np.array_equal(u32(pv[j]), b)


@pytest.mark.parametrize("n,m,k,R", [(400, 3000, 37, 3), (3000, 60_000, 512, 8), (150, 120, 60, 5)])
def test_estimate_matches_oracle(n, m, k, R):
    u, v, t = synth.uniform_events(n, m, t_range=m // 3, seed=k)
    du, dv, dt = dev_events(u, v, t)
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, 77)
    P = torch.empty((R, k, tn.tn_row_words(k)), dtype=torch.int64, device="cuda")
    plans = [tn.Plan(pu[j].contiguous(), pv[j].contiguous(), dt, k) for j in range(R)]
    tn.tn_plan_apply_batch(plans, [P[j] for j in range(R)])
    est = tn.tn_hash_estimate(P, R, k, H, n)
    src = torch.tensor([0, n - 1, n // 2, 3], dtype=torch.int32, device="cuda")
    est_sub = tn.tn_hash_estimate(P, R, k, H, n, src=src)
    torch.cuda.synchronize()
    Href = oracle.hash_nodes(77, R, k, n)
    Pref = oracle.proxy_matrices(u, v, t, Href, k)
    for j in range(R):
        assert np.array_equal(host_matrix(P[j], k), Pref[j])
    want = oracle.hash_estimate(Pref, Href, n)
    assert np.array_equal(u32(est), want)
    assert np.array_equal(u32(est_sub), want[[0, n - 1, n // 2, 3]])
    exact = oracle.column_counts(oracle.component_matrix(u, v, t, n), n)
    assert (want >= exact).all()  # containment (Section 4.2)


def test_estimate_global_table_path():
    """R * k beyond the shared-memory table: the per-CTA table lives in global memory."""
    n, m, k, R = 2000, 20_000, 40_000, 6
    u, v, t = synth.uniform_events(n, m, t_range=m, seed=31)
    du, dv, dt = dev_events(u, v, t)
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, 3)
    P = torch.empty((R, k, tn.tn_row_words(k)), dtype=torch.int64, device="cuda")
    for j in range(R):
        tn.tn_component_matrix(pu[j].contiguous(), pv[j].contiguous(), dt, k, S=P[j])
    src = torch.arange(0, n, 13, dtype=torch.int32, device="cuda")
    est = tn.tn_hash_estimate(P, R, k, H, n, src=src)
    torch.cuda.synchronize()
    Href = oracle.hash_nodes(3, R, k, n)
    Pref = oracle.proxy_matrices(u, v, t, Href, k)  # the oracle's own proxies, all R replicas
    for j in range(R):
        assert np.array_equal(host_matrix(P[j], k), Pref[j])
    ref_src = np.arange(0, n, 13, dtype=np.uint32)
    assert np.array_equal(u32(est), oracle.hash_estimate(Pref, Href, n, ref_src))


# --------------------------------------------------------------------------
# error of the estimate (Section 4.4)
# --------------------------------------------------------------------------
def _err_check(est, exact, maxv):
    g = tn.tn_error_stats(torch.from_numpy(est.view(np.int32)).cuda(),
                          torch.from_numpy(exact.view(np.int32)).cuda(), maxv)
    want = oracle.error_stats(est, exact)
    for key in ("count", "sum_abs", "max_abs", "w1_num"):
        assert g[key] == want[key], key
    assert g["max_rel"] == want["max_rel"]  # one correctly rounded division per source
    # the relative-error sum is a float sum in another order: |error| <= count * eps * sum
    assert g["rel_sum"] == pytest.approx(want["rel_sum"], rel=max(1e-15, len(est) * 2.3e-16), abs=1e-300)
    return g


@pytest.mark.parametrize("count,maxv,seed", [(1, 5, 0), (1000, 700, 1), (100_000, 1_000_000, 2), (4097, 3, 3)])
def test_error_stats_match_oracle(count, maxv, seed):
    rng = np.random.default_rng(seed)
    exact = rng.integers(1, maxv + 1, count).astype(np.uint32)
    est = np.minimum(exact + rng.integers(0, 50, count), maxv).astype(np.uint32)
    _err_check(est, exact, maxv)
    _err_check(exact, exact, maxv)


def test_error_stats_range_errors():
    a = torch.tensor([1, 2, 9], dtype=torch.int32, device="cuda")
    b = torch.tensor([1, 2, 3], dtype=torch.int32, device="cuda")
    with pytest.raises(tn.TnError) as exc:
        tn.tn_error_stats(a, b, 8)  # 9 > max_value
    assert exc.value.status == tn.TN_ERANGE
    with pytest.raises(tn.TnError) as exc:
        tn.tn_error_stats(b, torch.tensor([1, 0, 3], dtype=torch.int32, device="cuda"), 8)  # exact size 0
    assert exc.value.status == tn.TN_ERANGE


def test_estimate_error_end_to_end():
    """Hashed estimates against exact sizes of sampled sources, all on the GPU."""
    n, m, k, R = 3000, 40_000, 300, 4
    u, v, t = synth.activity_driven(n, m, seed=21)
    du, dv, dt = dev_events(u, v, t)
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, 9)
    P = torch.empty((R, k, tn.tn_row_words(k)), dtype=torch.int64, device="cuda")
    plans = [tn.Plan(pu[j].contiguous(), pv[j].contiguous(), dt, k) for j in range(R)]
    tn.tn_plan_apply_batch(plans, [P[j] for j in range(R)], init=True)
    rng = np.random.default_rng(21)
    src_np = np.sort(rng.choice(n, 256, replace=False)).astype(np.uint32)
    src = torch.from_numpy(src_np.view(np.int32)).cuda()
    est = tn.tn_hash_estimate(P, R, k, H, n, src=src)
    Sx = tn.tn_component_columns(du, dv, dt, n, src)
    exact, _, _ = tn.tn_out_sizes(Sx, n, len(src_np))
    g = tn.tn_error_stats(est, exact, n)
    Href = oracle.hash_nodes(9, R, k, n)
    want_est = oracle.hash_estimate(oracle.proxy_matrices(u, v, t, Href, k), Href, n, src_np)
    want_exact = oracle.column_counts(oracle.component_matrix(u, v, t, n, src_np), len(src_np))
    assert np.array_equal(u32(est), want_est) and np.array_equal(u32(exact), want_exact)
    want = oracle.error_stats(want_est, want_exact)
    for key in ("sum_abs", "max_abs", "w1_num"):
        assert g[key] == want[key]
    assert (want_est >= want_exact).all()


def test_estimate_bitsliced_chunks_and_both_paths_agree():
    """All 70,000 sources: the bit-sliced fusion in two source chunks (65,536 +
    4,464), several table CTAs per replica; sampled sources against the oracle
    and a few hundred against the byte-table fusion."""
    n, m, k, R = 70_000, 200_000, 700, 3
    u, v, t = synth.uniform_events(n, m, t_range=m // 2, seed=41)
    du, dv, dt = dev_events(u, v, t)
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, 17)
    P = torch.empty((R, k, tn.tn_row_words(k)), dtype=torch.int64, device="cuda")
    plans = [tn.Plan(pu[j].contiguous(), pv[j].contiguous(), dt, k) for j in range(R)]
    tn.tn_plan_apply_batch(plans, [P[j] for j in range(R)])
    est = u32(tn.tn_hash_estimate(P, R, k, H, n))
    Href = oracle.hash_nodes(17, R, k, n)
    Pref = oracle.proxy_matrices(u, v, t, Href, k)
    for j in range(R):
        assert np.array_equal(host_matrix(P[j], k), Pref[j])
    rng = np.random.default_rng(41)
    sample = np.unique(np.concatenate([rng.choice(n, 60, replace=False), [0, 65_535, 65_536, n - 1]])).astype(np.uint32)
    assert np.array_equal(est[sample], oracle.hash_estimate(Pref, Href, n, sample))
    few = torch.from_numpy(sample.view(np.int32)).cuda()
    small = torch.zeros(len(sample), dtype=torch.int32, device="cuda")
    tn.tn_hash_estimate_noalloc(P, R, k, H, n, small, src=few)  # byte-table fusion
    assert np.array_equal(u32(small), est[sample])


# --------------------------------------------------------------------------
# reversed sequence (Section 3.4)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,t_range,seed", [(300, 5000, 800, 1), (1500, 40_000, 30, 2), (70, 3000, 4000, 3)])
def test_reversed_matrix_is_transposed(n, m, t_range, seed):
    u, v, t = synth.uniform_events(n, m, t_range=t_range, seed=seed, self_loops=True)
    du, dv, dt = dev_events(u, v, t)
    R = tn.tn_component_matrix(du, dv, dt, n, reverse=True)
    torch.cuda.synchronize()
    got = host_matrix(R, n)
    assert np.array_equal(got, oracle.component_matrix_reversed(u, v, t, n))
    F = oracle.to_bool(oracle.component_matrix(u, v, t, n), n)
    assert np.array_equal(oracle.to_bool(got, n), F.T)
    # in-sizes of the reversed matrix are the out-sizes of the chronological one
    _, ins, _ = tn.tn_out_sizes(R, n, n, in_sizes=True)
    assert np.array_equal(u32(ins), oracle.column_counts(oracle.component_matrix(u, v, t, n), n))


def test_reversed_rejects_streaming_use():
    n = 50
    u, v, t = synth.uniform_events(n, 200, t_range=100, seed=4)
    du, dv, dt = dev_events(u, v, t)
    t_last = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    with pytest.raises(tn.TnError) as exc:
        tn.tn_component_matrix(du, dv, dt, n, t_last=t_last, reverse=True)
    assert exc.value.status == tn.TN_EINVAL
    with pytest.raises(tn.TnError):
        tn.tn_component_matrix(du, dv, dt, n, init=False, reverse=True)


# --------------------------------------------------------------------------
# failure handling: bounded device waits
# --------------------------------------------------------------------------
def test_bounded_wait_times_out_and_context_survives():
    """A wait on a barrier that nothing completes gives up with TN_ETIMEOUT
    (no trap, no hang), and the next call works."""
    assert tn.tn_selftest_wait_timeout() == tn.TN_ETIMEOUT
    u, v, t = synth.uniform_events(100, 500, t_range=200, seed=6)
    assert np.array_equal(gpu_matrix(u, v, t, 100), oracle.component_matrix(u, v, t, 100))


# --------------------------------------------------------------------------
# directed events (footnote to Section 3.1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,m,t_range,slab,smem_rows,seed", [
    (400, 8000, 8000, 16, 0, 1),    # mostly lone events: ONEWAY ops in shared memory
    (400, 8000, 300, 8, 0, 2),      # small tie groups: PULL runs with saved rows
    (900, 20_000, 12, 16, 0, 3),    # giant groups: global tiles
    (900, 20_000, 40, 4, 1, 4),     # every window through the global path
    (70, 5000, 9000, 2, 0, 5),
])
def test_directed_matches_oracle(n, m, t_range, slab, smem_rows, seed):
    u, v, t = synth.uniform_events(n, m, t_range=t_range, seed=seed, self_loops=True)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, slab_words=slab, smem_rows=smem_rows, directed=True)
    S = plan.apply(None, init=True)
    assert plan.status() == 0
    want = oracle.component_matrix_directed(u, v, t, n)
    assert np.array_equal(host_matrix(S, n), want)
    out, _, _ = tn.tn_out_sizes(S, n, n)
    assert np.array_equal(u32(out), oracle.column_counts(want, n))


def test_directed_doubled_equals_undirected_and_reverse_transposes():
    n, m = 600, 15_000
    u, v, t = synth.uniform_events(n, m, t_range=900, seed=9, self_loops=True)
    du2 = np.stack([u, v], 1).reshape(-1)
    dv2 = np.stack([v, u], 1).reshape(-1)
    dt2 = np.repeat(t, 2)
    a, b, c = dev_events(du2, dv2, dt2)
    D = host_matrix(tn.tn_component_matrix(a, b, c, n, directed=True), n)
    assert np.array_equal(D, oracle.component_matrix(u, v, t, n))
    du, dv, dt = dev_events(u, v, t)
    F = oracle.to_bool(host_matrix(tn.tn_component_matrix(du, dv, dt, n, directed=True), n), n)
    R = oracle.to_bool(host_matrix(tn.tn_component_matrix(du, dv, dt, n, directed=True, reverse=True), n), n)
    torch.cuda.synchronize()
    assert np.array_equal(R, F.T)


def test_directed_incremental_batches():
    n, m = 500, 12_000
    u, v, t = synth.uniform_events(n, m, t_range=3000, seed=10)
    parts = synth.split_batches(t, 4)
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    t_last = torch.full((1,), -(2**62), dtype=torch.int64, device="cuda")
    for k, (a, b) in enumerate(parts):
        du, dv, dt = dev_events(u[a:b], v[a:b], t[a:b])
        tn.tn_component_matrix(du, dv, dt, n, S=S, t_last=t_last, init=(k == 0), directed=True)
    torch.cuda.synchronize()
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix_directed(u, v, t, n))


# --------------------------------------------------------------------------
# the paper's synthetic experiments (Sections 3.5 and 4.4): ER G(n, 2/n)
# with an independent Poisson process on every link
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,m", [(100, 20_000), (500, 50_000), (2000, 100_000)])
def test_er_poisson_exact_and_hashed(n, m):
    """The exact matrix and sizes, and the hashed estimate with n_s = 0.3 n
    super-nodes and K = 5 replicas (the sweep's settings), bit-exact to the
    oracle on the paper's generator; the error statistics as the sweep
    reports them, against the oracle's."""
    u, v, t = synth.er_poisson(n, m, seed=60 + n)
    du, dv, dt = dev_events(u, v, t)
    S = tn.tn_component_matrix(du, dv, dt, n)
    exact, _, am = tn.tn_out_sizes(S, n, n, argmax=True)
    ref = oracle.component_matrix(u, v, t, n)
    assert np.array_equal(host_matrix(S, n), ref)
    want_exact = oracle.column_counts(ref, n)
    assert np.array_equal(u32(exact), want_exact) and int(am.item()) == oracle.argmax(want_exact)
    k, K = max(1, int(0.3 * n)), 5
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, K, 6)
    plans = [tn.Plan(pu[j].contiguous(), pv[j].contiguous(), dt, k) for j in range(K)]
    P = torch.empty((K, k, tn.tn_row_words(k)), dtype=torch.int64, device="cuda")
    tn.tn_plan_apply_batch(plans, [P[j] for j in range(K)])
    est = tn.tn_hash_estimate(P, K, k, H, n)
    err = tn.tn_error_stats(est, exact, n)
    Href = oracle.hash_nodes(6, K, k, n)
    Pref = oracle.proxy_matrices(u, v, t, Href, k)
    want_est = oracle.hash_estimate(Pref, Href, n)
    assert np.array_equal(u32(est), want_est)
    want_err = oracle.error_stats(want_est, want_exact)
    assert err["max_abs"] == want_err["max_abs"] and err["w1_num"] == want_err["w1_num"]
    assert abs(err["w1"] - want_err["w1"]) <= 1e-12 * max(1.0, want_err["w1"])


@pytest.mark.parametrize("n,m,t_range,window,smem_rows", [
    (300, 20_000, 50, 640, 0),        # groups of ~400 events, every node ~2.7 times per group
    (300, 20_000, 50, 4096, 1),       # the same through global windows
    (5000, 60_000, 300, 640, 0),      # groups of ~200, few repeats
    (40, 9_000, 3, 2048, 0),          # three giant groups on 40 nodes: long PULL lists, saved rows
    (2000, 30_000, 200, 64, 0),       # windows smaller than a group
])
def test_large_groups_scheduled_by_the_whole_cta(n, m, t_range, window, smem_rows):
    """Timestamp groups of 128 events or more are scheduled by every thread of
    the planner's CTA (roles, runs, saved rows and source lists through
    shared-memory atomics); the matrix must equal the oracle's."""
    u, v, t = synth.uniform_events(n, m, t_range=t_range, seed=n + t_range)
    du, dv, dt = dev_events(u, v, t)
    for slab in (16, 64):
        plan = tn.Plan(du, dv, dt, n, window_events=window, slab_words=slab, smem_rows=smem_rows)
        S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
        plan.apply(S, init=True)
        assert plan.status() == 0
        assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n)), slab


@pytest.mark.parametrize("slab,window", [(64, 3000), (26, 3000), (64, 200)])
def test_directed_through_wide_slabs_and_the_ring(slab, window):
    """Directed events (footnote to Section 3.1) with tie groups of about 500
    events: receivers' PULL runs, senders that also receive read from saved
    rows; through the per-thread ring (windows of 3,000 events, larger than the
    buffer) and through records (200), at wide slabs (96 row words: 64 + 32)."""
    n = 6000
    u, v, t = synth.uniform_events(n, 40_000, t_range=80, seed=41)
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, directed=True, slab_words=slab, window_events=window)
    S = plan.apply(None, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix_directed(u, v, t, n))


def test_reversed_stream_through_wide_slabs():
    """The reversed sequence (Section 3.4: the flipped stream, t -> ~t) of a
    bursty network through 64-word slabs and the ring equals the oracle's
    reversed matrix (rows = out-components)."""
    n = 6000
    u, v, t = synth.powerlaw_bursty(n, 60_000, seed=43)
    ru, rv, rt = u[::-1].copy(), v[::-1].copy(), ~t[::-1]
    du, dv, dt = dev_events(ru, rv, rt)
    plan = tn.Plan(du, dv, dt, n, slab_words=64, window_events=3000)
    S = plan.apply(None, init=True)
    assert plan.status() == 0
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix_reversed(u, v, t, n))
