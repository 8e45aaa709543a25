"""Parity of the resident-slab form with the CPU oracle (needs a GPU: -m gpu).

In the resident-slab form every CTA keeps 1 or 2 words of every row in
shared memory for the whole batch and streams only the schedule
(tn_plan_options.resident_words).  It computes the same component matrix as
the column-slab form, so every comparison is bit-exact, including the zero
padding: dense ties (saved rows, multi-source updates), directed events,
column subsets, incremental batches, one launch mixed with column-slab plans,
graph replay, levels larger than one tile, schedule chunks crossed by a tile,
the size limit, and the hashed proxies.
"""
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


def resident_matrix(u, v, t, n, rw, window=0, directed=False, src=None):
    du, dv, dt = dev_events(u, v, t)
    plan = tn.Plan(du, dv, dt, n, window_events=window, resident_words=rw, directed=directed)
    ncols = n if src is None else len(src)
    S = torch.full((n, tn.tn_row_words(ncols)), -1, dtype=torch.int64, device="cuda")  # stale bits
    dsrc = None if src is None else torch.from_numpy(np.asarray(src, np.uint32).view(np.int32)).cuda()
    plan.apply(S, ncols=ncols, src=dsrc, init=True)
    assert plan.status() == 0
    st = plan.stats()
    plan.destroy()
    return host_matrix(S, ncols), st


@pytest.mark.parametrize("rw", [1, 2])
@pytest.mark.parametrize("window", [40, 640, 4096])
def test_uniform_ties_identical_to_oracle(rw, window):
    n = 1500  # 24 words of columns: 24 / 12 CTAs, several windows, a ragged last window
    u, v, t = synth.uniform_events(n, 31_001, t_range=12_000, seed=3)
    got, _ = resident_matrix(u, v, t, n, rw, window)
    assert np.array_equal(got, oracle.component_matrix(u, v, t, n))


@pytest.mark.parametrize("seed", range(40))
def test_fuzz_dense_ties(seed):
    """Tiny networks with a few timestamps: big tie groups, saved rows and
    multi-source updates in every window."""
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(1, 300))
    m = int(rng.integers(1, 600))
    u = rng.integers(0, n, m).astype(np.uint32)
    v = rng.integers(0, n, m).astype(np.uint32)
    t = np.sort(rng.integers(0, int(rng.integers(1, 12)), m))
    rw = int(rng.choice([1, 2]))
    win = int(rng.choice([32, 64, 2048]))
    directed = bool(seed % 3 == 0)
    got, st = resident_matrix(u, v, t, n, rw, win, directed=directed)
    want = (oracle.component_matrix_directed if directed else oracle.component_matrix)(u, v, t, n)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("rw", [1, 2])
def test_directed_activity(rw):
    n = 3000
    u, v, t = synth.activity_driven(n, 200_000, seed=8)
    t = t // 50  # some ties
    got, _ = resident_matrix(u, v, t, n, rw, 640, directed=True)
    assert np.array_equal(got, oracle.component_matrix_directed(u, v, t, n))


@pytest.mark.parametrize("rw", [1, 2])
def test_column_subset_with_repeats(rw):
    n = 5000
    u, v, t = synth.uniform_events(n, 60_000, t_range=20_000, seed=5)
    rng = np.random.default_rng(1)
    src = np.concatenate([rng.choice(n, 700, replace=False), [3, 3, n - 1]]).astype(np.uint32)  # ragged: 703
    got, _ = resident_matrix(u, v, t, n, rw, 640, src=src)
    assert np.array_equal(got, oracle.component_matrix(u, v, t, n, src))


def test_incremental_batches_and_order_gate():
    n = 2000
    u, v, t = synth.uniform_events(n, 40_000, t_range=30_000, seed=6)
    cut = int(np.searchsorted(t, t[20_000], side="left"))  # at a group start
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    t_last = torch.full((1,), -(2 ** 62), dtype=torch.int64, device="cuda")
    du, dv, dt = dev_events(u, v, t)
    p1 = tn.Plan(du[:cut], dv[:cut], dt[:cut], n, resident_words=1)
    p2 = tn.Plan(du[cut:], dv[cut:], dt[cut:], n, resident_words=2)
    p1.apply(S, init=True, t_last=t_last)
    before = S.clone()
    p1.apply(S, t_last=t_last)  # the same batch again: out of order, S untouched
    assert p1.status() == tn.TN_EORDER
    assert torch.equal(S, before)
    p2.apply(S, t_last=t_last)
    assert p2.status() == 0
    assert int(t_last.item()) == int(t[-1])
    assert np.array_equal(host_matrix(S, n), oracle.component_matrix(u, v, t, n))


def test_one_launch_mixed_with_column_slabs_and_graph_replay():
    """Resident plans of uneven n and m beside column-slab plans (full matrix
    and a source subset) in one job-list launch, and the same batch replayed
    from a CUDA graph: identical to the oracle."""
    nets = []
    for i, (n, m) in enumerate([(700, 9_000), (4100, 50_000), (1300, 1), (9000, 80_000)]):
        u, v, t = synth.uniform_events(n, m, t_range=max(1, m // 3), seed=40 + i)
        nets.append((n, u, v, t))
    plans, mats, ncols, srcs, want = [], [], [], [], []
    for i, (n, u, v, t) in enumerate(nets):
        du, dv, dt = dev_events(u, v, t)
        if i == 1:  # a column-slab plan over a source subset
            src = np.arange(0, n, 7, dtype=np.uint32)
            plans.append(tn.Plan(du, dv, dt, n, slab_words=8))
            srcs.append(torch.from_numpy(src.view(np.int32)).cuda())
            ncols.append(len(src))
            want.append(oracle.component_matrix(u, v, t, n, src))
        elif i == 3:  # a column-slab plan, full matrix
            plans.append(tn.Plan(du, dv, dt, n))
            srcs.append(None)
            ncols.append(n)
            want.append(oracle.component_matrix(u, v, t, n))
        else:
            plans.append(tn.Plan(du, dv, dt, n, resident_words=1 if i == 0 else 2))
            srcs.append(None)
            ncols.append(n)
            want.append(oracle.component_matrix(u, v, t, n))
        mats.append(torch.full((n, tn.tn_row_words(ncols[-1])), -1, dtype=torch.int64, device="cuda"))
    # resident plans for the two column-slab networks too, in the same launch
    for i in (1, 3):
        n, u, v, t = nets[i]
        du, dv, dt = dev_events(u, v, t)
        plans.append(tn.Plan(du, dv, dt, n, resident_words=1))
        srcs.append(srcs[i])
        ncols.append(ncols[i])
        want.append(want[i])
        mats.append(torch.full_like(mats[i], -1))
    tn.tn_plan_apply_batch(plans, mats, ncols=ncols, init=True, srcs=srcs)
    assert all(p.status() == 0 for p in plans)
    for S, nc, w in zip(mats, ncols, want):
        assert np.array_equal(host_matrix(S, nc), w)
    full = [i for i in range(len(plans)) if srcs[i] is None]
    g = tn.BatchGraph([plans[i] for i in full], [mats[i] for i in full])
    for _ in range(2):
        for i in full:
            mats[i].fill_(-1)
        g.launch()
        torch.cuda.synchronize()
        for i in full:
            assert np.array_equal(host_matrix(mats[i], ncols[i]), want[i])
    g.destroy()


def test_levels_larger_than_a_tile_and_chunk_crossings():
    """Windows of 8,192 events of a perfect matching: one level of 4,096 ops
    (two tiles) per window, and tiles that straddle schedule chunks."""
    n = 16_384
    rng = np.random.default_rng(12)
    us, vs = [], []
    for _ in range(12):
        p = rng.permutation(n).astype(np.uint32)
        us.append(p[0::2])
        vs.append(p[1::2])
    u, v = np.concatenate(us), np.concatenate(vs)
    t = np.arange(len(u), dtype=np.int64) // 3  # groups of 3 events, distinct nodes inside most
    got, st = resident_matrix(u, v, t, n, 1, 8192)
    assert st["items"] > st["levels"]  # some levels span several tiles
    assert np.array_equal(got, oracle.component_matrix(u, v, t, n))


def test_size_limit():
    lim = tn.tn_resident_max_rows(1)
    assert lim > 16_384 and tn.tn_resident_max_rows(2) == lim // 2 and tn.tn_resident_max_rows(4) == 0
    u, v, t = synth.uniform_events(lim + 1, 1000, t_range=1000, seed=2)
    du, dv, dt = dev_events(u, v, t)
    with pytest.raises(tn.TnError) as exc:
        tn.Plan(du, dv, dt, lim + 1, resident_words=1)
    assert exc.value.status == tn.TN_EINVAL
    # the largest network: ragged column count, all rows resident
    n = lim
    u, v, _ = synth.uniform_events(n, 30_000, t_range=30_000, seed=9)
    t = np.arange(len(u), dtype=np.int64)  # no ties, so no saved rows beside the rows
    got, _ = resident_matrix(u, v, t, n, 1)
    rng = np.random.default_rng(3)
    cols = np.unique(np.concatenate([rng.choice(n, 60, replace=False), [0, n - 1]])).astype(np.uint32)
    ref = oracle.to_bool(oracle.component_matrix(u, v, t, n, cols), len(cols))
    B = ((got[:, cols // 64] >> (cols % 64).astype(np.uint64)) & np.uint64(1)).astype(bool)
    assert np.array_equal(B, ref)


def test_self_loops_only_and_single_event():
    n = 300
    u = np.arange(50, dtype=np.uint32)
    t = np.arange(50, dtype=np.int64)
    got, st = resident_matrix(u, u, t, n, 1)
    assert st["ops"] == 0
    assert np.array_equal(got, oracle.component_matrix(u, u, t, n))
    u1, v1, t1 = np.array([5], np.uint32), np.array([77], np.uint32), np.array([3], np.int64)
    got, _ = resident_matrix(u1, v1, t1, n, 2)
    assert np.array_equal(got, oracle.component_matrix(u1, v1, t1, n))


def test_hashed_proxies_resident():
    """Network hashing with the proxies in the resident form and the sampled
    exact columns in the column-slab form, in one launch: proxies, estimates
    and exact sizes equal the oracle's."""
    n, m, k, R = 20_000, 300_000, 2048, 4
    u, v, t = synth.activity_driven(n, m, seed=13)
    du, dv, dt = dev_events(u, v, t)
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, 5)
    Href = oracle.hash_nodes(5, R, k, n)
    assert np.array_equal(H.cpu().numpy().view(np.uint32), Href)
    rng = np.random.default_rng(2)
    src_np = np.sort(rng.choice(n, 3000, replace=False)).astype(np.uint32)
    src = torch.from_numpy(src_np.view(np.int32)).cuda()
    P = torch.empty((R, k, tn.tn_row_words(k)), dtype=torch.int64, device="cuda")
    Sx = torch.empty((n, tn.tn_row_words(len(src_np))), dtype=torch.int64, device="cuda")
    plans = [tn.Plan(pu[j].contiguous(), pv[j].contiguous(), dt, k, resident_words=2) for j in range(R)]
    plan_x = tn.Plan(du, dv, dt, n)
    tn.tn_plan_apply_batch(plans + [plan_x], [P[j] for j in range(R)] + [Sx], ncols=[k] * R + [len(src_np)],
                           init=True, srcs=[None] * R + [src])
    assert all(p.status() == 0 for p in plans + [plan_x])
    Pref = oracle.proxy_matrices(u, v, t, Href, k)
    for j in range(R):
        assert np.array_equal(host_matrix(P[j], k), Pref[j]), j
    est = tn.tn_hash_estimate(P, R, k, H, n, src=src).cpu().numpy().view(np.uint32)
    assert np.array_equal(est, oracle.hash_estimate(Pref, Href, n, src_np))
    exact = tn.tn_out_sizes(Sx, n, len(src_np))[0].cpu().numpy().view(np.uint32)
    assert np.array_equal(exact, oracle.column_counts(oracle.component_matrix(u, v, t, n, src_np), len(src_np)))
