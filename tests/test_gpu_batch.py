"""Batched application under a CUDA graph, and the autotuner (needs a GPU: -m gpu).

The graph replays one persistent launch over networks of uneven n and m
(hash proxies of two sizes, a plain network and a tie-heavy network whose
schedule needs saved-row slots); every replay must give the same matrices as
the direct batched call and the CPU oracle.  Options chosen by the autotuner
must not change any result.
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


def dev(a, dtype=np.int32):
    return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).cuda()


def host(S, ncols):
    return S.cpu().numpy().view(np.uint64)[:, : (ncols + 63) // 64]


def networks():
    """(plan, n, oracle matrix) for networks of uneven n and m."""
    nets = []
    n, m = 2000, 30_000
    u, v, t = synth.activity_driven(n, m, seed=3)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    for k, R, seed in ((300, 3, 4), (1500, 2, 8)):
        H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, seed)
        Href = oracle.hash_nodes(seed, R, k, n)
        Pref = oracle.proxy_matrices(u, v, t, Href, k)
        for j in range(R):
            nets.append((tn.Plan(pu[j].contiguous(), pv[j].contiguous(), dt, k), k, Pref[j]))
    nets.append((tn.Plan(du, dv, dt, n), n, oracle.component_matrix(u, v, t, n)))
    # giant tie groups: global windows with saved-row slots
    n2 = 700
    u2, v2, t2 = synth.uniform_events(n2, 9000, t_range=6, seed=5)
    p2 = tn.Plan(dev(u2), dev(v2), dev(t2, np.int64), n2, smem_rows=1)
    assert p2.stats()["temps"] > 0
    nets.append((p2, n2, oracle.component_matrix(u2, v2, t2, n2)))
    return nets


def test_graph_replay_equals_direct_and_oracle():
    nets = networks()
    plans = [p for p, _, _ in nets]
    mats = [torch.zeros((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda") for _, n, _ in nets]
    tn.tn_plan_apply_batch(plans, mats)
    torch.cuda.synchronize()
    direct = [host(S, n) for S, (_, n, _) in zip(mats, nets)]
    for d, (_, n, ref) in zip(direct, nets):
        assert np.array_equal(d, ref)
    g = tn.BatchGraph(plans, mats)
    for rep in range(2):
        for S in mats:
            S.fill_(-1)  # the replay must rebuild everything from the identity
        g.launch()
        torch.cuda.synchronize()
        for S, d, (_, n, _) in zip(mats, direct, nets):
            assert np.array_equal(host(S, n), d), rep
    assert all(p.status() == 0 for p in plans)
    g.destroy()


def test_graph_launch_counts_kernels():
    nets = networks()[:2]
    mats = [torch.zeros((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda") for _, n, _ in nets]
    g = tn.BatchGraph([p for p, _, _ in nets], mats)
    before = tn.tn_kernel_launches()
    g.launch()
    torch.cuda.synchronize()
    assert tn.tn_kernel_launches() - before >= 3  # two inits + the streaming launch


@pytest.mark.parametrize("n,m,replicas", [(1000, 50_000, 1), (16_384, 100_000, 4), (50_000, 300_000, 1)])
def test_autotune_keeps_results(n, m, replicas):
    u, v, t = synth.activity_driven(n, m, seed=n)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    res = tn.tn_autotune(du, dv, dt, n, replicas=replicas, sample_events=50_000)
    assert res["tried"] > 0 and not res["cached"]
    if res["resident_words"]:  # the resident-slab form: only for networks whose rows fit
        assert res["resident_words"] in (1, 2) and n <= tn.tn_resident_max_rows(res["resident_words"])
        assert res["window_events"] in (640, 2048) and res["slab_words"] == 0 and res["smem_rows"] == 0
    else:
        assert res["slab_words"] in (2, 4, 8, 12, 16, 24, 32, 48, 64) and res["window_events"] in (320, 640, 1024)
    again = tn.tn_autotune(du, dv, dt, n, replicas=replicas, sample_events=50_000)
    assert again["cached"] and again["slab_words"] == res["slab_words"]
    assert again["resident_words"] == res["resident_words"]
    tuned = tn.Plan(du, dv, dt, n, window_events=res["window_events"], slab_words=res["slab_words"],
                    smem_rows=res["smem_rows"], resident_words=res["resident_words"])
    plain = tn.Plan(du, dv, dt, n)
    a = tuned.apply(None, init=True)
    b = plain.apply(None, init=True)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    out_a, _, _ = tn.tn_out_sizes(a, n, n)
    if n * m <= 1e10:
        want = oracle.column_counts(oracle.component_matrix(u, v, t, n), n)
        assert np.array_equal(out_a.cpu().numpy().view(np.uint32), want)


def test_batch_with_source_columns_and_wide_slabs():
    """One launch over full matrices and column subsets (the hashed workload's
    proxies together with its sampled exact columns), at different slab widths
    and a wave spread: every matrix equals the oracle's."""
    n, m = 3000, 40_000
    u, v, t = synth.activity_driven(n, m, seed=17)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    rng = np.random.default_rng(17)
    src_np = np.sort(rng.choice(n, 700, replace=False)).astype(np.uint32)
    src2_np = rng.integers(0, n, 150).astype(np.uint32)  # repeated ids allowed
    plans = [tn.Plan(du, dv, dt, n, slab_words=16), tn.Plan(du, dv, dt, n, slab_words=8, smem_rows=640),
             tn.Plan(du, dv, dt, n, slab_words=2), tn.Plan(du, dv, dt, n, slab_words=32, wave_ctas=3)]
    ncols = [n, 700, 150, n]
    srcs = [None, dev(src_np), dev(src2_np), None]
    mats = [torch.empty((n, tn.tn_row_words(c)), dtype=torch.int64, device="cuda") for c in ncols]
    tn.tn_plan_apply_batch(plans, mats, ncols=ncols, init=True, srcs=srcs)
    torch.cuda.synchronize()
    full = oracle.component_matrix(u, v, t, n)
    want = [full, oracle.component_matrix(u, v, t, n, src_np), oracle.component_matrix(u, v, t, n, src2_np), full]
    for p, S, c, ref in zip(plans, mats, ncols, want):
        assert p.status() == 0
        assert np.array_equal(host(S, c), ref)
