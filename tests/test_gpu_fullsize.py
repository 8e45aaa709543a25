"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (needs a GPU: -m gpu).

Matrix columns are independent (column j is the out-component of source j),
so the oracle computes a seeded sample of columns exactly and the GPU matrix
must match them bit for bit; properties that hold at any size (diagonal set,
sum of in-sizes = sum of out-sizes, argmax attains the maximum) cover the
rest.  For the hashed estimate the oracle rebuilds only the proxy columns the
sampled sources need, which fixes their estimates exactly.
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


def gpu_columns(S, cols):
    """Bits of the listed columns of a GPU matrix, as a bool [rows, len(cols)]."""
    c = torch.from_numpy(np.asarray(cols, np.int64)).cuda()
    words = S[:, c // 64]
    return ((words >> (c % 64)) & 1).bool().cpu().numpy()


def check_sampled_columns(S, u, v, t, n, cols):
    ref = oracle.to_bool(oracle.component_matrix(u, v, t, n, np.asarray(cols, np.uint32)), len(cols))
    assert np.array_equal(gpu_columns(S, cols), ref)
    return ref.sum(axis=0)


def check_matrix_properties(S, n):
    out, ins, am = tn.tn_out_sizes(S, n, n, in_sizes=True, argmax=True)
    out = out.cpu().numpy().view(np.uint32)
    ins = ins.cpu().numpy().view(np.uint32)
    assert int(out.astype(np.int64).sum()) == int(ins.astype(np.int64).sum())  # Section 3.3
    assert out.min() >= 1 and ins.min() >= 1
    a = int(am.item())
    assert out[a] == out.max() and (out[:a] < out[a]).all()  # lowest id among the largest
    rows = np.random.default_rng(n).choice(n, 256, replace=False)
    r = torch.from_numpy(rows.astype(np.int64)).cuda()
    diag = ((S[r, r // 64] >> (r % 64)) & 1).cpu().numpy()
    assert diag.all()  # every node reaches itself
    return out


def test_activity_n1e5_m1e7_bench_config():
    n, m = 100_000, 10_000_000
    u, v, t = synth.activity_driven(n, m, seed=2)  # bench.py --workload activity
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    plan = tn.Plan(du, dv, dt, n)  # default options, as timed by bench.py
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    tn.tn_init_matrix(S, n)
    plan.apply(S)
    assert plan.status() == 0
    rng = np.random.default_rng(7)
    cols = np.unique(np.concatenate([rng.choice(n, 62, replace=False), [0, n - 1]]))
    sizes = check_sampled_columns(S, u, v, t, n, cols)
    out = check_matrix_properties(S, n)
    assert np.array_equal(out[cols], sizes)


def test_bursty_n5e5_m1e8_bench_config():
    n, m = 500_000, 100_000_000
    u, v, t = synth.powerlaw_bursty(n, m, seed=3)  # bench.py's default workload
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    # the plan options bench.py times: the autotuner's choice on the first 2e6 events
    tuned = tn.tn_autotune(du, dv, dt, n, sample_events=2_000_000)
    plan = tn.Plan(du, dv, dt, n, **{k: tuned[k] for k in ("window_events", "slab_words", "smem_rows")})
    st = plan.stats()
    assert st["big_windows"] > 0 and st["local_windows"] == 0  # every tie group is larger than a window
    S = torch.empty((n, tn.tn_row_words(n)), dtype=torch.int64, device="cuda")
    tn.tn_init_matrix(S, n)
    plan.apply(S)
    assert plan.status() == 0
    del du, dv, dt
    rng = np.random.default_rng(11)
    cols = np.unique(np.concatenate([rng.choice(n, 30, replace=False), [0, n - 1]]))
    sizes = check_sampled_columns(S, u, v, t, n, cols)
    out = check_matrix_properties(S, n)
    assert np.array_equal(out[cols], sizes)


def test_hashed_n1e6_m1e8_bench_config():
    n, m, k, R, nsrc = 1_000_000, 100_000_000, 16_384, 8, 65_536
    u, v, t = synth.activity_driven(n, m, seed=4)
    rng = np.random.default_rng(4)
    src_np = np.sort(rng.choice(n, nsrc, replace=False)).astype(np.uint32)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, 0)
    P = torch.empty((R, k, tn.tn_row_words(k)), dtype=torch.int64, device="cuda")
    src = dev(src_np)
    # the launch bench.py times: the 8 proxies (24-word slabs) and the sampled exact
    # columns (16-word slabs) in one job-list launch, one wave of 152 CTAs
    plans = [tn.Plan(pu[j].contiguous(), pv[j].contiguous(), dt, k, slab_words=24, window_events=480,
                     smem_rows=192 * 1024 // (8 * 24)) for j in range(R)]
    plan_x = tn.Plan(du, dv, dt, n, slab_words=16, window_events=640)
    Sx = torch.empty((n, tn.tn_row_words(nsrc)), dtype=torch.int64, device="cuda")
    tn.tn_plan_apply_batch(plans + [plan_x], [P[j] for j in range(R)] + [Sx], ncols=[k] * R + [nsrc], init=True,
                           srcs=[None] * R + [src])
    assert all(p.status() == 0 for p in plans + [plan_x])
    est = tn.tn_hash_estimate(P, R, k, H, n, src=src).cpu().numpy().view(np.uint32)
    exact = tn.tn_out_sizes(Sx, n, nsrc)[0].cpu().numpy().view(np.uint32)
    Hh = H.cpu().numpy().view(np.uint32)
    Href = oracle.hash_nodes(0, R, k, n)
    assert np.array_equal(Hh, Href)
    del du, dv, dt, pu, pv
    # sampled sources (positions in src), checked exactly
    pos = np.unique(np.concatenate([rng.choice(nsrc, 14, replace=False), [0, nsrc - 1]]))
    x = src_np[pos]
    # oracle: for every replica only the proxy columns h_j(x) are needed
    W = (k + 63) // 64
    Pcols = np.zeros((R, k, W), dtype=np.uint64)
    for j in range(R):
        cols = np.unique(Href[j][x]).astype(np.uint32)
        pu_j, pv_j = oracle.proxy_events(u, v, Href[j])
        part = oracle.to_bool(oracle.component_matrix(pu_j, pv_j, t, k, cols), len(cols))
        gpu_part = gpu_columns(P[j], cols)
        assert np.array_equal(gpu_part, part), j
        for ci, c in enumerate(cols):
            Pcols[j, part[:, ci], c // 64] |= np.uint64(1) << np.uint64(c % 64)
    want_est = oracle.hash_estimate(Pcols, Href, n, x)
    assert np.array_equal(est[pos], want_est)
    want_exact = oracle.column_counts(oracle.component_matrix(u, v, t, n, x), len(x))
    assert np.array_equal(exact[pos], want_exact)
    assert (est >= exact).all()  # containment (Section 4.2), on all 65,536 sources
    # exact sampled columns also match column by column for a few positions
    sub = pos[:4]
    assert np.array_equal(gpu_columns(Sx, sub), oracle.to_bool(oracle.component_matrix(u, v, t, n, src_np[sub]), len(sub)))
