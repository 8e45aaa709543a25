"""Online state and node growth (tn_online_*, tn_grow_matrix; needs a GPU: -m gpu).

Section 3.5: the matrix method takes new events and new nodes as they arrive.
Batches may split a timestamp group anywhere; after every push the matrix must
equal the oracle over the events before the held-back last group, and after a
flush the oracle over all of them.  Growth must equal the oracle's definition
(new rows and columns of zeros with the new diagonal bits set).
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


def gpu_bits(S, n):
    """bool [n, n] of a GPU matrix; the padding columns must be zero."""
    h = S.cpu().numpy().view(np.uint64)
    B = np.unpackbits(h.view(np.uint8).reshape(h.shape[0], -1), axis=1, bitorder="little").astype(bool)
    assert not B[:n, n:].any(), "bits set beyond column n"
    return B[:n, :n]


def cuts_through_groups(t, rng, count):
    """Batch boundaries: inside groups, at group starts, two inside the same
    group (a batch that only continues the pending group) and 1-event batches."""
    m = len(t)
    starts = np.flatnonzero(np.r_[True, t[1:] != t[:-1]])
    ends = np.r_[starts[1:], m]
    big = np.flatnonzero(ends - starts >= 4)
    cuts = set(rng.integers(1, m, count).tolist())
    cuts |= set(starts[rng.choice(len(starts), min(4, len(starts)), replace=False)].tolist())
    for g in rng.choice(big, min(3, len(big)), replace=False):
        cuts |= {int(starts[g]) + 1, int(starts[g]) + 3}  # a batch entirely inside group g
    c = int(rng.integers(1, m - 2))
    cuts |= {c, c + 1}  # a one-event batch
    cuts = sorted(x for x in cuts if 0 < x < m)
    return list(zip([0] + cuts, cuts + [m]))


@pytest.mark.parametrize("seed,t_range", [(0, 300), (1, 40), (2, 5000)])
def test_split_groups_equal_the_whole_sequence(seed, t_range):
    n, m = 700, 20_000
    u, v, t = synth.uniform_events(n, m, t_range=t_range, seed=seed)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    rng = np.random.default_rng(seed)
    batches = cuts_through_groups(t, rng, 25)
    check_at = set(rng.choice(len(batches), 6, replace=False).tolist()) | {len(batches) - 1}
    with tn.Online(n) as on:
        for i, (a, b) in enumerate(batches):
            on.push(du[a:b], dv[a:b], dt[a:b])
            st = on.state()
            held = int((t[:b] == t[b - 1]).sum())
            assert st["pending_events"] == held and st["pending_t"] == t[b - 1]
            done = int(np.searchsorted(t, t[b - 1], side="left"))
            assert st["applied_events"] == done
            if i in check_at:
                want = oracle.to_bool(oracle.component_matrix(u[:done], v[:done], t[:done], n), n)
                assert np.array_equal(gpu_bits(on.matrix(), n), want), (i, a, b)
        on.flush()
        assert on.status() == 0
        st = on.state()
        assert st["pending_events"] == 0 and st["applied_events"] == m and st["t_applied"] == t[-1]
        want = oracle.to_bool(oracle.component_matrix(u, v, t, n), n)
        assert np.array_equal(gpu_bits(on.matrix(), n), want)


def test_group_end_and_ordering_rules():
    n = 300
    u, v, t = synth.uniform_events(n, 4000, t_range=200, seed=3)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    c = int(np.searchsorted(t, t[2000], side="right"))  # a group boundary
    with tn.Online(n) as on:
        on.push(du[:c], dv[:c], dt[:c], group_end=True)
        st = on.state()
        assert st["pending_events"] == 0 and st["t_applied"] == t[c - 1]
        want = oracle.to_bool(oracle.component_matrix(u[:c], v[:c], t[:c], n), n)
        assert np.array_equal(gpu_bits(on.matrix(), n), want)
        # the group was declared complete: continuing it is an ordering error
        same_t = dt[c - 1:c].clone()
        with pytest.raises(tn.TnError) as exc:
            on.push(du[:1], dv[:1], same_t)
        assert exc.value.status == tn.TN_EORDER
        # an empty push changes nothing
        on.push(du[:0], dv[:0], dt[:0])
        on.push(du[c:3000], dv[c:3000], dt[c:3000])
        pend = on.state()["pending_events"]
        assert pend >= 1
        # a batch that starts before the pending timestamp is rejected, state unchanged
        before = on.matrix().clone()
        with pytest.raises(tn.TnError) as exc:
            on.push(du[c:c + 5], dv[c:c + 5], dt[c:c + 5])
        assert exc.value.status == tn.TN_EORDER
        # an endpoint >= n is rejected, state unchanged
        bad_u = du[3000:3010].clone()
        bad_u[4] = n
        with pytest.raises(tn.TnError) as exc:
            on.push(bad_u, dv[3000:3010], dt[3000:3010])
        assert exc.value.status == tn.TN_ERANGE
        # decreasing timestamps inside a batch are rejected
        rev = dt[3000:3010].flip(0).contiguous()
        if rev[0] > rev[-1]:
            with pytest.raises(tn.TnError) as exc:
                on.push(du[3000:3010], dv[3000:3010], rev)
            assert exc.value.status == tn.TN_EORDER
        assert on.state()["pending_events"] == pend
        assert torch.equal(on.matrix(), before)
        on.push(du[3000:], dv[3000:], dt[3000:])
        on.flush()
        want = oracle.to_bool(oracle.component_matrix(u, v, t, n), n)
        assert np.array_equal(gpu_bits(on.matrix(), n), want)


def test_growth_between_batches_in_place_and_reallocated():
    """n: 1000 -> 1020 (same row stride: in place) -> 2500 (new stride), with a
    timestamp group pending across each growth; new nodes join later batches."""
    rng = np.random.default_rng(4)
    sizes = [1000, 1020, 2500]
    us, vs, ts = [], [], []
    t0 = 0
    for n_k in sizes:
        m_k = 8 * n_k
        us.append(rng.integers(0, n_k, m_k).astype(np.uint32))
        vs.append(rng.integers(0, n_k, m_k).astype(np.uint32))
        ts.append(np.sort(rng.integers(t0, t0 + 400, m_k)).astype(np.int64))
        t0 += 400
    # each batch ends inside a group that the next batch (same t) continues
    for k in range(len(sizes) - 1):
        ts[k + 1][:5] = ts[k][-1]
    u, v, t = np.concatenate(us), np.concatenate(vs), np.concatenate(ts)
    with tn.Online(sizes[0]) as on:
        S_first = on.state()["S"]
        for k, n_k in enumerate(sizes):
            if k:
                on.grow(n_k)
                st = on.state()
                assert st["n"] == n_k and st["pending_events"] > 0
                assert (st["S"] == S_first) == (tn.tn_row_words(n_k) == tn.tn_row_words(sizes[0]))
            on.push(dev(us[k]), dev(vs[k]), dev(ts[k], np.int64))
        on.flush()
        got = gpu_bits(on.matrix(), sizes[-1])
    # the oracle's definition, step by step: complete groups, grow, continue
    S = oracle.init_sources(sizes[0])
    n_prev, done = sizes[0], 0
    for k, n_k in enumerate(sizes):
        if k:
            S = oracle.grow_matrix(S, n_prev, n_k)
            n_prev = n_k
        end = len(np.concatenate(ts[:k + 1]))
        upto = end if k == len(sizes) - 1 else int(np.searchsorted(t, t[end - 1], side="left"))
        oracle.apply_events(u[done:upto], v[done:upto], t[done:upto], n_k, S)
        done = upto
    assert np.array_equal(got, oracle.to_bool(S, sizes[-1]))
    # nodes that join later have no earlier events: same as the whole network from the start
    assert np.array_equal(got, oracle.to_bool(oracle.component_matrix(u, v, t, sizes[-1]), sizes[-1]))


@pytest.mark.parametrize("n_old,n_new", [(0, 700), (1500, 1500), (1500, 2100), (1024, 1025), (3000, 3070)])
def test_grow_matrix_out_of_place(n_old, n_new):
    if n_old:
        u, v, t = synth.uniform_events(n_old, 6 * n_old, t_range=3 * n_old, seed=n_old)
        S = tn.tn_component_matrix(dev(u), dev(v), dev(t, np.int64), n_old)
        ref = oracle.component_matrix(u, v, t, n_old)
    else:
        S = torch.empty((0, 0), dtype=torch.int64, device="cuda")
        ref = np.zeros((0, 1), np.uint64)
    G = tn.tn_grow_matrix(S, n_old, n_new)
    assert np.array_equal(gpu_bits(G, n_new), oracle.to_bool(oracle.grow_matrix(ref, n_old, n_new), n_new))


@pytest.mark.parametrize("n_old,n_new", [(1100, 2048), (64, 1000), (1000, 1001)])
def test_grow_matrix_in_place_clears_stale_columns(n_old, n_new):
    assert tn.tn_row_words(n_old) == tn.tn_row_words(n_new)
    W = tn.tn_row_words(n_new)
    u, v, t = synth.uniform_events(n_old, 5 * n_old, t_range=2 * n_old, seed=7)
    buf = torch.full((n_new, W), -1, dtype=torch.int64, device="cuda")  # stale bits everywhere
    tn.tn_component_matrix(dev(u), dev(v), dev(t, np.int64), n_old, S=buf[:n_old])
    # stale bits in the columns the old matrix does not own
    w = n_old // 64
    if n_old % 64:
        buf[:n_old, w] |= torch.tensor(-(1 << (n_old % 64)), dtype=torch.int64, device="cuda")
        w += 1
    buf[:n_old, w:] = -1
    out = tn.tn_grow_matrix(buf[:n_old], n_old, n_new, out=buf)
    assert out.data_ptr() == buf.data_ptr()
    ref = oracle.grow_matrix(oracle.component_matrix(u, v, t, n_old), n_old, n_new)
    assert np.array_equal(gpu_bits(buf, n_new), oracle.to_bool(ref, n_new))


def test_grow_matrix_rejects_bad_arguments():
    u, v, t = synth.uniform_events(100, 300, t_range=50, seed=1)
    S = tn.tn_component_matrix(dev(u), dev(v), dev(t, np.int64), 100)
    with pytest.raises(tn.TnError) as exc:
        tn.tn_grow_matrix(S, 100, 50)
    assert exc.value.status == tn.TN_EINVAL
    big = torch.zeros((2000, tn.tn_row_words(2000)), dtype=torch.int64, device="cuda")
    old = big.view(-1)[: 1000 * tn.tn_row_words(1000)].view(1000, tn.tn_row_words(1000))
    with pytest.raises(tn.TnError) as exc:  # in place, but the row stride would change
        tn.tn_grow_matrix(old, 1000, 2000, out=big)
    assert exc.value.status == tn.TN_EINVAL
    with pytest.raises(tn.TnError) as exc:  # partially overlapping buffers
        tn.tn_grow_matrix(old, 1000, 1500, out=big.view(-1)[16:16 + 1500 * 32].view(1500, 32))
    assert exc.value.status == tn.TN_EINVAL
    on = tn.Online(100)
    with pytest.raises(tn.TnError) as exc:
        on.grow(99)
    assert exc.value.status == tn.TN_EINVAL
    on.close()


@pytest.mark.parametrize("seed", [0, 1])
def test_online_directed_split_groups(seed):
    n, m = 500, 12_000
    u, v, t = synth.uniform_events(n, m, t_range=150, seed=10 + seed)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    with tn.Online(n, directed=True) as on:
        for a, b in cuts_through_groups(t, np.random.default_rng(seed), 12):
            on.push(du[a:b], dv[a:b], dt[a:b])
        on.flush()
        got = gpu_bits(on.matrix(), n)
    assert np.array_equal(got, oracle.to_bool(oracle.component_matrix_directed(u, v, t, n), n))


def test_online_equals_one_shot_at_scale():
    """Activity-driven events over 20,000 nodes split into 7 batches at arbitrary
    points; the result must equal the one-shot library call bit for bit."""
    n, m = 20_000, 2_000_000
    u, v, t = synth.activity_driven(n, m, seed=6)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    ref = tn.tn_component_matrix(du, dv, dt, n)
    cuts = np.sort(np.random.default_rng(6).choice(np.arange(1, m), 6, replace=False))
    with tn.Online(n, slab_words=8) as on:
        for a, b in zip(np.r_[0, cuts], np.r_[cuts, m]):
            on.push(du[a:b], dv[a:b], dt[a:b])
        on.flush()
        assert on.status() == 0
        assert torch.equal(on.matrix(), ref)
    rng = np.random.default_rng(16)
    cols = np.sort(rng.choice(n, 24, replace=False)).astype(np.uint32)
    want = oracle.to_bool(oracle.component_matrix(u, v, t, n, cols), len(cols))
    got = ((ref[:, torch.from_numpy(cols.astype(np.int64) // 64).cuda()]
            >> torch.from_numpy(cols.astype(np.int64) % 64).cuda()) & 1).bool().cpu().numpy()
    assert np.array_equal(got, want)


def test_hashed_network_streamed_with_new_nodes():
    """Section 4 with Section 3.5: the hash is a function of the node id, so the
    tables of a grown network extend those of the smaller one, and the k x k
    proxy matrices never grow.  Streaming the super-events of batches whose
    later part names new nodes through R online states (groups split across
    batches) gives the same proxies and estimates as the one-shot hashed path
    over the final network, and the oracle's."""
    n0, n1, k, R, seed = 1500, 2600, 256, 4, 9
    rng = np.random.default_rng(seed)
    m0, m1 = 20_000, 30_000
    u = np.r_[rng.integers(0, n0, m0), rng.integers(0, n1, m1)].astype(np.uint32)
    v = np.r_[rng.integers(0, n0, m0), rng.integers(0, n1, m1)].astype(np.uint32)
    t = np.r_[np.sort(rng.integers(0, 500, m0)), np.sort(rng.integers(499, 1000, m1))].astype(np.int64)
    du, dv, dt = dev(u), dev(v), dev(t, np.int64)
    H0, _, _ = tn.tn_hash_proxy(None, None, n0, k, R, seed, events=False)
    H1, pu, pv = tn.tn_hash_proxy(du, dv, n1, k, R, seed)
    assert torch.equal(H1[:, :n0], H0)  # the grown network's tables extend the old ones
    states = [tn.Online(k) for _ in range(R)]
    for a, b in cuts_through_groups(t, rng, 10):
        for j in range(R):
            states[j].push(pu[j, a:b].contiguous(), pv[j, a:b].contiguous(), dt[a:b])
    P_stream = torch.empty((R, k, tn.tn_row_words(k)), dtype=torch.int64, device="cuda")
    for j in range(R):
        states[j].flush()
        P_stream[j].copy_(states[j].matrix())
        states[j].close()
    P_batch = torch.empty_like(P_stream)
    plans = [tn.Plan(pu[j].contiguous(), pv[j].contiguous(), dt, k) for j in range(R)]
    tn.tn_plan_apply_batch(plans, [P_batch[j] for j in range(R)])
    assert torch.equal(P_stream, P_batch)
    est = tn.tn_hash_estimate(P_stream, R, k, H1, n1).cpu().numpy().view(np.uint32)
    Href = oracle.hash_nodes(seed, R, k, n1)
    want = oracle.hash_estimate(oracle.proxy_matrices(u, v, t, Href, k), Href, n1)
    assert np.array_equal(est, want)
