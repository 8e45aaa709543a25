"""tn_hash_estimate_noalloc against tn_hash_estimate (needs a GPU: -m gpu).

The no-alloc variant serves callers that cannot allocate device memory during
a call (code inside another framework's memory budget, latency-bound loops).
The no-alloc entry point keeps its scratch in one fixed device array, so each
case calls it twice in a row and checks both results against the allocating
entry point on the same inputs: a first call that leaves stale scratch behind
would show up in the second.  Covers the shared-memory table, the global
table inside the fixed scratch, the size limit and the source-id check.
"""
import numpy as np
import pytest

from paper_2307_04890_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if torch.cuda.is_available():
    import paper_2307_04890_gb300 as tn
    from paper_2307_04890_gb300.build import build_library

    build_library()

TABLE_LIMIT = 8 << 20  # TN_NOALLOC_TABLE_BYTES


def proxies(n, m, k, R, seed):
    u, v, t = synth.uniform_events(n, m, t_range=m // 2, seed=seed)
    d = torch.device("cuda")
    du = torch.from_numpy(u.view(np.int32)).to(d)
    dv = torch.from_numpy(v.view(np.int32)).to(d)
    dt = torch.from_numpy(t).to(d)
    H, pu, pv = tn.tn_hash_proxy(du, dv, n, k, R, seed)
    P = torch.empty((R, k, tn.tn_row_words(k)), dtype=torch.int64, device=d)
    for j in range(R):
        tn.tn_component_matrix(pu[j].contiguous(), pv[j].contiguous(), dt, k, S=P[j])
    return P, H


def twice(P, R, k, H, n, src, nsrc):
    outs = []
    for _ in range(2):
        est = torch.full((nsrc,), -1, dtype=torch.int32, device="cuda")
        tn.tn_hash_estimate_noalloc(P, R, k, H, n, est, src=src)
        outs.append(est)
    torch.cuda.synchronize()
    return [e.cpu().numpy() for e in outs]


def test_shared_memory_table_all_sources():
    n, k, R = 3000, 257, 3
    P, H = proxies(n, 30_000, k, R, seed=4)
    ref = tn.tn_hash_estimate(P, R, k, H, n).cpu().numpy()
    for got in twice(P, R, k, H, n, None, n):
        assert np.array_equal(got, ref)


def test_global_table_in_fixed_scratch_and_limit():
    n, k, R = 5000, 3300, 64  # R * k = 211,200 B: beyond the shared-memory table
    assert R * k > 200 * 1024
    P, H = proxies(n, 20_000, k, R, seed=9)
    rng = np.random.default_rng(9)
    nsrc = 300  # 38 CTAs x 211,200 B = 8,025,600 B of table, inside the limit
    assert ((nsrc + 7) // 8) * R * k <= TABLE_LIMIT
    src = torch.from_numpy(rng.integers(0, n, nsrc).astype(np.int32)).cuda()
    ref = tn.tn_hash_estimate(P, R, k, H, n, src=src).cpu().numpy()
    for got in twice(P, R, k, H, n, src, nsrc):
        assert np.array_equal(got, ref)

    big = torch.from_numpy(rng.integers(0, n, 320).astype(np.int32)).cuda()  # 40 CTAs: 8,448,000 B
    assert ((320 + 7) // 8) * R * k > TABLE_LIMIT
    est = torch.zeros(320, dtype=torch.int32, device="cuda")
    with pytest.raises(tn.TnError) as exc:
        tn.tn_hash_estimate_noalloc(P, R, k, H, n, est, src=big)
    assert exc.value.status == tn.TN_ESCRATCH
    assert "fixed scratch" in str(exc.value)
    for got in twice(P, R, k, H, n, src, nsrc):  # still correct after the rejected call
        assert np.array_equal(got, ref)


def test_source_check_flag_is_cleared():
    n, k, R = 2000, 101, 4
    P, H = proxies(n, 10_000, k, R, seed=12)
    bad = torch.tensor([0, 5, n], dtype=torch.int32, device="cuda")
    est = torch.zeros(3, dtype=torch.int32, device="cuda")
    with pytest.raises(tn.TnError) as exc:
        tn.tn_hash_estimate_noalloc(P, R, k, H, n, est, src=bad)
    assert exc.value.status == tn.TN_ERANGE
    good = torch.tensor([0, 5, n - 1, 17], dtype=torch.int32, device="cuda")
    ref = tn.tn_hash_estimate(P, R, k, H, n, src=good).cpu().numpy()
    for got in twice(P, R, k, H, n, good, 4):
        assert np.array_equal(got, ref)
