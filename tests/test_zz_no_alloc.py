"""tn_hash_estimate_noalloc against tn_hash_estimate (needs a GPU: -m gpu).

The no-alloc variant serves callers that cannot allocate device memory during
a call (code inside another framework's memory budget, latency-bound loops).
The no-alloc entry point keeps its scratch in one fixed device array, so each
case calls it twice in a row and checks both results against the allocating
entry point on the same inputs: a first call that leaves stale scratch behind
would show up in the second.  Covers the shared-memory table, the global
table inside the fixed scratch, the size limit and the source-id check.
"""
import ctypes
import os

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


_USED_CURRENT, _USED_HIGH = 0x7, 0x8  # cudaMemPoolAttrUsedMemCurrent / cudaMemPoolAttrUsedMemHigh


def _cudart():
    for name in ("libcudart.so.13", "libcudart.so", os.path.join("/usr/local/cuda/lib64", "libcudart.so")):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("CUDA runtime library not found for the allocation check")


def _pool_reset_and_read(rt, reset):
    """Bytes in use from the current device's default stream-ordered pool (the
    pool the library's allocating entry points draw on) and its high-water
    mark; with `reset` the mark is first reset to the current use."""
    pool = ctypes.c_void_p()
    assert rt.cudaDeviceGetDefaultMemPool(ctypes.byref(pool), torch.cuda.current_device()) == 0
    if reset:
        zero = ctypes.c_uint64(0)
        assert rt.cudaMemPoolSetAttribute(pool, _USED_HIGH, ctypes.byref(zero)) == 0
    cur, high = ctypes.c_uint64(), ctypes.c_uint64()
    assert rt.cudaMemPoolGetAttribute(pool, _USED_CURRENT, ctypes.byref(cur)) == 0
    assert rt.cudaMemPoolGetAttribute(pool, _USED_HIGH, ctypes.byref(high)) == 0
    return cur.value, high.value


def twice(P, R, k, H, n, src, nsrc):
    """Two calls in a row; asserts that neither allocated device memory: the
    stream-ordered pool's high-water mark stays at its use before the calls,
    and torch's allocator hands out nothing beyond the two output tensors."""
    outs = [torch.full((nsrc,), -1, dtype=torch.int32, device="cuda") for _ in range(2)]
    rt = _cudart()
    torch.cuda.synchronize()
    used0, _ = _pool_reset_and_read(rt, reset=True)
    torch_before = torch.cuda.memory_allocated()
    for est in outs:
        tn.tn_hash_estimate_noalloc(P, R, k, H, n, est, src=src)
    torch.cuda.synchronize()
    used1, high = _pool_reset_and_read(rt, reset=False)
    assert used1 == used0 and high == used0, "the no-alloc entry point drew on the stream-ordered pool"
    assert torch.cuda.memory_allocated() == torch_before
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
