"""HyperLogLog sketches of the components on the GPU (Sections 3.3, 3.4; needs a GPU: -m gpu).

Registers are integers: bit-exact to the oracle in every mode.  Estimates are
doubles summed in another order: within 1e-12 relative.  Against the exact
component sizes they stay within the HLL error.
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


@pytest.mark.parametrize("n,m,t_range,p,reverse,directed", [
    (300, 6000, 6000, 6, False, False),
    (300, 6000, 40, 8, False, False),    # tie groups
    (500, 9000, 9000, 10, True, False),  # out-components
    (400, 8000, 200, 7, False, True),
    (400, 8000, 200, 7, True, True),
    (2000, 30_000, 15, 4, False, False), # giant groups: global tiles
    (150, 2000, 3000, 16, False, False), # widest sketch
])
def test_hll_registers_and_estimates_match_oracle(n, m, t_range, p, reverse, directed):
    u, v, t = synth.uniform_events(n, m, t_range=t_range, seed=p + n, self_loops=True)
    R = tn.tn_hll_sketches(dev(u), dev(v), dev(t, np.int64), n, p, 99, reverse=reverse, directed=directed)
    est = tn.tn_hll_estimate(R, n, p)
    torch.cuda.synchronize()
    s = 1 << p
    got = R.cpu().numpy()
    want = oracle.hll_sketches(u, v, t, n, p, 99, reverse=reverse, directed=directed)
    assert np.array_equal(got[:, :s], want)
    assert not got[:, s:].any()  # row padding stays zero
    assert np.allclose(est.cpu().numpy(), oracle.hll_estimate(want, p), rtol=1e-12, atol=0)


def test_hll_estimates_track_exact_sizes():
    n, m, p = 3000, 60_000, 10
    u, v, t = synth.activity_driven(n, m, seed=5)
    R = tn.tn_hll_sketches(dev(u), dev(v), dev(t, np.int64), n, p, 7, reverse=True)
    est = tn.tn_hll_estimate(R, n, p).cpu().numpy()
    exact = oracle.column_counts(oracle.component_matrix(u, v, t, n), n).astype(np.float64)
    rel = np.abs(est / exact - 1.0)
    assert rel.mean() < 3 * 1.04 / np.sqrt(1 << p)
    # the average size (Eq. s_t) from the sketches
    assert abs(est.mean() / exact.mean() - 1.0) < 0.05


def test_hll_rejects_bad_arguments():
    u = dev(np.array([0, 9], np.uint32)); v = dev(np.array([1, 2], np.uint32)); t = dev(np.array([0, 1], np.int64), np.int64)
    with pytest.raises(tn.TnError) as exc:
        tn.tn_hll_sketches(u, v, t, 5, 6, 1)  # endpoint 9 >= n
    assert exc.value.status == tn.TN_ERANGE
    with pytest.raises(ValueError):
        tn.tn_hll_sketches(u, v, t, 10, 3, 1)
