"""Pins for the CPU oracle (no GPU).

The oracle is checked against things fixed by the paper and by mathematics,
never against itself: hand-derived worked examples (tests/golden), brute-force
SI simulation (Section 1), closed forms, invariants of reachability, and
library routines for the special cases that reduce to them.
"""
import itertools

import numpy as np
import pytest

import oracle
from conftest import golden_names, load_golden
from paper_2307_04890_gb300 import synth


def _arrays(events):
    ev = np.array(events, dtype=np.int64).reshape(-1, 3)
    return ev[:, 0].astype(np.uint32), ev[:, 1].astype(np.uint32), ev[:, 2].astype(np.int64)


def _oc_sets(S, n):
    B = oracle.to_bool(S, n)
    return {j: sorted(np.flatnonzero(B[:, j]).tolist()) for j in range(n)}


# --------------------------------------------------------------------------
# hand-derived worked examples
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", golden_names())
def test_golden_examples(name):
    n, events, oc, rows = load_golden(name)
    u, v, t = _arrays(events)
    S = oracle.component_matrix(u, v, t, n)
    got = _oc_sets(S, n)
    for j, want in oc.items():
        assert got[j] == want, (name, j)
        # the SI simulation from the same source agrees
        assert sorted(np.flatnonzero(oracle.si_reach(u, v, t, n, j)).tolist()) == want
    B = oracle.to_bool(S, n)
    for i, want in rows.items():
        assert sorted(np.flatnonzero(B[i]).tolist()) == want, (name, "row", i)


# --------------------------------------------------------------------------
# brute force: SI simulation from every source equals every column
# --------------------------------------------------------------------------
def _matrix_equals_si(u, v, t, n):
    S = oracle.component_matrix(u, v, t, n)
    B = oracle.to_bool(S, n)
    for j in range(n):
        si = oracle.si_reach(u, v, t, n, j)
        if not np.array_equal(B[:, j], si):
            return False
    return True


def test_exhaustive_tiny_sequences():
    """Every event sequence of length <= 4 over the 6 links of 4 nodes, with
    non-decreasing timestamps drawn from {0, 1, 2}."""
    n = 4
    links = [(a, b) for a in range(n) for b in range(a + 1, n)]
    checked = 0
    for length in range(1, 5):
        for times in itertools.combinations_with_replacement(range(3), length):
            for seq in itertools.product(links, repeat=length):
                u = np.array([p[0] for p in seq], dtype=np.uint32)
                v = np.array([p[1] for p in seq], dtype=np.uint32)
                t = np.array(times, dtype=np.int64)
                assert _matrix_equals_si(u, v, t, n), (seq, times)
                checked += 1
    assert checked == 21834


@pytest.mark.parametrize("seed", range(60))
def test_random_dense_ties_vs_si(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(2, 71))
    m = int(rng.integers(1, 301))
    u = rng.integers(0, n, m)
    v = rng.integers(0, n, m)  # self-loops allowed
    t = np.sort(rng.integers(0, int(rng.integers(1, 12)), m))
    assert _matrix_equals_si(u.astype(np.uint32), v.astype(np.uint32), t, n)


def test_medium_random_vs_si_sampled():
    u, v, t = synth.uniform_events(800, 20000, t_range=5000, seed=7)
    n = 800
    S = oracle.component_matrix(u, v, t, n)
    B = oracle.to_bool(S, n)
    for j in np.random.default_rng(0).choice(n, 40, replace=False):
        assert np.array_equal(B[:, j], oracle.si_reach(u, v, t, n, int(j)))


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------
def test_star_distinct_times():
    k = 50
    u = np.zeros(k, np.uint32)
    v = np.arange(1, k + 1, dtype=np.uint32)
    t = np.arange(1, k + 1, dtype=np.int64)
    sizes = oracle.column_counts(oracle.component_matrix(u, v, t, k + 1), k + 1)
    assert sizes[0] == k + 1
    for i in range(1, k + 1):  # leaf i meets the centre at time i, then reaches later leaves
        assert sizes[i] == 2 + (k - i)


def test_path_forward_and_backward():
    k = 90
    # forward: link (j-1, j) at time j
    u = np.arange(0, k, dtype=np.uint32)
    v = np.arange(1, k + 1, dtype=np.uint32)
    t = np.arange(1, k + 1, dtype=np.int64)
    s = oracle.column_counts(oracle.component_matrix(u, v, t, k + 1), k + 1)
    assert s[0] == k + 1
    assert all(s[j] == k - j + 2 for j in range(1, k + 1))
    # backward: link (j, j+1) at time k - j, so time runs from node k down to 0
    t2 = (k - np.arange(0, k)).astype(np.int64)
    order = np.argsort(t2, kind="stable")
    s2 = oracle.column_counts(oracle.component_matrix(u[order], v[order], t2[order], k + 1), k + 1)
    assert all(s2[j] == min(j + 2, k + 1) for j in range(k + 1))


def test_single_group_is_identity_plus_adjacency():
    rng = np.random.default_rng(3)
    n, m = 60, 200
    u = rng.integers(0, n, m).astype(np.uint32)
    v = rng.integers(0, n, m).astype(np.uint32)
    t = np.full(m, 5, dtype=np.int64)
    B = oracle.to_bool(oracle.component_matrix(u, v, t, n), n)
    A = np.eye(n, dtype=bool)
    A[u, v] = True
    A[v, u] = True
    assert np.array_equal(B, A)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------
def _cfg_small(seed):
    return synth.uniform_events(300, 6000, t_range=2000, seed=seed), 300


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_diagonal_and_row_col_sums(seed):
    (u, v, t), n = _cfg_small(seed)
    S = oracle.component_matrix(u, v, t, n)
    B = oracle.to_bool(S, n)
    assert B.diagonal().all()
    assert oracle.column_counts(S, n).sum() == oracle.row_counts(S).sum() == B.sum()


@pytest.mark.parametrize("seed", [0, 1])
def test_concatenation_is_boolean_product(seed):
    """Split at a boundary between timestamp groups: S_full = S_suffix (x) S_prefix."""
    (u, v, t), n = _cfg_small(seed)
    cut = int(np.searchsorted(t, t[len(t) // 2], side="left"))
    Sp = oracle.to_bool(oracle.component_matrix(u[:cut], v[:cut], t[:cut], n), n).astype(np.int64)
    Ss = oracle.to_bool(oracle.component_matrix(u[cut:], v[cut:], t[cut:], n), n).astype(np.int64)
    Sf = oracle.to_bool(oracle.component_matrix(u, v, t, n), n)
    assert np.array_equal((Ss @ Sp) > 0, Sf)


def test_incremental_equals_one_shot_and_monotone():
    (u, v, t), n = _cfg_small(5)
    full = oracle.component_matrix(u, v, t, n)
    S = oracle.init_sources(n)
    prev = oracle.column_counts(S, n)
    for a, b in synth.split_batches(t, 4):
        oracle.apply_events(u[a:b], v[a:b], t[a:b], n, S)
        cur = oracle.column_counts(S, n)
        assert (cur >= prev).all()
        prev = cur
    assert np.array_equal(S, full)


# --------------------------------------------------------------------------
# node growth (Section 3.5: a new node is a new row and column of zeros with
# its own diagonal bit set)
# --------------------------------------------------------------------------
def _pack(B):
    B = np.asarray(B, dtype=bool)
    W = max(1, oracle.words(B.shape[1]))
    out = np.zeros((B.shape[0], W), dtype=np.uint64)
    for i, j in zip(*np.nonzero(B)):
        out[i, j // 64] |= np.uint64(1) << np.uint64(j % 64)
    return out


def test_grow_hand_example():
    old = [[1, 1, 0],
           [0, 1, 0],
           [0, 1, 1]]
    want = [[1, 1, 0, 0, 0],
            [0, 1, 0, 0, 0],
            [0, 1, 1, 0, 0],
            [0, 0, 0, 1, 0],
            [0, 0, 0, 0, 1]]
    G = oracle.grow_matrix(_pack(old), 3, 5)
    assert np.array_equal(oracle.to_bool(G, 5), np.array(want, dtype=bool))


@pytest.mark.parametrize("n_old,n_new", [(0, 4), (5, 5), (64, 65), (60, 130)])
def test_grow_identity_stays_identity(n_old, n_new):
    G = oracle.grow_matrix(oracle.init_sources(n_old) if n_old else np.zeros((0, 1), np.uint64), n_old, n_new)
    assert np.array_equal(oracle.to_bool(G, n_new), np.eye(n_new, dtype=bool))


@pytest.mark.parametrize("seed,n_old,n_new", [(0, 60, 130), (1, 10, 11), (2, 128, 200)])
def test_grow_then_stream_matches_si_on_the_larger_network(seed, n_old, n_new):
    """Nodes that join after the first batch: growing the matrix and streaming
    the second batch gives every source's SI reach over all events."""
    rng = np.random.default_rng(seed)
    m1, m2 = 3 * n_old, 3 * n_new
    u1 = rng.integers(0, n_old, m1).astype(np.uint32)
    v1 = rng.integers(0, n_old, m1).astype(np.uint32)
    t1 = np.sort(rng.integers(0, 50, m1)).astype(np.int64)
    u2 = rng.integers(0, n_new, m2).astype(np.uint32)
    v2 = rng.integers(0, n_new, m2).astype(np.uint32)
    t2 = np.sort(rng.integers(50, 100, m2)).astype(np.int64)
    S = oracle.grow_matrix(oracle.component_matrix(u1, v1, t1, n_old), n_old, n_new)
    oracle.apply_events(u2, v2, t2, n_new, S)
    B = oracle.to_bool(S, n_new)
    u, v, t = np.concatenate([u1, u2]), np.concatenate([v1, v2]), np.concatenate([t1, t2])
    for j in range(n_new):
        assert np.array_equal(B[:, j], oracle.si_reach(u, v, t, n_new, j)), j


def test_grow_rejects_shrinking():
    with pytest.raises(oracle.OracleError):
        oracle.grow_matrix(oracle.init_sources(5), 5, 4)


def test_split_group_needs_the_whole_group():
    """A timestamp group is one snapshot: applying its two halves as separate
    batches (what an incremental caller would do without carrying the group)
    lets a path run through it, which the whole group does not."""
    u, v, t = _arrays([(0, 1, 1), (1, 2, 1)])
    whole = oracle.to_bool(oracle.component_matrix(u, v, t, 3), 3)
    assert sorted(np.flatnonzero(whole[:, 0]).tolist()) == [0, 1]
    S = oracle.init_sources(3)
    oracle.apply_events(u[:1], v[:1], t[:1], 3, S)
    oracle.apply_events(u[1:], v[1:], t[1:], 3, S)
    assert sorted(np.flatnonzero(oracle.to_bool(S, 3)[:, 0]).tolist()) == [0, 1, 2]


def test_order_inside_groups_is_irrelevant():
    (u, v, t), n = _cfg_small(9)
    rng = np.random.default_rng(1)
    perm = np.lexsort((rng.random(len(t)), t))  # shuffle inside each group
    assert np.array_equal(oracle.component_matrix(u, v, t, n),
                          oracle.component_matrix(u[perm], v[perm], t[perm], n))


def test_sequential_semantics_differs_on_ties():
    """The snapshot reading matters: processing a tie group event by event
    (plain Algorithm 1 order) would give a different matrix here."""
    n, events, oc, _ = load_golden("star_tie.txt")
    u, v, t = _arrays(events)
    distinct = np.arange(len(t), dtype=np.int64)
    B = oracle.to_bool(oracle.component_matrix(u, v, distinct, n), n)
    assert sorted(np.flatnonzero(B[:, 2]).tolist()) != oc[2]


def test_source_subset_equals_columns():
    (u, v, t), n = _cfg_small(4)
    full = oracle.to_bool(oracle.component_matrix(u, v, t, n), n)
    src = np.random.default_rng(2).choice(n, 100, replace=False).astype(np.uint32)
    sub = oracle.to_bool(oracle.component_matrix(u, v, t, n, src=src), len(src))
    assert np.array_equal(sub, full[:, src])


def test_validation_errors():
    u = np.array([0, 1], np.uint32)
    v = np.array([1, 5], np.uint32)
    t = np.array([0, 1], np.int64)
    assert oracle.validate(u, v, t, 5) == oracle.ERANGE
    assert oracle.validate(u, v, t[::-1].copy(), 6) == oracle.EORDER
    with pytest.raises(oracle.OracleError):
        oracle.component_matrix(u, v, t, 5)


def test_argmax_lowest_index():
    assert oracle.argmax(np.array([3, 7, 7, 1], np.uint32)) == 1


# --------------------------------------------------------------------------
# hashing (Section 4.1)
# --------------------------------------------------------------------------
P61 = (1 << 61) - 1


M64 = (1 << 64) - 1


def test_splitmix64_known_answer():
    """SplitMix64 (Steele, Lea and Flood, OOPSLA 2014; Vigna's reference C
    implementation splitmix64.c) started at state 1234567 gives the sequence
    below, the known-answer values that ports of the generator check in their
    test suites.  A mistyped increment, multiplier or shift changes every one."""
    want = [6457827717110365317, 3203168211198807973, 9817491932198370423,
            4593380528125082431, 16408922859458223821]
    assert [int(x) for x in oracle.splitmix64_stream(1234567, 5)] == want


def _splitmix64_py(state, count):
    """The published generator in Python integers: a Weyl step of the golden
    gamma 0x9E3779B97F4A7C15, then the variant-13 finaliser (30, 27, 31)."""
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_matches_big_integer_generator():
    assert _splitmix64_py(1234567, 5) == [int(x) for x in oracle.splitmix64_stream(1234567, 5)]
    for state in (0, 1, 2**63, M64, 0xDEADBEEFCAFEF00D):
        assert _splitmix64_py(state, 64) == [int(x) for x in oracle.splitmix64_stream(state, 64)]


def test_hash_coeffs_match_big_integer_restatement():
    """The coefficient rule (Section 4.1, with the reading of the unnamed rand
    as SplitMix64 reduced mod 2^31 - 1): replica j's stream starts at
    splitmix64(seed XOR j); A(i, c) = ((r1 << 32) + r2) mod p, drawn for
    i = 0..2, c = 0..3, r1 before r2.  Written here in unbounded integers."""
    for seed in (0, 1, 123, 2**40 + 7, M64):
        for j in range(4):
            stream = _splitmix64_py(seed ^ j, 1)[0]
            draws = _splitmix64_py(stream, 24)
            want = [(((draws[2 * q] % (2**31 - 1)) << 32) + draws[2 * q + 1] % (2**31 - 1)) % P61
                    for q in range(12)]
            assert [int(a) for a in oracle.hash_coeffs(seed, j)] == want


def test_table_value_matches_big_integer_horner():
    """T_i[x] = ((A0 x + A1) x + A2) x + A3 mod 2^61 - 1 (MultAddMod applied
    order - 1 = 3 times), in unbounded integers, over coefficients anywhere in
    the field (including p - 1) and every key size the hash uses (x < 2^17)."""
    rng = np.random.default_rng(5)
    rows = [[P61 - 1] * 4, [0, 0, 0, P61 - 1], [1, 0, 0, 0]]
    rows += [[int(a) for a in rng.integers(0, P61, 4, dtype=np.uint64)] for _ in range(40)]
    xs = [0, 1, 2, 65535, 65536, 131069, 131070] + [int(x) for x in rng.integers(0, 131071, 20)]
    for A in rows:
        arr = np.array(A, dtype=np.uint64)
        for x in xs:
            acc = A[0]
            for c in range(1, 4):
                acc = (acc * x + A[c]) % P61
            assert oracle.table_value(arr, 0, x) == acc


def test_hash_coefficients_in_field_and_distinct():
    A0 = oracle.hash_coeffs(123, 0)
    A1 = oracle.hash_coeffs(123, 1)
    assert (A0 < P61).all() and (A1 < P61).all()
    assert not np.array_equal(A0, A1)
    assert np.array_equal(A0, oracle.hash_coeffs(123, 0))
    assert len(set(A0.tolist())) == 12


def test_hash_range_and_uniformity():
    from scipy import stats
    k, n = 64, 200_000
    H = oracle.hash_nodes(11, 2, k, n)
    assert H.max() < k
    for j in range(2):
        counts = np.bincount(H[j], minlength=k)
        assert stats.chisquare(counts).pvalue > 1e-4


def test_hash_pairwise_collisions():
    k, n = 97, 4000
    rates = []
    for seed in range(40):
        H = oracle.hash_nodes(seed, 1, k, n)[0]
        rates.append((H[:-1] == H[1:]).mean())
    assert abs(np.mean(rates) - 1 / k) < 0.25 / k


def test_hash_tables_are_cubics_mod_p():
    """Each table is the polynomial A0 x^3 + A1 x^2 + A2 x + A3 over GF(p)
    (Horner recursion of MultAddMod, order 4): its constant term is A3 and its
    third finite difference is the constant 3! * A0 (mod p)."""
    for seed in range(5):
        A = [int(a) for a in oracle.hash_coeffs(seed, 2)]
        for i in range(3):
            a0, a3 = A[4 * i], A[4 * i + 3]
            assert oracle.table_value(oracle.hash_coeffs(seed, 2), i, 0) == a3
            for x in (0, 1, 1000, 65530, 131068):
                T = [oracle.table_value(oracle.hash_coeffs(seed, 2), i, x + d) for d in range(4)]
                d3 = (T[3] - 3 * T[2] + 3 * T[1] - T[0]) % P61
                assert d3 == (6 * a0) % P61


def test_hash_combines_three_tables():
    """h(u) = T0[u & 0xFFFF] ^ T1[u >> 16] ^ T2[(u & 0xFFFF) + (u >> 16)]."""
    A = oracle.hash_coeffs(77, 0)
    for x in (0, 1, 65535, 65536, 123456789, 2**32 - 1):
        x0, x1 = x & 0xFFFF, x >> 16
        want = oracle.table_value(A, 0, x0) ^ oracle.table_value(A, 1, x1) ^ oracle.table_value(A, 2, x0 + x1)
        assert oracle.hash_raw(A, x) == want


def test_hash_rectangle_breaks_simple_tabulation():
    """Keys (a,c),(a,d),(b,c),(b,d) (16-bit characters) always XOR to zero under
    simple two-table tabulation; the derived third character T2[x0+x1]
    (Thorup-Zhang) removes that dependence, making the family 4-universal."""
    keys = [a | (c << 16) for a in (1, 2) for c in (10, 20)]
    zero = 0
    patterns = np.zeros(16, dtype=np.int64)
    seeds = 4000
    for seed in range(seeds):
        A = oracle.hash_coeffs(seed, 0)
        h = [oracle.hash_raw(A, x) for x in keys]
        zero += (h[0] ^ h[1] ^ h[2] ^ h[3]) == 0
        bits = [x & 1 for x in h]
        patterns[bits[0] | bits[1] << 1 | bits[2] << 2 | bits[3] << 3] += 1
    assert zero == 0
    from scipy import stats
    assert stats.chisquare(patterns).pvalue > 1e-4


# --------------------------------------------------------------------------
# fusion (Section 4.2)
# --------------------------------------------------------------------------
def _hashed_case(seed, n=120, m=60, k=45, R=3):
    """Sparse hashed networks: proxy out-components are small and the proxy
    matrices far from symmetric, so a swapped row/column test would show."""
    u, v, t = synth.uniform_events(n, m, t_range=300, seed=seed)
    H = oracle.hash_nodes(seed, R, k, n)
    P = oracle.proxy_matrices(u, v, t, H, k)
    for j in range(R):
        B = oracle.to_bool(P[j], k)
        assert not np.array_equal(B, B.T) and B.mean() < 0.5
    return u, v, t, n, k, R, H, P


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_estimate_contains_exact(seed):
    u, v, t, n, k, R, H, P = _hashed_case(seed)
    exact = oracle.column_counts(oracle.component_matrix(u, v, t, n), n)
    est = oracle.hash_estimate(P, H, n)
    assert (est >= exact).all()


def test_estimate_matches_set_formula():
    """|intersection_j h_j^-1(OC_j(h_j(u)))| by Python sets, with proxy
    out-components from the SI simulation on the super-events."""
    u, v, t, n, k, R, H, P = _hashed_case(5, n=40, m=24, k=20, R=3)
    est = oracle.hash_estimate(P, H, n)
    for x in range(n):
        acc = set(range(n))
        for j in range(R):
            pu, pv = oracle.proxy_events(u, v, H[j])
            oc = set(np.flatnonzero(oracle.si_reach(pu, pv, t, k, int(H[j, x]))).tolist())
            acc &= {w for w in range(n) if int(H[j, w]) in oc}
        assert est[x] == len(acc)


def test_injective_hash_gives_exact():
    u, v, t = synth.uniform_events(80, 700, t_range=200, seed=8)
    n = 80
    H = np.stack([np.random.default_rng(s).permutation(n) for s in range(2)]).astype(np.uint32)
    P = oracle.proxy_matrices(u, v, t, H, n)
    exact = oracle.column_counts(oracle.component_matrix(u, v, t, n), n)
    assert np.array_equal(oracle.hash_estimate(P, H, n), exact)


def test_single_replica_is_fibre_count():
    u, v, t, n, k, R, H, P = _hashed_case(6, R=1)
    fibre = np.bincount(H[0], minlength=k)
    B = oracle.to_bool(P[0], k)  # B[row b, column c]: b reached from c
    est = oracle.hash_estimate(P, H, n)
    for x in range(n):
        c = H[0, x]
        assert est[x] == int((B[:, c] * fibre).sum())


def test_more_replicas_never_increase_estimate():
    u, v, t, n, k, R, H, P = _hashed_case(7, R=4)
    prev = None
    for r in range(1, R + 1):
        est = oracle.hash_estimate(P[:r], H[:r], n)
        if prev is not None:
            assert (est <= prev).all()
        prev = est


def test_estimate_source_subset():
    u, v, t, n, k, R, H, P = _hashed_case(2)
    src = np.array([5, 0, 77, 119], np.uint32)
    assert np.array_equal(oracle.hash_estimate(P, H, n, src), oracle.hash_estimate(P, H, n)[src])


# --------------------------------------------------------------------------
# error metric (Section 4.4)
# --------------------------------------------------------------------------
def test_emd_matches_scipy():
    from scipy import stats
    rng = np.random.default_rng(0)
    a = rng.integers(1, 500, 1000)
    b = rng.integers(1, 700, 1000)
    assert oracle.emd_w1(a, b) == pytest.approx(stats.wasserstein_distance(a, b), rel=1e-12)
    assert oracle.emd_w1(a, a) == 0.0


def test_error_stats_hand_example():
    # est = (3, 1, 4), exact = (1, 1, 2): |d| = (2, 0, 2), d/exact = (2, 0, 1)
    # sorted: (1, 3, 4) vs (1, 1, 2) -> W1 * 3 = 0 + 2 + 2
    st = oracle.error_stats([3, 1, 4], [1, 1, 2])
    assert (st["sum_abs"], st["max_abs"], st["w1_num"]) == (4, 2, 4)
    assert st["rel_sum"] == 3.0 and st["max_rel"] == 2.0
    assert st["mean_abs"] == pytest.approx(4 / 3) and st["w1"] == pytest.approx(4 / 3)


def test_error_stats_closed_forms():
    rng = np.random.default_rng(3)
    b = rng.integers(1, 10_000, 5000).astype(np.uint32)
    # a constant shift moves the whole distribution: W1 = shift = mean |d|
    st = oracle.error_stats(b + 7, b)
    assert st["w1_num"] == 7 * 5000 and st["sum_abs"] == 7 * 5000 and st["max_abs"] == 7
    assert st["max_rel"] == pytest.approx(7.0 / b.min(), rel=1e-15)
    # a permutation keeps the distribution: W1 = 0 while the per-source error is not
    p = rng.permutation(b)
    st = oracle.error_stats(p, b)
    assert st["w1_num"] == 0 and st["sum_abs"] == int(np.abs(p.astype(np.int64) - b).sum()) > 0
    # identical samples: no error at all
    st = oracle.error_stats(b, b)
    assert st["sum_abs"] == st["w1_num"] == st["max_abs"] == 0 and st["rel_sum"] == 0.0


def test_error_stats_w1_is_emd():
    from scipy import stats
    rng = np.random.default_rng(5)
    a = rng.integers(1, 900, 3000).astype(np.uint32)
    b = rng.integers(1, 400, 3000).astype(np.uint32)
    st = oracle.error_stats(a, b)
    assert st["w1"] == pytest.approx(stats.wasserstein_distance(a, b), rel=1e-12)
    assert st["w1"] == pytest.approx(oracle.emd_w1(a, b), rel=1e-12)
    # W1 never exceeds the mean per-source error (the identity matching is a transport plan)
    assert st["w1_num"] <= st["sum_abs"]


def test_error_stats_rejects_zero_exact_size():
    with pytest.raises(Exception):
        oracle.error_stats([1, 2], [1, 0])


# --------------------------------------------------------------------------
# reversed-sequence variant (Section 3.4)
# --------------------------------------------------------------------------
def test_reversed_hand_example():
    # 0-1 at t=1, 1-2 at t=2: forward, 0 reaches 1 and 2, 1 reaches 0 (t=1) and 2 (t=2), 2 reaches 1 only
    u = np.array([0, 1], np.uint32); v = np.array([1, 2], np.uint32); t = np.array([1, 2], np.int64)
    R = oracle.to_bool(oracle.component_matrix_reversed(u, v, t, 3), 3)
    assert R.tolist() == [[True, True, True], [True, True, True], [False, True, True]]


@pytest.mark.parametrize("seed", range(12))
def test_reversed_is_transpose_of_forward(seed):
    """Reversing time turns in-components into out-components: row i of the
    reversed result is column i of the forward matrix (ties stay snapshots in
    both directions, so the relation is exact)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 90))
    m = int(rng.integers(1, 400))
    u, v, t = synth.uniform_events(n, m, t_range=int(rng.integers(1, 60)), seed=seed, self_loops=True)
    F = oracle.to_bool(oracle.component_matrix(u, v, t, n), n)
    R = oracle.to_bool(oracle.component_matrix_reversed(u, v, t, n), n)
    assert np.array_equal(R, F.T)


def test_reversed_rows_match_brute_force_si():
    """Row i of the reversed result is the set the SI process from i infects."""
    rng = np.random.default_rng(77)
    n, m = 40, 300
    u, v, t = synth.uniform_events(n, m, t_range=50, seed=77)
    R = oracle.to_bool(oracle.component_matrix_reversed(u, v, t, n), n)
    for i in rng.choice(n, 10, replace=False):
        assert np.array_equal(R[i], oracle.si_reach(u, v, t, n, int(i)).astype(bool))


# --------------------------------------------------------------------------
# directed events (footnote to Section 3.1: S[v] |= S[u] only)
# --------------------------------------------------------------------------
def test_directed_hand_example():
    # 0->1 at t=1, 1->2 at t=2, 2->0 at t=2: 0 reaches 1 and 2; 1 reaches 2; 2 reaches 0 only;
    # 1 -> 2 and 2 -> 0 share t=2, so 1 does not reach 0 through 2
    u = np.array([0, 1, 2], np.uint32); v = np.array([1, 2, 0], np.uint32); t = np.array([1, 2, 2], np.int64)
    B = oracle.to_bool(oracle.component_matrix_directed(u, v, t, 3), 3)  # B[i, j]: i reached from j
    assert B[:, 0].tolist() == [True, True, True]
    assert B[:, 1].tolist() == [False, True, True]
    assert B[:, 2].tolist() == [True, False, True]


@pytest.mark.parametrize("seed", range(20))
def test_directed_matches_directed_si(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 40))
    m = int(rng.integers(1, 200))
    u, v, t = synth.uniform_events(n, m, t_range=int(rng.integers(1, 30)), seed=seed, self_loops=True)
    B = oracle.to_bool(oracle.component_matrix_directed(u, v, t, n), n)
    for j in range(n):
        assert np.array_equal(B[:, j], oracle.si_reach_directed(u, v, t, n, j)), j


@pytest.mark.parametrize("seed", range(12))
def test_undirected_is_both_directions_at_once(seed):
    """An undirected event is the two directed events u->v and v->u at the
    same timestamp (one snapshot), so the directed rule on the doubled stream
    must give the undirected matrix."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(2, 120))
    m = int(rng.integers(1, 500))
    u, v, t = synth.uniform_events(n, m, t_range=int(rng.integers(1, 80)), seed=seed, self_loops=True)
    du = np.stack([u, v], 1).reshape(-1)
    dv = np.stack([v, u], 1).reshape(-1)
    dt = np.repeat(t, 2)
    assert np.array_equal(oracle.component_matrix_directed(du, dv, dt, n), oracle.component_matrix(u, v, t, n))


def test_directed_exhaustive_tiny():
    """Every directed sequence of up to 3 events on 3 nodes over 2 timestamps."""
    pairs = [(a, b) for a in range(3) for b in range(3)]
    for k in range(1, 4):
        for evs in itertools.product(pairs, repeat=k):
            for ts in itertools.product(range(2), repeat=k):
                t = np.sort(np.array(ts, np.int64))
                u = np.array([e[0] for e in evs], np.uint32)
                v = np.array([e[1] for e in evs], np.uint32)
                B = oracle.to_bool(oracle.component_matrix_directed(u, v, t, 3), 3)
                for j in range(3):
                    assert np.array_equal(B[:, j], oracle.si_reach_directed(u, v, t, 3, j))


# --------------------------------------------------------------------------
# HyperLogLog sketches of the components (Section 3.3; reversed, Section 3.4)
# --------------------------------------------------------------------------
def _singletons(seed, p, n):
    s = 1 << p
    S1 = np.zeros((n, s), np.uint8)
    for x in range(n):
        reg, rank = oracle.hll_singleton(seed, p, x)
        S1[x, reg] = rank
    return S1


@pytest.mark.parametrize("reverse,directed", [(False, False), (True, False), (False, True), (True, True)])
def test_hll_sketch_is_the_union_of_its_members(reverse, directed):
    """A node's sketch equals the register-wise maximum of the singleton
    sketches of exactly the members of its component (the exact matrix), in
    every mode: the merge rule commutes with set union."""
    n, m, p, seed = 60, 700, 6, 11
    u, v, t = synth.uniform_events(n, m, t_range=120, seed=3, self_loops=True)
    R = oracle.hll_sketches(u, v, t, n, p, seed, reverse=reverse, directed=directed)
    if directed:
        F = oracle.to_bool(oracle.component_matrix_directed(u, v, t, n), n)
    else:
        F = oracle.to_bool(oracle.component_matrix(u, v, t, n), n)
    members = F.T if reverse else F  # row i: members of i's component
    S1 = _singletons(seed, p, n)
    for i in range(n):
        assert np.array_equal(R[i], S1[members[i]].max(axis=0)), i


def test_hll_rank_distribution():
    """P(rank = r) = 2^-r and registers are uniform (the hash's job)."""
    p, N = 8, 40_000
    regs = np.zeros(N, np.int64)
    ranks = np.zeros(N, np.int64)
    for x in range(N):
        regs[x], ranks[x] = oracle.hll_singleton(17, p, x)
    for r in range(1, 6):
        assert abs((ranks == r).mean() - 2.0 ** -r) < 4 * np.sqrt(2.0 ** -r / N)
    counts = np.bincount(regs, minlength=1 << p)
    assert counts.min() > 0.6 * N / (1 << p) and counts.max() < 1.4 * N / (1 << p)


@pytest.mark.parametrize("p", [7, 10])
def test_hll_estimate_accuracy(p):
    """Estimates of sets of many sizes stay within the HLL error: the mean
    relative error is a few times 1.04 / sqrt(2^p), small sets are exact-ish
    (linear counting)."""
    s = 1 << p
    rng = np.random.default_rng(p)
    S1 = _singletons(23, p, 30_000)
    rel = []
    for N in (5, 50, 500, 5000, 30_000):
        for _ in range(4):
            idx = rng.choice(30_000, N, replace=False)
            e = oracle.hll_estimate(S1[idx].max(axis=0)[None, :], p)[0]
            rel.append(abs(e / N - 1.0))
            if N <= s // 10:
                assert abs(e - N) <= max(1.0, 0.05 * N)
    assert np.mean(rel) < 3 * 1.04 / np.sqrt(s)


def test_hll_estimate_formula_hand_values():
    p = 4  # s = 16, alpha = 0.673
    empty = np.zeros((1, 16), np.uint8)
    assert oracle.hll_estimate(empty, p)[0] == 0.0  # linear counting: 16 ln(16/16)
    one = empty.copy(); one[0, 3] = 1
    assert oracle.hll_estimate(one, p)[0] == pytest.approx(16 * np.log(16 / 15), rel=1e-15)
    full = np.full((1, 16), 5, np.uint8)  # no zero register: the raw estimate
    assert oracle.hll_estimate(full, p)[0] == pytest.approx(0.673 * 256 / (16 * 2.0 ** -5), rel=1e-15)
