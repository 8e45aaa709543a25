"""Model check of the scheduling rules used by the GPU planner (host logic, no GPU).

The GPU planner turns a time-ordered batch into levels of row operations:
  EVENT(u, v): r = S[u] | S[v] into both rows        (both ends occur once in their group)
  ONEWAY(y<-x): S[y] |= S[x]                           (y once, x several times in the group)
  COPY(x->T):  T = S[x]                                (x several times, has such a partner)
  PULL(x; srcs): S[x] |= OR srcs                       (x several times in the group)
with levels restarting in every window.  This model applies the same rules in
Python, executes every level's operations in a random order (they must not
conflict) and compares with the oracle's group-snapshot semantics.
"""
import numpy as np
import pytest

import oracle
from paper_2307_04890_gb300 import synth


def schedule(u, v, t, window):
    m = len(t)
    starts = [0]
    for w in range(1, (m + window - 1) // window):
        s = w * window
        while s < m and t[s] == t[s - 1]:
            s += 1
        starts.append(min(s, m))
    starts.append(m)
    levels = []  # list of lists of ops
    for w in range(len(starts) - 1):
        s, e = starts[w], starts[w + 1]
        lev = {}
        wl = {}
        ntemp = 0
        i = s
        while i < e:
            j = i
            while j < e and t[j] == t[i]:
                j += 1
            cnt = {}
            for q in range(i, j):
                if u[q] != v[q]:
                    cnt[u[q]] = cnt.get(u[q], 0) + 1
                    cnt[v[q]] = cnt.get(v[q], 0) + 1
            runs, temps, Lc, pending = {}, {}, 0, []
            for q in range(i, j):
                x, y = int(u[q]), int(v[q])
                if x == y:
                    continue
                if cnt[x] == 1 and cnt[y] == 1:
                    L = 1 + max(lev.get(x, 0), lev.get(y, 0))
                    lev[x] = lev[y] = L
                    wl.setdefault(L, []).append(("EVENT", x, y))
                    continue
                Lc = max(Lc, lev.get(x, 0), lev.get(y, 0))
                pending.append((x, y))
            if pending:
                L = Lc + 1
                for x, y in pending:
                    for a, b in ((x, y), (y, x)):
                        if cnt[a] == 1:
                            wl.setdefault(L, []).append(("ONEWAY", a, b))
                        else:
                            runs.setdefault(a, [])
                            if cnt[b] > 1:
                                if b not in temps:
                                    temps[b] = ntemp
                                    ntemp += 1
                                runs[a].append(("T", temps[b]))
                            else:
                                runs[a].append(("S", b))
                for x in temps:
                    wl.setdefault(L, []).append(("COPY", x, temps[x]))
                for a, srcs in runs.items():
                    wl.setdefault(L + 1, []).append(("PULL", a, srcs))
                for x, y in pending:
                    lev[x] = lev[y] = L + 1
            i = j
        for L in sorted(wl):
            levels.append(wl[L])
    return levels


def execute(levels, n, rng):
    S = oracle.to_bool(oracle.init_sources(n), n)
    T = {}
    for ops in levels:
        # every op of a level reads only values that no other op of the level writes
        reads, writes = set(), []
        for op in ops:
            if op[0] == "EVENT":
                reads |= {op[1], op[2]}; writes += [op[1], op[2]]
            elif op[0] == "ONEWAY":
                reads |= {op[1], op[2]}; writes.append(op[1])
            elif op[0] == "COPY":
                reads.add(op[1])
            else:
                reads.add(op[1]); writes.append(op[1])
                reads |= {r for kind, r in op[2] if kind == "S"}
        assert len(writes) == len(set(writes)), "two ops of one level write the same row"
        for op in ops:
            if op[0] != "PULL":
                continue
            for kind, r in op[2]:
                assert kind == "T" or r not in set(writes), "a pull reads a row written in its level"
        for k in rng.permutation(len(ops)):
            op = ops[k]
            if op[0] == "EVENT":
                r = S[op[1]] | S[op[2]]
                S[op[1]] = r
                S[op[2]] = r
            elif op[0] == "ONEWAY":
                S[op[1]] = S[op[1]] | S[op[2]]
            elif op[0] == "COPY":
                T[op[2]] = S[op[1]].copy()
            else:
                acc = S[op[1]].copy()
                for kind, r in op[2]:
                    acc |= T[r] if kind == "T" else S[r]
                S[op[1]] = acc
    return S


@pytest.mark.parametrize("seed", range(80))
def test_schedule_model_matches_oracle(seed):
    rng = np.random.default_rng(9000 + seed)
    n = int(rng.integers(2, 60))
    m = int(rng.integers(1, 400))
    u = rng.integers(0, n, m).astype(np.uint32)
    v = rng.integers(0, n, m).astype(np.uint32)
    t = np.sort(rng.integers(0, int(rng.integers(1, 30)), m))
    window = int(rng.choice([8, 32, 1000]))
    S = execute(schedule(u, v, t, window), n, rng)
    assert np.array_equal(S, oracle.to_bool(oracle.component_matrix(u, v, t, n), n))


def test_schedule_model_bursty():
    u, v, t = synth.powerlaw_bursty(3000, 20_000, seed=2)
    rng = np.random.default_rng(0)
    S = execute(schedule(u, v, t, 512), 3000, rng)
    assert np.array_equal(S, oracle.to_bool(oracle.component_matrix(u, v, t, 3000), 3000))
