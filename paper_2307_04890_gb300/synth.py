"""Seeded synthetic temporal-network generators.

Every workload in this project is synthetic: the paper's real datasets (SNAP
Superuser and Reddit, Section 4.4) are not available, so these generators stand
in for them with the shapes and statistics the workloads call for.  They only
produce inputs -- event arrays -- and contain none of the method's arithmetic
(no component matrix, no hashing); both the GPU path and the CPU oracle consume
their output.

Every generator returns ``(u, v, t)``: ``u`` and ``v`` are ``uint32`` endpoint
arrays and ``t`` an ``int64`` timestamp array, all of length ``m``, sorted by
``t`` with a stable sort (the order inside a group of equal timestamps is the
generation order).  Events are undirected interactions (Section 2.1).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "uniform_events",
    "activity_driven",
    "powerlaw_bursty",
    "er_poisson",
    "er_links",
    "er_poisson_stream",
    "serving_jobs",
    "job_events",
    "split_batches",
]


def _finish(u, v, t):
    order = np.argsort(t, kind="stable")
    return (np.ascontiguousarray(u[order], dtype=np.uint32),
            np.ascontiguousarray(v[order], dtype=np.uint32),
            np.ascontiguousarray(t[order], dtype=np.int64))


def uniform_events(n: int, m: int, t_range: int, seed: int = 0, self_loops: bool = False):
    """Uniform random endpoint pairs with uniform integer timestamps in [0, t_range).

    With ``self_loops=False`` the pair is uniform over ordered pairs u != v.
    A small ``t_range`` relative to ``m`` makes equal-timestamp groups frequent.
    """
    rng = np.random.default_rng(seed)
    u = rng.integers(0, n, size=m, dtype=np.int64)
    if self_loops or n < 2:
        v = rng.integers(0, n, size=m, dtype=np.int64)
    else:
        v = (u + rng.integers(1, n, size=m, dtype=np.int64)) % n
    t = rng.integers(0, t_range, size=m, dtype=np.int64)
    return _finish(u, v, t)


def activity_driven(n: int, m: int, gamma: float = 2.1, a_min: float = 1e-3,
                    ticks_per_unit: float = 1e6, seed: int = 0):
    """Activity-driven temporal network.

    Node activities follow a power law p(a) ~ a^-gamma on [a_min, 1], drawn by
    inverse CDF.  The superposition of the nodes' Poisson processes has rate
    sum(a): each event picks its active node with probability a_i / sum(a) and a
    partner uniformly among the other nodes; inter-event gaps are exponential
    with mean 1/sum(a).  Times are quantised to integer ticks
    (``floor(time * ticks_per_unit)``), so with the default microsecond ticks
    equal timestamps are rare.
    """
    rng = np.random.default_rng(seed)
    e = 1.0 - gamma
    a = (a_min ** e + rng.random(n) * (1.0 - a_min ** e)) ** (1.0 / e)
    total = float(a.sum())
    cdf = np.cumsum(a)
    cdf /= cdf[-1]
    act = np.searchsorted(cdf, rng.random(m), side="right").astype(np.int64)
    np.minimum(act, n - 1, out=act)
    partner = (act + rng.integers(1, n, size=m, dtype=np.int64)) % n
    gaps = rng.exponential(1.0 / total, size=m)
    time = np.cumsum(gaps)
    t = np.floor(time * ticks_per_unit).astype(np.int64)
    return _finish(act, partner, t)


def _discrete_powerlaw(rng, size, gamma, k_min, k_max):
    k = np.arange(k_min, k_max + 1, dtype=np.float64)
    pmf = k ** (-gamma)
    cdf = np.cumsum(pmf)
    cdf /= cdf[-1]
    idx = np.searchsorted(cdf, rng.random(size), side="right")
    return (np.minimum(idx, len(k) - 1) + k_min).astype(np.int64)


def powerlaw_bursty(n: int, m: int, gamma: float = 2.5, k_min: int = 1,
                    shape: float = 1.5, x_m: float = 60.0, seed: int = 0):
    """Power-law static graph with bursty (Pareto) link activity.

    Degrees follow a discrete power law p(k) ~ k^-gamma on [k_min, k_max] with
    the natural cutoff k_max = floor(n^(1/(gamma-1))).  Edges come from the
    configuration model (random stub matching); self-loops and multi-edges are
    dropped.  Every edge carries an independent renewal process whose gaps are
    Pareto(shape, scale x_m) seconds; its first event comes one gap after 0.
    The m earliest events over all edges are kept and their times are rounded
    down to integer seconds, which creates large groups of equal timestamps.
    """
    rng = np.random.default_rng(seed)
    k_max = int(np.floor(n ** (1.0 / (gamma - 1.0))))
    deg = _discrete_powerlaw(rng, n, gamma, k_min, k_max)
    if deg.sum() % 2:
        deg[rng.integers(0, n)] += 1
    stubs = np.repeat(np.arange(n, dtype=np.int64), deg)
    rng.shuffle(stubs)
    a, b = stubs[0::2], stubs[1::2]
    keep = a != b
    a, b = a[keep], b[keep]
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo * n + hi)
    ea, eb = (key // n), (key % n)
    n_edges = len(key)

    mean_gap = shape * x_m / (shape - 1.0)
    horizon = 1.2 * mean_gap * m / n_edges
    while True:
        times, owners = [], []
        cur = x_m / rng.random(n_edges) ** (1.0 / shape)
        alive = np.arange(n_edges)
        count = 0
        while alive.size:
            inside = cur <= horizon
            alive, cur = alive[inside], cur[inside]
            if not alive.size:
                break
            times.append(cur.copy())
            owners.append(alive.copy())
            count += alive.size
            cur = cur + x_m / rng.random(alive.size) ** (1.0 / shape)
        if count >= m:
            break
        horizon *= 1.5
    times = np.concatenate(times)
    owners = np.concatenate(owners)
    sel = np.argpartition(times, m - 1)[:m]
    times, owners = times[sel], owners[sel]
    order = np.argsort(times, kind="stable")
    times, owners = times[order], owners[order]
    t = np.floor(times).astype(np.int64)
    return (np.ascontiguousarray(ea[owners], dtype=np.uint32),
            np.ascontiguousarray(eb[owners], dtype=np.uint32),
            np.ascontiguousarray(t, dtype=np.int64))


def _draw_er_links(rng, n, p):
    """A binomial number of distinct pairs a < b, drawn uniformly (G(n, p))."""
    if p is None:
        p = 2.0 / n
    n_pairs = n * (n - 1) // 2
    n_links = rng.binomial(n_pairs, p)
    links = set()
    while len(links) < n_links:
        need = n_links - len(links)
        a = rng.integers(0, n, size=2 * need)
        b = rng.integers(0, n, size=2 * need)
        for x, y in zip(a.tolist(), b.tolist()):
            if x != y:
                links.add((min(x, y), max(x, y)))
                if len(links) == n_links:
                    break
    return np.array(sorted(links), dtype=np.int64).reshape(-1, 2)


def er_poisson(n: int, m: int, p: float | None = None, seed: int = 0,
               ticks_per_unit: float = 1e6):
    """Erdos-Renyi G(n, p) (default p = 2/n) with an independent unit-rate Poisson
    process on every link, as in the paper's synthetic experiments (Section 3.5).
    The superposed process is simulated directly: each event picks a uniform
    link and gaps are exponential with mean 1/|links|.  Times are integer ticks."""
    rng = np.random.default_rng(seed)
    links = _draw_er_links(rng, n, p)
    pick = rng.integers(0, len(links), size=m)
    gaps = rng.exponential(1.0 / len(links), size=m)
    t = np.floor(np.cumsum(gaps) * ticks_per_unit).astype(np.int64)
    return _finish(links[pick, 0], links[pick, 1], t)


def er_links(n: int, p: float | None = None, seed: int = 0) -> np.ndarray:
    """The links (a < b) of an Erdos-Renyi G(n, p) draw, p = 2/n by default,
    drawn exactly as ``er_poisson`` draws them for the same seed."""
    return _draw_er_links(np.random.default_rng(seed), n, p)


def er_poisson_stream(n: int, m: int, chunk: int = 100_000_000, p: float | None = None, seed: int = 0,
                      ticks_per_unit: float = 1e6):
    """The ER G(n, p) + per-link Poisson model of ``er_poisson`` (same links for
    the same seed) as a stream of about ``chunk`` events at a time, for event
    counts too large to hold at once.  The superposed process continues across
    chunks (one running clock); every yielded chunk ends at a timestamp-group
    boundary (the events of its last timestamp are held back and lead the next
    chunk), so chunk k + 1 starts strictly after chunk k ends.  Yields
    (u, v, t) arrays, m events in total."""
    links = er_links(n, p, seed)
    rng = np.random.default_rng([seed, 1])
    clock, done = 0.0, 0
    held = None
    while done < m:
        c = min(chunk, m - done)
        pick = rng.integers(0, len(links), size=c)
        gaps = rng.exponential(1.0 / len(links), size=c)
        times = clock + np.cumsum(gaps)
        clock = float(times[-1])
        u, v = links[pick, 0].astype(np.uint32), links[pick, 1].astype(np.uint32)
        t = np.floor(times * ticks_per_unit).astype(np.int64)
        done += c
        if held is not None:
            u, v, t = np.concatenate([held[0], u]), np.concatenate([held[1], v]), np.concatenate([held[2], t])
        if done < m:
            cut = int(np.searchsorted(t, t[-1], side="left"))  # the last timestamp group stays behind
            held = (u[cut:], v[cut:], t[cut:])
            u, v, t = u[:cut], v[:cut], t[:cut]
        if len(t):
            yield u, v, t


def serving_jobs(n_jobs: int, rate: float = 200.0, n_range=(10**3, 10**5),
                 m_range=(10**4, 10**7), seed: int = 0):
    """Job descriptors for a Poisson stream of component-matrix requests.

    Returns a list of dicts with arrival time (seconds), n and m (log-uniform
    in the given ranges) and a per-job seed.  Each job's events come from
    ``job_events``."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=n_jobs))
    ln = np.exp(rng.uniform(np.log(n_range[0]), np.log(n_range[1]), size=n_jobs))
    lm = np.exp(rng.uniform(np.log(m_range[0]), np.log(m_range[1]), size=n_jobs))
    seeds = rng.integers(0, 2**31 - 1, size=n_jobs)
    return [dict(job=i, arrival=float(arrivals[i]), n=int(ln[i]), m=int(lm[i]),
                 seed=int(seeds[i])) for i in range(n_jobs)]


def job_events(job: dict):
    """Events of one serving job: uniform endpoints (u != v) and integer
    timestamps spread uniformly over [0, about m), so equal-timestamp groups
    average one event.  The endpoints are independent of the times, so the
    sorted times are drawn directly, with no sort of m values: the m events of
    a unit-rate Poisson process (exponential gaps), floored to integer ticks,
    so the number of events at each tick is Poisson with mean 1."""
    rng = np.random.default_rng(job["seed"])
    n, m = job["n"], job["m"]
    u = rng.integers(0, n, size=m, dtype=np.int64)
    v = (u + rng.integers(1, n, size=m, dtype=np.int64)) % n if n > 1 else u.copy()
    t = np.floor(np.cumsum(rng.exponential(1.0, size=m))).astype(np.int64)
    return (np.ascontiguousarray(u, dtype=np.uint32), np.ascontiguousarray(v, dtype=np.uint32),
            np.ascontiguousarray(t, dtype=np.int64))


def split_batches(t: np.ndarray, parts: int = 4):
    """Split a time-sorted stream into ``parts`` contiguous batches at
    timestamp quantiles, never inside a group of equal timestamps.  Returns the
    list of (start, end) index pairs."""
    m = len(t)
    bounds = [0]
    for q in range(1, parts):
        i = (m * q) // parts
        if i <= 0 or i >= m:
            continue
        i = int(np.searchsorted(t, t[i], side="left"))
        if i > bounds[-1]:
            bounds.append(i)
    bounds.append(m)
    return [(bounds[i], bounds[i + 1]) for i in range(len(bounds) - 1)]
