"""CPU oracle for temporal out-components and network hashing.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct reference that the
GPU library is checked against.  Only the test suite, the package smoke check
and the benchmark's CPU-baseline leg may import it; the product path never
does.  It shares no code with the GPU library: the arithmetic lives in
``tnref.c`` (plain C, compiled with gcc) and this module only marshals numpy
arrays.  Functions cite the paper passage they follow:

* ``component_matrix``  -- Algorithm 1 (Section 3.1) with equal-timestamp
  groups applied as snapshots (adjacency needs dt > 0, Section 2.1).
* ``component_matrix_reversed`` -- the reversed-sequence variant (Section 3.4).
* ``component_matrix_directed`` / ``si_reach_directed`` -- directed events
  (footnote to Section 3.1: only the receiver's row is updated).
* ``hll_singleton`` / ``hll_sketches`` / ``hll_estimate`` -- HyperLogLog
  sketches of the components and their size estimates (Section 3.3; with
  the reversed sequence, Section 3.4).
* ``grow_matrix``       -- node growth: a new row and column of zeros with the
  new node's diagonal bit set (Section 3.5, advantages and limitations of the
  matrix method).
* ``si_reach``          -- the deterministic SI process (Section 1).
* ``column_counts`` / ``row_counts`` / ``argmax`` -- component sizes
  (Section 3.1, eq. for the mean size s_t in Section 3.3).
* ``splitmix64_stream`` / ``hash_*`` -- network hashing (Section 4.1; reading
  of the garbled construction documented in tnref.c).  The generator is
  pinned by its known-answer values, the coefficients and tables by big-integer
  restatements; agreement with the authors' own unpublished hash values cannot
  be checked.
* ``hash_estimate``     -- fusion by intersection (Section 4.2, eqs.
  DefInvHComp, DefEstOCMerge).
* ``emd_w1``            -- Earth-Mover (Wasserstein-1) distance between two
  equal-size samples of sizes (Section 4.4).
* ``error_stats``       -- absolute, relative and W1 error of estimates against
  exact sizes (Section 4.4).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tnref.c")
_LIB = os.path.join(_HERE, "libtnref.so")

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")

OK, EINVAL, ERANGE, EORDER, ENOMEM = 0, -1, -2, -3, -4


def build_oracle(force: bool = False) -> str:
    """Compile tnref.c into libtnref.so next to it (plain gcc, no CUDA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        lib.tnref_validate.argtypes = [_u32p, _u32p, _i64p, ctypes.c_uint64, ctypes.c_uint32]
        lib.tnref_validate.restype = ctypes.c_int
        lib.tnref_init_sources.argtypes = [_u64p, ctypes.c_uint32, ctypes.c_uint64,
                                           ctypes.c_void_p, ctypes.c_uint64]
        lib.tnref_init_sources.restype = None
        lib.tnref_apply_events.argtypes = [_u32p, _u32p, _i64p, ctypes.c_uint64, ctypes.c_uint32,
                                           _u64p, ctypes.c_uint64]
        lib.tnref_apply_events.restype = ctypes.c_int
        lib.tnref_apply_events_reversed.argtypes = lib.tnref_apply_events.argtypes
        lib.tnref_apply_events_reversed.restype = ctypes.c_int
        lib.tnref_apply_events_directed.argtypes = lib.tnref_apply_events.argtypes
        lib.tnref_apply_events_directed.restype = ctypes.c_int
        lib.tnref_grow_matrix.argtypes = [_u64p, ctypes.c_uint32, ctypes.c_uint64,
                                          _u64p, ctypes.c_uint32, ctypes.c_uint64]
        lib.tnref_grow_matrix.restype = ctypes.c_int
        lib.tnref_si_reach_directed.argtypes = [_u32p, _u32p, _i64p, ctypes.c_uint64, ctypes.c_uint32,
                                                ctypes.c_uint32, _u8p]
        lib.tnref_hll_singleton.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                            ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint8)]
        lib.tnref_hll_singleton.restype = None
        lib.tnref_hll_sketches.argtypes = [_u32p, _u32p, _i64p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           ctypes.c_uint64, ctypes.c_int, ctypes.c_int, _u8p]
        lib.tnref_hll_sketches.restype = ctypes.c_int
        lib.tnref_hll_estimate.argtypes = [_u8p, ctypes.c_uint32, ctypes.c_uint32,
                                           np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")]
        lib.tnref_hll_estimate.restype = None
        lib.tnref_si_reach_directed.restype = ctypes.c_int
        lib.tnref_si_reach.argtypes = [_u32p, _u32p, _i64p, ctypes.c_uint64, ctypes.c_uint32,
                                       ctypes.c_uint32, _u8p]
        lib.tnref_si_reach.restype = ctypes.c_int
        lib.tnref_column_counts.argtypes = [_u64p, ctypes.c_uint32, ctypes.c_uint64,
                                            ctypes.c_uint64, _u32p]
        lib.tnref_column_counts.restype = None
        lib.tnref_row_counts.argtypes = [_u64p, ctypes.c_uint32, ctypes.c_uint64, _u32p]
        lib.tnref_row_counts.restype = None
        lib.tnref_argmax.argtypes = [_u32p, ctypes.c_uint64]
        lib.tnref_argmax.restype = ctypes.c_uint64
        lib.tnref_splitmix64_stream.argtypes = [ctypes.c_uint64, ctypes.c_uint64, _u64p]
        lib.tnref_splitmix64_stream.restype = None
        lib.tnref_hash_coeffs.argtypes = [ctypes.c_uint64, ctypes.c_uint32, _u64p]
        lib.tnref_hash_coeffs.restype = None
        lib.tnref_table_value.argtypes = [_u64p, ctypes.c_uint64]
        lib.tnref_table_value.restype = ctypes.c_uint64
        lib.tnref_hash_raw.argtypes = [_u64p, ctypes.c_uint32]
        lib.tnref_hash_raw.restype = ctypes.c_uint64
        lib.tnref_hash_nodes.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                         ctypes.c_uint32, _u32p]
        lib.tnref_hash_nodes.restype = ctypes.c_int
        lib.tnref_proxy_events.argtypes = [_u32p, _u32p, ctypes.c_uint64, _u32p, _u32p, _u32p]
        lib.tnref_proxy_events.restype = None
        lib.tnref_hash_estimate.argtypes = [_u64p, ctypes.c_uint32, ctypes.c_uint32, _u32p,
                                            ctypes.c_uint32, ctypes.c_void_p, ctypes.c_uint64, _u32p]
        lib.tnref_hash_estimate.restype = ctypes.c_int
        _u64o = ctypes.POINTER(ctypes.c_uint64)
        _f64o = ctypes.POINTER(ctypes.c_double)
        lib.tnref_error_stats.argtypes = [_u32p, _u32p, ctypes.c_uint64, _u64o, _u64o, _u64o, _f64o, _f64o]
        lib.tnref_error_stats.restype = ctypes.c_int
        _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != OK:
        raise OracleError({EINVAL: "EINVAL", ERANGE: "ERANGE", EORDER: "EORDER",
                           ENOMEM: "ENOMEM"}.get(rc, str(rc)))


def _ev(u, v, t):
    return (np.ascontiguousarray(u, dtype=np.uint32), np.ascontiguousarray(v, dtype=np.uint32),
            np.ascontiguousarray(t, dtype=np.int64))


def words(bits: int) -> int:
    return (bits + 63) // 64


def validate(u, v, t, n) -> int:
    u, v, t = _ev(u, v, t)
    return _load().tnref_validate(u, v, t, len(u), n)


def init_sources(n: int, src=None) -> np.ndarray:
    """S <- I_n (Algorithm 1), or the columns of the listed sources only."""
    ncols = n if src is None else len(src)
    width = max(1, words(ncols))
    S = np.zeros((n, width), dtype=np.uint64)
    if src is None:
        _load().tnref_init_sources(S.reshape(-1), n, width, None, 0)
    else:
        s = np.ascontiguousarray(src, dtype=np.uint32)
        _load().tnref_init_sources(S.reshape(-1), n, width, s.ctypes.data, len(s))
    return S


def apply_events(u, v, t, n, S: np.ndarray) -> np.ndarray:
    """Stream events into S in place (Algorithm 1 with group snapshots)."""
    u, v, t = _ev(u, v, t)
    assert S.dtype == np.uint64 and S.flags.c_contiguous and S.shape[0] == n
    _check(_load().tnref_apply_events(u, v, t, len(u), n, S.reshape(-1), S.shape[1]))
    return S


def component_matrix(u, v, t, n, src=None) -> np.ndarray:
    """Component matrix from the identity (or from the listed source columns)."""
    S = init_sources(n, src)
    return apply_events(u, v, t, n, S)


def component_matrix_reversed(u, v, t, n) -> np.ndarray:
    """Reversed-sequence variant (Section 3.4): the identity, then the timestamp
    groups from the last to the first; row i ends as the out-component of i."""
    u, v, t = _ev(u, v, t)
    S = init_sources(n)
    _check(_load().tnref_apply_events_reversed(u, v, t, len(u), n, S.reshape(-1), S.shape[1]))
    return S


def component_matrix_directed(u, v, t, n, src=None) -> np.ndarray:
    """Directed events (footnote to Section 3.1): S[v] |= S[u] only, timestamp
    groups as snapshots; from the identity (or the listed source columns)."""
    u, v, t = _ev(u, v, t)
    S = init_sources(n, src)
    _check(_load().tnref_apply_events_directed(u, v, t, len(u), n, S.reshape(-1), S.shape[1]))
    return S


def si_reach_directed(u, v, t, n, source) -> np.ndarray:
    """Deterministic SI process over directed events from one source; bool[n]."""
    u, v, t = _ev(u, v, t)
    out = np.zeros(n, dtype=np.uint8)
    _check(_load().tnref_si_reach_directed(u, v, t, len(u), n, source, out))
    return out.astype(bool)


def si_reach(u, v, t, n, source) -> np.ndarray:
    """Deterministic SI process from one source (Section 1); bool[n]."""
    u, v, t = _ev(u, v, t)
    out = np.zeros(n, dtype=np.uint8)
    _check(_load().tnref_si_reach(u, v, t, len(u), n, source, out))
    return out.astype(bool)


def grow_matrix(S: np.ndarray, n_old: int, n_new: int) -> np.ndarray:
    """Node growth (Section 3.5): the n_old x n_old matrix S extended to n_new
    nodes, each new node a new row and column of zeros with its own diagonal
    bit set.  Returns a new n_new x words(n_new) matrix."""
    S = np.ascontiguousarray(S, dtype=np.uint64)
    assert S.shape[0] == n_old
    out = np.zeros((n_new, max(1, words(n_new))), dtype=np.uint64)
    _check(_load().tnref_grow_matrix(S.reshape(-1), n_old, S.shape[1], out.reshape(-1), n_new, out.shape[1]))
    return out


def column_counts(S: np.ndarray, ncols: int) -> np.ndarray:
    out = np.zeros(ncols, dtype=np.uint32)
    _load().tnref_column_counts(np.ascontiguousarray(S).reshape(-1), S.shape[0], S.shape[1], ncols, out)
    return out


def row_counts(S: np.ndarray) -> np.ndarray:
    out = np.zeros(S.shape[0], dtype=np.uint32)
    _load().tnref_row_counts(np.ascontiguousarray(S).reshape(-1), S.shape[0], S.shape[1], out)
    return out


def argmax(sizes) -> int:
    s = np.ascontiguousarray(sizes, dtype=np.uint32)
    return int(_load().tnref_argmax(s, len(s)))


def to_bool(S: np.ndarray, ncols: int) -> np.ndarray:
    """Unpack a component matrix into bool[n_rows, ncols] (bit c of row i)."""
    bits = np.unpackbits(np.ascontiguousarray(S).view(np.uint8).reshape(S.shape[0], -1),
                         axis=1, bitorder="little")
    return bits[:, :ncols].astype(bool)


def splitmix64_stream(state: int, count: int) -> np.ndarray:
    """The first `count` outputs of SplitMix64 started at `state` (the generator
    behind the hash coefficients and the HyperLogLog singletons)."""
    out = np.zeros(count, dtype=np.uint64)
    _load().tnref_splitmix64_stream(state, count, out)
    return out


def hash_coeffs(seed: int, replica: int) -> np.ndarray:
    A = np.zeros(12, dtype=np.uint64)
    _load().tnref_hash_coeffs(seed, replica, A)
    return A


def table_value(A: np.ndarray, table: int, x: int) -> int:
    """T_table[x]: the degree-3 polynomial of coefficient row A(table, .) at x."""
    row = np.ascontiguousarray(np.asarray(A, dtype=np.uint64)[4 * table:4 * table + 4])
    return int(_load().tnref_table_value(row, x))


def hash_raw(A: np.ndarray, x: int) -> int:
    return int(_load().tnref_hash_raw(np.ascontiguousarray(A, dtype=np.uint64), x))


def hash_nodes(seed: int, R: int, k: int, n: int) -> np.ndarray:
    """H[j, x] = h_j(x) for j < R, x < n (Section 4.1)."""
    H = np.zeros((R, n), dtype=np.uint32)
    _check(_load().tnref_hash_nodes(seed, R, k, n, H.reshape(-1)))
    return H


def proxy_events(u, v, Hj):
    u = np.ascontiguousarray(u, dtype=np.uint32)
    v = np.ascontiguousarray(v, dtype=np.uint32)
    Hj = np.ascontiguousarray(Hj, dtype=np.uint32)
    pu = np.zeros(len(u), dtype=np.uint32)
    pv = np.zeros(len(u), dtype=np.uint32)
    _load().tnref_proxy_events(u, v, len(u), Hj, pu, pv)
    return pu, pv


def proxy_matrices(u, v, t, H: np.ndarray, k: int) -> np.ndarray:
    """Component matrix of every hashed network (Section 4.2): P[j] is k x ceil(k/64)."""
    R = H.shape[0]
    P = np.zeros((R, k, words(k)), dtype=np.uint64)
    for j in range(R):
        pu, pv = proxy_events(u, v, H[j])
        P[j] = component_matrix(pu, pv, t, k)
    return P


def hash_estimate(P: np.ndarray, H: np.ndarray, n: int, src=None) -> np.ndarray:
    """|OC-hat(u)| for the listed sources (Section 4.2, eq. DefEstOCMerge)."""
    R, k = P.shape[0], P.shape[1]
    count = n if src is None else len(src)
    est = np.zeros(count, dtype=np.uint32)
    Pc = np.ascontiguousarray(P, dtype=np.uint64).reshape(-1)
    Hc = np.ascontiguousarray(H, dtype=np.uint32).reshape(-1)
    if src is None:
        _check(_load().tnref_hash_estimate(Pc, R, k, Hc, n, None, 0, est))
    else:
        s = np.ascontiguousarray(src, dtype=np.uint32)
        _check(_load().tnref_hash_estimate(Pc, R, k, Hc, n, s.ctypes.data, len(s), est))
    return est


def emd_w1(a, b) -> float:
    """Wasserstein-1 (Earth-Mover) distance between two equal-size samples:
    the mean absolute difference of the sorted samples (Section 4.4)."""
    a = np.sort(np.asarray(a, dtype=np.float64))
    b = np.sort(np.asarray(b, dtype=np.float64))
    if a.shape != b.shape:
        raise ValueError("emd_w1 expects equal-size samples")
    return float(np.abs(a - b).mean()) if a.size else 0.0


def error_stats(est, exact) -> dict:
    """Error of estimated against exact out-component sizes over the same
    sources (Section 4.4): sum / max absolute error, mean / max relative error
    (relative to the exact size) and the Wasserstein-1 distance between the two
    size distributions (``w1_num`` = count * W1, an integer)."""
    a = np.ascontiguousarray(est, dtype=np.uint32)
    b = np.ascontiguousarray(exact, dtype=np.uint32)
    if a.shape != b.shape:
        raise ValueError("error_stats expects equal-size samples")
    sa, ma, wn = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
    rs, mr = ctypes.c_double(), ctypes.c_double()
    _check(_load().tnref_error_stats(a, b, len(a), ctypes.byref(sa), ctypes.byref(ma), ctypes.byref(wn),
                                     ctypes.byref(rs), ctypes.byref(mr)))
    c = len(a)
    return dict(count=c, sum_abs=sa.value, max_abs=ma.value, w1_num=wn.value, rel_sum=rs.value,
                max_rel=mr.value, mean_abs=sa.value / c if c else 0.0, mean_rel=rs.value / c if c else 0.0,
                w1=wn.value / c if c else 0.0)


def hll_singleton(seed: int, p: int, x: int):
    """(register, rank) of element x in a sketch of 2^p registers (Section 3.3)."""
    reg, rank = ctypes.c_uint32(), ctypes.c_uint8()
    _load().tnref_hll_singleton(seed, p, x, ctypes.byref(reg), ctypes.byref(rank))
    return reg.value, rank.value


def hll_sketches(u, v, t, n: int, p: int, seed: int, reverse: bool = False, directed: bool = False) -> np.ndarray:
    """uint8[n, 2^p]: node i's sketch of its in-component (out-component with
    reverse=True), merged by register-wise maximum per event (Sections 3.3, 3.4)."""
    u, v, t = _ev(u, v, t)
    R = np.zeros((n, 1 << p), dtype=np.uint8)
    _check(_load().tnref_hll_sketches(u, v, t, len(u), n, p, seed, int(reverse), int(directed), R.reshape(-1)))
    return R


def hll_estimate(R: np.ndarray, p: int) -> np.ndarray:
    """float64[n] HyperLogLog size estimates of the sketches."""
    R = np.ascontiguousarray(R, dtype=np.uint8)
    est = np.zeros(R.shape[0], dtype=np.float64)
    _load().tnref_hll_estimate(R.reshape(-1), R.shape[0], p, est)
    return est
