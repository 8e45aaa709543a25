"""GB300-native temporal out-components and network hashing (arXiv 2307.04890).

Thin binding over the C ABI of ``libtn.so`` (declared in ``include/tn.h``).
Every function here only marshals arguments -- torch tensors for device
memory, the current CUDA stream -- and calls the native entry point of the
same name; all computation runs in the library's CUDA kernels.  Importing the
package does not need a GPU; calling anything that launches work does, and
raises if the native library is missing (it is never replaced by a CPU path).

Matrix layout (all entry points): a component matrix with ``n_rows`` rows and
``ncols`` source columns is an int64 tensor of shape
``(n_rows, tn_row_words(ncols))`` holding packed bits; bit ``c`` of row ``i``
means "node i has been reached from source column c" (Section 3.1: rows are
in-components, columns out-components).
"""
from __future__ import annotations

import ctypes
import os

__all__ = [
    "TnError", "load_library", "tn_row_words", "tn_status_string", "tn_kernel_launches", "tn_init_matrix",
    "tn_component_matrix", "tn_component_columns", "tn_out_sizes",
    "tn_hash_proxy", "tn_hash_estimate", "tn_hash_estimate_noalloc", "tn_error_stats",
    "tn_out_component_sizes_host",
    "Plan", "tn_plan_apply_batch", "Server", "BatchGraph", "tn_autotune", "tn_selftest_wait_timeout",
    "tn_hll_sketches", "tn_hll_estimate", "tn_grow_matrix", "Online",
    "TN_OK", "TN_EINVAL", "TN_ERANGE", "TN_EORDER", "TN_ENOMEM", "TN_ECUDA", "TN_ETIMEOUT", "TN_ESCRATCH",
    "TN_INIT_IDENTITY", "TN_REVERSE", "TN_DIRECTED", "TN_GROUP_END", "TN_LAST_BATCH", "tn_server_job_bytes",
]

TN_OK, TN_EINVAL, TN_ERANGE, TN_EORDER, TN_ENOMEM, TN_ECUDA, TN_ETIMEOUT = 0, -1, -2, -3, -4, -5, -6
TN_ESCRATCH = -7
TN_INIT_IDENTITY = 1
TN_REVERSE = 2
TN_DIRECTED = 4
TN_GROUP_END = 8
TN_LAST_BATCH = 16

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBRARY_PATH = os.path.join(_HERE, "libtn.so")

_c_u32p = ctypes.c_void_p
_lib = None


class TnError(RuntimeError):
    """A libtn entry point returned a non-zero tn_status."""

    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.tn_status_string(status).decode() if _lib else str(status)
        if _lib and status in (TN_ECUDA, TN_ENOMEM):
            msg += f" ({_lib.tn_last_cuda_error().decode()})"
        super().__init__(f"{where}: {msg}")


class _Options(ctypes.Structure):
    _fields_ = [("window_events", ctypes.c_uint32), ("slab_words", ctypes.c_uint32),
                ("smem_rows", ctypes.c_uint32), ("directed", ctypes.c_uint32), ("wave_ctas", ctypes.c_uint32),
                ("resident_words", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 2)]


class _ErrorStats(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint64), ("sum_abs", ctypes.c_uint64), ("max_abs", ctypes.c_uint64),
                ("w1_num", ctypes.c_uint64), ("rel_sum", ctypes.c_double), ("max_rel", ctypes.c_double),
                ("mean_abs", ctypes.c_double), ("mean_rel", ctypes.c_double), ("w1", ctypes.c_double)]


class _ServerOptions(ctypes.Structure):
    _fields_ = [("memory_budget", ctypes.c_uint64), ("max_active", ctypes.c_uint32),
                ("window_events", ctypes.c_uint32), ("slab_words", ctypes.c_uint32),
                ("workers", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 2)]


class _JobRecord(ctypes.Structure):
    _fields_ = [("job_id", ctypes.c_uint64), ("status", ctypes.c_int32), ("n", ctypes.c_uint32),
                ("events", ctypes.c_uint64), ("t_submit_ns", ctypes.c_uint64), ("t_admit_ns", ctypes.c_uint64),
                ("t_done_ns", ctypes.c_uint64), ("t_last_push_ns", ctypes.c_uint64),
                ("t_enqueued_ns", ctypes.c_uint64)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_uint64) for name in ("queued", "active", "admitted", "completed", "bytes_in_use",
                                                     "budget", "peak_active", "peak_bytes", "batches", "admit_ns",
                                                     "copy_ns", "schedule_ns", "result_ns", "retire_ns")]


class _TuneResult(ctypes.Structure):
    _fields_ = [("best", _Options), ("best_ms", ctypes.c_float), ("tried", ctypes.c_uint32),
                ("cached", ctypes.c_uint32), ("pad", ctypes.c_uint32), ("sample_events", ctypes.c_uint64)]


class _Stats(ctypes.Structure):
    _fields_ = [("events", ctypes.c_uint64), ("windows", ctypes.c_uint64), ("levels", ctypes.c_uint64),
                ("ops", ctypes.c_uint64), ("aux", ctypes.c_uint64), ("temps", ctypes.c_uint64),
                ("big_windows", ctypes.c_uint64), ("local_windows", ctypes.c_uint64), ("items", ctypes.c_uint64),
                ("t_first", ctypes.c_int64), ("t_last", ctypes.c_int64)]


def load_library(path: str | None = None):
    """Load libtn.so (built by ``build.build_library``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIBRARY_PATH
    if not os.path.exists(path):
        raise ImportError(f"libtn native library not found at {path}; build it with "
                          "paper_2307_04890_gb300.build.build_library() (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, u32, u64, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32
    sigs = {
        "tn_status_string": ([i32], ctypes.c_char_p),
        "tn_last_cuda_error": ([], ctypes.c_char_p),
        "tn_row_words": ([u64], u64),
        "tn_resident_max_rows": ([u32], u32),
        "tn_kernel_launches": ([], u64),
        "tn_init_matrix": ([vp, u32, u32, vp, vp], i32),
        "tn_component_matrix": ([vp, vp, vp, u64, u32, vp, vp, u32, vp], i32),
        "tn_component_columns": ([vp, vp, vp, u64, u32, vp, u32, vp, vp, u32, vp], i32),
        "tn_out_sizes": ([vp, u32, u32, vp, vp, vp, vp], i32),
        "tn_plan_create": ([vp, vp, vp, u64, u32, vp, vp, vp, ctypes.POINTER(vp)], i32),
        "tn_plan_apply": ([vp, vp, u32, vp, vp, u32, vp], i32),
        "tn_plan_apply_batch": ([vp, vp, vp, vp, u32, u32, vp], i32),
        "tn_plan_status": ([vp, vp], i32),
        "tn_plan_get_stats": ([vp, ctypes.POINTER(_Stats)], i32),
        "tn_plan_destroy": ([vp, vp], i32),
        "tn_hash_proxy": ([vp, vp, u64, u32, u32, u32, u64, vp, vp, vp, vp], i32),
        "tn_hash_estimate": ([vp, u32, u32, vp, u32, vp, u32, vp, vp], i32),
        "tn_hash_estimate_noalloc": ([vp, u32, u32, vp, u32, vp, u32, vp, vp], i32),
        "tn_error_stats_compute": ([vp, vp, u32, u32, ctypes.POINTER(_ErrorStats), vp], i32),
        "tn_graph_capture_batch": ([vp, vp, vp, u32, u32, ctypes.POINTER(vp)], i32),
        "tn_graph_launch": ([vp, vp], i32),
        "tn_graph_destroy": ([vp], i32),
        "tn_autotune": ([vp, vp, vp, u64, u32, u32, u32, u64, vp, ctypes.POINTER(_TuneResult)], i32),
        "tn_selftest_wait_timeout": ([vp], i32),
        "tn_hll_row_bytes": ([u32], u64),
        "tn_hll_sketches": ([vp, vp, vp, u64, u32, u32, u64, u32, vp, vp], i32),
        "tn_hll_estimate": ([vp, u32, u32, vp, vp], i32),
        "tn_server_create": ([ctypes.POINTER(_ServerOptions), ctypes.POINTER(vp)], i32),
        "tn_server_submit": ([vp, u64, u32, vp, vp, vp, vp, u32, vp, vp], i32),
        "tn_server_open": ([vp, u64, u32, u64, vp, vp], i32),
        "tn_server_push": ([vp, u64, vp, vp, vp, u64, u32], i32),
        "tn_server_job_bytes": ([u32, u64], u64),
        "tn_server_poll": ([vp, ctypes.POINTER(_JobRecord), u32, ctypes.POINTER(u32), u32], i32),
        "tn_server_get_stats": ([vp, ctypes.POINTER(_ServerStats)], i32),
        "tn_server_destroy": ([vp], i32),
        "tn_out_component_sizes_host": ([vp, vp, vp, u64, u32, vp, vp, vp, vp], i32),
        "tn_grow_matrix": ([vp, u32, vp, u32, vp], i32),
        "tn_online_create": ([u32, ctypes.POINTER(_Options), vp, ctypes.POINTER(vp)], i32),
        "tn_online_push": ([vp, vp, vp, vp, u64, u32, vp], i32),
        "tn_online_flush": ([vp, vp], i32),
        "tn_online_grow": ([vp, u32, vp], i32),
        "tn_online_status": ([vp, vp], i32),
        "tn_online_get_state": ([vp, ctypes.POINTER(_OnlineState)], i32),
        "tn_online_destroy": ([vp, vp], i32),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != TN_OK:
        raise TnError(status, where)


def _torch():
    import torch
    return torch


def _stream(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(x):
    return None if x is None else ctypes.c_void_p(x.data_ptr())


def _dev(x, dtype_names, what):
    torch = _torch()
    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if not x.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if str(x.dtype).replace("torch.", "") not in dtype_names:
        raise TypeError(f"{what} has dtype {x.dtype}, expected one of {dtype_names}")
    return x


def tn_row_words(ncols: int) -> int:
    return int(load_library().tn_row_words(ncols))


def tn_resident_max_rows(resident_words: int) -> int:
    """Largest node count whose rows fit the resident-slab form (no saved rows)."""
    return int(load_library().tn_resident_max_rows(resident_words))


def tn_kernel_launches() -> int:
    """Kernels launched by libtn in this process so far."""
    return int(load_library().tn_kernel_launches())


def tn_init_matrix(S, n_rows: int, ncols: int | None = None, src=None, stream=None):
    """Initial state of Algorithm 1: identity, or the listed source columns."""
    lib = load_library()
    ncols = n_rows if ncols is None else ncols
    S = _matrix(S, n_rows, ncols, S.device)
    _check(lib.tn_init_matrix(_ptr(S), n_rows, ncols, _ptr(src), _stream(stream)), "tn_init_matrix")
    return S


def tn_status_string(status: int) -> str:
    return load_library().tn_status_string(status).decode()


def _events(u, v, t):
    _dev(u, ("int32", "uint32"), "u")
    _dev(v, ("int32", "uint32"), "v")
    _dev(t, ("int64",), "t")
    if not (u.numel() == v.numel() == t.numel()):
        raise ValueError("u, v, t must have the same length")
    return u.numel()


def _matrix(S, n_rows, ncols, device):
    torch = _torch()
    shape = (n_rows, tn_row_words(ncols))
    if S is None:
        return torch.empty(shape, dtype=torch.int64, device=device)
    _dev(S, ("int64", "uint64"), "S")
    if tuple(S.shape) != shape:
        raise ValueError(f"S must have shape {shape}")
    return S


def tn_component_matrix(u, v, t, n: int, S=None, t_last=None, init: bool = True, reverse: bool = False,
                        directed: bool = False, stream=None):
    """Algorithm 1 (Section 3.1) over one event batch; returns S (int64 [n, W]).
    reverse=True processes the sequence backwards (Section 3.4): row i is then
    the out-component of i (the transpose of the chronological matrix)."""
    lib = load_library()
    m = _events(u, v, t)
    S = _matrix(S, n, n, u.device)
    if t_last is not None:
        _dev(t_last, ("int64",), "t_last")
    flags = (TN_INIT_IDENTITY if init else 0) | (TN_REVERSE if reverse else 0) | (TN_DIRECTED if directed else 0)
    _check(lib.tn_component_matrix(_ptr(u), _ptr(v), _ptr(t), m, n, _ptr(S), _ptr(t_last), flags,
                                   _stream(stream)), "tn_component_matrix")
    return S


def tn_component_columns(u, v, t, n: int, src, S=None, t_last=None, init: bool = True, reverse: bool = False,
                         directed: bool = False, stream=None):
    """Out-components of the listed sources only (column c = source src[c]);
    with reverse=True, column c is the in-component of src[c]."""
    lib = load_library()
    m = _events(u, v, t)
    _dev(src, ("int32", "uint32"), "src")
    S = _matrix(S, n, src.numel(), u.device)
    flags = (TN_INIT_IDENTITY if init else 0) | (TN_REVERSE if reverse else 0) | (TN_DIRECTED if directed else 0)
    _check(lib.tn_component_columns(_ptr(u), _ptr(v), _ptr(t), m, n, _ptr(src), src.numel(), _ptr(S),
                                    _ptr(t_last), flags, _stream(stream)), "tn_component_columns")
    return S


def tn_out_sizes(S, n_rows: int, ncols: int, in_sizes: bool = False, argmax: bool = False, stream=None):
    """Column (out-component) and row (in-component) sizes; returns
    (out int32[ncols], in int32[n_rows] or None, argmax int32[1] or None)."""
    torch = _torch()
    lib = load_library()
    S = _matrix(S, n_rows, ncols, S.device)
    out = torch.empty(ncols, dtype=torch.int32, device=S.device)
    ins = torch.empty(n_rows, dtype=torch.int32, device=S.device) if in_sizes else None
    am = torch.empty(1, dtype=torch.int32, device=S.device) if argmax else None
    _check(lib.tn_out_sizes(_ptr(S), n_rows, ncols, _ptr(out), _ptr(ins), _ptr(am), _stream(stream)),
           "tn_out_sizes")
    return out, ins, am


def tn_hash_proxy(u, v, n: int, k: int, R: int, seed: int, events: bool = True, stream=None):
    """Hash tables H (int32 [R, n]) and super-events (pu, pv: int32 [R, m])."""
    torch = _torch()
    lib = load_library()
    device = u.device if u is not None else torch.device("cuda")
    H = torch.empty((R, n), dtype=torch.int32, device=device)
    pu = pv = None
    m = 0
    if events and u is not None:
        m = u.numel()
        _dev(u, ("int32", "uint32"), "u")
        _dev(v, ("int32", "uint32"), "v")
        pu = torch.empty((R, m), dtype=torch.int32, device=device)
        pv = torch.empty((R, m), dtype=torch.int32, device=device)
    _check(lib.tn_hash_proxy(_ptr(u) if m else None, _ptr(v) if m else None, m, n, k, R, seed & (2**64 - 1),
                             _ptr(H), _ptr(pu), _ptr(pv), _stream(stream)), "tn_hash_proxy")
    return H, pu, pv


def tn_hash_estimate(P, R: int, k: int, H, n: int, src=None, stream=None):
    """Fusion by intersection (Section 4.2); est int32[nsrc]."""
    torch = _torch()
    lib = load_library()
    _dev(P, ("int64", "uint64"), "P")
    _dev(H, ("int32", "uint32"), "H")
    nsrc = n if src is None else src.numel()
    if src is not None:
        _dev(src, ("int32", "uint32"), "src")
    est = torch.empty(nsrc, dtype=torch.int32, device=P.device)
    _check(lib.tn_hash_estimate(_ptr(P), R, k, _ptr(H), n, _ptr(src), nsrc, _ptr(est), _stream(stream)),
           "tn_hash_estimate")
    return est


def tn_hash_estimate_noalloc(P, R: int, k: int, H, n: int, est, src=None, stream=None):
    """Fusion by intersection into the caller's est int32[nsrc]; the library
    allocates nothing (its scratch is one fixed device array per device)."""
    lib = load_library()
    _dev(P, ("int64", "uint64"), "P")
    _dev(H, ("int32", "uint32"), "H")
    _dev(est, ("int32", "uint32"), "est")
    nsrc = n if src is None else src.numel()
    if src is not None:
        _dev(src, ("int32", "uint32"), "src")
    if est.numel() < nsrc:
        raise ValueError("est is smaller than the number of sources")
    _check(lib.tn_hash_estimate_noalloc(_ptr(P), R, k, _ptr(H), n, _ptr(src), nsrc, _ptr(est), _stream(stream)),
           "tn_hash_estimate_noalloc")
    return est


def tn_error_stats(est, exact, max_value: int, stream=None) -> dict:
    """Error of estimated against exact sizes of the same sources (Section 4.4):
    absolute, relative and Wasserstein-1 (``w1_num`` = count * W1, exact)."""
    lib = load_library()
    _dev(est, ("int32", "uint32"), "est")
    _dev(exact, ("int32", "uint32"), "exact")
    if est.numel() != exact.numel():
        raise ValueError("est and exact must have the same length")
    out = _ErrorStats()
    _check(lib.tn_error_stats_compute(_ptr(est), _ptr(exact), est.numel(), max_value, ctypes.byref(out),
                                      _stream(stream)), "tn_error_stats")
    return {name: getattr(out, name) for name, _ in _ErrorStats._fields_}


def _plan_options(window_events=0, slab_words=0, smem_rows=0, directed=False, wave_ctas=0, resident_words=0):
    return _Options(window_events, slab_words, smem_rows, 1 if directed else 0, wave_ctas, resident_words)


def tn_out_component_sizes_host(u, v, t, n: int, **plan_options):
    """Whole exact path from host numpy arrays; returns (sizes uint32[n], argmax).
    ``plan_options``: window_events, slab_words, smem_rows, directed, wave_ctas, resident_words."""
    import numpy as np
    lib = load_library()
    u = np.ascontiguousarray(u, dtype=np.uint32)
    v = np.ascontiguousarray(v, dtype=np.uint32)
    t = np.ascontiguousarray(t, dtype=np.int64)
    out = np.empty(n, dtype=np.uint32)
    am = np.zeros(1, dtype=np.uint32)
    opt = _plan_options(**plan_options)
    _check(lib.tn_out_component_sizes_host(u.ctypes.data, v.ctypes.data, t.ctypes.data, len(u), n,
                                           ctypes.byref(opt), out.ctypes.data, am.ctypes.data, _stream()),
           "tn_out_component_sizes_host")
    return out, int(am[0])


def tn_out_component_sizes_host_ptrs(u_ptr: int, v_ptr: int, t_ptr: int, m: int, n: int, out_ptr: int,
                                     argmax_ptr: int | None = None, stream=None, **plan_options):
    """Same as ``tn_out_component_sizes_host`` on raw host pointers (pinned buffers)."""
    lib = load_library()
    opt = _plan_options(**plan_options)
    _check(lib.tn_out_component_sizes_host(u_ptr, v_ptr, t_ptr, m, n, ctypes.byref(opt), out_ptr, argmax_ptr,
                                           _stream(stream)), "tn_out_component_sizes_host")


class _OnlineState(ctypes.Structure):
    _fields_ = [("S", ctypes.c_void_p), ("n", ctypes.c_uint32), ("has_applied", ctypes.c_uint32),
                ("row_words", ctypes.c_uint64), ("pending_events", ctypes.c_uint64), ("pending_t", ctypes.c_int64),
                ("t_applied", ctypes.c_int64), ("applied_events", ctypes.c_uint64), ("batches", ctypes.c_uint64)]


class Plan:
    """A validated, scheduled event batch (tn_plan_create / tn_plan_apply)."""

    def __init__(self, u, v, t, n: int, t_after=None, window_events: int = 0, slab_words: int = 0,
                 smem_rows: int = 0, directed: bool = False, wave_ctas: int = 0, resident_words: int = 0,
                 stream=None):
        lib = load_library()
        self.m = _events(u, v, t)
        self.n = n
        self.device = u.device
        opt = _Options(window_events, slab_words, smem_rows, 1 if directed else 0, wave_ctas, resident_words)
        h = ctypes.c_void_p()
        if t_after is not None:
            _dev(t_after, ("int64",), "t_after")
        _check(lib.tn_plan_create(_ptr(u), _ptr(v), _ptr(t), self.m, n, _ptr(t_after), ctypes.byref(opt),
                                  _stream(stream), ctypes.byref(h)), "tn_plan_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def apply(self, S, ncols: int | None = None, src=None, t_last=None, init: bool = False, stream=None):
        lib = load_library()
        ncols = self.n if ncols is None else ncols
        S = _matrix(S, self.n, ncols, self.device)
        _check(lib.tn_plan_apply(self._h, _ptr(S), ncols, _ptr(src), _ptr(t_last),
                                 TN_INIT_IDENTITY if init else 0, _stream(stream)), "tn_plan_apply")
        return S

    def status(self, stream=None) -> int:
        return int(load_library().tn_plan_status(self._h, _stream(stream)))

    def stats(self) -> dict:
        st = _Stats()
        _check(load_library().tn_plan_get_stats(self._h, ctypes.byref(st)), "tn_plan_get_stats")
        return {f: getattr(st, f) for f, _ in _Stats._fields_}

    def destroy(self, stream=None):
        if self._h:
            load_library().tn_plan_destroy(self._h, _stream(stream))
            self._h = None

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.tn_plan_destroy(self._h, None)
                self._h = None
        except Exception:
            pass


def tn_plan_apply_batch(plans, mats, ncols=None, init: bool = True, srcs=None, stream=None):
    """One launch over several (plan, matrix) pairs; ``srcs``: None, or one
    entry per pair (None = all nodes, else a device int32 tensor of the
    matrix's source ids, used with ``init``)."""
    lib = load_library()
    count = len(plans)
    ncols = ncols or [p.n for p in plans]
    hp = (ctypes.c_void_p * count)(*[p.handle for p in plans])
    hs = (ctypes.c_void_p * count)(*[m.data_ptr() for m in mats])
    hn = (ctypes.c_uint32 * count)(*ncols)
    hsrc = None
    if srcs is not None:
        for s_ in srcs:
            if s_ is not None:
                _dev(s_, ("int32", "uint32"), "srcs")
        hsrc = (ctypes.c_void_p * count)(*[None if s_ is None else s_.data_ptr() for s_ in srcs])
    _check(lib.tn_plan_apply_batch(hp, hs, hn, hsrc, count, TN_INIT_IDENTITY if init else 0, _stream(stream)),
           "tn_plan_apply_batch")
    return mats


def tn_server_job_bytes(n: int, max_batch_events: int) -> int:
    """Device bytes a serving job of n nodes and batches of at most
    ``max_batch_events`` events is charged against the server's budget."""
    return int(load_library().tn_server_job_bytes(n, max_batch_events))


class Server:
    """Continuous admission of component-matrix jobs (tn_server_*).

    ``submit`` (all batches at once) or ``open`` + ``push`` (batches as they
    arrive) take host numpy arrays and keep them (and the result buffer)
    alive until the job's record comes back from ``poll``;
    ``results[job_id]`` then holds ``(out_sizes, argmax)``.
    """

    def __init__(self, memory_budget: int = 0, max_active: int = 0, window_events: int = 0, slab_words: int = 0,
                 workers: int = 0):
        lib = load_library()
        opt = _ServerOptions(memory_budget, max_active, window_events, slab_words, workers)
        h = ctypes.c_void_p()
        _check(lib.tn_server_create(ctypes.byref(opt), ctypes.byref(h)), "tn_server_create")
        self._h = h
        self._keep = {}
        self.results = {}

    def submit(self, job_id: int, n: int, u, v, t, batch_offsets):
        import numpy as np
        lib = load_library()
        u = np.ascontiguousarray(u, dtype=np.uint32)
        v = np.ascontiguousarray(v, dtype=np.uint32)
        t = np.ascontiguousarray(t, dtype=np.int64)
        offs = np.ascontiguousarray(batch_offsets, dtype=np.uint64)
        if offs[-1] != len(u) or len(v) != len(u) or len(t) != len(u):
            raise ValueError("batch offsets must end at the number of events")
        out = np.zeros(n, dtype=np.uint32)
        am = np.zeros(1, dtype=np.uint32)
        _check(lib.tn_server_submit(self._h, job_id, n, u.ctypes.data, v.ctypes.data, t.ctypes.data,
                                    offs.ctypes.data, len(offs) - 1, out.ctypes.data, am.ctypes.data),
               "tn_server_submit")
        self._keep[job_id] = [out, am, (u, v, t, offs)]

    def open(self, job_id: int, n: int, max_batch_events: int):
        """Opens a job whose batches (at most ``max_batch_events`` events each)
        follow with ``push``."""
        import numpy as np
        out = np.zeros(n, dtype=np.uint32)
        am = np.zeros(1, dtype=np.uint32)
        _check(load_library().tn_server_open(self._h, job_id, n, max_batch_events, out.ctypes.data, am.ctypes.data),
               "tn_server_open")
        self._keep[job_id] = [out, am]  # only once the job is open: a refused open keeps the old job's buffers

    def push(self, job_id: int, u, v, t, last: bool = False):
        """Appends a batch of host events to an open job (``last``: the job's
        final batch, after which its results follow)."""
        import numpy as np
        u = np.ascontiguousarray(u, dtype=np.uint32)
        v = np.ascontiguousarray(v, dtype=np.uint32)
        t = np.ascontiguousarray(t, dtype=np.int64)
        if len(v) != len(u) or len(t) != len(u):
            raise ValueError("u, v and t must have the same length")
        _check(load_library().tn_server_push(self._h, job_id, u.ctypes.data, v.ctypes.data, t.ctypes.data, len(u),
                                             TN_LAST_BATCH if last else 0), "tn_server_push")
        self._keep[job_id].append((u, v, t))  # alive until the job's record is polled

    def poll(self, wait_ms: int = 0, capacity: int = 256):
        """Records of finished jobs: dicts with job_id, status, n, events and
        the submit / admit / done host times in ns."""
        lib = load_library()
        recs = (_JobRecord * capacity)()
        cnt = ctypes.c_uint32()
        _check(lib.tn_server_poll(self._h, recs, capacity, ctypes.byref(cnt), wait_ms), "tn_server_poll")
        out = []
        for r in recs[: cnt.value]:
            d = {name: getattr(r, name) for name, _ in _JobRecord._fields_}
            kept = self._keep.pop(d["job_id"], None)
            if kept is not None:
                self.results[d["job_id"]] = (kept[0], int(kept[1][0]))
            out.append(d)
        return out

    def stats(self) -> dict:
        st = _ServerStats()
        _check(load_library().tn_server_get_stats(self._h, ctypes.byref(st)), "tn_server_get_stats")
        return {name: getattr(st, name) for name, _ in _ServerStats._fields_}

    def close(self):
        if self._h:
            _check(load_library().tn_server_destroy(self._h), "tn_server_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tn_autotune(u, v, t, n: int, replicas: int = 1, sample_events: int = 200_000, ncols: int = 0,
                stream=None) -> dict:
    """Plan options for a batch of ``replicas`` networks shaped like (u, v, t, n)
    with ``ncols`` source columns each (0 = n), chosen by timing the candidates
    on the first ``sample_events`` events (scored as waves x one wave's time)."""
    lib = load_library()
    m = _events(u, v, t)
    res = _TuneResult()
    _check(lib.tn_autotune(_ptr(u), _ptr(v), _ptr(t), m, n, ncols, replicas, sample_events, _stream(stream),
                           ctypes.byref(res)), "tn_autotune")
    return {"window_events": res.best.window_events, "slab_words": res.best.slab_words,
            "smem_rows": res.best.smem_rows, "wave_ctas": res.best.wave_ctas,
            "resident_words": res.best.resident_words, "best_ms": res.best_ms, "tried": res.tried,
            "cached": bool(res.cached), "sample_events": res.sample_events}


class BatchGraph:
    """One batched application (tn_plan_apply_batch) captured as a CUDA graph;
    ``launch()`` replays it with a single graph launch."""

    def __init__(self, plans, mats, ncols=None, init: bool = True):
        lib = load_library()
        count = len(plans)
        ncols = ncols or [p.n for p in plans]
        self._plans, self._mats = list(plans), list(mats)  # keep them alive
        hp = (ctypes.c_void_p * count)(*[p.handle for p in plans])
        hs = (ctypes.c_void_p * count)(*[m.data_ptr() for m in mats])
        hn = (ctypes.c_uint32 * count)(*ncols)
        h = ctypes.c_void_p()
        _check(lib.tn_graph_capture_batch(hp, hs, hn, count, TN_INIT_IDENTITY if init else 0, ctypes.byref(h)),
               "tn_graph_capture_batch")
        self._h = h

    def launch(self, stream=None):
        _check(load_library().tn_graph_launch(self._h, _stream(stream)), "tn_graph_launch")

    def destroy(self):
        if self._h:
            load_library().tn_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def tn_selftest_wait_timeout(stream=None) -> int:
    """Runs the bounded-wait self-test; returns its status (TN_ETIMEOUT expected)."""
    return int(load_library().tn_selftest_wait_timeout(_stream(stream)))


def tn_hll_sketches(u, v, t, n: int, p: int, seed: int, reverse: bool = False, directed: bool = False, stream=None):
    """HyperLogLog sketches of the components (Section 3.3; reversed, Section 3.4): uint8 [n, row_bytes];
    the first 2^p bytes of row i are node i's registers."""
    torch = _torch()
    lib = load_library()
    m = _events(u, v, t)
    rb = int(lib.tn_hll_row_bytes(p))
    if rb == 0:
        raise ValueError("p must be in [4, 16]")
    R = torch.empty((n, rb), dtype=torch.uint8, device=u.device)
    flags = (TN_REVERSE if reverse else 0) | (TN_DIRECTED if directed else 0)
    _check(lib.tn_hll_sketches(_ptr(u), _ptr(v), _ptr(t), m, n, p, seed & (2**64 - 1), flags, _ptr(R),
                               _stream(stream)), "tn_hll_sketches")
    return R


def tn_hll_estimate(R, n: int, p: int, stream=None):
    """float64[n] size estimates of the sketches."""
    torch = _torch()
    lib = load_library()
    est = torch.empty(n, dtype=torch.float64, device=R.device)
    _check(lib.tn_hll_estimate(_ptr(R), n, p, _ptr(est), _stream(stream)), "tn_hll_estimate")
    return est


def tn_grow_matrix(S, n_old: int, n_new: int, out=None, stream=None):
    """Node growth (Section 3.5): S (n_old x n_old) extended by new rows and
    columns of zeros with only the new nodes' diagonal bits set.  Writes into ``out`` (a new
    n_new x tn_row_words(n_new) tensor when None; ``out is S`` grows in place,
    which needs an unchanged row stride and room for n_new rows)."""
    lib = load_library()
    torch = _torch()
    S = _matrix(S, S.shape[0], n_old, S.device) if n_old else S
    if out is None:
        out = torch.empty((n_new, tn_row_words(n_new)), dtype=torch.int64, device=S.device)
    _dev(out, ("int64", "uint64"), "out")
    if out.shape[1] != tn_row_words(n_new) or out.shape[0] < n_new:
        raise ValueError("out must have tn_row_words(n_new) columns and at least n_new rows")
    _check(lib.tn_grow_matrix(_ptr(S) if n_old else None, n_old, _ptr(out), n_new, _stream(stream)),
           "tn_grow_matrix")
    return out


class _DeviceView:
    """Exposes library-owned device memory to torch without a copy."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<i8", "data": (ptr, False),
                                         "version": 3, "strides": None}


class Online:
    """Online component matrix (tn_online_*, Section 3.5): batches of device
    events in time order, timestamp groups may be split across batches, nodes
    may be added between batches."""

    def __init__(self, n: int, window_events: int = 0, slab_words: int = 0, smem_rows: int = 0,
                 directed: bool = False, wave_ctas: int = 0, stream=None):
        lib = load_library()
        opt = _Options(window_events, slab_words, smem_rows, 1 if directed else 0, wave_ctas)
        h = ctypes.c_void_p()
        _check(lib.tn_online_create(n, ctypes.byref(opt), _stream(stream), ctypes.byref(h)), "tn_online_create")
        self._h = h

    def push(self, u, v, t, group_end: bool = False, stream=None):
        """Applies every complete timestamp group; the batch's last group stays
        pending unless ``group_end``."""
        m = _events(u, v, t)
        _check(load_library().tn_online_push(self._h, _ptr(u), _ptr(v), _ptr(t), m,
                                             TN_GROUP_END if group_end else 0, _stream(stream)),
               "tn_online_push")

    def flush(self, stream=None):
        _check(load_library().tn_online_flush(self._h, _stream(stream)), "tn_online_flush")

    def grow(self, n_new: int, stream=None):
        _check(load_library().tn_online_grow(self._h, n_new, _stream(stream)), "tn_online_grow")

    def status(self, stream=None) -> int:
        return load_library().tn_online_status(self._h, _stream(stream))

    def state(self) -> dict:
        st = _OnlineState()
        _check(load_library().tn_online_get_state(self._h, ctypes.byref(st)), "tn_online_get_state")
        return {name: getattr(st, name) for name, _ in _OnlineState._fields_}

    def matrix(self):
        """The current matrix as an int64 [n, tn_row_words(n)] tensor that
        aliases the library's buffer (valid until the next grow or close)."""
        torch = _torch()
        st = self.state()
        return torch.as_tensor(_DeviceView(st["S"], (st["n"], st["row_words"])), device="cuda")

    def close(self, stream=None):
        if self._h:
            _check(load_library().tn_online_destroy(self._h, _stream(stream)), "tn_online_destroy")
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
