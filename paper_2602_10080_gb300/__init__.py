"""Python binding of libsssp.so (the C ABI in include/sssp.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  Arrays are torch tensors (CUDA or CPU) or numpy arrays; their data
pointers go straight to the C entry points.  There is no fallback: if the
shared library is missing or fails to load, importing a function raises.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsssp.so")

SSSP_OK = 0
SSSP_E_INVAL = -1
SSSP_E_NOMEM = -2
SSSP_E_CUDA = -3
SSSP_E_TIMEOUT = -4
SSSP_E_BADGRAPH = -5
SSSP_E_BUSY = -6
SSSP_E_NODEV = -7
SSSP_E_NOTFOUND = -8
SSSP_E_CANCELLED = -9
SSSP_NOALLOC_MAX_VERTICES = 2097152

SSSP_W_U32 = 0
SSSP_W_F32 = 1
L1_VECTOR, L1_NEARFAR, L1_FILTER, L1_SLF = 0, 1, 2, 3
L2_VECTOR, L2_BUCKET = 0, 1
Q_QUEUED, Q_RUNNING, Q_DONE, Q_ERROR = 0, 1, 2, 3
SERVE_MIGRATE_EACH_SLICE, SERVE_INJECT_OVERFLOW, SERVE_INJECT_TIMEOUT, SERVE_INJECT_NEGATIVE = 1, 2, 4, 8


class SsspError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class sssp_config(ctypes.Structure):
    _fields_ = [
        ("l1_type", ctypes.c_int32), ("l2_type", ctypes.c_int32), ("l0_rows", ctypes.c_int32),
        ("l1_cap", ctypes.c_int32), ("wb", ctypes.c_int32), ("delta_u32", ctypes.c_uint32),
        ("delta_f32", ctypes.c_float), ("bnum", ctypes.c_int32), ("bmax", ctypes.c_int32),
        ("filter_deltas", ctypes.c_float), ("near_deltas", ctypes.c_float), ("max_arcs", ctypes.c_int32),
        ("claim", ctypes.c_int32), ("shards", ctypes.c_int32), ("refillers", ctypes.c_int32),
        ("stage", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
        ("timeout_ms", ctypes.c_int32), ("l2_only", ctypes.c_int32), ("split_arcs", ctypes.c_int32),
        ("hub_bnum", ctypes.c_int32), ("dedup", ctypes.c_int32), ("pending_marks", ctypes.c_int32),
        ("direct_buckets", ctypes.c_int32),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class sssp_serve_options(ctypes.Structure):
    _fields_ = [
        ("mem_budget_bytes", ctypes.c_size_t), ("max_slots", ctypes.c_int32), ("slice_us", ctypes.c_int32),
        ("max_queued", ctypes.c_int32), ("ring_shift", ctypes.c_int32), ("query_timeout_ms", ctypes.c_int32),
        ("flags", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2),
    ]


class sssp_serve_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
        ("cancelled", ctypes.c_int64), ("slices", ctypes.c_int64), ("joined_running", ctypes.c_int64),
        ("ring_growths", ctypes.c_int64), ("restarts", ctypes.c_int64), ("max_resident", ctypes.c_int64),
        ("kernel_ms", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class sssp_features(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64), ("m", ctypes.c_int64), ("avg_deg", ctypes.c_double),
        ("max_deg", ctypes.c_double), ("std_deg", ctypes.c_double), ("avg_w", ctypes.c_double),
        ("max_w", ctypes.c_double), ("std_w", ctypes.c_double), ("min_w", ctypes.c_double),
        ("symmetric", ctypes.c_int32), ("has_zero_w", ctypes.c_int32), ("shadows", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class sssp_stats(ctypes.Structure):
    CYCLE_NAMES = ("relax", "l1_read", "l2_write", "global_read", "idle", "l0_read")

    _fields_ = [
        ("kernel_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("reached", ctypes.c_int64),
        ("reached_arcs", ctypes.c_int64), ("pops_l0", ctypes.c_int64), ("pops_l1", ctypes.c_int64),
        ("pops_l2", ctypes.c_int64), ("pops_heavy", ctypes.c_int64), ("relax_arcs", ctypes.c_int64),
        ("improved", ctypes.c_int64), ("stale", ctypes.c_int64),
        ("l2_chunks_written", ctypes.c_int64), ("l1_flushes", ctypes.c_int64),
        ("far_pushes", ctypes.c_int64), ("cas_fail", ctypes.c_int64), ("refills", ctypes.c_int64),
        ("deferred", ctypes.c_int64), ("relax_shadow", ctypes.c_int64), ("cycles", ctypes.c_int64 * 6),
        ("grid_blocks", ctypes.c_int32),
        ("block_threads", ctypes.c_int32), ("attempts", ctypes.c_int32), ("pad0", ctypes.c_int32),
        ("dup_targets", ctypes.c_int64), ("rounds", ctypes.c_int64), ("refill_tries", ctypes.c_int64),
        ("wait_spins", ctypes.c_int64), ("idle_iters", ctypes.c_int64), ("window_pull_backs", ctypes.c_int64),
        ("window_advances", ctypes.c_int64), ("lock_spins", ctypes.c_int64),
        ("cycles_fine", ctypes.c_int64 * 8), ("not_queued", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k not in ("cycles", "pad0", "cycles_fine")}
        d["cycles"] = dict(zip(self.CYCLE_NAMES, list(self.cycles)))
        d["cycles_fine"] = dict(zip(("rounds", "push", "batch", "far_flush", "lock", "claim", "chunks", "stage"),
                                    list(self.cycles_fine)))
        return d


_lib = None


def build(force: bool = False) -> str:
    from . import buildlib
    return buildlib.build(force=force)


def lib():
    """Loads libsssp.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsssp.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    sig = {
        "sssp_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "sssp_version": (ctypes.c_int, []),
        "sssp_config_default": (ctypes.c_int, [ctypes.POINTER(sssp_config)]),
        "sssp_graph_create": (ctypes.c_int, [P, P, P, I32, I64, I32, ctypes.POINTER(P)]),
        "sssp_graph_destroy": (ctypes.c_int, [P]),
        "sssp_graph_features": (ctypes.c_int, [P, ctypes.POINTER(sssp_features)]),
        "sssp_solve": (ctypes.c_int, [P, I32, P, P, ctypes.POINTER(sssp_config), P]),
        "sssp_solve_batch": (ctypes.c_int, [P, P, I32, P, P, ctypes.POINTER(sssp_config), P]),
        "sssp_bfs": (ctypes.c_int, [P, I32, P, P, ctypes.POINTER(sssp_config), P]),
        "sssp_solve_sampled": (ctypes.c_int, [P, I32, P, P, ctypes.POINTER(sssp_config), P, I32, I32,
                                              ctypes.POINTER(I32)]),
        "sssp_last_stats": (ctypes.c_int, [P, ctypes.POINTER(sssp_stats)]),
        "sssp_autotune": (ctypes.c_int, [P, P, I32, I32, ctypes.POINTER(sssp_config)]),
        "sssp_autotune_batch": (ctypes.c_int, [P, P, I32, I32, ctypes.POINTER(sssp_config)]),
        "sssp_serve_options_default": (ctypes.c_int, [ctypes.POINTER(sssp_serve_options)]),
        "sssp_serve_create": (ctypes.c_int, [ctypes.POINTER(sssp_serve_options), ctypes.POINTER(P)]),
        "sssp_serve_submit": (ctypes.c_int, [P, P, I32, P, P, ctypes.POINTER(ctypes.c_uint64)]),
        "sssp_serve_poll": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "sssp_serve_wait": (ctypes.c_int, [P, ctypes.c_uint64, I32, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "sssp_serve_latency_us": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
        "sssp_serve_cancel": (ctypes.c_int, [P, ctypes.c_uint64]),
        "sssp_serve_release": (ctypes.c_int, [P, ctypes.c_uint64]),
        "sssp_serve_get_stats": (ctypes.c_int, [P, ctypes.POINTER(sssp_serve_stats)]),
        "sssp_serve_destroy": (ctypes.c_int, [P]),
        "sssp_solve_noalloc": (ctypes.c_int, [P, P, I32, I64, I32, I32, P, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().sssp_strerror(code).decode()
    except Exception:  # pragma: no cover
        return str(code)


def _check(rc: int, where: str):
    if rc != SSSP_OK:
        raise SsspError(rc, where)


def _ptr(x):
    """Data pointer of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("array must be contiguous")
        return x.data_ptr()
    if hasattr(x, "ctypes"):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return x.ctypes.data
    raise TypeError(f"unsupported array type {type(x)}")


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def sssp_config_default() -> sssp_config:
    c = sssp_config()
    _check(lib().sssp_config_default(ctypes.byref(c)), "sssp_config_default")
    return c


def sssp_graph_create(row_ptr, col_idx, weights, n: int, m: int, wtype: int):
    h = ctypes.c_void_p()
    _check(lib().sssp_graph_create(_ptr(row_ptr), _ptr(col_idx), _ptr(weights), n, m, wtype,
                                   ctypes.byref(h)), "sssp_graph_create")
    return h


def sssp_graph_destroy(h) -> None:
    _check(lib().sssp_graph_destroy(h), "sssp_graph_destroy")


def sssp_graph_features(h) -> sssp_features:
    f = sssp_features()
    _check(lib().sssp_graph_features(h, ctypes.byref(f)), "sssp_graph_features")
    return f


def sssp_solve(h, src: int, dist_out, pred_out=None, cfg: sssp_config | None = None, stream=None) -> None:
    _check(lib().sssp_solve(h, int(src), _ptr(dist_out), _ptr(pred_out),
                            ctypes.byref(cfg) if cfg is not None else None, _stream_ptr(stream)),
           "sssp_solve")


def sssp_solve_batch(h, srcs, dist_out, pred_out=None, cfg: sssp_config | None = None,
                     stream=None) -> None:
    nq = int(srcs.numel() if hasattr(srcs, "numel") else srcs.size)
    _check(lib().sssp_solve_batch(h, _ptr(srcs), nq, _ptr(dist_out), _ptr(pred_out),
                                  ctypes.byref(cfg) if cfg is not None else None, _stream_ptr(stream)),
           "sssp_solve_batch")


def sssp_last_stats(h) -> sssp_stats:
    s = sssp_stats()
    _check(lib().sssp_last_stats(h, ctypes.byref(s)), "sssp_last_stats")
    return s


def sssp_autotune(h, srcs=None, budget_ms: int = 0) -> sssp_config:
    c = sssp_config()
    nsrc = 0 if srcs is None else int(srcs.numel() if hasattr(srcs, "numel") else srcs.size)
    _check(lib().sssp_autotune(h, _ptr(srcs), nsrc, int(budget_ms), ctypes.byref(c)), "sssp_autotune")
    return c


def sssp_autotune_batch(h, srcs, budget_ms: int = 0) -> sssp_config:
    """Tunes (and caches on the graph) the configuration of multi-query
    launches of len(srcs) queries."""
    c = sssp_config()
    nq = int(srcs.numel() if hasattr(srcs, "numel") else srcs.size)
    _check(lib().sssp_autotune_batch(h, _ptr(srcs), nq, int(budget_ms), ctypes.byref(c)), "sssp_autotune_batch")
    return c


def sssp_bfs(h, src: int, level_out, pred_out=None, cfg=None, stream=None) -> None:
    """Breadth-first levels (uint32 hops) and smallest-index parents."""
    _check(lib().sssp_bfs(h, int(src), _ptr(level_out), _ptr(pred_out), None if cfg is None else ctypes.byref(cfg),
                          _stream_ptr(stream)), "sssp_bfs")


SAMPLE_FIELDS = ("ns", "l2_written", "l2_done", "processed", "window", "busy_warps_block0")


def sssp_solve_sampled(h, src: int, dist_out, pred_out=None, cfg=None, cap: int = 4096, period_us: int = 20):
    """sssp_solve plus its run-time timeline: a numpy uint64 array [samples, 6]
    with the columns of SAMPLE_FIELDS."""
    import numpy as np
    out = np.zeros((cap, len(SAMPLE_FIELDS)), np.uint64)
    n = ctypes.c_int32()
    _check(lib().sssp_solve_sampled(h, int(src), _ptr(dist_out), _ptr(pred_out),
                                    None if cfg is None else ctypes.byref(cfg), out.ctypes.data, int(cap),
                                    int(period_us), ctypes.byref(n)), "sssp_solve_sampled")
    return out[:n.value]


def sssp_solve_noalloc(row_ptr, arcs, n: int, m: int, wtype: int, src: int, dist_out, pred_out=None,
                       stream=None) -> None:
    """Single-source solve with no allocation (all arrays device memory; `arcs`
    holds (column, weight bits) uint32 pairs)."""
    _check(lib().sssp_solve_noalloc(_ptr(row_ptr), _ptr(arcs), int(n), int(m), int(wtype), int(src),
                                    _ptr(dist_out), _ptr(pred_out), _stream_ptr(stream)), "sssp_solve_noalloc")


def sssp_serve_options_default() -> sssp_serve_options:
    o = sssp_serve_options()
    _check(lib().sssp_serve_options_default(ctypes.byref(o)), "sssp_serve_options_default")
    return o


def sssp_serve_create(opt: sssp_serve_options | None = None, **kw):
    """Starts a server; `opt` (or keyword overrides of the defaults) as in
    sssp_serve_options."""
    if opt is None:
        opt = sssp_serve_options_default()
    for k, v in kw.items():
        setattr(opt, k, v)
    h = ctypes.c_void_p()
    _check(lib().sssp_serve_create(ctypes.byref(opt), ctypes.byref(h)), "sssp_serve_create")
    return h


def sssp_serve_submit(s, g, src: int, dist_out, pred_out=None) -> int:
    t = ctypes.c_uint64()
    _check(lib().sssp_serve_submit(s, g, int(src), _ptr(dist_out), _ptr(pred_out), ctypes.byref(t)),
           "sssp_serve_submit")
    return t.value


def sssp_serve_poll(s, ticket: int) -> tuple[int, int]:
    st, code = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sssp_serve_poll(s, ticket, ctypes.byref(st), ctypes.byref(code)), "sssp_serve_poll")
    return st.value, code.value


def sssp_serve_wait(s, ticket: int, timeout_ms: int = 60000) -> tuple[int, int]:
    st, code = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().sssp_serve_wait(s, ticket, timeout_ms, ctypes.byref(st), ctypes.byref(code)),
           "sssp_serve_wait")
    return st.value, code.value


def sssp_serve_latency_us(s, ticket: int) -> float:
    v = ctypes.c_double()
    _check(lib().sssp_serve_latency_us(s, ticket, ctypes.byref(v)), "sssp_serve_latency_us")
    return v.value


def sssp_serve_cancel(s, ticket: int) -> int:
    """Returns the status code (SSSP_OK, SSSP_E_BUSY or SSSP_E_INVAL) without raising."""
    return lib().sssp_serve_cancel(s, ticket)


def sssp_serve_release(s, ticket: int) -> None:
    _check(lib().sssp_serve_release(s, ticket), "sssp_serve_release")


def sssp_serve_get_stats(s) -> dict:
    st = sssp_serve_stats()
    _check(lib().sssp_serve_get_stats(s, ctypes.byref(st)), "sssp_serve_get_stats")
    return st.as_dict()


def sssp_serve_destroy(s) -> None:
    _check(lib().sssp_serve_destroy(s), "sssp_serve_destroy")


class Graph:
    """Owning wrapper of an sssp_graph handle."""

    def __init__(self, row_ptr, col_idx, weights, wtype: int | str):
        if isinstance(wtype, str):
            wtype = SSSP_W_F32 if wtype == "f32" else SSSP_W_U32
        n = int((row_ptr.numel() if hasattr(row_ptr, "numel") else row_ptr.size) - 1)
        m = int(col_idx.numel() if hasattr(col_idx, "numel") else col_idx.size)
        self.n, self.m, self.wtype = n, m, wtype
        self.handle = sssp_graph_create(row_ptr, col_idx, weights, n, m, wtype)

    def close(self):
        if self.handle is not None and self.handle.value:
            sssp_graph_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def features(self) -> dict:
        return sssp_graph_features(self.handle).as_dict()

    def solve(self, src, dist_out, pred_out=None, cfg=None, stream=None):
        sssp_solve(self.handle, src, dist_out, pred_out, cfg, stream)

    def bfs(self, src, level_out, pred_out=None, cfg=None, stream=None):
        sssp_bfs(self.handle, src, level_out, pred_out, cfg, stream)

    def solve_batch(self, srcs, dist_out, pred_out=None, cfg=None, stream=None):
        sssp_solve_batch(self.handle, srcs, dist_out, pred_out, cfg, stream)

    def stats(self) -> dict:
        return sssp_last_stats(self.handle).as_dict()

    def autotune(self, srcs=None, budget_ms: int = 0) -> sssp_config:
        return sssp_autotune(self.handle, srcs, budget_ms)

    def autotune_batch(self, srcs, budget_ms: int = 0) -> sssp_config:
        return sssp_autotune_batch(self.handle, srcs, budget_ms)
