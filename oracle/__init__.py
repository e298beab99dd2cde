"""CPU oracle for single-source shortest paths -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU product path neither imports
nor links it, and the two share no code.

Functions follow Section 2.1 of the paper (the SSSP problem, Dijkstra's
algorithm and Bellman-Ford as the two classical end points).  The arithmetic
lives in ``sssp_oracle.c``; this module only marshals numpy arrays.

Pins (see ``tests/test_oracle.py``): hand-worked graphs under
``tests/golden/`` (including an instance of the redundant-wavefront example
of Fig. 5), closed forms on unit-weight grids and paths, brute-force path
enumeration on tiny graphs (u32 sums and the f32 left-fold), SciPy's
independent Dijkstra/Bellman-Ford, and the invariant checker.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsssp_oracle.so")
_lib = None

U32_INF = 0xFFFFFFFF
U32_SAT = 0xFFFFFFFE

CHECK_CODES = {
    0: "ok", 1: "source", 2: "edge-violation", 3: "no-tight-in-arc", 4: "pred-range",
    5: "pred-not-tight", 6: "pred-cycle", 7: "bad-args",
}


def build(force: bool = False) -> str:
    """Compile the oracle with strict IEEE single-precision semantics."""
    src = os.path.join(_HERE, "sssp_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                    "-fexcess-precision=standard", "-fno-fast-math", src, "-o", _SO, "-lm"],
                   check=True)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    _lib = _configure(ctypes.CDLL(_SO))
    return _lib


def use_library(path: str):
    """Point this module at another build of sssp_oracle.c (mutation tests)."""
    global _lib
    _lib = _configure(ctypes.CDLL(path))


def _configure(lib):
    P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    for name in ("oracle_dijkstra_u32", "oracle_dijkstra_f32", "oracle_dijkstra_f64"):
        f = getattr(lib, name)
        f.restype = I64
        f.argtypes = [I32, P, P, P, I32, P]
    for name in ("oracle_bellman_ford_u32", "oracle_bellman_ford_f32"):
        f = getattr(lib, name)
        f.restype = I32
        f.argtypes = [I32, P, P, P, I32, P]
    lib.oracle_pred_canonical_u32.restype = ctypes.c_int
    lib.oracle_pred_canonical_u32.argtypes = [I32, P, P, P, I32, P, P]
    lib.oracle_check.restype = ctypes.c_int
    lib.oracle_check.argtypes = [ctypes.c_int, I32, P, P, P, I32, P, P, P]
    lib.oracle_reached_counts.restype = ctypes.c_int
    lib.oracle_reached_counts.argtypes = [ctypes.c_int, I32, P, P, P, P]
    return lib


def _csr(row_ptr, col):
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    if col.size == 0:
        col = np.zeros(1, np.int32)
    return row_ptr, col


def _w(w, dtype):
    w = np.ascontiguousarray(w)
    if w.dtype != dtype:
        w = w.view(dtype) if w.dtype.itemsize == 4 else w.astype(dtype)
    if w.size == 0:
        w = np.zeros(1, dtype)
    return w


def dijkstra_u32(row_ptr, col, w, src: int) -> np.ndarray:
    """Shortest u32 path lengths (saturating at 2^32-2; 0xFFFFFFFF = unreachable)."""
    row_ptr, col = _csr(row_ptr, col)
    w = _w(w, np.uint32)
    n = row_ptr.size - 1
    dist = np.empty(n, np.uint32)
    if _load().oracle_dijkstra_u32(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                                   src, dist.ctypes.data) < 0:
        raise ValueError("oracle_dijkstra_u32 failed")
    return dist


def dijkstra_f32(row_ptr, col, w, src: int) -> np.ndarray:
    """Shortest paths with one rounded f32 add per arc (+inf = unreachable)."""
    row_ptr, col = _csr(row_ptr, col)
    w = _w(w, np.float32)
    n = row_ptr.size - 1
    dist = np.empty(n, np.float32)
    if _load().oracle_dijkstra_f32(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                                   src, dist.ctypes.data) < 0:
        raise ValueError("oracle_dijkstra_f32 failed")
    return dist


def dijkstra_f64(row_ptr, col, w, src: int) -> np.ndarray:
    """Shortest paths in double precision over the (f32) weights."""
    row_ptr, col = _csr(row_ptr, col)
    w = _w(w, np.float32)
    n = row_ptr.size - 1
    dist = np.empty(n, np.float64)
    if _load().oracle_dijkstra_f64(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                                   src, dist.ctypes.data) < 0:
        raise ValueError("oracle_dijkstra_f64 failed")
    return dist


def bellman_ford_u32(row_ptr, col, w, src: int) -> np.ndarray:
    row_ptr, col = _csr(row_ptr, col)
    w = _w(w, np.uint32)
    n = row_ptr.size - 1
    dist = np.empty(n, np.uint32)
    if _load().oracle_bellman_ford_u32(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                                       src, dist.ctypes.data) < 0:
        raise ValueError("oracle_bellman_ford_u32 failed")
    return dist


def bellman_ford_f32(row_ptr, col, w, src: int) -> np.ndarray:
    row_ptr, col = _csr(row_ptr, col)
    w = _w(w, np.float32)
    n = row_ptr.size - 1
    dist = np.empty(n, np.float32)
    if _load().oracle_bellman_ford_f32(n, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                                       src, dist.ctypes.data) < 0:
        raise ValueError("oracle_bellman_ford_f32 failed")
    return dist


def pred_canonical_u32(row_ptr, col, w, src: int, dist) -> np.ndarray:
    """Smallest-index tight in-neighbour for every reachable vertex."""
    row_ptr, col = _csr(row_ptr, col)
    w = _w(w, np.uint32)
    dist = np.ascontiguousarray(dist, np.uint32)
    pred = np.empty(row_ptr.size - 1, np.int32)
    _load().oracle_pred_canonical_u32(row_ptr.size - 1, row_ptr.ctypes.data, col.ctypes.data,
                                      w.ctypes.data, src, dist.ctypes.data, pred.ctypes.data)
    return pred


def check(row_ptr, col, w, src: int, dist, pred=None, kind: str = "u32") -> tuple[str, int]:
    """Invariant check of a claimed result; returns (status, first bad vertex)."""
    row_ptr, col = _csr(row_ptr, col)
    k = 0 if kind == "u32" else 1
    w = _w(w, np.uint32 if k == 0 else np.float32)
    dist = np.ascontiguousarray(dist, np.uint32 if k == 0 else np.float32)
    pp = None
    if pred is not None:
        pred = np.ascontiguousarray(pred, np.int32)
        pp = pred.ctypes.data
    bad = np.zeros(1, np.int32)
    rc = _load().oracle_check(k, row_ptr.size - 1, row_ptr.ctypes.data, col.ctypes.data,
                              w.ctypes.data, src, dist.ctypes.data, pp, bad.ctypes.data)
    return CHECK_CODES.get(rc, str(rc)), int(bad[0])


def reached_counts(row_ptr, dist, kind: str = "u32") -> tuple[int, int]:
    """(m_r, n_r): arcs out of reachable vertices, and reachable vertices."""
    row_ptr = np.ascontiguousarray(row_ptr, np.int32)
    k = 0 if kind == "u32" else 1
    dist = np.ascontiguousarray(dist, np.uint32 if k == 0 else np.float32)
    m_r = np.zeros(1, np.int64)
    n_r = np.zeros(1, np.int64)
    _load().oracle_reached_counts(k, row_ptr.size - 1, row_ptr.ctypes.data, dist.ctypes.data,
                                  m_r.ctypes.data, n_r.ctypes.data)
    return int(m_r[0]), int(n_r[0])


def dijkstra_many(row_ptr, col, w, sources, kind: str = "u32", threads: int = 1):
    """Independent single-source runs, one query per host thread."""
    fn = {"u32": dijkstra_u32, "f32": dijkstra_f32, "f64": dijkstra_f64}[kind]
    if threads <= 1:
        return [fn(row_ptr, col, w, int(s)) for s in sources]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda s: fn(row_ptr, col, w, int(s)), sources))
