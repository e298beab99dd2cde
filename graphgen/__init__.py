"""Seeded synthetic graph inputs shared by the CUDA path and the oracle.

This module only builds inputs (CSR arrays, weights, source lists, arrival
times).  It contains no shortest-path arithmetic.  The C core
(``graphgen.c``) draws every random number from SplitMix64 (Steele, Lea &
Flood 2014) as a pure function of (seed, stream, counter), so the same seed
gives the same graph on x86 and Arm and for any thread count.

The workload recipes stand in for the paper's datasets (Table 4: road
networks, meshes/circuits, power-law graphs), which are not available here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libgraphgen.so with gcc (OpenMP when available)."""
    src = os.path.join(_HERE, "graphgen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    base = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", src, "-o", _SO]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True)
    return _SO


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_SO)
    P = ctypes.c_void_p
    lib.gg_grid.restype = P
    lib.gg_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32,
                            ctypes.c_uint64, ctypes.c_int]
    lib.gg_road.restype = P
    lib.gg_road.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                            ctypes.c_int32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                            ctypes.c_uint64]
    lib.gg_rmat.restype = P
    lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                            ctypes.c_int]
    lib.gg_er.restype = P
    lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32,
                          ctypes.c_uint64, ctypes.c_int]
    lib.gg_random_directed.restype = P
    lib.gg_random_directed.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int]
    lib.gg_n.restype = ctypes.c_int32
    lib.gg_n.argtypes = [P]
    lib.gg_m.restype = ctypes.c_int64
    lib.gg_m.argtypes = [P]
    lib.gg_copy_out.restype = ctypes.c_int
    lib.gg_copy_out.argtypes = [P, P, P, P]
    lib.gg_free.restype = None
    lib.gg_free.argtypes = [P]
    lib.gg_giant_sources.restype = ctypes.c_int32
    lib.gg_giant_sources.argtypes = [P, P, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, P, P]
    lib.gg_uniform_f64.restype = ctypes.c_int
    lib.gg_uniform_f64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64,
                                   ctypes.c_int64, P]
    _lib = lib
    return lib


@dataclass
class Graph:
    """CSR graph: row_ptr int32[n+1], col int32[m], w uint32[m] or float32[m]."""
    name: str
    n: int
    m: int
    row_ptr: np.ndarray
    col: np.ndarray
    w: np.ndarray
    wtype: str  # "u32" or "f32"

    @property
    def w_bits(self) -> np.ndarray:
        return self.w.view(np.uint32)


def _take(h, name: str, wtype: str) -> Graph:
    lib = _load()
    if not h:
        raise MemoryError(f"graph generation failed: {name}")
    try:
        n, m = lib.gg_n(h), lib.gg_m(h)
        row_ptr = np.empty(n + 1, np.int32)
        col = np.empty(max(m, 1), np.int32)
        w = np.empty(max(m, 1), np.uint32)
        lib.gg_copy_out(h, row_ptr.ctypes.data, col.ctypes.data, w.ctypes.data)
    finally:
        lib.gg_free(h)
    col, w = col[:m], w[:m]
    if wtype == "f32":
        w = w.view(np.float32)
    return Graph(name, n, m, row_ptr, col, w, wtype)


def grid(W: int, H: int, lo: int = 1, hi: int = 100, seed: int = 1, wtype: str = "u32") -> Graph:
    """W x H 4-neighbour grid, both directions stored; vertex id = y*W + x."""
    h = _load().gg_grid(W, H, lo, hi, seed, int(wtype == "f32"))
    return _take(h, f"grid{W}x{H}", wtype)


def road(W: int, H: int, pdrop: float = 0.05, plong: float = 0.005, maxlen: int = 64,
         lo: int = 1, hi: int = 1000, longmul: int = 20, seed: int = 1) -> Graph:
    """Road-network-shaped high-diameter graph (u32 weights)."""
    h = _load().gg_road(W, H, pdrop, plong, maxlen, lo, hi, longmul, seed)
    return _take(h, f"road{W}x{H}", "u32")


def rmat(scale: int, ef: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         lo: int = 1, hi: int = 255, seed: int = 1, wtype: str = "u32") -> Graph:
    """Symmetrised R-MAT graph, self-loops and duplicates removed."""
    h = _load().gg_rmat(scale, ef, a, b, c, lo, hi, seed, int(wtype == "f32"))
    return _take(h, f"rmat{scale}", wtype)


def erdos_renyi(n: int, m: int, lo: int = 1, hi: int = 1, seed: int = 1, wtype: str = "f32") -> Graph:
    """G(n, m) with exactly m distinct undirected pairs, stored both ways."""
    h = _load().gg_er(n, m, lo, hi, seed, int(wtype == "f32"))
    return _take(h, f"er{n}_{m}", wtype)


def random_directed(n: int, m: int, lo: int = 1, hi: int = 100, seed: int = 1,
                    wtype: str = "u32") -> Graph:
    """Random directed multigraph (self-loops and parallel arcs allowed)."""
    h = _load().gg_random_directed(n, m, lo, hi, seed, int(wtype == "f32"))
    return _take(h, f"randdir{n}_{m}", wtype)


def from_edges(n: int, edges, wtype: str = "u32", name: str = "edges") -> Graph:
    """CSR from an explicit arc list [(u, v, w), ...] (kept in given order per row)."""
    edges = list(edges)
    deg = np.zeros(n + 1, np.int64)
    for u, _, _ in edges:
        deg[u + 1] += 1
    row_ptr = np.cumsum(deg).astype(np.int32)
    col = np.empty(len(edges), np.int32)
    w = np.empty(len(edges), np.float32 if wtype == "f32" else np.uint32)
    fill = row_ptr[:-1].astype(np.int64).copy()
    for u, v, wt in edges:
        col[fill[u]] = v
        w[fill[u]] = wt
        fill[u] += 1
    return Graph(name, n, len(edges), row_ptr, col, w, wtype)


def giant_sources(g: Graph, k: int, seed: int = 2) -> tuple[np.ndarray, int]:
    """k distinct seeded sources from the largest weakly connected component."""
    out = np.empty(max(k, 1), np.int32)
    gs = np.zeros(1, np.int32)
    got = _load().gg_giant_sources(g.row_ptr.ctypes.data, g.col.ctypes.data, g.n, k, seed,
                                   out.ctypes.data, gs.ctypes.data)
    if got < 0:
        raise RuntimeError("giant_sources failed")
    return out[:got].copy(), int(gs[0])


def uniform_stream(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """count seeded uniforms in [0, 1) (SplitMix64 counter stream)."""
    out = np.empty(max(count, 1), np.float64)
    _load().gg_uniform_f64(seed, stream, start, count, out.ctypes.data)
    return out[:count]


def poisson_arrivals(rate_qps: float, count: int, seed: int = 3, stream: int = 8) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process: cumulative exponential gaps."""
    u = uniform_stream(seed, stream, count)
    gaps = -np.log1p(-u) / rate_qps
    return np.cumsum(gaps)


# Workload recipes (graph seed 1, sources seed 2, arrivals seed 3).
def workload(name: str) -> Graph:
    if name == "grid256":
        return grid(256, 256, 1, 100, seed=1)
    if name == "rmat22":
        return rmat(22, 16, lo=1, hi=255, seed=1)
    if name == "road4096":
        return road(4096, 4096, 0.05, 0.005, 64, 1, 1000, 20, seed=1)
    if name == "rmat20":
        return rmat(20, 16, lo=1, hi=255, seed=1)
    if name == "rmat20f":
        return rmat(20, 16, seed=1, wtype="f32")
    if name == "grid1024":
        return grid(1024, 1024, 1, 100, seed=1)
    if name == "rmat18":
        return rmat(18, 16, lo=1, hi=255, seed=1)
    if name == "er21":
        return erdos_renyi(1 << 21, 1 << 25, seed=1, wtype="f32")
    raise KeyError(name)
