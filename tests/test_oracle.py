"""Pins for the CPU oracle (no GPU).

The oracle is checked against things other than itself: hand-worked
fixtures (tests/golden), closed forms, brute-force enumeration of simple
paths, SciPy's independent shortest-path routines, and the invariant
checker's ability to reject corrupted results.
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle
from golden_io import all_cases

U32_INF = 0xFFFFFFFF
U32_SAT = 0xFFFFFFFE


# ------------------------------------------------------------ fixtures --

@pytest.mark.parametrize("case", all_cases(), ids=lambda c: c["name"])
def test_golden_dist_and_pred(case):
    rp, col, src = case["row_ptr"], case["col"], case["src"]
    if case["kind"] == "u32":
        w = case["w_bits"]
        d = oracle.dijkstra_u32(rp, col, w, src)
        np.testing.assert_array_equal(d, case["dist_bits"])
        np.testing.assert_array_equal(oracle.bellman_ford_u32(rp, col, w, src), case["dist_bits"])
        if case["pred"] is not None:
            p = oracle.pred_canonical_u32(rp, col, w, src, d)
            np.testing.assert_array_equal(p, case["pred"])
            assert oracle.check(rp, col, w, src, d, p, "u32")[0] == "ok"
    else:
        w = case["w_bits"].view(np.float32)
        d = oracle.dijkstra_f32(rp, col, w, src)
        np.testing.assert_array_equal(d.view(np.uint32), case["dist_bits"])
        np.testing.assert_array_equal(oracle.bellman_ford_f32(rp, col, w, src).view(np.uint32),
                                      case["dist_bits"])
        assert oracle.check(rp, col, w, src, d, None, "f32")[0] == "ok"


# -------------------------------------------------------- closed forms --

@pytest.mark.parametrize("W,H", [(1, 1), (1, 7), (9, 1), (13, 11), (64, 40)])
def test_unit_grid_is_manhattan(W, H):
    g = gg.grid(W, H, 1, 1, seed=5)
    rng = np.random.default_rng(W * 100 + H)
    ys, xs = np.divmod(np.arange(W * H), W)
    for src in rng.integers(0, W * H, size=3):
        d = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, int(src))
        sy, sx = divmod(int(src), W)
        np.testing.assert_array_equal(d, np.abs(xs - sx) + np.abs(ys - sy))


def test_unit_weights_are_bfs_levels():
    """Unit weights reduce SSSP to BFS hop counts (the paper's BFS case study)."""
    g = gg.rmat(10, 8, lo=1, hi=1, seed=3)
    src = int(gg.giant_sources(g, 1, seed=4)[0][0])
    d = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, src)
    level = np.full(g.n, -1, np.int64)
    level[src] = 0
    frontier = [src]
    while frontier:
        nxt = []
        for u in frontier:
            for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
                if level[v] < 0:
                    level[v] = level[u] + 1
                    nxt.append(int(v))
        frontier = nxt
    expect = np.where(level < 0, U32_INF, level).astype(np.uint32)
    np.testing.assert_array_equal(d, expect)


def test_weighted_path_prefix_sums():
    rng = np.random.default_rng(7)
    n = 300
    w = rng.integers(0, 1000, size=n - 1).astype(np.uint32)
    g = gg.from_edges(n, [(i, i + 1, int(w[i])) for i in range(n - 1)])
    d = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, 0)
    np.testing.assert_array_equal(d, np.concatenate([[0], np.cumsum(w)]).astype(np.uint32))
    # from the middle: everything before is unreachable on a directed path
    d = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, 150)
    assert (d[:150] == U32_INF).all() and d[150] == 0


def test_saturating_chain():
    big = 0x7FFFFFFF
    g = gg.from_edges(5, [(0, 1, big), (1, 2, big), (2, 3, big), (3, 4, 0)])
    d = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, 0)
    np.testing.assert_array_equal(d, [0, big, 2 * big, U32_SAT, U32_SAT])


# ---------------------------------------------------- brute force paths --

def _simple_path_min(n, arcs, src, add, inf):
    """Minimum over all simple paths src -> v of the left-to-right fold."""
    adj = [[] for _ in range(n)]
    for u, v, w in arcs:
        adj[u].append((v, w))
    best = [inf] * n
    best[src] = add.zero

    def dfs(u, acc, seen):
        for v, w in adj[u]:
            if v in seen:
                continue
            nd = add(acc, w)
            if add.less(nd, best[v]):
                best[v] = nd
            dfs(v, nd, seen | {v})

    dfs(src, add.zero, {src})
    return best


class _U32Add:
    zero = 0

    def __call__(self, a, w):
        return min(a + w, U32_SAT)

    @staticmethod
    def less(a, b):
        return a < b


class _F32Add:
    zero = np.float32(0)

    def __call__(self, a, w):
        return np.float32(np.float32(a) + np.float32(w))

    @staticmethod
    def less(a, b):
        return a < b


@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_u32(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 8))
    m = int(rng.integers(0, 16))
    arcs = [(int(rng.integers(n)), int(rng.integers(n)), int(rng.integers(0, 20))) for _ in range(m)]
    g = gg.from_edges(n, arcs)
    src = int(rng.integers(n))
    expect = _simple_path_min(n, arcs, src, _U32Add(), U32_INF)
    np.testing.assert_array_equal(oracle.dijkstra_u32(g.row_ptr, g.col, g.w, src),
                                  np.array(expect, np.uint32))


@pytest.mark.parametrize("seed", range(40))
def test_bruteforce_f32_left_fold(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(1, 8))
    m = int(rng.integers(0, 16))
    # weights with many significant bits so that rounding matters
    arcs = [(int(rng.integers(n)), int(rng.integers(n)),
             np.float32(rng.uniform(1e-8, 1.0))) for _ in range(m)]
    g = gg.from_edges(n, arcs, wtype="f32")
    src = int(rng.integers(n))
    expect = _simple_path_min(n, arcs, src, _F32Add(), np.float32(np.inf))
    got = oracle.dijkstra_f32(g.row_ptr, g.col, g.w, src)
    np.testing.assert_array_equal(got.view(np.uint32), np.array(expect, np.float32).view(np.uint32))


# ----------------------------------------------------------- scipy pin --

def _scipy_dist(g, src):
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    # collapse parallel arcs to their minimum weight (scipy would sum them)
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    key = rows.astype(np.int64) * g.n + g.col
    order = np.lexsort((g.w.astype(np.float64), key))
    key, w = key[order], g.w.astype(np.float64)[order]
    first = np.ones(key.size, bool)
    first[1:] = key[1:] != key[:-1]
    key, w = key[first], w[first]
    mat = sp.csr_matrix((w, (key // g.n, key % g.n)), shape=(g.n, g.n))
    return csgraph.dijkstra(mat, directed=True, indices=src)


@pytest.mark.parametrize("seed", range(12))
def test_scipy_dijkstra_u32(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(2, 400))
    g = gg.random_directed(n, int(rng.integers(0, 6 * n)), lo=1, hi=1000, seed=seed)
    src = int(rng.integers(n))
    ref = _scipy_dist(g, src)
    got = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, src)
    expect = np.where(np.isinf(ref), U32_INF, ref).astype(np.uint64)
    np.testing.assert_array_equal(got.astype(np.uint64), expect)


@pytest.mark.parametrize("seed", range(6))
def test_scipy_dijkstra_f64(seed):
    g = gg.random_directed(500, 4000, seed=100 + seed, wtype="f32")
    ref = _scipy_dist(g, seed)
    got = oracle.dijkstra_f64(g.row_ptr, g.col, g.w, seed)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    assert (np.isinf(got) == np.isinf(ref)).all()


def test_scipy_on_generated_families():
    for g in (gg.grid(31, 17, 1, 100, seed=2), gg.road(40, 30, seed=2), gg.rmat(11, 8, seed=2)):
        src = int(gg.giant_sources(g, 1)[0][0])
        ref = _scipy_dist(g, src)
        got = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, src)
        np.testing.assert_array_equal(got.astype(np.float64), np.where(np.isinf(ref), U32_INF, ref))


# ------------------------------------------------- two algorithms agree --

@pytest.mark.parametrize("seed", range(20))
def test_bellman_ford_equals_dijkstra(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 120))
    wt = "f32" if seed % 2 else "u32"
    g = gg.random_directed(n, int(rng.integers(0, 5 * n)), lo=0, hi=50, seed=seed, wtype=wt)
    src = int(rng.integers(n))
    if wt == "u32":
        a = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, src)
        b = oracle.bellman_ford_u32(g.row_ptr, g.col, g.w, src)
    else:
        a = oracle.dijkstra_f32(g.row_ptr, g.col, g.w, src).view(np.uint32)
        b = oracle.bellman_ford_f32(g.row_ptr, g.col, g.w, src).view(np.uint32)
    np.testing.assert_array_equal(a, b)


def test_f32_close_to_f64():
    g = gg.erdos_renyi(1 << 12, 1 << 15, seed=9)
    d32 = oracle.dijkstra_f32(g.row_ptr, g.col, g.w, 0).astype(np.float64)
    d64 = oracle.dijkstra_f64(g.row_ptr, g.col, g.w, 0)
    fin = np.isfinite(d64)
    assert (np.isfinite(d32) == fin).all()
    rel = np.abs(d32[fin] - d64[fin]) / np.maximum(d64[fin], 1e-30)
    assert rel.max() <= 1e-6


# ---------------------------------------------------------- invariants --

def _solved(seed=0):
    g = gg.rmat(9, 8, lo=1, hi=30, seed=seed)
    src = int(gg.giant_sources(g, 1)[0][0])
    d = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, src)
    p = oracle.pred_canonical_u32(g.row_ptr, g.col, g.w, src, d)
    return g, src, d, p


def test_check_accepts_and_pred_is_canonical_tree():
    g, src, d, p = _solved()
    assert oracle.check(g.row_ptr, g.col, g.w, src, d, p) == ("ok", -1)
    reach = d != U32_INF
    assert (p[~reach] == -1).all() and p[src] == src
    # following pred from any reachable vertex reaches src with strictly decreasing dist
    for v in np.flatnonzero(reach)[:200]:
        x, steps = int(v), 0
        while x != src:
            assert d[p[x]] < d[x]
            x = int(p[x])
            steps += 1
            assert steps <= g.n


def test_check_rejects_corruptions():
    g, src, d, p = _solved(1)
    reach = np.flatnonzero((d != U32_INF) & (np.arange(g.n) != src))
    v = int(reach[len(reach) // 2])
    bad = d.copy(); bad[v] += 1                  # too long: no tight in-arc
    assert oracle.check(g.row_ptr, g.col, g.w, src, bad)[0] in ("no-tight-in-arc", "edge-violation")
    bad = d.copy(); bad[v] -= 1                  # too short
    assert oracle.check(g.row_ptr, g.col, g.w, src, bad)[0] in ("no-tight-in-arc", "edge-violation")
    bad = d.copy(); bad[src] = 1
    assert oracle.check(g.row_ptr, g.col, g.w, src, bad)[0] == "source"
    bad = d.copy(); bad[v] = U32_INF             # reachable vertex marked unreachable
    assert oracle.check(g.row_ptr, g.col, g.w, src, bad)[0] == "edge-violation"
    bp = p.copy(); bp[v] = v                     # self-loop predecessor
    assert oracle.check(g.row_ptr, g.col, g.w, src, d, bp)[0] in ("pred-not-tight", "pred-cycle")
    bp = p.copy(); bp[v] = -1
    assert oracle.check(g.row_ptr, g.col, g.w, src, d, bp)[0] == "pred-range"


def test_check_rejects_pred_cycle_on_zero_weights():
    # 0 -> 1 (w 0), 1 <-> 2 (w 0): dist all 0; pred 1->2, 2->1 is a tight cycle
    g = gg.from_edges(3, [(0, 1, 0), (1, 2, 0), (2, 1, 0)])
    d = np.zeros(3, np.uint32)
    assert oracle.check(g.row_ptr, g.col, g.w, 0, d, np.array([0, 2, 1], np.int32))[0] == "pred-cycle"
    assert oracle.check(g.row_ptr, g.col, g.w, 0, d, np.array([0, 0, 1], np.int32))[0] == "ok"


def test_reached_counts():
    g = gg.from_edges(4, [(0, 1, 1), (1, 2, 1), (3, 0, 1), (3, 2, 1)])
    d = oracle.dijkstra_u32(g.row_ptr, g.col, g.w, 0)
    assert oracle.reached_counts(g.row_ptr, d) == (2, 3)
