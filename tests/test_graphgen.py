"""Input generator properties (no GPU): sizes, symmetry, weights, seeds."""
import numpy as np
import pytest

import graphgen as gg


def _arcs(g):
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    return rows, g.col.astype(np.int64)


def _assert_simple_symmetric(g):
    r, c = _arcs(g)
    assert (r != c).all(), "self-loop"
    key = r * g.n + c
    assert np.unique(key).size == key.size, "duplicate arc"
    rev = c * g.n + r
    order = np.argsort(key)
    pos = np.searchsorted(key[order], rev)
    assert (key[order][np.minimum(pos, key.size - 1)] == rev).all(), "missing reverse arc"
    # shared weight per undirected edge
    wb = g.w_bits
    np.testing.assert_array_equal(wb[order][pos], wb)
    assert (np.diff(g.row_ptr) >= 0).all() and g.row_ptr[0] == 0 and g.row_ptr[-1] == g.m


def test_grid_shape_and_weights():
    g = gg.grid(256, 256, 1, 100, seed=1)
    assert g.n == 65536 and g.m == 261120
    _assert_simple_symmetric(g)
    assert g.w.min() >= 1 and g.w.max() <= 100
    assert np.unique(g.w).size == 100
    # 4-neighbourhood: every arc joins cells at Manhattan distance 1
    r, c = _arcs(g)
    assert (np.abs(r % 256 - c % 256) + np.abs(r // 256 - c // 256) == 1).all()


def test_seed_reproducible_and_distinct():
    a = gg.grid(64, 32, 1, 100, seed=1)
    b = gg.grid(64, 32, 1, 100, seed=1)
    c = gg.grid(64, 32, 1, 100, seed=2)
    np.testing.assert_array_equal(a.w, b.w)
    assert not np.array_equal(a.w, c.w)
    r1, r2 = gg.rmat(12, seed=5), gg.rmat(12, seed=5)
    np.testing.assert_array_equal(r1.col, r2.col)
    np.testing.assert_array_equal(r1.w, r2.w)


def test_rmat_properties():
    g = gg.rmat(14, 16, seed=1)
    assert g.n == 1 << 14
    assert g.m <= 2 * 16 * (1 << 14)
    _assert_simple_symmetric(g)
    assert g.w.min() >= 1 and g.w.max() <= 255
    deg = np.diff(g.row_ptr)
    assert deg.max() > 20 * deg.mean(), "R-MAT should be heavily skewed"


def test_rmat_f32_weights_exact_grid():
    g = gg.rmat(10, 8, seed=1, wtype="f32")
    k = g.w.astype(np.float64) * (1 << 24)
    assert (g.w > 0).all() and (g.w <= 1).all()
    np.testing.assert_array_equal(k, np.round(k))


def test_road_properties():
    g = gg.road(128, 96, 0.05, 0.005, 64, 1, 1000, 20, seed=1)
    _assert_simple_symmetric(g)
    r, c = _arcs(g)
    man = np.abs(r % 128 - c % 128) + np.abs(r // 128 - c // 128)
    grid_arcs = man == 1
    full = 2 * (2 * 128 * 96 - 128 - 96)
    kept = grid_arcs.sum()
    assert 0.93 * full < kept < 0.97 * full
    assert (g.w[grid_arcs] <= 1000).all() and (g.w[grid_arcs] >= 1).all()
    lr = ~grid_arcs
    assert lr.sum() > 0 and (man[lr] >= 2).all() and (man[lr] <= 64).all()
    np.testing.assert_array_equal(g.w[lr], 20 * man[lr])


def test_er_exact_edge_count():
    g = gg.erdos_renyi(1 << 10, 5000, seed=4)
    assert g.m == 2 * 5000
    _assert_simple_symmetric(g)


def test_giant_sources_in_component():
    g = gg.rmat(12, 4, seed=3)
    src, gsize = gg.giant_sources(g, 16, seed=2)
    assert len(src) == 16 and len(set(src.tolist())) == 16
    # BFS from the first source covers exactly the giant component, which holds all sources
    seen = np.zeros(g.n, bool)
    seen[src[0]] = True
    frontier = [int(src[0])]
    while frontier:
        nxt = []
        for u in frontier:
            for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
                if not seen[v]:
                    seen[v] = True
                    nxt.append(int(v))
        frontier = nxt
    assert seen.sum() == gsize and seen[src].all()


def test_poisson_arrivals():
    t = gg.poisson_arrivals(100.0, 20000, seed=3)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert (gaps > 0).all()
    assert abs(gaps.mean() - 0.01) < 0.0005


@pytest.mark.parametrize("n,m", [(1, 0), (5, 0), (3, 7)])
def test_random_directed_small(n, m):
    g = gg.random_directed(n, m, seed=1)
    assert g.n == n and g.m == m and g.row_ptr[-1] == m
