"""GPU parity at the full sizes of the five workloads, in the launch
configuration the benchmark times (the graph's prior configuration, 512
threads x resident blocks per SM, predecessors on).

The workloads: grid 256^2 from vertex 0; R-MAT-22 from all 64 benchmark
sources; road 4096^2 from all 16 sources under both the prior and the
autotuned configuration; 256 sources of R-MAT-20 in one launch (u32 with
predecessors, and f32); and the served mix over the resident graphs (grid
1024^2, R-MAT 18/20/22, ER(2^21, 2^25) f32), with and without predecessors.
Every query a test runs is compared with the oracle (the oracle runs spread
over the host cores), and every compared vector is complete: bit-exact u32
distances, canonical u32 predecessors (weights >= 1), f32 distances
bit-exact against the f32 Dijkstra and within 1e-6 relative of f64, and the
tight-arc / reaches-the-source invariants for the other predecessors.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2602_10080_gb300 as S
from gpu_util import assert_exact, assert_exact_many, gpu_batch, gpu_solve, oracle_threads, upload

pytestmark = pytest.mark.gpu

_cache = {}


def workload(name):
    if name not in _cache:
        S.build()
        oracle.build()
        g = gg.workload(name)
        _cache[name] = (g, upload(g))
    return _cache[name]


@pytest.fixture(scope="module", autouse=True)
def _release():
    yield
    for _, G in _cache.values():
        G.close()
    _cache.clear()


def _f64_close(g, src, dist_bits):
    ref = oracle.dijkstra_f64(g.row_ptr, g.col, g.w.astype(np.float64), int(src))
    got = dist_bits.view(np.float32).astype(np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(got), fin)
    rel = np.abs(got[fin] - ref[fin]) / np.maximum(ref[fin], 1e-30)
    assert rel.max(initial=0.0) <= 1e-6, rel.max()


def test_grid256_source0():
    g, G = workload("grid256")
    d, p = gpu_solve(G, 0)
    assert_exact(g, 0, d, p)


def _solve_all(G, srcs, cfg=None):
    """Single-source solves with predecessors for every source (results on the host)."""
    ds, ps = [], []
    for s in srcs:
        d, p = gpu_solve(G, int(s), config=cfg)
        ds.append(d)
        ps.append(p)
    return ds, ps


def test_rmat22_single_source():
    """All 64 benchmark sources, in the benchmark's launch configuration."""
    g, G = workload("rmat22")
    srcs, _ = gg.giant_sources(g, 64, seed=2)
    ds, ps = _solve_all(G, srcs)
    assert_exact_many(g, srcs, ds, ps)


@pytest.mark.parametrize("tuned", [False, True])
def test_road4096(tuned):
    g, G = workload("road4096")
    srcs, _ = gg.giant_sources(g, 16, seed=2)
    cfg = None
    if tuned:
        cfg = G.autotune(torch.from_numpy(srcs[:2].astype(np.int32)).cuda(), 3000)
    ds, ps = _solve_all(G, srcs, cfg)
    assert_exact_many(g, srcs, ds, ps)


def test_rmat20_batch256_u32():
    g, G = workload("rmat20")
    srcs, _ = gg.giant_sources(g, 256, seed=2)
    d, p = gpu_batch(G, srcs, pred=True)
    assert_exact_many(g, srcs, d, p)


def test_rmat20_batch256_f32():
    g, G = workload("rmat20f")
    srcs, _ = gg.giant_sources(g, 256, seed=2)
    d, _ = gpu_batch(G, srcs, pred=False)
    assert_exact_many(g, srcs, d)
    with ThreadPoolExecutor(max_workers=oracle_threads()) as ex:
        list(ex.map(lambda q: _f64_close(g, int(srcs[q]), d[q]), range(len(srcs))))


def test_served_mix_resident_graphs():
    """Six queries per resident graph, submitted together; the odd ones ask
    for predecessors (a second lane per graph)."""
    names = ("grid1024", "rmat18", "rmat20", "rmat22", "er21")
    srv = S.sssp_serve_create()
    try:
        jobs = []
        for name in names:
            g, G = workload(name)
            srcs, _ = gg.giant_sources(g, 4096, seed=2)
            for k, s in enumerate(int(srcs[i]) for i in (5, 900, 17, 2000, 333, 4000)):
                dist = torch.empty(g.n, dtype=torch.int32, device="cuda")
                pred = torch.empty(g.n, dtype=torch.int32, device="cuda") if k % 2 else None
                t = S.sssp_serve_submit(srv, G.handle, s, dist, pred)
                jobs.append((name, s, dist, pred, t))
        for name, s, _, _, t in jobs:
            st, code = S.sssp_serve_wait(srv, t, 600000)
            assert st == S.Q_DONE, (name, s, S.strerror(code))
        stats = S.sssp_serve_get_stats(srv)
    finally:
        S.sssp_serve_destroy(srv)
    assert stats["max_resident"] >= 2
    torch.cuda.synchronize()
    for name in names:
        g, _ = _cache[name]
        mine = [j for j in jobs if j[0] == name]
        srcs = [j[1] for j in mine]
        dists = [j[2].cpu().numpy().view(np.uint32) for j in mine]
        for with_pred in (False, True):
            sel = [i for i, j in enumerate(mine) if (j[3] is not None) == with_pred]
            preds = [mine[i][3].cpu().numpy() for i in sel] if with_pred else None
            assert_exact_many(g, [srcs[i] for i in sel], [dists[i] for i in sel], preds)
        if g.wtype == "f32":
            for s, bits in zip(srcs, dists):
                _f64_close(g, s, bits)
