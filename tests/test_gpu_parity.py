"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

u32 distances must be bit-exact; u32 predecessors (all weights >= 1) must
equal the canonical smallest-index tight in-neighbour; f32 distances must be
bit-exact against the f32 Dijkstra and within 1e-6 relative of the f64 one;
other predecessors are checked by the invariants (tight arc, chains reach
the source).
"""
import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2602_10080_gb300 as S
from golden_io import all_cases
from gpu_util import assert_exact, assert_exact_many, cfg, gpu_batch, gpu_solve, oracle_dist, upload

pytestmark = pytest.mark.gpu

L1_ALL = [S.L1_VECTOR, S.L1_NEARFAR, S.L1_FILTER, S.L1_SLF]


@pytest.fixture(scope="module", autouse=True)
def _built():
    S.build()
    S.lib()


def _golden_graph(case):
    w = case["w_bits"]
    g = gg.Graph(case["name"], case["n"], len(case["col"]), case["row_ptr"], case["col"],
                 w.view(np.float32) if case["kind"] == "f32" else w, case["kind"])
    return g


@pytest.mark.parametrize("case", all_cases(), ids=lambda c: c["name"])
@pytest.mark.parametrize("host", [False, True])
def test_golden_fixtures(case, host):
    g = _golden_graph(case)
    G = upload(g, device_inputs=not host)
    d, p = gpu_solve(G, case["src"], pred=True, host=host)
    np.testing.assert_array_equal(d, case["dist_bits"])
    if case["pred"] is not None and g.wtype == "u32" and int(g.w.min()) >= 1:
        np.testing.assert_array_equal(p, case["pred"])
    assert_exact(g, case["src"], d, p)


@pytest.mark.parametrize("l1", L1_ALL)
@pytest.mark.parametrize("l2", [S.L2_VECTOR, S.L2_BUCKET])
def test_grid256_all_queue_configs(l1, l2):
    """Config 1 (grid 256x256, u32 [1,100], seed 1, source 0) under every L1 x L2 policy."""
    g = gg.workload("grid256")
    G = upload(g)
    c = cfg(l1_type=l1, l2_type=l2, wb=8 if l1 == S.L1_VECTOR else 0)
    d, p = gpu_solve(G, 0, pred=True, config=c)
    assert_exact(g, 0, d, p)
    d2, _ = gpu_solve(G, 0, pred=False, config=c)
    np.testing.assert_array_equal(d2, d)


def with_hubs(g, hubs, seed):
    """g plus `hubs` extra out-arcs from a few vertices (targets and weights
    from seeded streams, weights within g's range), rows kept in order."""
    if g.n < 2 or hubs == 0:
        return g
    u = gg.uniform_stream(seed, 60, hubs)
    t = gg.uniform_stream(seed, 61, hubs)
    x = gg.uniform_stream(seed, 62, hubs)
    heads = np.array([(seed * 7919 + 104729 * i) % g.n for i in range(3)], np.int64)
    src = heads[np.minimum((u * 3).astype(np.int64), 2)]
    dst = np.minimum((t * g.n).astype(np.int64), g.n - 1)
    if g.wtype == "f32":
        lo, hi = (float(g.w.min()), float(g.w.max())) if g.m else (0.0, 1.0)
        wx = (lo + x * (hi - lo)).astype(np.float32)
    else:
        lo, hi = (int(g.w.min()), int(g.w.max())) if g.m else (1, 100)
        wx = (lo + np.minimum((x * (hi - lo + 1)).astype(np.int64), hi - lo)).astype(np.uint32)
    u0 = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))
    uu = np.concatenate([u0, src])
    order = np.argsort(uu, kind="stable")
    col = np.concatenate([g.col.astype(np.int64), dst])[order].astype(np.int32)
    w = np.concatenate([g.w, wx])[order]
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(uu, minlength=g.n))]).astype(np.int32)
    return gg.Graph(g.name + "+hubs", g.n, len(col), row_ptr, col, w, g.wtype)


@pytest.mark.parametrize("seed", range(24))
def test_random_graphs_stress(seed):
    """Tiny queue capacities force constant spill/refill; a 32-arc hub split
    threshold turns every vertex above 32 arcs (the planted hubs) into
    shadow vertices, with and without their own hub rings.  Claims of up to
    32 chunks go to the block as descriptors (the 256-slot L1 would hold 8),
    and 0-3 front buckets bypass the block staging."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 3000))
    m = int(rng.integers(0, 12 * n))
    wt = "f32" if seed % 3 == 2 else "u32"
    lo = 0 if seed % 4 == 1 else 1
    g = gg.random_directed(n, m, lo=lo, hi=int(rng.integers(1, 1000)), seed=seed, wtype=wt)
    g = with_hubs(g, 0 if seed % 6 == 5 else int(rng.integers(100, 1500)), seed)
    G = upload(g)
    c = cfg(l1_type=L1_ALL[seed % 4], l2_type=seed % 2, l1_cap=256, bmax=int(rng.choice([1, 2, 8, 32])),
            bnum=int(rng.choice([1, 2, 4])), split_arcs=32, hub_bnum=int(rng.choice([0, 1, 2])),
            dedup=int(seed % 2), wb=int(rng.choice([0, 1, 4])), block_threads=int(rng.choice([256, 512, 1024])),
            pending_marks=int(seed % 5 == 0), claim=int(rng.choice([1, 4, 16, 32])),
            direct_buckets=int(rng.choice([0, 1, 2, 3])), shards=int(rng.choice([2, 4, 16])))
    if wt == "u32":
        c.delta_u32 = int(rng.integers(1, 200))
    else:
        c.delta_f32 = float(rng.uniform(0.01, 2.0))
    max_deg = int(np.diff(g.row_ptr).max()) if g.n else 0
    for src in rng.integers(0, n, size=2):
        d, p = gpu_solve(G, src, pred=True, config=c)
        assert_exact(g, src, d, p)
        # the layout is rebuilt for the 32-arc threshold at the first solve
        shadows = G.features()["shadows"]
        assert (shadows > 0) == (max_deg > 32), (shadows, max_deg)
        d2, _ = gpu_solve(G, src, pred=False, config=c)
        np.testing.assert_array_equal(d2, d)
    # back to the graph's own configuration: the layout is rebuilt with its threshold
    d3, p3 = gpu_solve(G, int(src), pred=True)
    assert_exact(g, int(src), d3, p3)
    own = G.autotune(None, 0).split_arcs or 1024
    assert (G.features()["shadows"] > 0) == (max_deg > own)


def test_rmat_f32_exact_and_close_to_f64():
    g = gg.rmat(14, 16, seed=3, wtype="f32")
    G = upload(g)
    srcs, _ = gg.giant_sources(g, 3, seed=2)
    for s in srcs:
        d, p = gpu_solve(G, s, pred=True)
        assert_exact(g, s, d, p)
        d64 = oracle.dijkstra_f64(g.row_ptr, g.col, g.w, int(s))
        df = d.view(np.float32).astype(np.float64)
        fin = np.isfinite(d64)
        assert (np.isfinite(df) == fin).all()
        rel = np.abs(df[fin] - d64[fin]) / np.maximum(d64[fin], 1e-300)
        assert rel.max() <= 1e-6


def test_heavy_vertex_shadows():
    """Hubs (degree 200k and 3000) are split into shadow vertices at creation;
    their arcs are relaxed by many warps through the ordinary queues."""
    n = 200_001
    edges = [(0, v, (v * 7919) % 1000 + 1) for v in range(1, n)]
    edges += [(v, v + 1, 3) for v in range(1, n - 1)]
    edges += [(777, v, 1 + v % 13) for v in range(1000, 4000)]
    g = gg.from_edges(n, edges)
    G = upload(g)
    # every vertex above the graph's split threshold becomes ceil(arcs / threshold) shadows
    split = G.autotune(None, 0).split_arcs or 1024
    deg = np.diff(g.row_ptr)
    assert G.features()["shadows"] == int(sum(-(-d // split) for d in deg if d > split))
    assert G.features()["shadows"] >= 199
    for src in (0, 777, 5):
        for ma in (32, 4096):
            d, p = gpu_solve(G, src, pred=True, config=cfg(max_arcs=ma))
            assert_exact(g, src, d, p)
            d2, _ = gpu_solve(G, src, pred=False, config=cfg(max_arcs=ma, near_deltas=0.0))
            np.testing.assert_array_equal(d2, d)
        # hub slices in their own rings, read only near the front
        for hb in (1, 2):
            d3, p3 = gpu_solve(G, src, pred=True, config=cfg(hub_bnum=hb))
            assert_exact(g, src, d3, p3)
    # batch on the split layout (query slices are padded with shadow vertices)
    db, pb = gpu_batch(G, np.array([0, 777, 5, 0], np.int32), pred=True)
    for q, s in enumerate([0, 777, 5, 0]):
        assert_exact(g, s, db[q], pb[q])


@pytest.mark.parametrize("wt", ["u32", "f32"])
@pytest.mark.parametrize("pred", [False, True])
def test_batch_equals_single(wt, pred):
    g = gg.rmat(13, 16, seed=5, wtype=wt)
    G = upload(g)
    srcs, _ = gg.giant_sources(g, 40, seed=2)
    srcs = np.concatenate([srcs, srcs[:3]])  # repeated sources are independent queries
    d, p = gpu_batch(G, srcs, pred=pred)
    for q, s in enumerate(srcs):
        assert_exact(g, s, d[q], p[q] if pred else None)


def test_batch_host_buffers_and_tiny_capacity():
    g = gg.grid(64, 48, 1, 100, seed=7)
    G = upload(g, device_inputs=False)
    srcs = np.array([0, 5, 3071, 100, 2000], np.int32)
    d, p = gpu_batch(G, srcs, pred=True, host=True, config=cfg(l1_cap=256, bmax=4, bnum=2))
    for q, s in enumerate(srcs):
        assert_exact(g, s, d[q], p[q])


def test_edge_cases():
    # a single vertex, no arcs
    g = gg.from_edges(1, [])
    G = upload(g)
    d, p = gpu_solve(G, 0)
    assert d.tolist() == [0] and p.tolist() == [0]
    # source without out-arcs
    g = gg.from_edges(4, [(1, 2, 5), (2, 3, 1)])
    G = upload(g)
    d, p = gpu_solve(G, 0)
    assert d.tolist() == [0, 0xFFFFFFFF, 0xFFFFFFFF, 0xFFFFFFFF] and p.tolist() == [0, -1, -1, -1]
    # f32 -0.0 weight reads as +0.0
    g = gg.from_edges(2, [(0, 1, np.float32(-0.0))], wtype="f32")
    G = upload(g)
    d, _ = gpu_solve(G, 0, pred=False)
    assert d.tolist() == [0, 0]


def test_invalid_inputs():
    lib = S.lib()
    import ctypes
    h = ctypes.c_void_p()
    rp = np.array([0, 1, 2], np.int32)
    col_bad = np.array([1, 7], np.int32)
    w = np.array([1, 1], np.uint32)
    assert lib.sssp_graph_create(rp.ctypes.data, col_bad.ctypes.data, w.ctypes.data, 2, 2, 0,
                                 ctypes.byref(h)) == S.SSSP_E_BADGRAPH
    rp_bad = np.array([0, 2, 1], np.int32)
    col = np.array([1, 0], np.int32)
    assert lib.sssp_graph_create(rp_bad.ctypes.data, col.ctypes.data, w.ctypes.data, 2, 2, 0,
                                 ctypes.byref(h)) == S.SSSP_E_BADGRAPH
    for bad in (np.nan, -1.0, np.inf):
        wf = np.array([1.0, bad], np.float32)
        assert lib.sssp_graph_create(rp.ctypes.data, col.ctypes.data, wf.ctypes.data, 2, 2, 1,
                                     ctypes.byref(h)) == S.SSSP_E_BADGRAPH
    G = S.Graph(rp, col, w, "u32")
    d = torch.empty(2, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SsspError) as ei:
        G.solve(2, d)
    assert ei.value.code == S.SSSP_E_INVAL
    with pytest.raises(S.SsspError) as ei:
        G.solve(0, d, cfg=cfg(l1_cap=300))
    assert ei.value.code == S.SSSP_E_INVAL
    for bad in (dict(claim=0), dict(claim=33), dict(direct_buckets=-1), dict(direct_buckets=33),
                dict(shards=3), dict(block_threads=768)):
        with pytest.raises(S.SsspError) as ei:
            G.solve(0, d, cfg=cfg(**bad))
        assert ei.value.code == S.SSSP_E_INVAL, bad
    G.solve(0, d, cfg=cfg(claim=32, direct_buckets=32))   # the bounds themselves are valid


def test_watchdog_timeout_then_recovers():
    """A 1 ms watchdog on a long solve returns SSSP_E_TIMEOUT; the handle stays usable."""
    g = gg.grid(1024, 1024, 1, 100, seed=11)
    G = upload(g)
    c = cfg(timeout_ms=1, l2_type=S.L2_VECTOR)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    with pytest.raises(S.SsspError) as ei:
        G.solve(0, d, None, c)
    assert ei.value.code == S.SSSP_E_TIMEOUT
    d2, p2 = gpu_solve(G, 0, pred=True)
    assert_exact(g, 0, d2, p2)


def test_autotune_prior_and_search():
    g = gg.rmat(13, 16, seed=9)
    G = upload(g)
    prior = G.autotune(None, 0)
    assert prior.delta_u32 >= 1
    srcs = torch.from_numpy(gg.giant_sources(g, 2, seed=2)[0]).cuda()
    tuned = G.autotune(srcs, 1500)
    assert S.sssp_graph_features(G.handle).n == g.n
    s = int(srcs[0])
    d, p = gpu_solve(G, s, pred=True)  # cfg=None uses the tuned configuration
    assert_exact(g, s, d, p)
    d, p = gpu_solve(G, s, pred=True, config=tuned)
    assert_exact(g, s, d, p)


def test_autotune_batch_exact():
    """A multi-query configuration tuned on whole batch launches is cached on
    the graph for its size class; a later batch with cfg=None uses it and
    stays exact, with and without predecessors."""
    g = gg.rmat(14, 16, seed=12)
    G = upload(g)
    srcs, _ = gg.giant_sources(g, 64, seed=2)
    st = torch.from_numpy(srcs.astype(np.int32)).cuda()
    tuned = G.autotune_batch(st, 1500)
    heuristic = S.sssp_autotune_batch(G.handle, srcs.astype(np.int32), 0)   # untimed starting point
    assert tuned.delta_u32 >= 1 and heuristic.delta_u32 >= 1
    tuned = G.autotune_batch(st, 1500)
    d, p = gpu_batch(G, srcs, pred=True)
    assert_exact_many(g, srcs, d, p)
    d2, _ = gpu_batch(G, srcs, pred=False, config=tuned)
    np.testing.assert_array_equal(d2, d)
    G.close()


@pytest.mark.parametrize("l2", [S.L2_BUCKET, S.L2_VECTOR])
def test_single_queue_baselines(l2):
    """The single-queue baselines (every write straight to L2: a bucketed
    delta-stepping queue, or one FIFO) give the same exact results."""
    for g, src in ((gg.workload("grid256"), 0), (gg.rmat(14, 16, lo=1, hi=255, seed=3), None),
                   (gg.random_directed(3000, 20000, 0, 50, seed=9), 5)):
        G = upload(g)
        if src is None:
            src = int(gg.giant_sources(g, 1)[0][0])
        c = cfg(l2_only=1, l2_type=l2)
        d, p = gpu_solve(G, src, config=c)
        assert_exact(g, src, d, p)
        G.close()


def _bfs_reference(g, src):
    """Levels = unit-weight distances (pinned to BFS levels by the oracle
    tests), parents = the canonical smallest-index tight in-neighbour."""
    unit = np.ones(g.m, np.uint32)
    lev = oracle.dijkstra_u32(g.row_ptr, g.col, unit, int(src))
    par = oracle.pred_canonical_u32(g.row_ptr, g.col, unit, int(src), lev)
    return lev, par


@pytest.mark.parametrize("name", ["grid256", "rmat14", "randdir_zero", "rmat14f", "hubs"])
def test_bfs_levels_and_parents(name):
    if name == "grid256":
        g, src = gg.workload("grid256"), 0
    elif name == "rmat14":
        g, src = gg.rmat(14, 16, lo=1, hi=255, seed=5), None
    elif name == "randdir_zero":
        g, src = gg.random_directed(4000, 30000, 0, 20, seed=4), 3
    elif name == "rmat14f":
        g, src = gg.rmat(14, 16, seed=6, wtype="f32"), None
    else:
        # hub vertices are split into shadows in the device layout
        g, src = gg.rmat(16, 32, a=0.65, b=0.15, c=0.15, lo=1, hi=9, seed=2), None
    if src is None:
        src = int(gg.giant_sources(g, 1)[0][0])
    G = upload(g)
    lev_ref, par_ref = _bfs_reference(g, src)
    for host in (False, True):
        if host:
            lev = np.empty(G.n, np.uint32)
            par = np.empty(G.n, np.int32)
            G.bfs(src, lev, par)
        else:
            lt = torch.empty(G.n, dtype=torch.int32, device="cuda")
            pt = torch.empty(G.n, dtype=torch.int32, device="cuda")
            G.bfs(src, lt, pt)
            torch.cuda.synchronize()
            lev, par = lt.cpu().numpy().view(np.uint32), pt.cpu().numpy()
        assert np.array_equal(lev, lev_ref), name
        assert np.array_equal(par, par_ref), name
    G.close()


def test_solve_sampled_timeline():
    """Run-time sampling: same results as sssp_solve, and a timeline whose
    counters move the right way."""
    g = gg.grid(512, 512, 1, 100, seed=3)
    G = upload(g)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    p = torch.empty(g.n, dtype=torch.int32, device="cuda")
    tl = S.sssp_solve_sampled(G.handle, 0, d, p, cap=8192, period_us=10)
    torch.cuda.synchronize()
    assert_exact(g, 0, d.cpu().numpy().view(np.uint32), p.cpu().numpy())
    assert len(tl) >= 3
    t, written, done, processed, window = (tl[:, i].astype(np.int64) for i in range(5))
    assert (np.diff(t) > 0).all()
    assert (np.diff(written) >= 0).all() and (np.diff(processed) >= 0).all() and (np.diff(done) >= 0).all()
    assert (done <= written).all()
    assert processed[-1] > 0 and window.max() > 0
    assert (tl[:, 5] <= 32).all()
    G.close()
