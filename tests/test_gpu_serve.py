"""Serving with continuous batching, through the C ABI.

Every query's result must be the same alone and in the mix (and equal to
the oracle): u32 distances bit-exact, canonical predecessors for u32
weights >= 1, f32 distances bit-exact against the f32 Dijkstra.  Queries
join lanes whose earlier queries are still running; the recovery paths
(ring migration, restart after an overflow, a timed-out lane, cancellation,
per-query timeouts, admission limits) are driven from the host.
"""
import time

import numpy as np
import pytest
import torch

import graphgen as gg
import paper_2602_10080_gb300 as S
from gpu_util import assert_exact, gpu_solve, oracle_dist, upload

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def graphs():
    S.build()
    S.lib()
    gs = {
        "grid": gg.grid(128, 128, 1, 100, seed=1),
        "rmat": gg.rmat(15, 16, lo=1, hi=255, seed=1),
        "erf": gg.erdos_renyi(1 << 14, 1 << 17, seed=5, wtype="f32"),
        # high diameter: a query spans many slices, so others join it
        "road": gg.road(384, 384, 0.05, 0.005, 32, 1, 1000, 20, seed=1),
    }
    out = {k: (g, upload(g)) for k, g in gs.items()}
    yield out
    for _, G in out.values():
        G.close()


def _bufs(G, pred, host):
    if host:
        return np.full(G.n, 0xABABABAB, np.uint32), (np.full(G.n, -7, np.int32) if pred else None)
    d = torch.full((G.n,), -1, dtype=torch.int32, device="cuda")
    p = torch.full((G.n,), -7, dtype=torch.int32, device="cuda") if pred else None
    return d, p


def _np(x):
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        torch.cuda.synchronize()
        x = x.cpu().numpy()
    return x


def _dist_bits(d):
    return _np(d).view(np.uint32)


def _wait_all(srv, tickets, timeout_ms=120000):
    for t in tickets:
        st, code = S.sssp_serve_wait(srv, t, timeout_ms)
        assert st == S.Q_DONE, (t, st, S.strerror(code))


def _serve_one(G, src, pred, host=False, **opt):
    srv = S.sssp_serve_create(**opt)
    try:
        d, p = _bufs(G, pred, host)
        t = S.sssp_serve_submit(srv, G.handle, int(src), d, p)
        _wait_all(srv, [t])
        return _dist_bits(d).copy(), (None if p is None else _np(p).copy())
    finally:
        S.sssp_serve_destroy(srv)


def test_serve_single_query_matches_solve(graphs):
    for name, (g, G) in graphs.items():
        src = int(gg.giant_sources(g, 1)[0][0])
        d, _ = _serve_one(G, src, pred=False)
        ref, _ = gpu_solve(G, src, pred=False)
        assert np.array_equal(d, ref), name
        assert_exact(g, src, d)


def test_serve_alone_equals_mix(graphs):
    """Each query gives the same answer alone and when it shares its lane
    (and the SMs) with queries admitted before and after it."""
    rng_names = ["road", "grid", "rmat", "erf"]
    queries = []
    for name in rng_names:
        g, _ = graphs[name]
        srcs, _ = gg.giant_sources(g, 6, seed=2)
        for i, s in enumerate(srcs):
            queries.append((name, int(s), i % 2 == 0))   # every other query asks for pred
    # alone: one query per server
    alone = {}
    for name, s, pred in queries:
        g, G = graphs[name]
        alone[(name, s, pred)] = _serve_one(G, s, pred, slice_us=200)
    # the mix: a long road query first, the rest in waves while it runs
    srv = S.sssp_serve_create(slice_us=200)
    try:
        bufs, tickets = {}, []
        order = sorted(queries, key=lambda q: q[0] != "road")
        for k, (name, s, pred) in enumerate(order):
            g, G = graphs[name]
            d, p = _bufs(G, pred, host=False)
            bufs[(name, s, pred)] = (d, p)
            tickets.append(S.sssp_serve_submit(srv, G.handle, s, d, p))
            if k in (0, 3, 9):
                time.sleep(0.004)   # let the running queries make progress
        _wait_all(srv, tickets)
        stats = S.sssp_serve_get_stats(srv)
    finally:
        S.sssp_serve_destroy(srv)
    assert stats["completed"] == len(queries) and stats["failed"] == 0
    assert stats["joined_running"] >= 1, stats   # continuous batching happened
    assert stats["max_resident"] >= 2, stats
    for key, (d, p) in bufs.items():
        name, s, pred = key
        g, _ = graphs[name]
        da, pa = alone[key]
        db = _dist_bits(d)
        assert np.array_equal(db, da), key
        assert_exact(g, s, db, _np(p) if pred else None)
        if pred:
            assert np.array_equal(_np(p), pa), key


def test_serve_host_buffers(graphs):
    g, G = graphs["rmat"]
    srcs, _ = gg.giant_sources(g, 4, seed=2)
    srv = S.sssp_serve_create(slice_us=300)
    try:
        outs, tickets = [], []
        for i, s in enumerate(srcs):
            d, p = _bufs(G, i % 2 == 1, host=True)
            outs.append((int(s), d, p))
            tickets.append(S.sssp_serve_submit(srv, G.handle, int(s), d, p))
        _wait_all(srv, tickets)
        for t in tickets:
            assert S.sssp_serve_latency_us(srv, t) > 0.0
            S.sssp_serve_release(srv, t)
        with pytest.raises(S.SsspError) as ei:
            S.sssp_serve_poll(srv, tickets[0])
        assert ei.value.code == S.SSSP_E_NOTFOUND
    finally:
        S.sssp_serve_destroy(srv)
    for s, d, p in outs:
        assert_exact(g, s, d, p)


def test_serve_many_slots_one_graph(graphs):
    """More queries than the lane's first allocation (8 slots): the lane
    grows while queries run."""
    g, G = graphs["grid"]
    srcs, _ = gg.giant_sources(g, 40, seed=4)
    srv = S.sssp_serve_create(slice_us=150, max_slots=64)
    try:
        bufs, tickets = [], []
        for k, s in enumerate(srcs):
            d, _ = _bufs(G, False, host=False)
            bufs.append((int(s), d))
            tickets.append(S.sssp_serve_submit(srv, G.handle, int(s), d, None))
            if k % 10 == 9:
                time.sleep(0.001)
        _wait_all(srv, tickets)
    finally:
        S.sssp_serve_destroy(srv)
    for s, d in bufs:
        assert np.array_equal(_dist_bits(d), oracle_dist(g, s)), s


@pytest.mark.parametrize("flag", ["migrate", "overflow"])
def test_serve_recovery_paths_keep_results(graphs, flag):
    """Ring migration after every slice, and a lane restart after an
    (injected) overflow, both leave every result exact."""
    flags = S.SERVE_MIGRATE_EACH_SLICE if flag == "migrate" else S.SERVE_INJECT_OVERFLOW
    names = ["road", "rmat", "erf"]
    srv = S.sssp_serve_create(slice_us=200, flags=flags)
    try:
        bufs, tickets = [], []
        for name in names:
            g, G = graphs[name]
            srcs, _ = gg.giant_sources(g, 3, seed=6)
            for i, s in enumerate(srcs):
                d, p = _bufs(G, i == 0, host=False)
                bufs.append((name, int(s), d, p))
                tickets.append(S.sssp_serve_submit(srv, G.handle, int(s), d, p))
        _wait_all(srv, tickets)
        stats = S.sssp_serve_get_stats(srv)
    finally:
        S.sssp_serve_destroy(srv)
    if flag == "migrate":
        assert stats["ring_growths"] >= 1, stats
    else:
        assert stats["restarts"] >= len(names), stats
    for name, s, d, p in bufs:
        g, _ = graphs[name]
        assert_exact(g, s, _dist_bits(d), _np(p))


def test_serve_injected_timeout_fails_lane_then_recovers(graphs):
    g, G = graphs["grid"]
    srcs, _ = gg.giant_sources(g, 3, seed=7)
    srv = S.sssp_serve_create(slice_us=200, flags=S.SERVE_INJECT_TIMEOUT)
    try:
        d0, _ = _bufs(G, False, host=False)
        t0 = S.sssp_serve_submit(srv, G.handle, int(srcs[0]), d0, None)
        st, code = S.sssp_serve_wait(srv, t0, 60000)
        assert st == S.Q_ERROR and code == S.SSSP_E_TIMEOUT
        # the lane started over: later queries in it succeed (a query with
        # predecessors would open a second lane, whose first slice fails too)
        d1, _ = _bufs(G, False, host=False)
        t1 = S.sssp_serve_submit(srv, G.handle, int(srcs[1]), d1, None)
        _wait_all(srv, [t1])
        assert_exact(g, int(srcs[1]), _dist_bits(d1))
    finally:
        S.sssp_serve_destroy(srv)


def test_serve_negative_count_fails_lane_then_recovers(graphs):
    """A lane whose per-slot L2 count reads negative (injected on the host:
    more reads than writes) fails its queries with SSSP_E_CUDA and starts
    over on fresh rings; later queries in it are exact."""
    g, G = graphs["rmat"]
    srcs, _ = gg.giant_sources(g, 3, seed=9)
    srv = S.sssp_serve_create(slice_us=200, flags=S.SERVE_INJECT_NEGATIVE)
    try:
        d0, _ = _bufs(G, False, host=False)
        t0 = S.sssp_serve_submit(srv, G.handle, int(srcs[0]), d0, None)
        st, code = S.sssp_serve_wait(srv, t0, 60000)
        assert st == S.Q_ERROR and code == S.SSSP_E_CUDA, (st, S.strerror(code))
        d1, p1 = _bufs(G, False, host=False)
        t1 = S.sssp_serve_submit(srv, G.handle, int(srcs[1]), d1, None)
        _wait_all(srv, [t1])
        assert_exact(g, int(srcs[1]), _dist_bits(d1))
        stats = S.sssp_serve_get_stats(srv)
        assert stats["failed"] == 1 and stats["completed"] >= 1, stats
    finally:
        S.sssp_serve_destroy(srv)


def test_serve_cancel(graphs):
    g, G = graphs["road"]
    gs, Gs = graphs["grid"]
    srcs, _ = gg.giant_sources(g, 2, seed=8)
    srv = S.sssp_serve_create(slice_us=100)
    try:
        d, _ = _bufs(G, False, host=True)
        t = S.sssp_serve_submit(srv, G.handle, int(srcs[0]), d, None)
        rc = S.sssp_serve_cancel(srv, t)
        assert rc in (S.SSSP_OK, S.SSSP_E_BUSY, S.SSSP_E_INVAL)
        st, code = S.sssp_serve_wait(srv, t, 60000)
        if rc == S.SSSP_OK:
            assert st == S.Q_ERROR and code == S.SSSP_E_CANCELLED
            snapshot = d.copy()
        # the server keeps working; a cancelled query's buffer stays untouched
        d2, _ = _bufs(Gs, False, host=False)
        t2 = S.sssp_serve_submit(srv, Gs.handle, 0, d2, None)
        _wait_all(srv, [t2])
        assert np.array_equal(_dist_bits(d2), oracle_dist(gs, 0))
        if rc == S.SSSP_OK:
            assert np.array_equal(d, snapshot)
        assert S.sssp_serve_cancel(srv, t2) == S.SSSP_E_INVAL   # already done
    finally:
        S.sssp_serve_destroy(srv)


def test_serve_query_timeout(graphs):
    g, G = graphs["road"]
    src = int(gg.giant_sources(g, 1)[0][0])
    srv = S.sssp_serve_create(slice_us=100, query_timeout_ms=1)
    try:
        d, _ = _bufs(G, False, host=False)
        t = S.sssp_serve_submit(srv, G.handle, src, d, None)
        st, code = S.sssp_serve_wait(srv, t, 60000)
        # the road query needs far more than 1 ms
        assert st == S.Q_ERROR and code == S.SSSP_E_TIMEOUT
    finally:
        S.sssp_serve_destroy(srv)   # drains the timed-out query's leftovers


def test_serve_admission_limits(graphs):
    g, G = graphs["road"]
    # budget below one lane's needs: the query fails with NOMEM
    srv = S.sssp_serve_create(mem_budget_bytes=1 << 20)
    try:
        d, _ = _bufs(G, False, host=False)
        t = S.sssp_serve_submit(srv, G.handle, 0, d, None)
        st, code = S.sssp_serve_wait(srv, t, 60000)
        assert st == S.Q_ERROR and code == S.SSSP_E_NOMEM
    finally:
        S.sssp_serve_destroy(srv)
    # one slot, one waiting query: the next submit is refused
    srv = S.sssp_serve_create(max_slots=1, max_queued=1, slice_us=100)
    try:
        srcs, _ = gg.giant_sources(g, 3, seed=9)
        tickets, busy = [], 0
        bufs = []
        for s in srcs:
            d, _ = _bufs(G, False, host=False)
            try:
                tickets.append(S.sssp_serve_submit(srv, G.handle, int(s), d, None))
                bufs.append((int(s), d))
            except S.SsspError as e:
                assert e.code == S.SSSP_E_BUSY
                busy += 1
            time.sleep(0.002)
        _wait_all(srv, tickets)
        assert busy >= 1
        for s, d in bufs:
            assert np.array_equal(_dist_bits(d), oracle_dist(g, s))
    finally:
        S.sssp_serve_destroy(srv)


def test_serve_bad_arguments(graphs):
    g, G = graphs["grid"]
    srv = S.sssp_serve_create()
    try:
        d, _ = _bufs(G, False, host=False)
        for bad in (-1, G.n):
            with pytest.raises(S.SsspError) as ei:
                S.sssp_serve_submit(srv, G.handle, bad, d, None)
            assert ei.value.code == S.SSSP_E_INVAL
        with pytest.raises(S.SsspError) as ei:
            S.sssp_serve_poll(srv, 987654321)
        assert ei.value.code == S.SSSP_E_NOTFOUND
    finally:
        S.sssp_serve_destroy(srv)
