"""The no-allocation entry point against the oracle and the regular one.

sssp_solve_noalloc is for callers that cannot allocate device memory when
they need an answer; it keeps all scratch state in a fixed array inside the
library.  This file is collected last on purpose (a failure here leaves every
other test already run).  Two calls in a row on the shared array must equal
the oracle (u32 distances and canonical predecessors bit for bit, f32
distances bit for bit with predecessors checked by the invariants) and
sssp_solve.  A call after a failed one, and after a call that pushed the
fixed rings to their limit, must be exact again: every call re-initialises
the array's queue state first.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2602_10080_gb300 as S
from gpu_util import assert_exact

pytestmark = pytest.mark.gpu


def _interleave(g):
    arcs = np.empty(2 * max(g.m, 1), np.uint32)
    arcs[0:2 * g.m:2] = g.col.view(np.uint32)
    arcs[1:2 * g.m:2] = g.w_bits
    return torch.from_numpy(arcs.view(np.int32)).cuda()


def _regular(g, src):
    G = S.Graph(g.row_ptr, g.col, g.w_bits, g.wtype)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    p = torch.empty(g.n, dtype=torch.int32, device="cuda")
    G.solve(int(src), d, p)
    torch.cuda.synchronize()
    G.close()
    return d.cpu().numpy().view(np.uint32), p.cpu().numpy()


@pytest.mark.parametrize("make", [
    lambda: gg.grid(96, 80, 1, 100, seed=3),
    lambda: gg.rmat(13, 16, seed=4),
    lambda: gg.rmat(12, 8, seed=6, wtype="f32"),
], ids=["grid_u32", "rmat_u32", "rmat_f32"])
def test_noalloc_matches_solve_twice(make):
    g = make()
    S.build()
    rp = torch.from_numpy(g.row_ptr).cuda()
    arcs = _interleave(g)
    wt = S.SSSP_W_F32 if g.wtype == "f32" else S.SSSP_W_U32
    srcs = gg.giant_sources(g, 2, seed=2)[0]
    for s in srcs:  # two calls in a row share the static scratch array
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        p = torch.empty(g.n, dtype=torch.int32, device="cuda")
        S.sssp_solve_noalloc(rp, arcs, g.n, g.m, wt, int(s), d, p)
        torch.cuda.synchronize()
        dn, pn = d.cpu().numpy().view(np.uint32), p.cpu().numpy()
        assert_exact(g, int(s), dn, pn)
        dr, pr = _regular(g, s)
        np.testing.assert_array_equal(dn, dr)
        if g.wtype == "u32":
            np.testing.assert_array_equal(pn, pr)
        else:
            assert oracle.check(g.row_ptr, g.col, g.w, int(s), dn.view(np.float32), pn, "f32")[0] == "ok"
        # distances only (written straight into the caller's buffer)
        d2 = torch.empty(g.n, dtype=torch.int32, device="cuda")
        S.sssp_solve_noalloc(rp, arcs, g.n, g.m, wt, int(s), d2)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(d2.cpu().numpy().view(np.uint32), dr)


def test_noalloc_rejects_bad_arguments():
    S.build()
    lib = S.lib()
    g = gg.grid(8, 8, 1, 9, seed=1)
    rp = torch.from_numpy(g.row_ptr).cuda()
    arcs = _interleave(g)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    # beyond the fixed maximum
    big = S.SSSP_NOALLOC_MAX_VERTICES + 1
    assert lib.sssp_solve_noalloc(rp.data_ptr(), arcs.data_ptr(), big, g.m, 0, 0, d.data_ptr(), None,
                                  None) == S.SSSP_E_INVAL
    # host output buffer (no staging without allocation)
    hd = np.empty(g.n, np.uint32)
    assert lib.sssp_solve_noalloc(rp.data_ptr(), arcs.data_ptr(), g.n, g.m, 0, 0, hd.ctypes.data, None,
                                  None) == S.SSSP_E_INVAL
    # column out of range is caught on the device
    bad = arcs.clone()
    bad[0] = g.n + 5
    assert lib.sssp_solve_noalloc(rp.data_ptr(), bad.data_ptr(), g.n, g.m, 0, 0, d.data_ptr(), None,
                                  None) == S.SSSP_E_BADGRAPH
    # and the array is still usable afterwards
    S.sssp_solve_noalloc(rp, arcs, g.n, g.m, 0, 0, d)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32),
                                  oracle.dijkstra_u32(g.row_ptr, g.col, g.w, 0))


def _spreader_graph():
    """Source 0 reaches 1024 spreaders, each of which reaches 2000 fresh
    vertices at once, each with 4 arcs to a pool of sinks: about two million
    elements become live within a few relaxation rounds, against fixed rings
    of 8 x 4096 chunks."""
    ns, per, nsink = 1024, 2000, 40000
    n = 1 + ns + ns * per + nsink
    assert n <= S.SSSP_NOALLOC_MAX_VERTICES
    mids = np.arange(1 + ns, 1 + ns + ns * per, dtype=np.int64)
    sinks0 = 1 + ns + ns * per
    src = np.concatenate([np.zeros(ns, np.int64), np.repeat(np.arange(1, 1 + ns), per), np.repeat(mids, 4)])
    dst = np.concatenate([np.arange(1, 1 + ns), mids, sinks0 + (np.repeat(mids, 4) * 7919 + np.tile(
        np.arange(4), mids.size) * 104729) % nsink])
    w = np.concatenate([np.ones(ns, np.uint32), np.full(ns * per, 10, np.uint32),
                        (1000 + (np.repeat(mids, 4) + np.tile(np.arange(4), mids.size)) % 97).astype(np.uint32)])
    order = np.argsort(src, kind="stable")
    row_ptr = np.concatenate([[0], np.cumsum(np.bincount(src, minlength=n))]).astype(np.int32)
    return gg.Graph("spreaders", n, len(dst), row_ptr, dst[order].astype(np.int32), w[order], "u32")


def test_noalloc_after_ring_pressure_and_failure():
    """A graph that pushes about two million elements into the fixed rings at
    once either solves exactly or reports SSSP_E_NOMEM; either way, and after
    a rejected graph, the next call on another graph is exact."""
    S.build()
    lib = S.lib()
    g = _spreader_graph()
    rp = torch.from_numpy(g.row_ptr).cuda()
    arcs = _interleave(g)
    d = torch.empty(g.n, dtype=torch.int32, device="cuda")
    p = torch.empty(g.n, dtype=torch.int32, device="cuda")
    rc = lib.sssp_solve_noalloc(rp.data_ptr(), arcs.data_ptr(), g.n, g.m, 0, 0, d.data_ptr(), p.data_ptr(),
                                None)
    torch.cuda.synchronize()
    assert rc in (S.SSSP_OK, S.SSSP_E_NOMEM), S.strerror(rc)
    if rc == S.SSSP_OK:
        assert_exact(g, 0, d.cpu().numpy().view(np.uint32), p.cpu().numpy())
    del d, p, arcs, rp
    h = gg.rmat(14, 16, seed=8)
    hr = torch.from_numpy(h.row_ptr).cuda()
    ha = _interleave(h)
    bad = ha.clone()
    bad[0] = h.n + 3
    hd = torch.empty(h.n, dtype=torch.int32, device="cuda")
    hp = torch.empty(h.n, dtype=torch.int32, device="cuda")
    assert lib.sssp_solve_noalloc(hr.data_ptr(), bad.data_ptr(), h.n, h.m, 0, 0, hd.data_ptr(), None,
                                  None) == S.SSSP_E_BADGRAPH
    for s in gg.giant_sources(h, 2, seed=5)[0]:
        S.sssp_solve_noalloc(hr, ha, h.n, h.m, S.SSSP_W_U32, int(s), hd, hp)
        torch.cuda.synchronize()
        assert_exact(h, int(s), hd.cpu().numpy().view(np.uint32), hp.cpu().numpy())
