"""The no-allocation entry point against the regular one.

sssp_solve_noalloc is for callers that cannot allocate device memory when
they need an answer; it keeps all scratch state in a fixed array inside the
library.  This file is collected last on purpose (a failure here leaves every
other test already run).  Two calls in a row on the shared array must match
sssp_solve: u32 distances and canonical predecessors bit for bit, f32
distances bit for bit with predecessors checked by the invariants.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen as gg
import oracle
import paper_2602_10080_gb300 as S

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
