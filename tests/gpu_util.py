"""Helpers for the GPU tests: run the C ABI through the Python binding on
torch CUDA buffers and compare with the oracle."""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

import oracle
import paper_2602_10080_gb300 as S

U32_INF = 0xFFFFFFFF


def cfg(**kw):
    """The library's default configuration with the given fields set.  A key
    that is not a field of sssp_config raises (ctypes would accept any
    attribute name silently)."""
    c = S.sssp_config_default()
    fields = {name for name, _ in S.sssp_config._fields_}
    for k, v in kw.items():
        if k not in fields:
            raise KeyError(f"sssp_config has no field {k!r}")
        setattr(c, k, v)
    return c


def upload(g, device_inputs=True):
    """Creates a library graph from a graphgen.Graph (device or host input arrays)."""
    w = g.w_bits
    if device_inputs and g.m > 0:
        rp = torch.from_numpy(g.row_ptr).cuda()
        col = torch.from_numpy(g.col).cuda()
        wt = torch.from_numpy(w.view(np.int32)).cuda()
        G = S.Graph(rp, col, wt, g.wtype)
    else:
        G = S.Graph(g.row_ptr, g.col, w, g.wtype)
    return G


def gpu_solve(G, src, pred=True, config=None, host=False):
    """dist bits (uint32 numpy) and pred (int32 numpy or None)."""
    if host:
        d = np.empty(G.n, np.uint32)
        p = np.empty(G.n, np.int32) if pred else None
        G.solve(int(src), d, p, config)
        return d, p
    d = torch.empty(G.n, dtype=torch.int32, device="cuda")
    p = torch.empty(G.n, dtype=torch.int32, device="cuda") if pred else None
    G.solve(int(src), d, p, config)
    torch.cuda.synchronize()
    return d.cpu().numpy().view(np.uint32), (p.cpu().numpy() if pred else None)


def gpu_batch(G, srcs, pred=True, config=None, host=False):
    nq = len(srcs)
    s = np.ascontiguousarray(srcs, np.int32)
    if host:
        d = np.empty(nq * G.n, np.uint32)
        p = np.empty(nq * G.n, np.int32) if pred else None
        G.solve_batch(s, d, p, config)
        return d.reshape(nq, G.n), (p.reshape(nq, G.n) if pred else None)
    st = torch.from_numpy(s).cuda()
    d = torch.empty(nq * G.n, dtype=torch.int32, device="cuda")
    p = torch.empty(nq * G.n, dtype=torch.int32, device="cuda") if pred else None
    G.solve_batch(st, d, p, config)
    torch.cuda.synchronize()
    d = d.cpu().numpy().view(np.uint32).reshape(nq, G.n)
    return d, (p.cpu().numpy().reshape(nq, G.n) if pred else None)


def oracle_dist(g, src):
    if g.wtype == "f32":
        return oracle.dijkstra_f32(g.row_ptr, g.col, g.w, int(src)).view(np.uint32)
    return oracle.dijkstra_u32(g.row_ptr, g.col, g.w, int(src))


def assert_exact(g, src, dist_bits, pred=None, canonical=None):
    """Bit-exact distances; canonical pred for u32 positive weights, else invariants."""
    ref = oracle_dist(g, src)
    bad = np.flatnonzero(dist_bits != ref)
    assert bad.size == 0, (f"{bad.size} mismatches, first v={bad[0]} gpu={dist_bits[bad[0]]:#x} "
                           f"oracle={ref[bad[0]]:#x}")
    if pred is None:
        return
    if canonical is None:
        canonical = g.wtype == "u32" and (g.m == 0 or int(g.w.min()) >= 1)
    if canonical:
        pref = oracle.pred_canonical_u32(g.row_ptr, g.col, g.w, int(src), ref)
        bad = np.flatnonzero(pred != pref)
        assert bad.size == 0, f"pred mismatch at {bad[:5]}: gpu={pred[bad[:5]]} oracle={pref[bad[:5]]}"
    dist_view = dist_bits if g.wtype == "u32" else dist_bits.view(np.float32)
    status, v = oracle.check(g.row_ptr, g.col, g.w, int(src), dist_view, pred, g.wtype)
    assert status == "ok", (status, v)


def oracle_threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def assert_exact_many(g, srcs, dists, preds=None):
    """assert_exact for every query (row q of dists/preds from srcs[q]), with
    the oracle runs spread over the host cores."""
    srcs = [int(s) for s in srcs]

    def one(q):
        assert_exact(g, srcs[q], dists[q], None if preds is None else preds[q])
        return q

    with ThreadPoolExecutor(max_workers=oracle_threads()) as ex:
        done = list(ex.map(one, range(len(srcs))))
    assert done == list(range(len(srcs)))
