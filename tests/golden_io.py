"""Reader for the hand-worked fixtures in tests/golden/*.txt."""
import glob
import os

import numpy as np

GOLDEN_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok: str, kind: str):
    if tok == "INF":
        return 0xFFFFFFFF if kind == "u32" else 0x7F800000
    if tok.startswith("0x"):
        return int(tok, 16)
    return int(tok)


def load(path):
    kind, n, src, arcs, dist, pred = "u32", 0, 0, [], None, None
    section = None
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        head = line.split()
        if head[0] in ("kind", "n", "src") and len(head) == 2:
            if head[0] == "kind":
                kind = head[1]
            elif head[0] == "n":
                n = int(head[1])
            else:
                src = int(head[1])
            continue
        if head[0] in ("arcs", "dist", "pred") and len(head) == 1:
            section = head[0]
            continue
        if section == "arcs":
            u, v, w = head
            arcs.append((int(u), int(v), _num(w, kind)))
        elif section == "dist":
            dist = [_num(t, kind) for t in head]
        elif section == "pred":
            pred = [int(t) for t in head]
    deg = np.zeros(n + 1, np.int64)
    for u, _, _ in arcs:
        deg[u + 1] += 1
    row_ptr = np.cumsum(deg).astype(np.int32)
    fill = row_ptr[:-1].astype(np.int64).copy()
    col = np.zeros(len(arcs), np.int32)
    w = np.zeros(len(arcs), np.uint32)
    for u, v, wt in arcs:
        col[fill[u]] = v
        w[fill[u]] = wt
        fill[u] += 1
    case = dict(name=os.path.basename(path), kind=kind, n=n, src=src, row_ptr=row_ptr, col=col,
                w_bits=w, dist_bits=np.array(dist, np.uint32),
                pred=None if pred is None else np.array(pred, np.int32))
    return case


def all_cases():
    return [load(p) for p in sorted(glob.glob(os.path.join(GOLDEN_DIR, "*.txt")))]
