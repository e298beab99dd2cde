"""Planted mistakes: each mutated copy of the oracle must fail some pin.

Every mutant is compiled from a textual edit of oracle/sssp_oracle.c into a
temporary directory (CPU only); the pins of test_oracle.py are re-run
against it and at least one must fail.
"""
import os
import subprocess

import numpy as np
import pytest

import graphgen as gg
import oracle
from golden_io import all_cases

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "sssp_oracle.c")

MUTANTS = {
    "wrap-instead-of-saturate": ("uint64_t s = (uint64_t)d + (uint64_t)w;",
                                 "uint64_t s = (uint32_t)(d + w);"),
    "drop-last-arc": ("for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; e++) {\n"
                      "            int32_t v = col[e];\n            uint32_t nd",
                      "for (int32_t e = row_ptr[u]; e < row_ptr[u + 1] - 1; e++) {\n"
                      "            int32_t v = col[e];\n            uint32_t nd"),
    "pred-max-index": ("(pred[v] < 0 || u < pred[v])", "(pred[v] < 0 || u > pred[v])"),
    "f32-wrong-endpoint": ("volatile float nd = dist[u] + w[e]; /* one rounded f32 add */",
                           "volatile float nd = dist[v] + w[e];"),
    "source-not-zero": ("    dist[src] = 0;\n    if (heap_push(&h, 0.0, src)) return -1;\n    while",
                        "    dist[src] = 1;\n    if (heap_push(&h, 0.0, src)) return -1;\n    while"),
}


def _pins_pass() -> bool:
    try:
        for case in all_cases():
            rp, col, src = case["row_ptr"], case["col"], case["src"]
            if case["kind"] == "u32":
                d = oracle.dijkstra_u32(rp, col, case["w_bits"], src)
                if not np.array_equal(d, case["dist_bits"]):
                    return False
                if case["pred"] is not None:
                    p = oracle.pred_canonical_u32(rp, col, case["w_bits"], src, d)
                    if not np.array_equal(p, case["pred"]):
                        return False
            else:
                d = oracle.dijkstra_f32(rp, col, case["w_bits"].view(np.float32), src)
                if not np.array_equal(d.view(np.uint32), case["dist_bits"]):
                    return False
        g = gg.grid(20, 9, 1, 1, seed=1)
        ys, xs = np.divmod(np.arange(g.n), 20)
        if not np.array_equal(oracle.dijkstra_u32(g.row_ptr, g.col, g.w, 0), xs + ys):
            return False
    except ValueError:
        return False
    return True


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    before, after = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(before) >= 1, f"mutation anchor missing for {name}"
    mutated = text.replace(before, after, 1)
    src = tmp_path / "mut.c"
    so = tmp_path / "libmut.so"
    src.write_text(mutated)
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                    "-fexcess-precision=standard", str(src), "-o", str(so), "-lm"], check=True)
    saved = oracle._lib
    try:
        oracle.use_library(str(so))
        assert not _pins_pass(), f"mutant {name} survived every pin"
    finally:
        oracle._lib = saved


# Equivalent mutants: they change the order of work, not the result.  A
# mis-ordered heap turns Dijkstra into a label-correcting solver (every
# improvement is re-queued and stale entries are skipped), which converges to
# the same lengths -- the premise of Section 2.1 that the queue policy trades
# work against parallelism without changing l_su.
EQUIVALENT = {
    "heap-picks-larger-child": ("h->a[c + 1].key < h->a[c].key", "h->a[c + 1].key > h->a[c].key"),
}


@pytest.mark.parametrize("name", sorted(EQUIVALENT))
def test_equivalent_mutant_keeps_results(name, tmp_path):
    before, after = EQUIVALENT[name]
    text = open(SRC).read()
    assert before in text
    src = tmp_path / "eq.c"
    so = tmp_path / "libeq.so"
    src.write_text(text.replace(before, after, 1))
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off",
                    "-fexcess-precision=standard", str(src), "-o", str(so), "-lm"], check=True)
    saved = oracle._lib
    try:
        oracle.use_library(str(so))
        assert _pins_pass()
    finally:
        oracle._lib = saved


def test_unmutated_passes_pins():
    oracle._lib = None
    assert _pins_pass()
