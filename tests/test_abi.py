"""C ABI checks that need no GPU: the library loads, exports every function
include/sssp.h declares, the ctypes structs match the C layout, and calls
that need a device fail loudly without one."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2602_10080_gb300 as sssp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sssp.h")


@pytest.fixture(scope="module")
def lib():
    sssp.build()
    return sssp.lib()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"SSSP_API\s+[\w\s\*]*?\b(sssp_\w+)\s*\(", text)))


def test_header_declares_api():
    names = declared_functions()
    for must in ("sssp_graph_create", "sssp_solve", "sssp_solve_batch", "sssp_serve_submit",
                 "sssp_serve_poll", "sssp_autotune"):
        assert must in names


def test_every_declared_symbol_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", sssp.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    # nothing else leaks out of the library
    extra = [s for s in exported if s.startswith("sssp_") and s not in declared_functions()]
    assert not extra, extra


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(sssp_config), sizeof(sssp_features), sizeof(sssp_stats),
         offsetof(sssp_config, timeout_ms), offsetof(sssp_stats, attempts), offsetof(sssp_features, has_zero_w));
  printf("%zu %zu %zu %zu\\n", offsetof(sssp_config, shards), offsetof(sssp_stats, cycles),
         offsetof(sssp_config, l2_only), offsetof(sssp_stats, window_advances));
  return 0;
}}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [ctypes.sizeof(sssp.sssp_config), ctypes.sizeof(sssp.sssp_features),
                    ctypes.sizeof(sssp.sssp_stats), sssp.sssp_config.timeout_ms.offset,
                    sssp.sssp_stats.attempts.offset, sssp.sssp_features.has_zero_w.offset,
                    sssp.sssp_config.shards.offset, sssp.sssp_stats.cycles.offset,
                    sssp.sssp_config.l2_only.offset, sssp.sssp_stats.window_advances.offset]


def test_host_only_calls(lib):
    assert sssp.strerror(0) == "ok"
    assert "timed out" in sssp.strerror(sssp.SSSP_E_TIMEOUT)
    assert lib.sssp_version() >= 10000
    c = sssp.sssp_config_default()
    assert c.l0_rows == 2 and c.block_threads in (256, 512, 1024)
    # defaults: the first two buckets of the window bypass the block staging,
    # claims within the 1..32 chunks a refill can hand over
    assert c.direct_buckets == 2 and 1 <= c.claim <= 32
    assert c.stage == 1 and c.split_arcs == 0 and c.pending_marks == 0
    assert lib.sssp_config_default(None) == sssp.SSSP_E_INVAL
    assert lib.sssp_graph_destroy(None) == sssp.SSSP_OK


def test_no_device_fails_loudly(lib):
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rp = np.array([0, 1, 1], np.int32)
    col = np.array([1], np.int32)
    w = np.array([3], np.uint32)
    with pytest.raises(sssp.SsspError) as ei:
        sssp.sssp_graph_create(rp, col, w, 2, 1, sssp.SSSP_W_U32)
    assert ei.value.code == sssp.SSSP_E_NODEV


def test_bad_arguments_rejected_before_device(lib):
    h = ctypes.c_void_p()
    assert lib.sssp_graph_create(None, None, None, 0, 0, 0, ctypes.byref(h)) == sssp.SSSP_E_INVAL
    assert lib.sssp_solve(None, 0, None, None, None, None) == sssp.SSSP_E_INVAL
    assert lib.sssp_solve_batch(None, None, 0, None, None, None, None) == sssp.SSSP_E_INVAL


def test_serve_options_rejected_before_device(lib):
    o = sssp.sssp_serve_options_default()
    assert o.max_slots == 128 and o.slice_us == 1000 and o.flags == 0
    assert lib.sssp_serve_options_default(None) == sssp.SSSP_E_INVAL
    h = ctypes.c_void_p()
    for field, value in (("max_slots", 0), ("max_slots", 5000), ("slice_us", 10), ("ring_shift", 17),
                         ("query_timeout_ms", -1), ("flags", 64), ("max_queued", 0)):
        bad = sssp.sssp_serve_options_default()
        setattr(bad, field, value)
        assert lib.sssp_serve_create(ctypes.byref(bad), ctypes.byref(h)) == sssp.SSSP_E_INVAL, field
    bad = sssp.sssp_serve_options_default()
    bad.reserved[0] = 1
    assert lib.sssp_serve_create(ctypes.byref(bad), ctypes.byref(h)) == sssp.SSSP_E_INVAL
    assert lib.sssp_serve_create(None, None) == sssp.SSSP_E_INVAL
    assert lib.sssp_serve_destroy(None) == sssp.SSSP_OK
    assert lib.sssp_serve_submit(None, None, 0, None, None, None) == sssp.SSSP_E_INVAL


def test_serve_struct_layouts_match_c(tmp_path):
    src = tmp_path / "serve_layout.c"
    src.write_text(f'''
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu\\n", sizeof(sssp_serve_options), sizeof(sssp_serve_stats),
         offsetof(sssp_serve_options, flags), offsetof(sssp_serve_stats, kernel_ms));
  return 0;
}}
''')
    exe = tmp_path / "serve_layout"
    subprocess.run(["gcc", str(src), "-o", str(exe)], check=True)
    vals = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [ctypes.sizeof(sssp.sssp_serve_options), ctypes.sizeof(sssp.sssp_serve_stats),
                    sssp.sssp_serve_options.flags.offset, sssp.sssp_serve_stats.kernel_ms.offset]


def test_sampled_rejects_bad_arguments(lib):
    n = ctypes.c_int32()
    buf = (ctypes.c_uint64 * 12)()
    assert lib.sssp_solve_sampled(None, 0, None, None, None, buf, 2, 10, ctypes.byref(n)) == sssp.SSSP_E_INVAL
    assert lib.sssp_bfs(None, 0, None, None, None, None) == sssp.SSSP_E_INVAL
