"""Host-side helpers of bench.py: the kernel-code hash ignores comments,
the recorded DRAM traffic is reported only for the kernel code and the
configuration it was captured with."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import paper_2602_10080_gb300 as S  # noqa: E402


def test_strip_comments_keeps_code_only():
    src = "int a; // one\n/* two\n   lines */ int b;\n\n   // only a comment\nint c; /* x */ int d;\n"
    assert bench._strip_comments(src) == "int a;\n int b;\nint c;  int d;"


def test_traffic_keyed_to_code_and_config():
    path = os.path.join(ROOT, "profiles", "mlmq_kernel_rmat22_traffic.txt")
    vals = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals["kernel_source_hash"] == bench.kernel_source_hash():
        assert bench.profiled_traffic(vals["config"]) == float(vals["dram_bytes_per_launch"])
    else:
        # the kernel changed since the capture: no traffic is reported
        assert bench.profiled_traffic(vals["config"]) is None
    assert bench.profiled_traffic("l1_type=0,l2_type=1") is None
    # the signature has the format bench.py builds from a configuration
    c = S.sssp_config_default()
    sig = bench.config_signature(c)
    assert sig.split(",")[0].startswith("l1_type=") and len(sig.split(",")) == len(bench.TRAFFIC_CONFIG_KEYS)


def test_rank_sources_cover_and_are_disjoint():
    srcs = list(range(10))
    shares = [bench.rank_sources(srcs, r, 3) for r in range(3)]
    assert sorted(sum(shares, [])) == srcs


def test_percentiles_and_cpu_model():
    p = bench.percentiles([1.0, 2.0, 3.0, 4.0, 100.0])
    assert p["p50"] == 3.0 and p["mean"] == 22.0 and 4.0 < p["p99"] <= 100.0
    assert bench.percentiles([]) == {"p50": None, "p99": None, "mean": None}
    m = bench.cpu_model()
    assert isinstance(m, str) and m
