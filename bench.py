"""Benchmark: GTEPS and HBM-roofline fraction of single-source SSSP on a
symmetrised R-MAT scale-22 graph (edge factor 16, a/b/c/d .57/.19/.19/.05,
uint32 weights in [1, 255]; 64 seeded sources from the giant component,
each solved alone), plus batched and served throughput as extra keys.

A step = one sssp_solve (distance init, the persistent MLMQ relaxation loop,
predecessors) for the next source.  Inputs (the CSR, 1.07 GB of (col, w)
pairs) are larger than L2 and resident in HBM before timing.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank solves its own sources (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GTEPS & HBM-roofline fraction per SSSP; serving p50/p99 latency vs plain solve"
BYTES_PER_ARC = 12      # col 4 B + weight 4 B + dist[v] check 4 B
BYTES_PER_VERTEX = 32   # row_ptr 8 B + dist 4 B + pred 4 B + queue push/pop of an 8 B element
WORKLOAD = "rmat22"
N_SOURCES = 64
WORK_KEYS = ("relax_arcs", "relax_shadow", "improved", "stale", "dup_targets", "rounds", "pops_l0", "pops_l1",
             "pops_l2", "refills", "refill_tries", "cas_fail", "l2_chunks_written", "far_pushes", "idle_iters",
             "wait_spins", "lock_spins")


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


def _strip_comments(src: str) -> str:
    """C/C++ source without comments and blank lines (the code the hash tracks)."""
    import re
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    lines = []
    for line in src.splitlines():
        line = re.sub(r"//.*", "", line).rstrip()
        if line:
            lines.append(line)
    return "\n".join(lines)


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("mlmq.cuh", "kernels_inst.cuh", "kernels_u32.cu"):
        text = open(os.path.join(ROOT, "paper_2602_10080_gb300", "csrc", f), encoding="utf-8").read()
        h.update(_strip_comments(text).encode())
    return h.hexdigest()[:16]


TRAFFIC_CONFIG_KEYS = ("l1_type", "l2_type", "delta_u32", "bnum", "bmax", "claim", "shards", "block_threads",
                       "split_arcs", "hub_bnum", "pending_marks", "direct_buckets")


def config_signature(cfg) -> str:
    d = cfg.as_dict()
    return ",".join(f"{k}={d[k]}" for k in TRAFFIC_CONFIG_KEYS)


def profiled_traffic(signature=None):
    """Per-launch DRAM bytes of the relaxation kernel from the committed ncu
    summary, or None if the kernel source or the configuration changed
    since it was captured."""
    p = os.path.join(ROOT, "profiles", "mlmq_kernel_rmat22_traffic.txt")
    if not os.path.exists(p):
        return None
    vals = {}
    for line in open(p):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel_source_hash") != kernel_source_hash():
        return None
    if signature is not None and vals.get("config") != signature:
        return None
    try:
        return float(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self) -> dict:
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sms)) if sms else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sms)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def percentiles(values) -> dict:
    """p50, p99 and mean of a list of numbers (3 decimals)."""
    a = np.asarray(values, dtype=np.float64)
    if a.size == 0:
        return {"p50": None, "p99": None, "mean": None}
    return {"p50": round(float(np.percentile(a, 50)), 3), "p99": round(float(np.percentile(a, 99)), 3),
            "mean": round(float(a.mean()), 3)}


def cpu_model() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or implementer/part on Arm)."""
    try:
        info = open("/proc/cpuinfo").read()
    except OSError:
        import platform
        return platform.machine()
    for line in info.splitlines():
        if line.lower().startswith("model name"):
            return line.split(":", 1)[1].strip()
    impl = part = None
    for line in info.splitlines():
        if line.startswith("CPU implementer") and impl is None:
            impl = line.split(":", 1)[1].strip()
        if line.startswith("CPU part") and part is None:
            part = line.split(":", 1)[1].strip()
    if impl or part:
        return f"implementer {impl}, part {part}"
    import platform
    return platform.machine()


def rank_sources(srcs, rank: int, ws: int) -> list:
    """This rank's share of the sources: every ws-th one from `rank` (weak
    scaling; the ranks' shares are disjoint and cover all sources)."""
    mine = [int(s) for s in srcs[rank::ws]]
    return mine or [int(srcs[0])]


def combine_over_ranks(t_ms: float, arcs: int, verts: int, device) -> tuple:
    """Whole-job figures: the slowest rank's time, the units all ranks
    processed.  No-op on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t_ms, arcs, verts
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    at = torch.tensor([arcs, verts], dtype=torch.float64, device=device)
    dist.all_reduce(at)
    return float(tt.item()), int(at[0].item()), int(at[1].item())


def cpu_oracle_gteps(g, srcs, threads: int, kind: str = "u32"):
    """The oracle as it stands: one Dijkstra per host thread, all at once."""
    import oracle
    t0 = time.perf_counter()
    dists = oracle.dijkstra_many(g.row_ptr, g.col, g.w, srcs, kind=kind, threads=threads)
    dt = time.perf_counter() - t0
    arcs = sum(oracle.reached_counts(g.row_ptr, d, kind)[0] for d in dists)
    return arcs / dt / 1e9, dt, arcs


def reached(row_ptr_t, dist_t, wtype: str):
    """(m_r, n_r) of one result, computed on the device (outside timing)."""
    import torch
    inf = 0x7F800000 if wtype == "f32" else -1  # int32 view of 0xFFFFFFFF
    r = dist_t != inf
    deg = (row_ptr_t[1:] - row_ptr_t[:-1]).to(torch.int64)
    return int(deg[r].sum().item()), int(r.sum().item())


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import graphgen as gg
    import oracle
    oracle.build()
    g = gg.workload(WORKLOAD)
    srcs, _ = gg.giant_sources(g, N_SOURCES, seed=2)
    cores = max(1, min(len(srcs), os.cpu_count() or 1))
    k = 0
    # each step: one query per host core (a bounded sample of the 64 sources)
    for _ in range(args.warmup):
        sub = [srcs[(k + i) % len(srcs)] for i in range(cores)]
        k += cores
        cpu_oracle_gteps(g, sub, cores)
    total_arcs, total_t = 0, 0.0
    for _ in range(args.steps):
        sub = [srcs[(k + i) % len(srcs)] for i in range(cores)]
        k += cores
        gteps, dt, arcs = cpu_oracle_gteps(g, sub, cores)
        total_arcs += arcs
        total_t += dt
    value = total_arcs / total_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GTEPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1000 * total_t / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "rmat22 single-source (R-MAT scale 22, ef 16, u32 [1,255]); "
                               f"{cores} sources per step, one per host core"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GTEPS", "cores": cores, "kind": "oracle",
                         "sample": f"{cores} single-source Dijkstra runs per step on {WORKLOAD}"},
        "e2e": {"value": round(value, 4), "unit": "GTEPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def batch_leg(S, gg, torch, wtype: str = "u32", nq: int = 256, seq_sample: int = 32, tune_ms: int = 8000):
    """Batched throughput: nq sources of R-MAT 20 in one persistent launch
    (sssp_solve_batch, dist nq x n on the device) against one-at-a-time
    sssp_solve calls on the same sources (a timed sample of them), first
    with the library's multi-query heuristic, then with the configuration
    sssp_autotune_batch picks for this batch size (timed whole launches)."""
    g = gg.workload("rmat20" if wtype == "u32" else "rmat20f")
    srcs, _ = gg.giant_sources(g, nq, seed=2)
    G = S.Graph(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(),
                torch.from_numpy(g.w_bits.view(np.int32)).cuda(), g.wtype)
    try:
        st = torch.from_numpy(srcs.astype(np.int32)).cuda()
        out = torch.empty(len(srcs) * g.n, dtype=torch.int32, device="cuda")
        stream = torch.cuda.current_stream()
        G.solve_batch(st, out, None, None, stream)           # warm-up
        torch.cuda.synchronize()
        reps = 3
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            G.solve_batch(st, out, None, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        batch_s = e0.elapsed_time(e1) / 1e3 / reps
        tuned = G.autotune_batch(st, tune_ms)          # cached on the graph for this size class
        G.solve_batch(st, out, None, None, stream)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            G.solve_batch(st, out, None, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        tuned_s = e0.elapsed_time(e1) / 1e3 / reps
        one = torch.empty(g.n, dtype=torch.int32, device="cuda")
        for s in srcs[:3]:
            G.solve(int(s), one, None, None, stream)
        torch.cuda.synchronize()
        k = min(seq_sample, len(srcs))
        e0.record(stream)
        for s in srcs[:k]:
            G.solve(int(s), one, None, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        seq_s = e0.elapsed_time(e1) / 1e3 / k
        return {"workload": f"{'rmat20' if wtype == 'u32' else 'rmat20f'} x{len(srcs)} sources, one launch",
                "dtype": wtype, "qps": round(len(srcs) / batch_s, 1), "ms_per_batch": round(batch_s * 1e3, 2),
                "sequential_qps": round(1.0 / seq_s, 1),
                "sequential_sample": f"{k} sssp_solve calls",
                "speedup": round(seq_s * len(srcs) / batch_s, 2),
                "tuned": {"qps": round(len(srcs) / tuned_s, 1), "ms_per_batch": round(tuned_s * 1e3, 2),
                          "speedup": round(seq_s * len(srcs) / tuned_s, 2), "budget_ms": tune_ms,
                          "config": {k2: v for k2, v in tuned.as_dict().items()
                                     if k2 in ("delta_u32", "delta_f32", "bnum", "l1_cap", "claim", "refillers",
                                               "hub_bnum")}}}
    finally:
        G.close()


def bfs_leg(S, G, g, srcs, torch, nsrc: int = 4):
    """Breadth-first search on the same engine (every arc counts 1), on the
    benchmark graph: levels and parents from `nsrc` of its sources."""
    lev = torch.empty(g.n, dtype=torch.int32, device="cuda")
    par = torch.empty(g.n, dtype=torch.int32, device="cuda")
    row_ptr_t = torch.from_numpy(g.row_ptr).cuda()
    G.bfs(int(srcs[0]), lev, par)
    ms, arcs = [], 0
    for s in srcs[1:1 + nsrc]:
        G.bfs(int(s), lev, par)
        ms.append(S.sssp_last_stats(G.handle).kernel_ms)
        arcs += reached(row_ptr_t, lev, "u32")[0]
    return {"workload": f"BFS on the benchmark graph, {nsrc} sources", "ms_per_bfs": round(float(np.mean(ms)), 3),
            "gteps": round(arcs / (sum(ms) / 1e3) / 1e9, 3)}


def road_leg(S, gg, torch, nsrc: int = 4, tune_ms: int = 3000):
    """Road-shaped high-diameter graph (4096^2 grid, 5% of edges dropped,
    0.5% long-range edges): the prior configuration against the autotuned
    one on the same sources (distances and predecessors)."""
    g = gg.workload("road4096")
    srcs, _ = gg.giant_sources(g, 16, seed=2)
    G = S.Graph(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(),
                torch.from_numpy(g.w_bits.view(np.int32)).cuda(), g.wtype)
    try:
        d = torch.empty(g.n, dtype=torch.int32, device="cuda")
        p = torch.empty(g.n, dtype=torch.int32, device="cuda")
        row_ptr_t = torch.from_numpy(g.row_ptr).cuda()
        prior = S.sssp_autotune(G.handle, None, 0)
        tuned = G.autotune(torch.from_numpy(srcs[:2].astype(np.int32)).cuda(), tune_ms)
        out = {"workload": f"road4096 (n={g.n}, m={g.m}), {nsrc} giant-component sources"}
        for name, cfg in (("prior", prior), ("autotuned", tuned)):
            G.solve(int(srcs[0]), d, p, cfg)
            ms, arcs = [], 0
            for s in srcs[2:2 + nsrc]:
                G.solve(int(s), d, p, cfg)
                ms.append(S.sssp_last_stats(G.handle).kernel_ms)
                arcs += reached(row_ptr_t, d, g.wtype)[0]
            out[name] = {"ms_per_solve": round(float(np.mean(ms)), 3),
                         "gteps": round(arcs / (sum(ms) / 1e3) / 1e9, 3),
                         "config": {k: v for k, v in cfg.as_dict().items()
                                    if k not in ("delta_f32", "l0_rows", "timeout_ms", "pending_marks",
                                                 "dedup", "l2_only")}}
        return out
    finally:
        G.close()


def queues_leg(S, gg, torch, nsrc: int = 4):
    """The paper's comparison of the multi-level queue with single-queue
    designs, on this GPU: the prior MLMQ configuration against every write
    going straight to a delta-bucketed L2 (L2DQ only) or to one FIFO."""
    out = {}
    for name in ("rmat20", "grid1024"):
        g = gg.workload(name)
        srcs, _ = gg.giant_sources(g, 8, seed=2)
        G = S.Graph(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(),
                    torch.from_numpy(g.w_bits.view(np.int32)).cuda(), g.wtype)
        try:
            d = torch.empty(g.n, dtype=torch.int32, device="cuda")
            prior = S.sssp_autotune(G.handle, None, 0)
            variants = {"mlmq": prior}
            for vname, l2 in (("l2dq_only", S.L2_BUCKET), ("fifo_only", S.L2_VECTOR)):
                c = S.sssp_autotune(G.handle, None, 0)
                c.l2_only, c.l2_type = 1, l2
                if l2 == S.L2_VECTOR:
                    c.bmax = c.bnum = 1
                variants[vname] = c
            res = {}
            for vname, c in variants.items():
                G.solve(int(srcs[0]), d, None, c)
                ms, rl = [], []
                for s in srcs[1:1 + nsrc]:
                    G.solve(int(s), d, None, c)
                    st = S.sssp_last_stats(G.handle)
                    ms.append(st.kernel_ms)
                    rl.append(st.relax_arcs)
                res[vname] = {"ms_per_solve": round(float(np.mean(ms)), 3),
                              "relaxed_arcs": int(np.mean(rl))}
            out[name] = res
        finally:
            G.close()
    return out


SERVE_GRAPHS = ("grid1024", "rmat18", "rmat20", "rmat22", "er21")


def serve_leg(S, gg, torch, rates, seconds: float, max_queries: int, graph_cache: dict):
    """Served latency/throughput: Poisson arrivals over the resident graphs
    (graph uniform per query, source uniform over its giant component),
    through the continuous-batching server, and the same arrival trace
    through a one-at-a-time sssp_solve loop (FIFO)."""
    graphs = []
    for name in SERVE_GRAPHS:
        if name not in graph_cache:
            g = gg.workload(name)
            G = S.Graph(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(),
                        torch.from_numpy(g.w_bits.view(np.int32)).cuda(), g.wtype)
            srcs, _ = gg.giant_sources(g, 4096, seed=2)
            graph_cache[name] = (g, G, srcs)
        graphs.append(graph_cache[name])
    out = []
    for ri, rate in enumerate(rates):
        count = int(max(20, min(max_queries, rate * seconds)))
        arr = gg.poisson_arrivals(rate, count, seed=3, stream=8 + ri)
        ug = gg.uniform_stream(3, 20 + ri, count)
        us = gg.uniform_stream(3, 40 + ri, count)
        trace = []
        for i in range(count):
            gi = min(int(ug[i] * len(graphs)), len(graphs) - 1)
            srcs = graphs[gi][2]
            trace.append((float(arr[i]), gi, int(srcs[min(int(us[i] * len(srcs)), len(srcs) - 1)])))
        # one output buffer per query: submission is never held back
        bufs = [torch.empty(graphs[gi][0].n, dtype=torch.int32, device="cuda") for _, gi, _ in trace]
        # --- served
        srv = S.sssp_serve_create(slice_us=1000)
        try:
            # warm the lanes (allocation, first launch) outside the trace
            wbufs = [torch.empty(g.n, dtype=torch.int32, device="cuda") for g, _, _ in graphs]
            warm = [S.sssp_serve_submit(srv, G.handle, int(srcs[0]), wb, None)
                    for (g, G, srcs), wb in zip(graphs, wbufs)]
            for t in warm:
                S.sssp_serve_wait(srv, t, -1)
            tickets, late = [], []
            t0 = time.perf_counter()
            for i, (at, gi, src) in enumerate(trace):
                now = time.perf_counter() - t0
                if at > now:
                    time.sleep(at - now)
                late.append(time.perf_counter() - t0 - at)     # submit time - scheduled arrival
                tickets.append(S.sssp_serve_submit(srv, graphs[gi][1].handle, src, bufs[i], None))
            for t in tickets:
                st, code = S.sssp_serve_wait(srv, t, -1)
                if st != S.Q_DONE:
                    raise RuntimeError(f"served query failed: {S.strerror(code)}")
            t_end = time.perf_counter() - t0
            # latency from the scheduled arrival: (submit - arrival) + (submit -> DONE)
            lat = np.array([S.sssp_serve_latency_us(srv, t) / 1e3 + 1e3 * lt for t, lt in zip(tickets, late)])
            sstats = S.sssp_serve_get_stats(srv)
        finally:
            S.sssp_serve_destroy(srv)
        # --- one at a time (FIFO over the same trace), latency from the scheduled arrival
        stream = torch.cuda.current_stream()
        plat = []
        t0 = time.perf_counter()
        for i, (at, gi, src) in enumerate(trace):
            now = time.perf_counter() - t0
            if at > now:
                time.sleep(at - now)
            graphs[gi][1].solve(src, bufs[i], None, None, stream)
            torch.cuda.synchronize()
            plat.append((time.perf_counter() - t0 - at) * 1e3)
        p_end = time.perf_counter() - t0
        plat = np.array(plat)
        del bufs
        out.append({"rate_qps": rate, "queries": count, "arrival_span_s": round(float(trace[-1][0]), 2),
                    "served": {"qps": round(count / t_end, 1), "p50_ms": round(float(np.percentile(lat, 50)), 3),
                               "p99_ms": round(float(np.percentile(lat, 99)), 3),
                               "joined_running": sstats["joined_running"],
                               "max_resident": sstats["max_resident"]},
                    "plain_solve": {"qps": round(count / p_end, 1),
                                    "p50_ms": round(float(np.percentile(plat, 50)), 3),
                                    "p99_ms": round(float(np.percentile(plat, 99)), 3)}})
    return {"graphs": list(SERVE_GRAPHS), "arrivals": "Poisson, seed 3; graph uniform, source uniform over "
                                                       "the giant component",
            "latency": "p50/p99 from each query's scheduled arrival to its result, both arms; served = "
                       "(submit - arrival) + the server's submit-to-DONE time",
            "results": out}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=64)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", default="mlmq", choices=["mlmq", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip batch/serving/cpu legs")
    ap.add_argument("--legs", default="cpu,batch,bfs,road,queues,serving",
                    help="extra legs to run after the metric (comma list; --no-extras runs none)")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--tune-ms", type=int, default=0,
                    help="timed autotune budget in ms (0 = the feature-based prior configuration)")
    ap.add_argument("--serve-rates", default="10,30,100,300,1000,2000", help="serving leg arrival rates (q/s)")
    ap.add_argument("--serve-seconds", type=float, default=20.0, help="arrival span per rate at most")
    ap.add_argument("--serve-max", type=int, default=2000, help="queries per rate at most")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    import graphgen as gg
    import paper_2602_10080_gb300 as S
    S.build()

    g = gg.workload(args.workload)
    srcs_all, giant = gg.giant_sources(g, N_SOURCES, seed=2)
    G = S.Graph(torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda(),
                torch.from_numpy(g.w_bits.view(np.int32)).cuda(), g.wtype)
    row_ptr_t = torch.from_numpy(g.row_ptr).cuda()
    # input-adaptive configuration (Section 3.5), cached on the graph
    tune_srcs = torch.from_numpy(srcs_all[:2].copy()).cuda()
    tuned = G.autotune(tune_srcs if args.tune_ms > 0 else None, args.tune_ms)

    my_srcs = rank_sources(srcs_all, rank, ws)
    stream = torch.cuda.current_stream()
    dist_t = torch.empty(g.n, dtype=torch.int32, device="cuda")
    pred_t = torch.empty(g.n, dtype=torch.int32, device="cuda")

    # reached arcs / vertices per source (outside timing)
    mr, nr = {}, {}
    for s in set(my_srcs[: args.steps + args.warmup] + my_srcs):
        G.solve(s, dist_t, pred_t)
        mr[s], nr[s] = reached(row_ptr_t, dist_t, g.wtype)

    def src_at(i):
        return my_srcs[i % len(my_srcs)]

    for i in range(args.warmup):
        G.solve(src_at(i), dist_t, pred_t, None, stream)
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kernel_ms, step_arcs, arcs, verts, relaxed = [], [], 0, 0, 0
    work_sum = {k: 0 for k in WORK_KEYS}
    cyc_sum = np.zeros(6)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for i in range(args.steps):
            s = src_at(args.warmup + i)
            G.solve(s, dist_t, pred_t, None, stream)
            st = S.sssp_last_stats(G.handle)
            kernel_ms.append(st.kernel_ms)
            step_arcs.append(mr[s])
            relaxed += st.relax_arcs
            for k in WORK_KEYS:
                work_sum[k] += getattr(st, k)
            cyc_sum += np.array(list(st.cycles), dtype=np.float64)
            arcs += mr[s]
            verts += nr[s]
        ev1.record(stream)
        torch.cuda.synchronize()
    t_ms = ev0.elapsed_time(ev1)
    t_ms, arcs, verts = combine_over_ranks(t_ms, arcs, verts, "cuda")
    value = arcs / (t_ms / 1e3) / 1e9
    stats = G.stats()

    # e2e: the same solves through the C ABI with pinned HOST output buffers
    hd = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
    hp = torch.empty(g.n, dtype=torch.int32, pin_memory=True)
    for i in range(2):
        G.solve(src_at(i), hd, hp, None, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_arcs = 0
    for i in range(args.steps):
        s = src_at(args.warmup + i)
        G.solve(s, hd, hp, None, stream)
        e2e_arcs += mr[s]
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_value = e2e_arcs / e2e_s / 1e9 * ws

    # L2 residency from the device's own L2 size: the CSR streamed from HBM,
    # the distance words (8 B per layout vertex with predecessors) re-used
    l2_bytes = int(torch.cuda.get_device_properties(local).L2_cache_size)
    csr_bytes = 8 * g.m + 4 * (g.n + 1)
    dist_bytes = 8 * G.features()["shadows"] + 8 * g.n
    l2_note = (f"inputs larger than L2 (CSR {csr_bytes / 1e9:.2f} GB > L2 {l2_bytes / 2**20:.0f} MiB), no flush"
               if csr_bytes > l2_bytes else f"CSR {csr_bytes / 1e6:.0f} MB fits in L2 ({l2_bytes / 2**20:.0f} MiB)")
    l2_res = {"l2_bytes": l2_bytes, "csr_bytes": csr_bytes, "dist_bytes": dist_bytes,
              "csr_fits": csr_bytes <= l2_bytes, "dist_fits": dist_bytes <= l2_bytes}

    peaks = measured_peaks()
    # roofline of the relaxation kernel: algorithmic bytes per launch / kernel time
    alg_bytes = (BYTES_PER_ARC * arcs + BYTES_PER_VERTEX * verts) / (args.steps * ws)
    kms = float(np.mean(kernel_ms))
    achieved = alg_bytes / (kms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": profiled_traffic(config_signature(tuned)),
            "peak_source": peaks["source"], "kernel": "mlmq_kernel", "kernel_ms_mean": round(kms, 4),
            "alg_bytes_per_launch": int(alg_bytes)}

    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GTEPS", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} single-source (R-MAT scale 22, ef 16, a/b/c/d .57/.19/.19/.05, "
                               "u32 [1,255], symmetrised, dedup); 64 giant-component sources, each solved alone",
                   "n": g.n, "m": g.m, "giant": giant, "l2_flush": l2_note,
                   "l2_residency": l2_res,
                   "queue": {k: v for k, v in tuned.as_dict().items()
                             if k in ("l1_type", "l2_type", "delta_u32", "bnum", "bmax", "wb", "claim", "shards",
                                      "filter_deltas", "th_heavy", "block_threads", "split_arcs",
                                      "hub_bnum", "direct_buckets")},
                   "parallelism": f"replicas x{ws}"},
        "e2e": {"value": round(e2e_value, 3), "unit": "GTEPS", "h2d_bytes_per_step": 4,
                "d2h_bytes_per_step": 8 * g.n},
        # per solve: distance fill, [pending-mark fill], seed, relaxation, unpack
        "gpu_launches": (4 + int(tuned.pending_marks)) * args.steps,
        "roofline": roof,
        "clocks": clk.summary(),
        "per_source": {"kernel_ms": percentiles(kernel_ms),
                       "gteps": percentiles([a / (k / 1e3) / 1e9 for a, k in zip(step_arcs, kernel_ms) if k > 0])},
        "work": {"relaxed_arcs_per_reached_arc": round(relaxed / max(1, arcs / ws), 3),
                 "per_solve_mean": {k: int(v / args.steps) for k, v in work_sum.items()},
                 "warp_cycle_split": {k: round(float(c / max(1.0, cyc_sum.sum())), 3)
                                      for k, c in zip(S.sssp_stats.CYCLE_NAMES, cyc_sum)},
                 "cas_fail_per_refill": round(work_sum["cas_fail"] / max(1, work_sum["refills"]), 2),
                 "grid_blocks": stats["grid_blocks"], "block_threads": stats["block_threads"]},
    }
    legs = set() if args.no_extras else {x for x in args.legs.split(",") if x}
    if rank == 0 and "cpu" in legs:
        # the oracle timed on this host's cores on a bounded sample of the same workload
        cores = max(1, min(16, os.cpu_count() or 1))
        sample = [int(s) for s in srcs_all[:cores]]
        cg, cdt, _ = cpu_oracle_gteps(g, sample, cores)
        # one query alone on one core (nothing else running), for a few sources
        single = []
        for s in srcs_all[:3]:
            _, dt1, _ = cpu_oracle_gteps(g, [int(s)], 1)
            single.append(dt1)
        line["cpu_baseline"] = {"value": round(cg, 4), "unit": "GTEPS", "cores": cores, "kind": "oracle",
                                "sample": f"{cores} single-source Dijkstra runs on {args.workload}, "
                                          f"one per thread, all at once ({cdt:.1f} s)",
                                "single_thread_s_per_query": {"p50": round(float(np.median(single)), 3),
                                                              "max": round(float(np.max(single)), 3),
                                                              "sample": f"{len(single)} sources, one at a time "
                                                                        "on one core"},
                                "all_core_s_per_query": round(cdt / cores, 3), "cpu_model": cpu_model()}
    if rank == 0 and "batch" in legs:
        line["batch"] = [batch_leg(S, gg, torch, "u32"), batch_leg(S, gg, torch, "f32")]
    if rank == 0 and "bfs" in legs:
        line["bfs"] = bfs_leg(S, G, g, srcs_all, torch)
    if rank == 0 and "road" in legs:
        line["road"] = road_leg(S, gg, torch)
    if rank == 0 and "queues" in legs:
        line["queues"] = queues_leg(S, gg, torch)
    if rank == 0 and "serving" in legs:
        cache = {}
        if args.workload in SERVE_GRAPHS:
            cache[args.workload] = (g, G, gg.giant_sources(g, 4096, seed=2)[0])
        rates = [float(r) for r in args.serve_rates.split(",") if r]
        line["serving"] = serve_leg(S, gg, torch, rates, args.serve_seconds, args.serve_max, cache)
        for name, (_, Gc, _) in cache.items():
            if Gc is not G:
                Gc.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    G.close()
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
