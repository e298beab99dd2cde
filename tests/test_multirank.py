"""The multi-rank host logic of bench.py on CPU: two gloo ranks shard the
sources without overlap and combine the slowest rank's time with the sum of
the work (weak scaling, no collective on the data path)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, srcs, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = bench.rank_sources(srcs, rank, ws)
        # rank r "took" 10 + r ms and processed 100 * (r + 1) arcs, 10 * (r + 1) vertices
        t, a, v = bench.combine_over_ranks(10.0 + rank, 100 * (rank + 1), 10 * (rank + 1), "cpu")
        q.put((rank, mine, t, a, v))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2])
def test_two_gloo_ranks_shard_and_combine(ws):
    srcs = list(range(100, 164))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, srcs, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out.sort()
    shares = [set(o[1]) for o in out]
    assert shares[0].isdisjoint(shares[1])
    assert shares[0] | shares[1] == set(srcs)
    for _, _, t, a, v in out:
        assert t == 10.0 + (ws - 1)          # the slowest rank
        assert a == sum(100 * (r + 1) for r in range(ws))
        assert v == sum(10 * (r + 1) for r in range(ws))


def test_single_rank_is_identity():
    assert bench.rank_sources([5, 6, 7], 0, 1) == [5, 6, 7]
    assert bench.combine_over_ranks(3.5, 7, 2, "cpu") == (3.5, 7, 2)
