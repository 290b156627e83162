"""Replica aggregation of bench.py on two CPU ranks (gloo): the job time is the maximum of the
ranks' timed regions and the work the sum of their bond updates."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms, upd = bench.reduce_over_ranks(100.0 + 50.0 * rank, 172 * (rank + 1), dist, "cpu")
    q.put((rank, ms, upd))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out == [(0, 150.0, 516.0), (1, 150.0, 516.0)]


def test_single_process_has_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(12.5, 7, None, "cpu") == (12.5, 7.0)
