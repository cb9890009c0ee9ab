"""The multi-rank (replicas) aggregation of bench.py, run as two gloo ranks
on the CPU: every rank gets the slowest rank's time and the whole-job rate."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow replica
    t_max, value = bench.aggregate_ranks(torch, dist, local_ms, 10, 1000, world, "cpu")
    q.put((rank, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, value in got:
        assert t_max == 150.0
        # 2 ranks x 10 steps x 1000 units in 150 ms
        assert abs(value - 2 * 10 * 1000 / 0.150) < 1e-6


def test_single_rank_aggregation():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    t_max, value = bench.aggregate_ranks(torch, None, 200.0, 4, 500, 1, "cpu")
    assert t_max == 200.0 and abs(value - 4 * 500 / 0.2) < 1e-9
