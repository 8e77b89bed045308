"""The multi-GPU bench path on CPU: two gloo ranks, each with its own
walker batch and step time; the job's throughput is all walkers over the
slowest rank's time (walkers are independent: no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t_local = 100.0 + 50.0 * rank           # rank 1 is the slow one
    t, v = bench.aggregate(t_local, 2048, world, dist, torch.device("cpu"))
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_rank_aggregate_is_weak_scaling_max_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 150.0
        assert abs(v - world * 2048 / 0.150) < 1e-6


def test_single_rank_aggregate():
    import bench
    t, v = bench.aggregate(200.0, 100, 1)
    assert t == 200.0 and abs(v - 500.0) < 1e-9
