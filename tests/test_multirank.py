"""The N > 1 path of bench.py on the CPU: two gloo ranks, each a replica;
the reported time is the max over ranks and the work the sum."""
import os
import socket

import pytest

torch = pytest.importorskip('torch')
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR='127.0.0.1', MASTER_PORT=str(port))
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    t, u = bench.aggregate(1.0 + rank, 10.0 * (rank + 1), dist)
    out[rank] = (t, u)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (2.0, 30.0)
