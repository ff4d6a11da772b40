"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): each rank takes distinct
minibatches at every step, and the reported time is the max over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = (bench.rank_batches(rank, world, 3, 10, 8), bench.max_over_ranks(1.5 + rank))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_distinct_minibatches_and_max_time():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    b0, t0 = res[0]
    b1, t1 = res[1]
    assert t0 == t1 == 2.5
    assert all(x != y for x, y in zip(b0, b1))
    assert set(b0) | set(b1) == set(range(8))
    import bench
    assert bench.rank_batches(0, 1, 0, 3, 8) == [0, 1, 2]
    assert bench.max_over_ranks(4.0) == 4.0
