"""bench.py's multi-rank bookkeeping on CPU with two gloo ranks: the whole-job
time is the slowest rank's, work counts add up, and rank 0 reports them."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    times = [10.0 + rank, 20.0 - rank]
    counts = [100.0 * (rank + 1), 7.0]
    out = bench.combine_ranks(times, counts, world, torch.device("cpu"))
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        assert res[r] == [11.0, 20.0, 300.0, 14.0]


def test_combine_ranks_single_process_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks([3.0], [5.0], 1, torch.device("cpu")) == [3.0, 5.0]
