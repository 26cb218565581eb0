"""Multi-rank bookkeeping of bench.py on CPU (gloo, world size 2): the step
time is the max over ranks and the value counts every rank's work (weak
scaling over independent subband sets; the path itself has no exchange)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [10.0, 14.0][rank]
    ops_local = [1e12, 2e12][rank]
    ms, value = bench.aggregate(ms_local, ops_local)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 14.0                               # max over ranks
        assert abs(value - 3e12 / 14e-3 / 1e12) < 1e-9   # all ranks' ops over the max time


def test_aggregate_single_process():
    import bench
    ms, value = bench.aggregate(20.0, 4e12)
    assert ms == 20.0 and abs(value - 200.0) < 1e-9
