"""The multi-GPU path is replicas only: every rank solves its own problems
and the job's figures are the slowest rank's time and the summed work. This
checks that bookkeeping with two gloo ranks on CPU (no GPU involved)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    sec, work = bench.reduce_over_ranks(1.0 + rank, 100 * (rank + 1))
    out[rank] = (sec, work)
    dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        for r in range(world):
            assert out[r] == (2.0, 300.0)


def test_reduce_over_ranks_single_process():
    import bench
    assert bench.reduce_over_ranks(3.5, 7) == (3.5, 7.0)
