"""The N > 1 path of bench.py on the CPU: two gloo ranks, each a replica,
agree on the slowest rank's time and report all ranks' updates over it."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [12.5, 17.25][rank]
    ms = bench._max_over_ranks(local_ms, world, torch.device("cpu"))
    out[rank] = (ms, bench._job_mlups(world, 1000, 10, ms * 1e-3))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        ms, mlups = out[r]
        assert ms == 17.25
        assert mlups == pytest.approx(2 * 1000 * 10 / 17.25e-3 / 1e6)
