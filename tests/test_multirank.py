"""The multi-GPU path of bench.py is replicas only: every rank runs its own
problem and the job combines the ranks' times and work.  These tests run that
logic as world-size-2 gloo process groups on the CPU."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: device time 1 + r, host time 2 + 3 r, work 100 (r + 1)
        res = bench.combine_ranks(1.0 + rank, 2.0 + 3 * rank, 100 * (rank + 1), world, device="cpu")
        dist.barrier()
        out[rank] = res
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_work_the_sum():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(world):
        assert out[r] == (2.0, 5.0, 300.0)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(1.5, 2.5, 7, 1, device="cpu") == (1.5, 2.5, 7.0)


def test_replicas_are_independent_problems():
    sys.path.insert(0, ROOT)
    import bench
    (c0, i0), (c1, i1) = bench.replica(0), bench.replica(1)
    assert c0.seed != c1.seed and i0 != i1
    assert (c0.nx, c0.ny, c0.n_particles, c0.n_obs) == (c1.nx, c1.ny, c1.n_particles, c1.n_obs) == \
        (1024, 1024, 1000, 1521)
