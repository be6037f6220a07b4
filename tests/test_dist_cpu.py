"""The multi-rank plumbing of bench.py (one process per GPU, weak-scaling replicas) on CPU:
two gloo ranks, no GPU.  Each rank gets its own seeded replica of the workload, the job time is
the max over ranks, and the job value counts the units of every rank."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    op = bench.rank_workload("small-2d", rank)
    ms = 10.0 + 5.0 * rank                       # the slower rank must time the job
    job_ms = bench.max_over_ranks(ms, torch.device("cpu"), world)
    value = bench.job_value(world, 1000, job_ms)
    checksum = float(np.abs(op.u).sum() + np.abs(op.v).sum())
    got = [None] * world
    dist.all_gather_object(got, (rank, job_ms, value, checksum))
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        out.put(got)


def test_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = q.get(timeout=240)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    got = sorted(got)
    assert [g[0] for g in got] == [0, 1]
    assert all(g[1] == 15.0 for g in got)                     # max over ranks, on every rank
    assert all(abs(g[2] - 2 * 1000 / 15e-3) < 1e-6 * g[2] for g in got)
    assert got[0][3] != got[1][3]                              # independent replicas


def test_single_rank_is_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, 1) == 3.5
    assert bench.job_value(1, 10, 2.0) == 10 / 2e-3
