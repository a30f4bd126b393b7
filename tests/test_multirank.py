"""The N > 1 bench path on CPU ranks (gloo, world size 2): independent replicas with distinct data,
the slowest rank's time as the run's time, the reference arm running on rank 0 only."""
import os
import socket
import sys

import numpy as np
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
        slow = bench.max_over_ranks(1.5 + rank, dist, device="cpu")
        wl, pr, th = bench.make_problem(seed_offset=bench.replica_seed(rank))
        # the reference arm prints and times on rank 0 only; other ranks leave at once
        class A:
            steps = 0
        ref = bench.run_reference(A, rank, world) if rank == 1 else 0
        out.put((rank, slow, float(pr.X[:4].sum()), pr.X.shape, pr.p, ref))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replicas_and_max_over_ranks_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=240) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, slow0, x0, shape0, p0, _), (r1, slow1, x1, shape1, p1, ref1) = res
    assert slow0 == slow1 == 2.5                  # every rank reports the slowest rank's time
    assert shape0 == shape1 and p0 == p1          # same workload shape on every replica
    assert x0 != x1                               # ... with its own points (weak scaling)
    assert ref1 == 0


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_seed(0) == 0 and bench.replica_seed(3) != bench.replica_seed(2)
