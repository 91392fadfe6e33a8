"""World-size-2 checks of the multi-rank path on CPU (gloo backend).

The factorisation has no exchange step between independent problems, so the
N > 1 path runs replicas: each rank factorises its own seeded matrix and the
only collectives are the bench's rendezvous, barrier and max-over-ranks time
(the slowest rank sets the reported time). The reference arm runs on rank 0
alone; the other ranks return without work."""

import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, queue):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), BENCH_BACKEND="gloo", BENCH_PG_TIMEOUT="120")
    import torch
    import torch.distributed as dist

    import bench
    w, r, loc = bench.dist_setup()
    assert (w, r, loc) == (world, rank, rank)
    assert bench.dist_setup() == (w, r, loc)  # joining again is a no-op
    bench.barrier(w)
    slowest = bench.max_over_ranks(10.0 + 5.0 * rank, w, torch.device("cpu"))
    f = bench.make_matrix("c1", seed=r)  # the replica this rank would factorise
    digest = float(np.sum(f.a[:8, :8]))

    class Args:
        workload = "c1"
        steps = 1
        warmup = 0

    rc = bench.run_reference(Args) if r != 0 else None  # rank 0 would run the oracle
    queue.put((r, slowest, digest, rc))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_replicas_and_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    queue = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, queue), nprocs=2, join=True, start_method="spawn")
    res = sorted(queue.get() for _ in range(2))
    (r0, s0, d0, _), (r1, s1, d1, rc1) = res
    assert (r0, r1) == (0, 1)
    assert s0 == s1 == 15.0          # every rank reports the slowest rank's time
    assert d0 != d1                  # the ranks factorise different (seeded) matrices
    assert rc1 == 0                  # the reference arm: rank 1 returns at once
