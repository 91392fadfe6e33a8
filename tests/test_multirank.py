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


def _sum_worker(rank, world, port, queue):
    """The exchange of the row-partitioned factorisation as the library drives
    it: a corutv_allreduce_fn built by the binding is called on a host buffer
    (the way the library calls it) on each of two gloo ranks."""
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import ctypes

    import torch.distributed as dist

    from paper_1906_04572_gb300 import corutv
    dist.init_process_group("gloo", rank=rank, world_size=world)
    cb = corutv.allreduce_callback(corutv.torch_distributed_sum)
    out = []
    for dtype, code in ((np.float64, corutv.F64), (np.float32, corutv.F32)):
        buf = (np.arange(37, dtype=dtype) + 1000 * rank).copy()
        st = cb(ctypes.c_void_p(buf.ctypes.data), buf.size, code, None)
        out.append((st, buf.copy()))
    # a failing sum is reported as a status, not raised through the C caller
    bad = corutv.allreduce_callback(lambda a: (_ for _ in ()).throw(RuntimeError("lost rank")))
    st_bad = bad(ctypes.c_void_p(np.zeros(4).ctypes.data), 4, corutv.F64, None)
    dist.destroy_process_group()
    queue.put((rank, out, st_bad))


def test_row_partition_exchange_sums_over_two_ranks():
    import multiprocessing as mp
    from paper_1906_04572_gb300 import corutv
    ctx = mp.get_context("spawn")
    port = _free_port()
    q = ctx.Queue()
    procs = [ctx.Process(target=_sum_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (o, b)) for r, o, b in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    for r in range(2):
        out, st_bad = res[r]
        for (st, buf), dtype in zip(out, (np.float64, np.float32)):
            assert st == corutv.OK
            want = 2 * np.arange(37, dtype=dtype) + 1000
            assert np.array_equal(buf, want)
        assert st_bad != corutv.OK
