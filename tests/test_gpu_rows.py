"""The row-partitioned factorisation (corutv_factor_rows): two processes on
the one GPU each hold half of A's rows and exchange the row sums (the Gram
matrices of the thin QRs of C1, C2 = sum A_i^T Q1_i, D = sum Q1_i^T A_i Q2)
over gloo on the host. No kernel waits on another rank: only the host
callback blocks. The stacked U, and T, V, perm, agree with one corutv_factor
call on the whole matrix with the same Psi: to FP64 rounding on the FP64 path
(only the order of the rows' sums differs), within the precision's budget on
the FP32 / tensor-core paths."""

import os
import socket
import sys

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, a, k, p, q, prec, queue):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist

    from paper_1906_04572_gb300 import Context, corutv
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m, n = a.shape
    rows = np.array_split(np.arange(m), world)[rank]
    tdt = torch.float64 if a.dtype == np.float64 else torch.float32
    a_i = torch.from_numpy(np.ascontiguousarray(a[rows])).to("cuda", tdt)
    ell = k + p
    U = torch.empty((len(rows), ell), device="cuda", dtype=tdt)
    T = torch.empty((ell, ell), device="cuda", dtype=tdt)
    V = torch.empty((n, ell), device="cuda", dtype=tdt)
    perm = torch.empty(ell, device="cuda", dtype=torch.int32)
    cb = corutv.allreduce_callback(corutv.torch_distributed_sum)
    with Context(0) as ctx:
        corutv.corutv_factor_rows(ctx.handle, a_i, m, k, p, q, prec, cb, U, T, V, perm, seed=5, stream=2)
        assert ctx.sync() == 0
        torch.cuda.synchronize()
        queue.put((rank, U.cpu().double().numpy(), T.cpu().double().numpy(), V.cpu().double().numpy(),
                   perm.cpu().numpy()))
    dist.destroy_process_group()


def _run_two(a, k, p, q, prec):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    port = _free_port()
    qu = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, a, k, p, q, prec, qu)) for r in range(2)]
    for pr in procs:
        pr.start()
    got = {}
    try:
        for _ in procs:
            r, u, t, v, perm = qu.get(timeout=300)
            got[r] = (u, t, v, perm)
    finally:
        for pr in procs:
            pr.join(timeout=60)
            if pr.is_alive():
                pr.kill()
    assert all(pr.exitcode == 0 for pr in procs)
    return got


@pytest.mark.parametrize("prec,dtype,tol", [("f64", np.float64, 1e-12), ("f32", np.float32, None),
                                            ("bf16", np.float32, None)])
def test_rows_on_two_ranks_equal_the_single_call(prec, dtype, tol):
    import torch

    from paper_1906_04572_gb300 import Context
    m, n, k, p, q = 900, 700, 20, 10, 2
    a = synth.spectrum_matrix(m, n, np.arange(1, min(m, n) + 1) ** -1.5, 1e-6, 61).astype(dtype)
    got = _run_two(a, k, p, q, prec)
    with Context(0) as c:
        ref = c.factor(torch.from_numpy(a).cuda(), k, p, q, prec, seed=5, stream=2)
        torch.cuda.synchronize()
        ref = {x: ref[x].cpu().double().numpy() for x in ("U", "T", "V", "perm")}
    u = np.vstack([got[0][0], got[1][0]])
    t0, v0, perm0 = got[0][1], got[0][2], got[0][3]
    # T, V, perm are replicated: bitwise the same on both ranks
    assert np.array_equal(t0, got[1][1]) and np.array_equal(v0, got[1][2]) and np.array_equal(perm0, got[1][3])
    a64 = a.astype(np.float64)
    na = np.linalg.norm(a64)
    approx, ref_approx = u @ t0 @ v0.T, ref["U"] @ ref["T"] @ ref["V"].T
    e_rows = np.linalg.norm(a64 - approx) / na
    e_ref = np.linalg.norm(a64 - ref_approx) / na
    ell = k + p
    if tol is not None:
        assert np.linalg.norm(approx - ref_approx) / na <= tol
        assert np.array_equal(perm0, ref["perm"].astype(np.int32))
        assert np.abs(t0 - ref["T"]).max() <= 1e-11 * np.abs(ref["T"]).max()
    else:
        u_p = 2.0 ** -24 if prec == "f32" else 2.0 ** -8
        budget = 4 * u_p * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
        assert abs(e_rows - e_ref) <= budget, (e_rows, e_ref, budget)
    assert np.linalg.norm(u.T @ u - np.eye(ell)) < (1e-12 if prec == "f64" else 1e-5)
    assert np.all(np.tril(t0, -1) == 0)
