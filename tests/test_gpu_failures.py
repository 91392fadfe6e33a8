"""Failure detection, driven from the host: admission over budget, queueing
until memory frees, polling an unfinished request, and a device wait that
runs out. Nothing here faults, traps or hangs the GPU: the over-budget cases
are refused before any work is enqueued, and the device wait is bounded by a
limit the test sets (a barrier nothing arrives on), after which the kernel
frees its tensor memory and reports CORUTV_ETIMEDOUT."""

import numpy as np
import pytest
import torch

import synth
from paper_1906_04572_gb300 import Context, corutv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1906_04572_gb300 import build
    build.build()


def _mat(m, n, seed, dtype=torch.float32):
    a = synth.spectrum_matrix(m, n, np.arange(1, min(m, n) + 1) ** -1.5, 0.0, seed)
    return torch.from_numpy(a).to("cuda", dtype)


def _outs(m, n, ell, dtype=torch.float32):
    return (torch.empty((m, ell), device="cuda", dtype=dtype), torch.empty((ell, ell), device="cuda", dtype=dtype),
            torch.empty((n, ell), device="cuda", dtype=dtype))


def test_submit_over_budget_is_refused():
    with Context(0, mem_budget_bytes=1 << 20) as c:
        a = _mat(1024, 1024, 1)
        u, t, v = _outs(1024, 1024, 30)
        req = corutv.make_request(a, 20, 10, 1, "bf16", u, t, v)
        with pytest.raises(corutv.CorutvError) as ei:
            corutv.corutv_submit(c.handle, req)
        assert ei.value.status == corutv.ENOMEM


def test_factor_over_budget_is_refused():
    with Context(0, mem_budget_bytes=1 << 20) as c:
        a = _mat(1024, 1024, 2)
        with pytest.raises(corutv.CorutvError) as ei:
            c.factor(a, 20, 10, 1, "bf16")
        assert ei.value.status == corutv.ENOMEM
        # a problem that fits still runs on the same context
        small = _mat(128, 96, 3)
        out = c.factor(small, 4, 4, 0, "f32")
        assert c.sync() == 0
        assert torch.isfinite(out["T"]).all()


def test_requests_queue_until_memory_frees():
    """A budget that holds one request's workspace but not two: the requests
    are admitted one after another as memory frees up, and each result equals
    the direct call's."""
    m, n, k, p, q = 1024, 768, 20, 10, 1
    mats = [_mat(m, n, 10 + i) for i in range(3)]
    with Context(0) as ref_ctx:
        refs = []
        for a in mats:
            o = ref_ctx.factor(a, k, p, q, "bf16", seed=5)
            torch.cuda.synchronize()
            refs.append({x: o[x].cpu().numpy() for x in ("U", "T", "V")})
    # the workspace one request needs, from a context that admitted one alone
    one = None
    for budget in (8 << 20, 16 << 20, 32 << 20, 64 << 20, 128 << 20):
        with Context(0, mem_budget_bytes=budget) as c:
            u, t, v = _outs(m, n, k + p)
            try:
                tk = corutv.corutv_submit(c.handle, corutv.make_request(mats[0], k, p, q, "bf16", u, t, v, seed=5))
            except corutv.CorutvError as e:
                assert e.status == corutv.ENOMEM
                continue
            assert corutv.corutv_poll(c.handle, tk, timeout_us=60_000_000)[0] == corutv.OK
            one = budget
            break
    assert one is not None
    with Context(0, mem_budget_bytes=one, max_slots=4) as c:
        bufs, tickets = [], []
        for a in mats:
            u, t, v = _outs(m, n, k + p)
            bufs.append((u, t, v))
            tickets.append(corutv.corutv_submit(c.handle, corutv.make_request(a, k, p, q, "bf16", u, t, v, seed=5)))
        for tk in tickets:
            assert corutv.corutv_poll(c.handle, tk, timeout_us=120_000_000)[0] == corutv.OK
        torch.cuda.synchronize()
        for (u, t, v), r in zip(bufs, refs):
            assert np.array_equal(u.cpu().numpy(), r["U"])
            assert np.array_equal(t.cpu().numpy(), r["T"])
            assert np.array_equal(v.cpu().numpy(), r["V"])


def test_poll_pending_and_timed_out_then_done():
    """A long FP64 request: polling without waiting says EPENDING, polling
    with a short timeout says ETIMEDOUT, waiting returns its result."""
    m = n = 4096
    with Context(0) as c:
        a = _mat(m, n, 20, torch.float64)
        u, t, v = _outs(m, n, 74, torch.float64)
        torch.cuda.synchronize()
        tk = corutv.corutv_submit(c.handle, corutv.make_request(a, 64, 10, 2, "f64", u, t, v))
        st0, _ = corutv.corutv_poll(c.handle, tk, timeout_us=0)
        st1, _ = corutv.corutv_poll(c.handle, tk, timeout_us=1000)
        st2, lat = corutv.corutv_poll(c.handle, tk, timeout_us=300_000_000)
        assert st0 == corutv.EPENDING
        assert st1 == corutv.ETIMEDOUT
        assert st2 == corutv.OK and lat > 0
        torch.cuda.synchronize()
        assert torch.isfinite(t).all()
        with pytest.raises(corutv.CorutvError) as ei:
            corutv.corutv_poll(c.handle, tk, timeout_us=0)  # a finished ticket is forgotten
        assert ei.value.status == corutv.EINVAL


def test_device_wait_runs_out_and_the_context_stays_usable():
    """A kernel holding tensor memory waits on a barrier nothing arrives on:
    after the test's 2 ms limit it reports the timeout and frees the tensor
    memory; a tensor-core factorisation (which allocates tensor memory in
    every block) then runs normally on the same context."""
    with Context(0) as c:
        corutv.corutv_selftest_wait(c.handle, 2_000_000)
        with pytest.raises(corutv.CorutvError) as ei:
            c.sync()
        assert ei.value.status == corutv.ETIMEDOUT
        assert c.sync() == 0  # the status was reported once and cleared
        a = _mat(900, 700, 30)
        out = c.factor(a, 20, 10, 1, "bf16")
        assert c.sync() == 0
        torch.cuda.synchronize()
    # bitwise the result of the same call on a context that never timed out
    with Context(0) as fresh:
        ref = fresh.factor(a, 20, 10, 1, "bf16")
        torch.cuda.synchronize()
    for x in ("U", "T", "V", "perm"):
        assert torch.equal(out[x], ref[x]), x
