"""Bitwise reproducibility of the factorisation (Algorithm 1) through the C
ABI: the same A and Psi give the same U, T, V, perm whatever the pointer kind
(host or device), the torch stream the call is enqueued on, and the calls
that came before -- 50 factorisations in a row per precision. Every sum on the
path has a fixed order (split-K partials and stream-K pieces added in index
order, cluster reductions in rank order), so nothing may differ."""

import numpy as np
import pytest
import torch

import synth
from paper_1906_04572_gb300 import Context, corutv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1906_04572_gb300 import build
    build.build()
    c = Context(0)
    yield c
    c.close()


def _run_device(ctx, a, psi, k, p, q, prec, stream):
    with torch.cuda.stream(stream):
        out = ctx.factor(a, k, p, q, prec, psi=psi)
    torch.cuda.synchronize()
    return tuple(out[x].cpu().numpy().copy() for x in ("U", "T", "V", "perm"))


def _run_host(ctx, a_np, psi_np, k, p, q, prec):
    m, n = a_np.shape
    ell = k + p
    u = np.empty((m, ell), dtype=a_np.dtype)
    t = np.empty((ell, ell), dtype=a_np.dtype)
    v = np.empty((n, ell), dtype=a_np.dtype)
    perm = np.empty(ell, dtype=np.int32)
    corutv.corutv_factor(ctx.handle, a_np, k, p, q, prec, u, t, v, perm, psi=psi_np)
    return u, t, v, perm


@pytest.mark.parametrize("prec,dtype", [("f64", np.float64), ("bf16", np.float32), ("tf32", np.float32)])
def test_fifty_factorisations_bitwise_equal(ctx, prec, dtype):
    m, n, k, p, q = 700, 520, 24, 8, 2
    a_np = synth.spectrum_matrix(m, n, np.arange(1, min(m, n) + 1) ** -1.5, 1e-6, 31).astype(dtype)
    psi_np = synth.gaussian_psi(n, k + p, seed=32)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    a = torch.from_numpy(a_np).to("cuda", tdt)
    psi = torch.from_numpy(psi_np).to("cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    default = torch.cuda.current_stream()
    ref = _run_device(ctx, a, psi, k, p, q, prec, default)
    for i in range(50):
        mode = i % 4
        if mode == 3:
            got = _run_host(ctx, a_np, psi_np, k, p, q, prec)
        else:
            got = _run_device(ctx, a, psi, k, p, q, prec, (s1, s2, default)[mode])
        for name, g, r in zip(("U", "T", "V", "perm"), got, ref):
            assert np.array_equal(g, r), f"run {i} (mode {mode}): {name} differs"
    assert ctx.sync() == 0


def test_calls_on_alternating_streams_do_not_overlap(ctx):
    """Calls queued back to back on two streams with no host synchronisation
    in between: each waits for the previous one (the workspace is shared), so
    all results equal the result of a lone call."""
    m, n, k, p, q = 900, 800, 30, 10, 1
    a_np = synth.spectrum_matrix(m, n, np.arange(1, min(m, n) + 1) ** -1.0, 0.0, 5).astype(np.float32)
    psi_np = synth.gaussian_psi(n, k + p, seed=6)
    a = torch.from_numpy(a_np).cuda()
    psi = torch.from_numpy(psi_np).cuda()
    ref = _run_device(ctx, a, psi, k, p, q, "bf16", torch.cuda.current_stream())
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for i in range(12):
        with torch.cuda.stream(streams[i % 2]):
            outs.append(ctx.factor(a, k, p, q, "bf16", psi=psi))
    torch.cuda.synchronize()
    for i, o in enumerate(outs):
        for name, r in zip(("U", "T", "V", "perm"), ref):
            assert np.array_equal(o[name].cpu().numpy(), r), f"call {i}: {name} differs"


def test_submit_waits_for_the_producer_of_a(ctx):
    """A is still being produced on the caller's stream (a large matrix
    product queued just before) when the request is submitted: the request
    waits for it on the device, without any host synchronisation."""
    m, n, k, p, q = 2048, 1536, 20, 10, 1
    u, s, v = synth.spectrum_factors(m, n, np.arange(1, 257) ** -1.5, seed=8)
    us = torch.from_numpy(u * s).cuda().float()
    vt = torch.from_numpy(v).cuda().float().t().contiguous()
    psi = torch.from_numpy(synth.gaussian_psi(n, k + p, seed=9)).cuda()
    torch.cuda.synchronize()
    ref_a = (us @ vt).contiguous()
    ref = _run_device(ctx, ref_a, psi, k, p, q, "bf16", torch.cuda.current_stream())
    side = torch.cuda.Stream()
    ell = k + p
    with torch.cuda.stream(side):
        # slow the producer down: a few large products ahead of A on the same stream
        big = torch.randn(8192, 8192, device="cuda")
        for _ in range(4):
            big = big @ big
            big = big / big.abs().max()
        a = (us @ vt).contiguous()
        U = torch.empty((m, ell), device="cuda")
        T = torch.empty((ell, ell), device="cuda")
        V = torch.empty((n, ell), device="cuda")
        perm = torch.empty(ell, dtype=torch.int32, device="cuda")
        req = corutv.make_request(a, k, p, q, "bf16", U, T, V, perm, psi=psi)
        ticket = corutv.corutv_submit(ctx.handle, req)
    st, _ = corutv.corutv_poll(ctx.handle, ticket, timeout_us=120_000_000)
    assert st == corutv.OK
    torch.cuda.synchronize()
    for name, g, r in zip(("U", "T", "V", "perm"), (U, T, V, perm), ref):
        assert np.array_equal(g.cpu().numpy(), r), f"{name} differs from the synchronous result"
    del big


@pytest.mark.parametrize("prec", ["bf16", "f64"])
def test_graph_replay_is_bitwise_the_direct_call(ctx, prec):
    """With graph replay on, the second occurrence of a call is captured and
    later ones are replayed: every result is bitwise the direct call's, and a
    replay reads the buffers' current contents (A overwritten in place)."""
    m, n, k, p, q = 900, 700, 20, 10, 2
    dtype = torch.float64 if prec == "f64" else torch.float32
    sig = np.arange(1, min(m, n) + 1) ** -1.2
    a1 = torch.from_numpy(synth.spectrum_matrix(m, n, sig, 1e-6, 41)).to("cuda", dtype)
    a2 = torch.from_numpy(synth.spectrum_matrix(m, n, sig, 1e-6, 42)).to("cuda", dtype)
    ell = k + p
    A = a1.clone()
    U = torch.empty((m, ell), device="cuda", dtype=dtype)
    T = torch.empty((ell, ell), device="cuda", dtype=dtype)
    V = torch.empty((n, ell), device="cuda", dtype=dtype)
    perm = torch.empty(ell, device="cuda", dtype=torch.int32)

    def run():
        corutv.corutv_factor(ctx.handle, A, k, p, q, prec, U, T, V, perm, seed=3, stream=0)
        torch.cuda.synchronize()
        return tuple(x.cpu().numpy().copy() for x in (U, T, V, perm))

    refs = []
    for src in (a1, a2):
        A.copy_(src)
        refs.append(run())
    corutv.corutv_set_graphs(ctx.handle, True)
    try:
        for i, src in enumerate((a1, a1, a1, a2, a1, a2)):
            A.copy_(src)
            got = run()
            want = refs[0] if src is a1 else refs[1]
            for name, g, r in zip(("U", "T", "V", "perm"), got, want):
                assert np.array_equal(g, r), f"call {i}: {name} differs"
    finally:
        corutv.corutv_set_graphs(ctx.handle, False)
    assert ctx.sync() == 0
