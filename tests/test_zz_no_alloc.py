"""The allocation-free thin QR, corutv_orth_noalloc, against corutv_orth.

corutv_orth_noalloc is for callers that cannot allocate device memory: a host
framework that owns all device memory through its own pool, a process that
forbids allocation once it has started, or a plug-in running inside another
library's step. It keeps its temporaries in a fixed 16 MiB device array
instead of allocating. Here it is called through the C ABI several times in a
row on one stream (different sizes, including an ill-conditioned input that
takes the shifted pass), and every result is checked against the existing
entry point corutv_orth with the tolerance the QR parity tests use; sizes
beyond the fixed array must be refused before any work is enqueued.
"""

import numpy as np
import pytest
import torch

import synth
from paper_1906_04572_gb300 import Context, corutv

pytestmark = pytest.mark.gpu


def _panel(rows, ell, cond, seed):
    rng = np.random.default_rng(seed)
    c = (synth.haar(rng, rows, ell) * np.logspace(0, -np.log10(cond), ell)) @ synth.haar(rng, ell, ell).T
    return torch.from_numpy(c).cuda()


def test_noalloc_orth_matches_orth_on_consecutive_calls():
    from paper_1906_04572_gb300 import build
    build.build()
    cases = [(4000, 100, 1e4, 1), (1000, 37, 1e2, 2), (2000, 20, 1e10, 3), (4096, 128, 10.0, 4)]
    with Context(0) as ctx:
        inputs = [_panel(r, l, k, s) for (r, l, k, s) in cases]
        refs = []
        for c in inputs:
            rows, ell = c.shape
            q = torch.empty((rows, ell), dtype=torch.float64, device="cuda")
            r = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
            corutv.corutv_orth(ctx.handle, c, q, r)
            refs.append((q, r))
        assert ctx.sync() == 0
        torch.cuda.synchronize()
        outs = []
        for c in inputs:  # enqueued back to back on the current stream
            rows, ell = c.shape
            q = torch.empty((rows, ell), dtype=torch.float64, device="cuda")
            r = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
            info = torch.full((1,), -1, dtype=torch.int32, device="cuda")
            corutv.corutv_orth_noalloc(c, q, r, info)
            outs.append((q, r, info))
        torch.cuda.synchronize()
    for (rows, ell, cond, _), (q_ref, r_ref), (q, r, info) in zip(cases, refs, outs):
        assert int(info.item()) == 0
        qg, qr_ = q.cpu().numpy(), q_ref.cpu().numpy()
        assert np.linalg.norm(qg.T @ qg - np.eye(ell)) < 1e-13 * max(ell, 10)
        # same tolerance as the QR parity test against the oracle
        assert np.linalg.norm(qg - qr_) < 1e-14 * ell * max(cond, 1e3)
        rg, rr = np.triu(r.cpu().numpy()), np.triu(r_ref.cpu().numpy())
        assert np.linalg.norm(rg - rr) <= 1e-13 * max(cond, 1e3) * np.linalg.norm(rr)


def test_noalloc_orth_refuses_sizes_beyond_its_fixed_scratch():
    c = torch.zeros((5000, 128), dtype=torch.float64, device="cuda")
    q = torch.empty_like(c)
    with pytest.raises(corutv.CorutvError) as ei:
        corutv.corutv_orth_noalloc(c, q)
    assert ei.value.status == corutv.EINVAL
    assert "16 MiB" in str(ei.value)
