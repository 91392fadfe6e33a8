"""GPU parity of the lower-triangular-T variant (the m < n form of Sec. 3:
Algorithm 1 on A^T, returned as U = V', T = T'^T, V = U') against the
oracle's `corutv_lower` on the same seeded inputs, through the C ABI: the
FP64 path within 1e-12 in relative reconstruction error, the mixed paths
within their precision's budget, T exactly lower triangular, and the
single-pass core and the serving path on the same variant."""

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1906_04572_gb300 import Context, corutv

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def ctx():
    from paper_1906_04572_gb300 import build
    build.build()
    oracle.build()
    c = Context(0)
    yield c
    c.close()


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _approx(o):
    return o["U"] @ o["T"] @ o["V"].T


def _case(m, n, seed):
    return synth.spectrum_matrix(m, n, 0.9 ** np.arange(min(m, n)), 1e-9, seed)


@pytest.mark.parametrize("m,n,k,p,q", [(211, 333, 12, 5, 2), (129, 4100, 60, 4, 1), (500, 700, 20, 6, 0),
                                       (333, 211, 12, 5, 1)])
def test_lower_f64_matches_oracle(ctx, m, n, k, p, q):
    a = _case(m, n, m + 3 * n)
    ell = k + p
    psi = synth.gaussian_psi(m, ell, seed=4)  # the test matrix of A^T: m x ell
    ref = oracle.corutv_lower(a, k, p, q, psi)
    out = ctx.factor(dev(a), k, p, q, "f64", psi=dev(psi), t_lower=1)
    assert ctx.sync() == 0
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    assert got["U"].shape == (m, ell) and got["V"].shape == (n, ell)
    na = np.linalg.norm(a)
    e_gpu = np.linalg.norm(a - _approx(got)) / na
    e_or = np.linalg.norm(a - _approx(ref)) / na
    assert abs(e_gpu - e_or) <= 1e-12
    assert np.linalg.norm(_approx(got) - _approx(ref)) / na <= 1e-12
    assert np.all(np.triu(got["T"], 1) == 0) and np.all(np.diag(got["T"]) >= 0)
    assert np.linalg.norm(got["U"].T @ got["U"] - np.eye(ell)) < 1e-12
    assert np.linalg.norm(got["V"].T @ got["V"] - np.eye(ell)) < 1e-12
    sv_o = np.linalg.svd(ref["T"], compute_uv=False)
    if np.array_equal(host(out["perm"]).astype(np.int32), ref["perm"]):
        assert np.abs(got["T"] - ref["T"]).max() <= 1e-11 * sv_o[0]
        # U = (Q2 of the run on A^T) P: the permutation acts on U's columns
        assert np.abs(got["U"] - ref["U"]).max() <= 1e-10


@pytest.mark.parametrize("prec", ["bf16", "tf32", "f32"])
def test_lower_mixed_error_budget(ctx, prec):
    m, n, k, p, q = 1500, 2000, 40, 10, 1
    a = synth.spectrum_matrix(m, n, np.arange(1, m + 1) ** -1.5, 0.0, 91)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    psi = synth.gaussian_psi(m, k + p, seed=22)
    ref = oracle.corutv_lower(a64, k, p, q, psi)
    out = ctx.factor(dev(a32, torch.float32), k, p, q, prec, psi=dev(psi), t_lower=1)
    assert ctx.sync() == 0
    u, t, v = (host(out[x]) for x in ("U", "T", "V"))
    assert np.all(np.triu(t, 1) == 0)
    na = np.linalg.norm(a64)
    e_gpu = np.linalg.norm(a64 - u @ t @ v.T) / na
    e_or = np.linalg.norm(a64 - _approx(ref)) / na
    unit = {"bf16": 2.0 ** -8, "tf32": 2.0 ** -10, "f32": 64 * U32}[prec]
    budget = 4 * unit * np.sqrt(k + p) * np.linalg.norm(a64, 2) / na
    assert e_gpu <= e_or + budget, (e_gpu, e_or, budget)
    assert np.linalg.norm(u.T @ u - np.eye(k + p)) < 1e-5
    assert np.linalg.norm(v.T @ v - np.eye(k + p)) < 1e-5


def test_lower_single_pass_core(ctx):
    """d_mode 1 with the lower variant: D_approx of the run on A^T (= R2^T
    there), compared with the oracle's single-pass core on A^T."""
    m, n, k, p, q = 450, 600, 8, 8, 2
    a = _case(m, n, 5)
    psi = synth.gaussian_psi(m, k + p, seed=6)
    ref = oracle.corutv_dapprox(np.ascontiguousarray(a.T), k, p, q, psi)
    out = ctx.factor(dev(a), k, p, q, "f64", psi=dev(psi), d_mode=1, t_lower=1)
    assert ctx.sync() == 0
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    ref_a = ref["V"] @ ref["T"].T @ ref["U"].T
    na = np.linalg.norm(a)
    assert np.linalg.norm(got["U"] @ got["T"] @ got["V"].T - ref_a) / na <= 1e-12
    assert np.all(np.triu(got["T"], 1) == 0)


def test_lower_serving_equals_direct_call(ctx):
    """The same request through submit/poll gives the direct call's factorisation."""
    m, n, k, p, q = 300, 520, 10, 6, 1
    a = _case(m, n, 8)
    ell = k + p
    A = dev(a)
    direct = ctx.factor(A, k, p, q, "f64", seed=3, t_lower=1)
    assert ctx.sync() == 0
    U = torch.empty((m, ell), dtype=torch.float64, device="cuda")
    T = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
    V = torch.empty((n, ell), dtype=torch.float64, device="cuda")
    perm = torch.empty(ell, dtype=torch.int32, device="cuda")
    rq = corutv.make_request(A, k, p, q, "f64", U, T, V, perm, seed=3, t_lower=1)
    ticket = corutv.corutv_submit(ctx.handle, rq)
    st, _ = corutv.corutv_poll(ctx.handle, ticket, timeout_us=30_000_000)
    assert st == corutv.OK
    got = {"U": host(U), "T": host(T), "V": host(V)}
    ref = {x: host(direct[x]) for x in ("U", "T", "V")}
    assert np.linalg.norm(_approx(got) - _approx(ref)) / np.linalg.norm(_approx(ref)) < 1e-13
    assert np.all(np.triu(got["T"], 1) == 0)


def test_lower_rejects_unknown_value(ctx):
    a = dev(_case(100, 150, 1))
    with pytest.raises(corutv.CorutvError):
        ctx.factor(a, 5, 5, 0, "f64", t_lower=2)
