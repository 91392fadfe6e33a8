"""Sketch widths 128 < ell <= 320 on the FP64 / FP32 paths (the paper's RPCA
runs at n = 2000 and 3000 use ell = 2k = 200 and 300, Table 1): every step
against the FP64 CPU oracle through the C ABI -- the products (column groups
of at most 128), the thin QR (one-block Cholesky in global memory, R^-1 and a
product for the triangular solve), the pivoted QR of D and its Q, and whole
factorisations -- with the tolerances of the narrow-width parity tests."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1906_04572_gb300 import Context, corutv

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53
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
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def approx_of(o):
    return o["U"] @ o["T"] @ o["V"].T


@pytest.mark.parametrize("m,n,ell", [(700, 500, 200), (333, 450, 320)])
@pytest.mark.parametrize("trans", [0, 1])
def test_sketch_f64_wide_within_rounding_bound(ctx, m, n, ell, trans):
    rng = np.random.default_rng(m + n + ell)
    a = rng.standard_normal((m, n))
    x = rng.standard_normal((m if trans else n, ell))
    c = torch.empty((n if trans else m, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_sketch(ctx.handle, dev(a), dev(x), c, trans, "f64")
    ref = oracle.gemm_aty(a, x) if trans else oracle.gemm_ax(a, x)
    k = m if trans else n
    bound = 2 * k * U64 * ((np.abs(a).T if trans else np.abs(a)) @ np.abs(x))
    assert np.all(np.abs(host(c) - ref) <= bound + 1e-300)


@pytest.mark.parametrize("rows,ell,cond", [(3000, 200, 1e4), (1500, 320, 1e2), (400, 129, 1.0)])
def test_orth_wide_matches_oracle_qr(ctx, rows, ell, cond):
    rng = np.random.default_rng(rows + ell)
    c = (synth.haar(rng, rows, ell) * np.logspace(0, -np.log10(cond), ell)) @ synth.haar(rng, ell, ell).T
    q = torch.empty((rows, ell), dtype=torch.float64, device="cuda")
    r = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_orth(ctx.handle, dev(c), q, r)
    assert ctx.sync() == 0
    qo, ro = oracle.qr(c)
    qg = host(q)
    assert np.linalg.norm(qg.T @ qg - np.eye(ell)) < 50 * ell * U64
    assert np.linalg.norm(qg - qo) < 1e-14 * ell * cond
    assert rel(np.triu(host(r)), ro) < 1e-13 * cond


def test_orth_wide_shift_recovers_ill_conditioned(ctx):
    """kappa ~ 1e10 at ell = 150: the shifted pass and the passes after it
    give an orthonormal Q spanning C."""
    rows, ell = 2000, 150
    rng = np.random.default_rng(6)
    c = (synth.haar(rng, rows, ell) * np.logspace(0, -10, ell)) @ synth.haar(rng, ell, ell).T
    q = torch.empty((rows, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_orth(ctx.handle, dev(c), q)
    assert ctx.sync() == 0
    qg = host(q)
    assert np.linalg.norm(qg.T @ qg - np.eye(ell)) < 1e-12
    assert rel(qg @ (qg.T @ c), c) < 1e-12


@pytest.mark.parametrize("ell", [129, 200, 320])
def test_qrcp_wide_matches_oracle(ctx, ell):
    rng = np.random.default_rng(ell)
    d = rng.standard_normal((ell, ell)) * np.logspace(0, -4, ell)
    qt = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
    rt = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
    perm = torch.empty(ell, dtype=torch.int32, device="cuda")
    corutv.corutv_qrcp(ctx.handle, dev(d), qt, rt, perm)
    qo, ro, po = oracle.qrcp(d)
    assert np.array_equal(host(perm).astype(np.int32), po)
    assert rel(host(rt), ro) < 1e-13
    assert np.linalg.norm(host(qt) - qo) < 1e-12


def test_qrcp_wide_ties_take_lowest_index(ctx):
    """Equal column norms at ell = 160 (columns of a scaled permutation
    matrix): the pivots are the oracle's, lowest index first."""
    ell = 160
    d = np.zeros((ell, ell))
    rng = np.random.default_rng(3)
    rows = rng.permutation(ell)
    for c in range(ell):
        d[rows[c], c] = 2.0 if c % 7 == 0 else 1.0
    qt = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
    rt = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
    perm = torch.empty(ell, dtype=torch.int32, device="cuda")
    corutv.corutv_qrcp(ctx.handle, dev(d), qt, rt, perm)
    assert np.array_equal(host(perm).astype(np.int32), oracle.qrcp(d)[2])


@pytest.mark.parametrize("m,n,k,p,q", [(900, 700, 150, 50, 1), (1100, 1000, 250, 50, 0), (700, 900, 180, 20, 2)])
def test_factor_wide_f64_matches_oracle(ctx, m, n, k, p, q):
    a = synth.spectrum_matrix(m, n, 0.97 ** np.arange(min(m, n)), 1e-9, m + n)
    ell = k + p
    psi = synth.gaussian_psi(n, ell, seed=2)
    ref = oracle.corutv(a, k, p, q, psi)
    out = ctx.factor(dev(a), k, p, q, "f64", psi=dev(psi))
    assert ctx.sync() == 0
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    na = np.linalg.norm(a)
    e_gpu = np.linalg.norm(a - approx_of(got)) / na
    e_or = np.linalg.norm(a - approx_of(ref)) / na
    assert abs(e_gpu - e_or) <= 1e-12
    assert np.linalg.norm(approx_of(got) - approx_of(ref)) / na <= 1e-12
    assert np.linalg.norm(got["U"].T @ got["U"] - np.eye(ell)) < 1e-12
    assert np.linalg.norm(got["V"].T @ got["V"] - np.eye(ell)) < 1e-12
    assert np.all(np.tril(got["T"], -1) == 0) and np.all(np.diag(got["T"]) >= 0)
    sv_g = np.linalg.svd(got["T"], compute_uv=False)
    sv_o = np.linalg.svd(ref["T"], compute_uv=False)
    assert np.all(np.abs(sv_g - sv_o) <= 1e-12 * sv_o[0])


def test_factor_wide_f32_error_budget(ctx):
    """FP32 data and sketches at ell = 200: FP32 Grams on 4 x 4 tiles (the
    upper ten), the global-memory Cholesky and the FP32 R^-1 product."""
    m, n, k, p, q = 1500, 1200, 180, 20, 1
    a = synth.spectrum_matrix(m, n, 0.98 ** np.arange(min(m, n)), 0.0, 17)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    ell = k + p
    psi = synth.gaussian_psi(n, ell, seed=4)
    ref = oracle.corutv(a64, k, p, q, psi)
    out = ctx.factor(dev(a32, torch.float32), k, p, q, "f32", psi=dev(psi))
    assert ctx.sync() == 0
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    na = np.linalg.norm(a64)
    e_gpu = np.linalg.norm(a64 - approx_of(got)) / na
    e_or = np.linalg.norm(a64 - approx_of(ref)) / na
    budget = 4 * U32 * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
    assert e_gpu <= e_or + budget, (e_gpu, e_or, budget)
    assert np.linalg.norm(got["U"].T @ got["U"] - np.eye(ell)) < 1e-4
    assert np.linalg.norm(got["V"].T @ got["V"] - np.eye(ell)) < 1e-4


def test_factor_wide_single_pass_core_f64(ctx):
    """d_mode = 1 at ell = 200: D_approx = R2^T from the pass factors."""
    m, n, k, p, q = 800, 700, 150, 50, 1
    a = synth.spectrum_matrix(m, n, 0.97 ** np.arange(min(m, n)), 1e-9, 8)
    ell = k + p
    psi = synth.gaussian_psi(n, ell, seed=9)
    ref = oracle.corutv_dapprox(a, k, p, q, psi)
    out = ctx.factor(dev(a), k, p, q, "f64", psi=dev(psi), d_mode=1)
    assert ctx.sync() == 0
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    na = np.linalg.norm(a)
    assert np.linalg.norm(approx_of(got) - approx_of(ref)) / na <= 1e-10


def test_tensor_core_sketches_stay_at_128(ctx):
    a = dev(synth.spectrum_matrix(600, 500, 0.9 ** np.arange(500), 0.0, 1), torch.float32)
    with pytest.raises(corutv.CorutvError) as ei:
        ctx.factor(a, 150, 10, 0, "bf16")
    assert ei.value.status == corutv.EINVAL
