"""GPU parity: every step of the CUDA path against the FP64 CPU oracle on the
same seeded inputs, through the C ABI.

Tolerances (FP64 path): products within the a-priori bound
2 K u (|A| |X|) elementwise (u = 2^-53, K = reduction length); QR / QRCP
factors within 1e-12 scaled by conditioning; factorisations within 1e-12 of
the oracle in relative Frobenius reconstruction error, the bar fixed for the
FP64 path.
"""

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


# ---------------------------------------------------------------- step 1
@pytest.mark.parametrize("n,ell,seed,stream", [(1000, 17, 0, 0), (257, 128, 12345678901, 7), (5, 1, 3, 1)])
def test_gaussian_matches_oracle(ctx, n, ell, seed, stream):
    psi = torch.empty((n, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_gaussian(ctx.handle, seed, stream, psi)
    ref = oracle.gauss_matrix(seed, stream, n, ell)
    got = host(psi)
    # same Philox words; log/cos/sqrt differ by at most a few ulp between libm and CUDA
    assert np.all(np.abs(got - ref) <= 1e-14 * np.maximum(1.0, np.abs(ref)))


# ---------------------------------------------------------------- eqs. 4, 5
@pytest.mark.parametrize("m,n,ell", [(1000, 700, 15), (333, 1021, 60), (130, 97, 128), (4100, 64, 1)])
@pytest.mark.parametrize("trans", [0, 1])
def test_sketch_f64_within_rounding_bound(ctx, m, n, ell, trans):
    rng = np.random.default_rng(m * 7 + n + ell)
    a = rng.standard_normal((m, n))
    x = rng.standard_normal((m if trans else n, ell))
    c = torch.empty((n if trans else m, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_sketch(ctx.handle, dev(a), dev(x), c, trans, "f64")
    ref = oracle.gemm_aty(a, x) if trans else oracle.gemm_ax(a, x)
    k = m if trans else n
    bound = 2 * k * U64 * ((np.abs(a).T if trans else np.abs(a)) @ np.abs(x))
    assert np.all(np.abs(host(c) - ref) <= bound + 1e-300)


@pytest.mark.parametrize("trans", [0, 1])
def test_sketch_f32_within_rounding_bound(ctx, trans):
    m, n, ell = 777, 513, 33
    rng = np.random.default_rng(11)
    a32 = rng.standard_normal((m, n)).astype(np.float32)
    x = rng.standard_normal((m if trans else n, ell))
    x32 = x.astype(np.float32).astype(np.float64)
    c = torch.empty((n if trans else m, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_sketch(ctx.handle, dev(a32, torch.float32), dev(x), c, trans, "f32")
    a64 = a32.astype(np.float64)
    ref = oracle.gemm_aty(a64, x32) if trans else oracle.gemm_ax(a64, x32)
    k = m if trans else n
    bound = 2 * k * U32 * ((np.abs(a64).T if trans else np.abs(a64)) @ np.abs(x32))
    assert np.all(np.abs(host(c) - ref) <= bound)


# ---------------------------------------------------------------- thin QR
@pytest.mark.parametrize("rows,ell,cond", [(1000, 60, 1e4), (513, 17, 1.0), (6000, 128, 1e6), (40, 40, 10.0)])
def test_orth_matches_oracle_qr(ctx, rows, ell, cond):
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


def test_orth_shift_recovers_ill_conditioned(ctx):
    """kappa ~ 1e10: the first Gram is not numerically SPD, the shifted pass
    plus two more passes still give an orthonormal Q spanning C."""
    rows, ell = 2000, 20
    rng = np.random.default_rng(5)
    c = (synth.haar(rng, rows, ell) * np.logspace(0, -10, ell)) @ synth.haar(rng, ell, ell).T
    q = torch.empty((rows, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_orth(ctx.handle, dev(c), q)
    assert ctx.sync() == 0
    qg = host(q)
    assert np.linalg.norm(qg.T @ qg - np.eye(ell)) < 1e-13
    assert rel(qg @ (qg.T @ c), c) < 1e-12


# ---------------------------------------------------------------- eq. 8
@pytest.mark.parametrize("ell", [1, 5, 15, 60, 110, 128])
def test_qrcp_matches_oracle(ctx, ell):
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


def test_qrcp_ties_take_lowest_index(ctx):
    d = np.array([[0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [0.5, 0.0, 0.0]])
    qt = torch.empty((3, 3), dtype=torch.float64, device="cuda")
    rt = torch.empty((3, 3), dtype=torch.float64, device="cuda")
    perm = torch.empty(3, dtype=torch.int32, device="cuda")
    corutv.corutv_qrcp(ctx.handle, dev(d), qt, rt, perm)
    assert list(host(perm).astype(int)) == list(oracle.qrcp(d)[2]) == [1, 2, 0]


# ---------------------------------------------------------------- Algorithm 1
CASES = [
    (1000, 1000, 10, 5, 0),   # the 1000 x 1000, ell = 15, q = 0 workload shape
    (333, 211, 12, 5, 1),     # ragged tails in both dimensions
    (211, 333, 12, 5, 2),     # m < n
    (300, 300, 20, 0, 1),     # p = 0
    (129, 4100, 60, 4, 1),    # very wide
    (70, 65, 63, 1, 0),       # ell = min(m, n) - 1
]


def _case_matrix(m, n, seed):
    r = min(m, n)
    return synth.spectrum_matrix(m, n, 0.9 ** np.arange(r), 1e-9, seed)


@pytest.mark.parametrize("m,n,k,p,q", CASES)
def test_factor_f64_matches_oracle(ctx, m, n, k, p, q):
    a = _case_matrix(m, n, m + n)
    psi = synth.gaussian_psi(n, k + p, seed=1)
    ref = oracle.corutv(a, k, p, q, psi)
    out = ctx.factor(dev(a), k, p, q, "f64", psi=dev(psi))
    assert ctx.sync() == 0
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    na = np.linalg.norm(a)
    e_gpu = np.linalg.norm(a - approx_of(got)) / na
    e_or = np.linalg.norm(a - approx_of(ref)) / na
    assert abs(e_gpu - e_or) <= 1e-12
    assert np.linalg.norm(approx_of(got) - approx_of(ref)) / na <= 1e-12
    ell = k + p
    assert np.linalg.norm(got["U"].T @ got["U"] - np.eye(ell)) < 1e-12
    assert np.linalg.norm(got["V"].T @ got["V"] - np.eye(ell)) < 1e-12
    assert np.all(np.tril(got["T"], -1) == 0) and np.all(np.diag(got["T"]) >= 0)
    sv_g = np.linalg.svd(got["T"], compute_uv=False)
    sv_o = np.linalg.svd(ref["T"], compute_uv=False)
    assert np.all(np.abs(sv_g - sv_o) <= 1e-12 * sv_o[0])
    if np.array_equal(host(out["perm"]).astype(np.int32), ref["perm"]):
        assert np.abs(got["T"] - ref["T"]).max() <= 1e-11 * sv_o[0]


def test_factor_c1_workload(ctx):
    """1000 x 1000, exact rank 10 + 1e-6 noise, ell = 15, q = 0, FP64."""
    f = synth.factor_c1()
    psi = synth.gaussian_psi(f.n, f.ell, seed=0)
    ref = oracle.corutv(f.a, f.k, f.p, f.q, psi)
    out = ctx.factor(dev(f.a), f.k, f.p, f.q, "f64", psi=dev(psi))
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    na = np.linalg.norm(f.a)
    assert abs(np.linalg.norm(f.a - approx_of(got)) - np.linalg.norm(f.a - approx_of(ref))) / na <= 1e-12
    assert np.array_equal(host(out["perm"]).astype(np.int32), ref["perm"])
    assert np.abs(got["T"] - ref["T"]).max() <= 1e-11


def test_factor_seeded_psi_matches_oracle(ctx):
    a = _case_matrix(400, 300, 9)
    ref = oracle.corutv(a, 10, 6, 1, None, seed=77, stream=5)
    out = ctx.factor(dev(a), 10, 6, 1, "f64", seed=77, stream=5)
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    assert rel(approx_of(got), approx_of(ref)) < 1e-12


def test_factor_host_pointers_equal_device(ctx):
    a = _case_matrix(300, 260, 4)
    psi = synth.gaussian_psi(260, 14, seed=2)
    outd = ctx.factor(dev(a), 10, 4, 1, "f64", psi=dev(psi))
    u = np.empty((300, 14))
    t = np.empty((14, 14))
    v = np.empty((260, 14))
    perm = np.empty(14, dtype=np.int32)
    corutv.corutv_factor(ctx.handle, a, 10, 4, 1, "f64", u, t, v, perm, psi=psi)
    assert np.array_equal(u, host(outd["U"])) and np.array_equal(t, host(outd["T"]))
    assert np.array_equal(v, host(outd["V"])) and np.array_equal(perm, host(outd["perm"]).astype(np.int32))


def test_factor_f32_error_budget(ctx):
    """FP32 input and FP32 products: error within the FP32 budget of the
    FP64 oracle's error on the rounded input."""
    m, n, k, p, q = 900, 700, 20, 6, 2
    a = synth.spectrum_matrix(m, n, np.arange(1, 301) ** -1.5, 0.0, 8)
    a32 = a.astype(np.float32)
    psi = synth.gaussian_psi(n, k + p, seed=3)
    ref = oracle.corutv(a32.astype(np.float64), k, p, q, psi)
    out = ctx.factor(dev(a32, torch.float32), k, p, q, "f32", psi=dev(psi))
    got = {x: host(out[x]) for x in ("U", "T", "V")}
    a64 = a32.astype(np.float64)
    na = np.linalg.norm(a64)
    e_gpu = np.linalg.norm(a64 - approx_of(got)) / na
    e_or = np.linalg.norm(a64 - approx_of(ref)) / na
    budget = 64 * U32 * np.sqrt(k + p) * np.linalg.norm(a64, 2) / na
    assert e_gpu <= e_or + budget
    ell = k + p
    assert np.linalg.norm(got["U"].T @ got["U"] - np.eye(ell)) < 1e-5


@pytest.mark.parametrize("m,n,k,p,q", [(500, 400, 10, 5, 0), (600, 450, 12, 6, 1), (450, 600, 8, 8, 2)])
def test_factor_single_pass_core_f64_matches_oracle(ctx, m, n, k, p, q):
    """d_mode 1 (Sec. 3.1's D_approx, formed on the device as R2^T from the
    CholeskyQR factors of the final thin QR, no third pass over A) against the
    oracle's literal D_approx = Q1^T C1 (Q2^T X)^+."""
    a = _case_matrix(m, n, m + q)
    psi = synth.gaussian_psi(n, k + p, seed=q + 20)
    ref = oracle.corutv_dapprox(a, k, p, q, psi)
    got = ctx.factor(dev(a), k, p, q, "f64", psi=dev(psi), d_mode=1)
    assert ctx.sync() == 0
    got = {x: host(got[x]) for x in ("U", "T", "V")}
    na = np.linalg.norm(a)
    assert np.linalg.norm(approx_of(got) - approx_of(ref)) / na <= 1e-12
    assert np.linalg.norm(got["U"].T @ got["U"] - np.eye(k + p)) < 1e-12
    assert np.all(np.tril(got["T"], -1) == 0)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_factor_single_pass_core_mixed_budget(ctx, prec):
    """d_mode 1 on the mixed paths: D comes from the sketch products'
    precision (no FP32 refinement pass), so the reconstruction error stays
    within that precision's budget of the oracle's."""
    m, n, k, p, q = 2000, 1500, 40, 10, 1
    sigma = np.arange(1, min(m, n) + 1) ** -1.5
    a = synth.spectrum_matrix(m, n, sigma, 0.0, 77)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    psi = synth.gaussian_psi(n, k + p, seed=21)
    ref = oracle.corutv_dapprox(a64, k, p, q, psi)
    out = ctx.factor(dev(a32, torch.float32), k, p, q, prec, psi=dev(psi), d_mode=1)
    assert ctx.sync() == 0
    u, t, v = (host(out[x]) for x in ("U", "T", "V"))
    na = np.linalg.norm(a64)
    e_gpu = np.linalg.norm(a64 - u @ t @ v.T) / na
    e_or = np.linalg.norm(a64 - ref["U"] @ ref["T"] @ ref["V"].T) / na
    unit = 2.0 ** -8 if prec == "bf16" else 2.0 ** -10
    budget = 4 * unit * np.sqrt(k + p) * np.linalg.norm(a64, 2) / na
    assert e_gpu <= e_or + budget, (e_gpu, e_or, budget)
    assert np.linalg.norm(u.T @ u - np.eye(k + p)) < 1e-5


def test_factor_rejects_unknown_d_mode(ctx):
    a = dev(_case_matrix(60, 50, 3))
    with pytest.raises(corutv.CorutvError) as ei:
        ctx.factor(a, 5, 3, 0, "f64", d_mode=2)
    assert ei.value.status == corutv.EINVAL


@pytest.mark.parametrize("bad", ["ell_too_big", "mixed_memory", "null_t"])
def test_factor_rejects_bad_arguments(ctx, bad):
    a = dev(_case_matrix(50, 40, 1))
    t = torch.empty((10, 10), dtype=torch.float64, device="cuda")
    with pytest.raises(corutv.CorutvError) as ei:
        if bad == "ell_too_big":
            corutv.corutv_factor(ctx.handle, a, 30, 10, 0, "f64", None, torch.empty((40, 40), dtype=torch.float64,
                                                                                     device="cuda"))
        elif bad == "mixed_memory":
            corutv.corutv_factor(ctx.handle, a, 8, 2, 0, "f64", None, np.empty((10, 10)))
        else:
            corutv.corutv_factor(ctx.handle, a, 8, 2, 0, "f64", None, None)
    assert ei.value.status == corutv.EINVAL
    del t


# ---------------------------------------------------------------- Algorithm 2
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_rpca_matches_oracle(ctx, dtype):
    pr = synth.rpca_problem(480, 120, 5, 0.10, "uniform", seed=0, amplitude=50.0)
    mobs = pr.m_obs.astype(dtype)
    d = oracle.rpca_defaults(mobs.astype(np.float64))
    ref = oracle.rpca(mobs.astype(np.float64), 5, d["lam"], d["mu0"], d["mu_bar"], d["rho"], 1e-5, 50)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    res = ctx.rpca(dev(mobs, tdt), 5, lam=d["lam"], mu0=d["mu0"], mu_bar=d["mu_bar"], rho=d["rho"],
                   tol=1e-5, max_iter=50, prec="f64" if dtype == np.float64 else "f32")
    assert res["iters"] == ref["iters"]
    assert res["rank"] == ref["rank"] == 5
    assert res["zeta"] < 1e-5
    lg, sg = host(res["L"]), host(res["S"])
    tol = 1e-9 if dtype == np.float64 else 1e-4
    assert rel(lg, ref["L"]) < tol
    assert abs(res["zeta"] - ref["zeta"]) <= tol * 10 + 1e-3 * ref["zeta"]
    assert np.array_equal(sg != 0, ref["S"] != 0)
    # the reported zeta is the definition of Sec. 5.3 on the returned L, S
    mm = mobs.astype(np.float64)
    assert abs(np.linalg.norm(mm - lg - sg) / np.linalg.norm(mm) - res["zeta"]) < 1e-3 * res["zeta"] + 1e-7


def test_rpca_fixed_iterations_report_notconv(ctx):
    pr = synth.rpca_problem(300, 100, 3, 0.05, "uniform", seed=1)
    res = ctx.rpca(dev(pr.m_obs), 3, tol=1e-30, max_iter=7, prec="f64", allow_notconv=True)
    assert res["status"] == corutv.ENOTCONV and res["iters"] == 7


def test_rpca_f32_past_convergence_keeps_shifting(ctx):
    """Once L is exactly rank 5 the sketches (ell = 10) are rank-deficient and
    their FP32 Gram matrices singular to FP32 rounding: the shift must be sized
    by the FP32 unit roundoff, so the run continues instead of breaking down."""
    pr = synth.rpca_problem(1200, 300, 5, 0.10, "uniform", seed=2, amplitude=50.0)
    m = dev(pr.m_obs, torch.float32)
    res = ctx.rpca(m, 5, tol=1e-30, max_iter=50, prec="f32", allow_notconv=True)
    assert res["status"] == corutv.ENOTCONV and res["iters"] == 50
    assert res["rank"] == 5
    assert rel(host(res["L"]), pr.l_true) < 1e-4


def test_rpca_tf32_sketches_track_f32(ctx):
    """Algorithm 2 with TF32 sketch products (FP32 data, FP32-accurate
    projection) converges to the same tolerance as the FP32 run, with L within
    the TF32 span error (about 2^-10 relative) of it. It may take more
    iterations: the span error of each low-rank step enters the residual."""
    pr = synth.rpca_problem(480, 120, 5, 0.10, "uniform", seed=0, amplitude=50.0)
    m32 = dev(pr.m_obs.astype(np.float32), torch.float32)
    d = oracle.rpca_defaults(pr.m_obs.astype(np.float32).astype(np.float64))
    kw = dict(lam=d["lam"], mu0=d["mu0"], mu_bar=d["mu_bar"], rho=d["rho"], tol=1e-5, max_iter=50)
    r32 = ctx.rpca(m32, 5, prec="f32", **kw)
    rtf = ctx.rpca(m32, 5, prec="tf32", **kw)
    print("iters", r32["iters"], rtf["iters"], "zeta", r32["zeta"], rtf["zeta"],
          "dL", rel(host(rtf["L"]), host(r32["L"])))
    assert rtf["rank"] == 5
    assert r32["status"] == rtf["status"] == corutv.OK and rtf["zeta"] < 1e-5
    assert rel(host(rtf["L"]), host(r32["L"])) < 4 * 2.0 ** -10


# ---------------------------------------------------------------- serving
def test_serving_results_equal_alone_and_in_the_mix(ctx):
    rng = np.random.default_rng(0)
    shapes = [(300, 200, 10, 5, 0), (512, 700, 20, 10, 1), (257, 263, 5, 10, 2), (1000, 333, 30, 10, 1),
              (640, 640, 64, 10, 2), (260, 1200, 12, 10, 0)]
    mats, alone, bufs, tickets = [], [], [], []
    for i, (m, n, k, p, q) in enumerate(shapes):
        a = dev(synth.spectrum_matrix(m, n, np.arange(1, min(m, n) + 1) ** -1.5, 0.0, i))
        mats.append(a)
        o = ctx.factor(a, k, p, q, "f64", seed=i)
        alone.append({x: host(o[x]) for x in ("U", "T", "V")})
    for i, (m, n, k, p, q) in enumerate(shapes):
        ell = k + p
        u = torch.empty((m, ell), dtype=torch.float64, device="cuda")
        t = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
        v = torch.empty((n, ell), dtype=torch.float64, device="cuda")
        bufs.append((u, t, v))
        req = corutv.make_request(mats[i], k, p, q, "f64", u, t, v, seed=i)
        tickets.append(corutv.corutv_submit(ctx.handle, req))
    del rng
    for i, tk in enumerate(tickets):
        st, lat = corutv.corutv_poll(ctx.handle, tk, timeout_us=60_000_000)
        assert st == corutv.OK and lat > 0
        u, t, v = (host(x) for x in bufs[i])
        a_alone = alone[i]
        assert rel(u @ t @ v.T, approx_of(a_alone)) < 1e-13


def test_rpca_c4_workload_matches_oracle(ctx):
    """Algorithm 2 on the full RPCA workload (4800 x 1200, rank 5, 10 % of the
    entries replaced by uniform [-50, 50] outliers), FP32 data, against the
    FP64 oracle run on the same FP32-rounded M with the same parameters:
    the same number of iterations, rank 5, zeta < tol, the exact support of
    S, and L within 1e-5 relative."""
    pr = synth.rpca_c4(0)
    m32 = pr.m_obs.astype(np.float32)
    mm = m32.astype(np.float64)
    d = oracle.rpca_defaults(mm)
    ref = oracle.rpca(mm, 5, d["lam"], d["mu0"], d["mu_bar"], d["rho"], 1e-5, 50)
    res = ctx.rpca(dev(m32, torch.float32), 5, lam=d["lam"], mu0=d["mu0"], mu_bar=d["mu_bar"], rho=d["rho"],
                   tol=1e-5, max_iter=50, prec="f32")
    lg, sg = host(res["L"]), host(res["S"])
    print("C4 iters", res["iters"], ref["iters"], "zeta", res["zeta"], ref["zeta"], "dL", rel(lg, ref["L"]))
    assert res["iters"] == ref["iters"]
    assert res["rank"] == ref["rank"] == 5
    assert res["zeta"] < 1e-5
    assert np.array_equal(sg != 0, ref["S"] != 0)
    assert rel(lg, ref["L"]) < 1e-5
    assert rel(lg, pr.l_true) < 1e-4
