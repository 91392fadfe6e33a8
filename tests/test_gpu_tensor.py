"""GPU parity of the tcgen05 sketch products and of the BF16 mixed-precision
factorisation against the FP64 oracle.

Bounds: the tensor cores multiply bf16 operands exactly and accumulate in
FP32, so against the oracle's product of the same bf16-rounded operands
|C - C_ref| <= 2 K 2^-24 (|A_r| |X_r|) elementwise. TF32 operands keep 10
mantissa bits (the low 13 bits of the FP32 input are dropped), which adds
2^-10 (|A| |X|). A^T Y in TF32 runs on a transposed FP32 copy of A."""

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
    c = Context(0)
    yield c
    c.close()


def dev(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def bf16_round(x):
    """Round float64 values to the nearest bf16 (ties to even) in one step,
    from the float64 bit pattern: bf16 keeps the sign, an 8-bit exponent and
    7 of the 52 mantissa bits (values here are normal and in range).
    torch's float64 -> bfloat16 conversion passes through float32 and can
    round twice, so it is not used as the reference."""
    b = np.ascontiguousarray(x, dtype=np.float64).view(np.uint64)
    drop = np.uint64(45)
    keep = b >> drop
    half = (b >> np.uint64(44)) & np.uint64(1)
    sticky = (b & np.uint64((1 << 44) - 1)) != 0
    up = (half == 1) & (sticky | ((keep & np.uint64(1)) == 1))
    return ((keep + up.astype(np.uint64)) << drop).view(np.float64)


def test_bf16_reference_rounding_is_exact():
    h = float.fromhex
    v = np.array([h("-0x1.3d0000fa4d343p-1"), h("0x1.3dp-1"), h("0x1.3c8p-1"), h("0x1.3d8p-1"), 1.0, -3.75])
    want = [h("-0x1.3ep-1"), h("0x1.3cp-1"), h("0x1.3cp-1"), h("0x1.3ep-1"), 1.0, -3.75]
    assert list(bf16_round(v)) == want


@pytest.mark.parametrize("m,n,ell", [(1000, 700, 15), (333, 1021, 60), (4100, 130, 110), (256, 200, 128),
                                     (129, 65, 16)])
@pytest.mark.parametrize("trans", [0, 1])
def test_sketch_bf16_within_bound(ctx, m, n, ell, trans):
    rng = np.random.default_rng(m + 3 * n + ell + trans)
    a32 = rng.standard_normal((m, n)).astype(np.float32)
    x = rng.standard_normal((m if trans else n, ell))
    c = torch.empty((n if trans else m, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_sketch(ctx.handle, dev(a32, torch.float32), dev(x), c, trans, "bf16")
    assert ctx.sync() == 0
    ar, xr = bf16_round(a32.astype(np.float64)), bf16_round(x)
    ref = oracle.gemm_aty(ar, xr) if trans else oracle.gemm_ax(ar, xr)
    k = m if trans else n
    bound = 2 * k * U32 * ((np.abs(ar).T if trans else np.abs(ar)) @ np.abs(xr))
    err = np.abs(host(c) - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("m,n,ell", [(1000, 700, 16), (333, 1021, 60)])
def test_sketch_tf32_within_bound(ctx, m, n, ell):
    rng = np.random.default_rng(m + n)
    a32 = rng.standard_normal((m, n)).astype(np.float32)
    x = rng.standard_normal((n, ell))
    c = torch.empty((m, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_sketch(ctx.handle, dev(a32, torch.float32), dev(x), c, 0, "tf32")
    assert ctx.sync() == 0
    a64 = a32.astype(np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle.gemm_ax(a64, x32)
    bound = (2 * 2.0 ** -10 + 2 * n * U32) * (np.abs(a64) @ np.abs(x32))
    assert np.all(np.abs(host(c) - ref) <= bound)


@pytest.mark.parametrize("m,n,ell", [(1000, 700, 60), (333, 1021, 110), (4100, 130, 16), (256, 64, 128)])
def test_sketch_bf16x3_has_fp32_accuracy(ctx, m, n, ell):
    """A X from exact three-way bf16 splits of A and X on the tensor cores:
    within the rounding bound of an FP32 dot product (the SIMT FP32 bound)."""
    rng = np.random.default_rng(m * 3 + n + ell)
    a32 = rng.standard_normal((m, n)).astype(np.float32)
    x = rng.standard_normal((n, ell))
    c = torch.empty((m, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_sketch(ctx.handle, dev(a32, torch.float32), dev(x), c, 0, "bf16x3")
    assert ctx.sync() == 0
    a64 = a32.astype(np.float64)
    x32 = x.astype(np.float32).astype(np.float64)
    ref = oracle.gemm_ax(a64, x32)
    bound = 2 * n * U32 * (np.abs(a64) @ np.abs(x32))
    err = np.abs(host(c) - ref)
    assert np.all(err <= bound), float((err / bound).max())


@pytest.mark.parametrize("m,n,ell", [(700, 1000, 16), (1021, 333, 60), (130, 4100, 110)])
def test_sketch_tf32_transposed_within_bound(ctx, m, n, ell):
    """A^T Y in TF32 runs as (A^T) Y on a transposed FP32 copy of A (K-major
    operands): the same TF32 bound as A X, with K = m."""
    rng = np.random.default_rng(3 * m + n)
    a32 = rng.standard_normal((m, n)).astype(np.float32)
    y = rng.standard_normal((m, ell))
    c = torch.empty((n, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_sketch(ctx.handle, dev(a32, torch.float32), dev(y), c, 1, "tf32")
    assert ctx.sync() == 0
    a64 = a32.astype(np.float64)
    y32 = y.astype(np.float32).astype(np.float64)
    ref = oracle.gemm_aty(a64, y32)
    bound = (2 * 2.0 ** -10 + 2 * m * U32) * (np.abs(a64).T @ np.abs(y32))
    assert np.all(np.abs(host(c) - ref) <= bound)


def test_sketch_bf16_stream_k_many_pieces(ctx):
    """Few tiles and a long K: each tile is split over many CTAs."""
    m, n, ell = 200, 30000, 32
    rng = np.random.default_rng(1)
    a32 = rng.standard_normal((m, n)).astype(np.float32)
    x = rng.standard_normal((n, ell))
    c = torch.empty((m, ell), dtype=torch.float64, device="cuda")
    corutv.corutv_sketch(ctx.handle, dev(a32, torch.float32), dev(x), c, 0, "bf16")
    ar, xr = bf16_round(a32.astype(np.float64)), bf16_round(x)
    ref = oracle.gemm_ax(ar, xr)
    bound = 2 * n * U32 * (np.abs(ar) @ np.abs(xr))
    assert np.all(np.abs(host(c) - ref) <= bound)


@pytest.mark.parametrize("m,n,k,p,q,pad", [(2000, 1500, 50, 10, 2, 0), (1500, 2000, 30, 10, 1, 1),
                                           (777, 513, 10, 5, 0, 3)])
def test_factor_tf32_error_budget(ctx, m, n, k, p, q, pad):
    """TF32 sketches (A X on A, A^T Y on its transposed copy) + CholeskyQR2 +
    the FP32-accurate split projection: within the TF32 budget of the FP64
    oracle's error. pad > 0 gives A a row stride that is not a multiple of
    16 bytes (the padded-copy path)."""
    sigma = np.arange(1, min(m, n) + 1) ** -1.5
    a = synth.spectrum_matrix(m, n, sigma, 0.0, m + n + 1)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    psi = synth.gaussian_psi(n, k + p, seed=9)
    ref = oracle.corutv(a64, k, p, q, psi)
    big = torch.zeros((m, n + pad), dtype=torch.float32, device="cuda")
    big[:, :n] = dev(a32, torch.float32)
    out = ctx.factor(big[:, :n], k, p, q, "tf32", psi=dev(psi))
    assert ctx.sync() == 0
    u, t, v = (host(out[x]) for x in ("U", "T", "V"))
    na = np.linalg.norm(a64)
    e_gpu = np.linalg.norm(a64 - u @ t @ v.T) / na
    e_or = np.linalg.norm(a64 - ref["U"] @ ref["T"] @ ref["V"].T) / na
    ell = k + p
    budget = 4 * 2.0 ** -10 * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
    assert e_gpu <= e_or + budget, (e_gpu, e_or, budget)
    assert np.linalg.norm(u.T @ u - np.eye(ell)) < 1e-5
    assert np.linalg.norm(v.T @ v - np.eye(ell)) < 1e-5
    assert np.all(np.tril(t, -1) == 0)


@pytest.mark.parametrize("m,n,k,p,q", [(2000, 1500, 50, 10, 2), (1500, 2000, 30, 10, 1), (777, 513, 10, 5, 0)])
def test_factor_bf16_error_budget(ctx, m, n, k, p, q):
    """BF16 sketches + CholeskyQR2 + FP32 projection: the reconstruction
    error stays within the BF16 budget of the FP64 oracle's error."""
    sigma = np.arange(1, min(m, n) + 1) ** -1.5
    a = synth.spectrum_matrix(m, n, sigma, 0.0, m + n)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    psi = synth.gaussian_psi(n, k + p, seed=7)
    ref = oracle.corutv(a64, k, p, q, psi)
    out = ctx.factor(dev(a32, torch.float32), k, p, q, "bf16", psi=dev(psi))
    assert ctx.sync() == 0
    u, t, v = (host(out[x]) for x in ("U", "T", "V"))
    na = np.linalg.norm(a64)
    e_gpu = np.linalg.norm(a64 - u @ t @ v.T) / na
    e_or = np.linalg.norm(a64 - ref["U"] @ ref["T"] @ ref["V"].T) / na
    ell = k + p
    budget = 4 * 2.0 ** -8 * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
    assert e_gpu <= e_or + budget, (e_gpu, e_or, budget)
    assert np.linalg.norm(u.T @ u - np.eye(ell)) < 1e-5
    assert np.linalg.norm(v.T @ v - np.eye(ell)) < 1e-5
    assert np.all(np.tril(t, -1) == 0)


@pytest.mark.parametrize("prec,u_p", [("bf16", 2.0 ** -8), ("tf32", 2.0 ** -10)])
@pytest.mark.parametrize("k,p", [(100, 10), (118, 10)])
def test_factor_mixed_wide_sketch_matches_oracle(ctx, prec, u_p, k, p):
    """The mixed paths at the sketch widths of the 20000 x 20000 workload
    (ell = 110) and at the largest supported one (ell = 128), on a 3000 x 2500
    matrix with its spectrum sigma_i = exp(-i/20), q = 2. At these widths the
    FP32 Gram runs on 2 x 2 output tiles and adds the products' split tiles
    (pieces) with write-back for the off-diagonal tiles too. Against the FP64
    oracle: the reconstruction error within the per-precision budget, the
    rank-ell approximation itself within that budget of the oracle's, and
    orthonormal factors."""
    m, n, q = 3000, 2500, 2
    a = synth.spectrum_matrix(m, n, synth.c3_sigma(min(m, n)), 0.0, 11)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    ell = k + p
    psi = synth.gaussian_psi(n, ell, seed=3)
    ref = oracle.corutv(a64, k, p, q, psi)
    out = ctx.factor(dev(a32, torch.float32), k, p, q, prec, psi=dev(psi))
    assert ctx.sync() == 0
    u, t, v = (host(out[x]) for x in ("U", "T", "V"))
    na = np.linalg.norm(a64)
    approx = u @ t @ v.T
    ref_approx = ref["U"] @ ref["T"] @ ref["V"].T
    e_gpu = np.linalg.norm(a64 - approx) / na
    e_or = np.linalg.norm(a64 - ref_approx) / na
    budget = 4 * u_p * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
    assert e_gpu <= e_or + budget, (e_gpu, e_or, budget)
    assert np.linalg.norm(approx - ref_approx) / na <= e_or + budget
    assert np.linalg.norm(u.T @ u - np.eye(ell)) < 1e-5
    assert np.linalg.norm(v.T @ v - np.eye(ell)) < 1e-5
    assert np.all(np.tril(t, -1) == 0) and np.all(np.diag(t) >= 0)


@pytest.mark.parametrize("prec", ["bf16", "tf32"])
def test_serving_mixed_results_equal_alone_and_in_the_mix(ctx, prec):
    """Requests of different m, n, k, q with FP32 data and tensor-core
    sketches, submitted together so that they overlap on the device: each
    result is bitwise the result of the same request run alone (every kernel's
    summation order depends only on the request's own sizes)."""
    shapes = [(300, 200, 10, 5, 0), (512, 700, 20, 10, 1), (257, 263, 5, 10, 2), (1000, 333, 30, 10, 1),
              (640, 640, 64, 10, 2), (260, 1200, 12, 10, 0), (2048, 1024, 40, 10, 2), (900, 1500, 50, 14, 1)]
    mats, alone = [], []
    for i, (m, n, k, p, q) in enumerate(shapes):
        a = dev(synth.spectrum_matrix(m, n, np.arange(1, min(m, n) + 1) ** -1.5, 0.0, 40 + i), torch.float32)
        mats.append(a)
        o = ctx.factor(a, k, p, q, prec, seed=i)
        alone.append({x: host(o[x]) for x in ("U", "T", "V", "perm")})
    bufs, tickets = [], []
    for i, (m, n, k, p, q) in enumerate(shapes):
        ell = k + p
        u = torch.empty((m, ell), dtype=torch.float32, device="cuda")
        t = torch.empty((ell, ell), dtype=torch.float32, device="cuda")
        v = torch.empty((n, ell), dtype=torch.float32, device="cuda")
        perm = torch.empty(ell, dtype=torch.int32, device="cuda")
        bufs.append((u, t, v, perm))
        tickets.append(corutv.corutv_submit(ctx.handle, corutv.make_request(mats[i], k, p, q, prec, u, t, v, perm,
                                                                            seed=i)))
    for i, tk in enumerate(tickets):
        st, lat = corutv.corutv_poll(ctx.handle, tk, timeout_us=60_000_000)
        assert st == corutv.OK and lat > 0
        for name, x in zip(("U", "T", "V", "perm"), bufs[i]):
            assert np.array_equal(host(x), alone[i][name]), f"request {i}: {name} differs from the lone run"


@pytest.mark.parametrize("spectrum", ["c2", "c3"])
@pytest.mark.parametrize("prec,u_p", [("f32", 2.0 ** -24), ("tf32", 2.0 ** -10)])
def test_power_form_one_qr_per_round(ctx, spectrum, prec, u_p):
    """power_form 1 (X = qr(A^T (A X)), C1 used as it is) on the spectra of
    the 8000 x 6000 (sigma_i = i^-2, i <= 200) and 20000 x 20000 (sigma_i =
    exp(-i/20)) workloads, 2000 x 1500, q = 2. The three forms are equal in
    exact arithmetic; in floating point the printed loop without any
    re-orthonormalisation loses the weak directions on the steep i^-2
    spectrum (the oracle's FP64 literal form is several times less accurate
    there). power_form 1 keeps one thin QR per round: its error lies within the
    precision's budget of the literal FP64 form's or better, and on the
    exp(-i/20) spectrum within budget of the re-orthonormalised form's."""
    m, n, k, p, q = 2000, 1500, 50, 10, 2
    sigma = np.arange(1, 201) ** -2.0 if spectrum == "c2" else synth.c3_sigma(n)
    a = synth.spectrum_matrix(m, n, sigma, 0.0, 17)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    psi = synth.gaussian_psi(n, k + p, seed=18)
    na = np.linalg.norm(a64)
    budget = 4 * u_p * np.sqrt(k + p) * np.linalg.norm(a64, 2) / na
    e_or = {}
    for lit in (False, True):
        r = oracle.corutv(a64, k, p, q, psi, literal=lit)
        e_or[lit] = np.linalg.norm(a64 - r["U"] @ r["T"] @ r["V"].T) / na
    e = {}
    for pf in (0, 1):
        out = ctx.factor(dev(a32, torch.float32), k, p, q, prec, psi=dev(psi), power_form=pf)
        assert ctx.sync() == 0
        u, t, v = (host(out[x]) for x in ("U", "T", "V"))
        e[pf] = np.linalg.norm(a64 - u @ t @ v.T) / na
        assert np.linalg.norm(u.T @ u - np.eye(k + p)) < 1e-5
    print(spectrum, prec, "pf0", e[0], "pf1", e[1], "oracle", e_or[False], "literal", e_or[True])
    assert e[0] <= e_or[False] + budget
    assert e[1] <= e_or[True] + budget
    if spectrum == "c3":
        assert e[1] <= e_or[False] + budget


def test_bf16_last_round_refinement_reaches_fp64_error(ctx):
    """BF16 sketches on the spectrum of the 20000 x 20000 workload, same Psi
    as the FP64 oracle: with every round on A_h (the default) and with the last
    power round on A_h + A_m (bf16_last_round = 1) the reconstruction error is
    within 1 % of the oracle's (equal error); the refinement is not worse."""
    m, n, k, p, q = 3000, 2500, 100, 10, 2
    a = synth.spectrum_matrix(m, n, synth.c3_sigma(min(m, n)), 0.0, 11)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    psi = synth.gaussian_psi(n, k + p, seed=3)
    ref = oracle.corutv(a64, k, p, q, psi)
    na = np.linalg.norm(a64)
    e_or = np.linalg.norm(a64 - ref["U"] @ ref["T"] @ ref["V"].T) / na
    e = {}
    for last in (0, 1):
        out = ctx.factor(dev(a32, torch.float32), k, p, q, "bf16", psi=dev(psi), bf16_last_round=last)
        assert ctx.sync() == 0
        u, t, v = (host(out[x]) for x in ("U", "T", "V"))
        e[last] = np.linalg.norm(a64 - u @ t @ v.T) / na
    print("bf16 plain", e[0] / e_or, "last round x2", e[1] / e_or)
    assert e[0] <= 1.01 * e_or
    assert e[1] <= 1.01 * e_or and e[1] <= e[0] * (1 + 1e-3)


@pytest.mark.parametrize("prec,u_p", [("bf16", 2.0 ** -8), ("tf32", 2.0 ** -10)])
def test_autotuned_products_meet_the_budget(ctx, prec, u_p):
    """With the stage-shape autotuner on, the first factorisation tunes each
    product shape (timed candidates, then the chosen launch), the second
    reuses the choices: both stay within the per-precision budget of the FP64
    oracle, the second is bitwise the first (same choices, fixed sums), and
    every choice is one of the candidate shapes."""
    m, n, k, p, q = 2600, 2100, 60, 10, 2
    a = synth.spectrum_matrix(m, n, synth.c3_sigma(min(m, n)), 0.0, 21)
    a32 = a.astype(np.float32)
    a64 = a32.astype(np.float64)
    ell = k + p
    psi = synth.gaussian_psi(n, ell, seed=5)
    ref = oracle.corutv(a64, k, p, q, psi)
    na = np.linalg.norm(a64)
    e_or = np.linalg.norm(a64 - ref["U"] @ ref["T"] @ ref["V"].T) / na
    budget = 4 * u_p * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
    corutv.corutv_set_autotune(True)
    try:
        outs = []
        for _ in range(2):
            out = ctx.factor(dev(a32, torch.float32), k, p, q, prec, psi=dev(psi))
            assert ctx.sync() == 0
            outs.append({x: host(out[x]) for x in ("U", "T", "V")})
    finally:
        corutv.corutv_set_autotune(False)
    for o in outs:
        e_gpu = np.linalg.norm(a64 - o["U"] @ o["T"] @ o["V"].T) / na
        assert e_gpu <= e_or + budget, (e_gpu, e_or, budget)
    for x in ("U", "T", "V"):
        assert np.array_equal(outs[0][x], outs[1][x]), x
    entries = corutv.corutv_autotune_entries()
    assert entries
    for ent in entries:
        assert ent["kgroup"] in (1, 2) and 2 <= ent["stages"] <= 8 and ent["us"] > 0
        stage_bytes = ent["kgroup"] * (128 * 128 + ent["panel_cols"] * 128)
        assert ent["stages"] * stage_bytes <= 200 * 1024


@pytest.mark.parametrize("pad", [0, 12])
def test_factor_bf16_pinned_host_input_equals_device(ctx, pad):
    """FP32 A in page-locked host memory on the split BF16 path: the tiled
    three-part cast reads A where it lies (row stride n + pad) instead of a
    staged device copy; pageable host memory takes the staged copy. Both give
    bitwise the results of the same call on device data."""
    m, n, k, p, q = 1300, 1100, 40, 10, 2
    ell = k + p
    a = synth.spectrum_matrix(m, n, synth.c3_sigma(min(m, n)), 0.0, 31).astype(np.float32)
    psi = synth.gaussian_psi(n, ell, seed=8)
    want = ctx.factor(dev(a, torch.float32), k, p, q, "bf16", psi=dev(psi))
    assert ctx.sync() == 0
    want = {x: host(want[x]) for x in ("U", "T", "V", "perm")}
    hbuf = torch.zeros((m, n + pad), dtype=torch.float32).pin_memory()
    hbuf[:, :n] = torch.from_numpy(a)
    pinned = hbuf.numpy()[:, :n]
    for src in (pinned, np.ascontiguousarray(a)):
        u = np.empty((m, ell), dtype=np.float32)
        t = np.empty((ell, ell), dtype=np.float32)
        v = np.empty((n, ell), dtype=np.float32)
        perm = np.empty(ell, dtype=np.int32)
        corutv.corutv_factor(ctx.handle, src, k, p, q, "bf16", u, t, v, perm, psi=psi)
        assert np.array_equal(u.astype(np.float64), want["U"])
        assert np.array_equal(t.astype(np.float64), want["T"])
        assert np.array_equal(v.astype(np.float64), want["V"])
        assert np.array_equal(perm, want["perm"].astype(np.int32))
