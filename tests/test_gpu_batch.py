"""The batched factorisation (corutv_factor_batch): every step of Algorithm 1
one grouped launch over problems of uneven m, n, k, q.

Each problem is checked against the FP64 CPU oracle run on the same FP32
matrix with the same seeded Gaussian test matrix (Alg. 1 step 1; the oracle
draws it in FP64, the GPU in FP32 rounded to the bf16 operand), within the
BF16 error budget of the single-call tests; its results must be bitwise the
same alone (a batch of one) and inside the batch, in any order of the
batch; and they must agree with a corutv_factor call on the same request
(BF16 sketches) to the budget."""
import numpy as np
import pytest
import torch

import oracle
import synth
from paper_1906_04572_gb300 import Context, corutv

pytestmark = pytest.mark.gpu
U_BF16 = 2.0 ** -8

# (m, n, k, p, q, seed): uneven shapes, both orientations, q in {0, 1, 2},
# widths below and above 64 (the QRCP's one-block range), ragged tails
SHAPES = [(700, 520, 20, 10, 2, 1), (333, 900, 8, 10, 0, 2), (1500, 1300, 60, 10, 1, 3),
          (450, 450, 5, 10, 2, 4), (1030, 610, 64, 10, 2, 5), (260, 300, 33, 10, 1, 6)]


@pytest.fixture(scope="module")
def ctx():
    from paper_1906_04572_gb300 import build
    build.build()
    oracle.build()
    c = Context(0)
    yield c
    c.close()


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def matrix(m, n, seed):
    sigma = np.arange(1, min(m, n) + 1, dtype=np.float64) ** -1.5  # the serving stream's spectrum
    return synth.spectrum_matrix(m, n, sigma, 0.0, 100 + seed).astype(np.float32)


def request(a, k, p, q, seed):
    m, n = a.shape
    ell = k + p
    out = {"U": torch.empty((m, ell), dtype=torch.float32, device="cuda"),
           "T": torch.empty((ell, ell), dtype=torch.float32, device="cuda"),
           "V": torch.empty((n, ell), dtype=torch.float32, device="cuda"),
           "perm": torch.empty(ell, dtype=torch.int32, device="cuda")}
    rq = corutv.make_request(a, k, p, q, "bf16", out["U"], out["T"], out["V"], out["perm"], seed=seed, stream=7)
    return rq, out


def run_batch(ctx, mats, shapes):
    reqs, outs = [], []
    for a, (m, n, k, p, q, seed) in zip(mats, shapes):
        rq, out = request(a, k, p, q, seed)
        reqs.append(rq)
        outs.append(out)
    corutv.corutv_factor_batch(ctx.handle, reqs)
    assert ctx.sync() == 0
    return [{x: host(o[x]) for x in ("U", "T", "V", "perm")} for o in outs]


@pytest.fixture(scope="module")
def batch(ctx):
    mats = [torch.from_numpy(matrix(m, n, s)).cuda() for (m, n, k, p, q, s) in SHAPES]
    return mats, run_batch(ctx, mats, SHAPES)


def test_batch_matches_oracle_within_bf16_budget(batch):
    mats, res = batch
    for a, got, (m, n, k, p, q, seed) in zip(mats, res, SHAPES):
        a64 = a.cpu().numpy().astype(np.float64)
        ell = k + p
        ref = oracle.corutv(a64, k, p, q, seed=seed, stream=7)
        na = np.linalg.norm(a64)
        e_gpu = np.linalg.norm(a64 - got["U"] @ got["T"] @ got["V"].T) / na
        e_or = np.linalg.norm(a64 - ref["U"] @ ref["T"] @ ref["V"].T) / na
        budget = 4 * U_BF16 * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
        assert e_gpu <= e_or + budget, (m, n, k, q, e_gpu, e_or, budget)
        assert np.linalg.norm(got["U"].T @ got["U"] - np.eye(ell)) < 1e-5
        assert np.linalg.norm(got["V"].T @ got["V"] - np.eye(ell)) < 1e-5
        assert np.all(np.tril(got["T"], -1) == 0) and np.all(np.diag(got["T"]) >= 0)
        assert sorted(got["perm"].astype(int)) == list(range(ell))


def test_batch_results_are_the_same_alone_and_in_the_mix(ctx, batch):
    mats, res = batch
    for i in (0, 2, 5):
        alone = run_batch(ctx, [mats[i]], [SHAPES[i]])[0]
        for x in ("U", "T", "V", "perm"):
            assert np.array_equal(alone[x], res[i][x]), (i, x)
    # another order and another company
    idx = [5, 3, 0, 2]
    mixed = run_batch(ctx, [mats[i] for i in idx], [SHAPES[i] for i in idx])
    for j, i in enumerate(idx):
        for x in ("U", "T", "V", "perm"):
            assert np.array_equal(mixed[j][x], res[i][x]), (i, x)


def test_batch_agrees_with_single_calls(ctx, batch):
    mats, res = batch
    for a, got, (m, n, k, p, q, seed) in zip(mats, res, SHAPES):
        ell = k + p
        one = ctx.factor(a, k, p, q, "bf16", seed=seed, stream=7)
        assert ctx.sync() == 0
        u, t, v = (host(one[x]) for x in ("U", "T", "V"))
        a64 = a.cpu().numpy().astype(np.float64)
        na = np.linalg.norm(a64)
        budget = 4 * U_BF16 * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
        diff = np.linalg.norm(u @ t @ v.T - got["U"] @ got["T"] @ got["V"].T) / na
        assert diff <= budget, (m, n, k, q, diff, budget)


def test_batch_rejects_what_the_grouped_path_does_not_take(ctx):
    a = torch.from_numpy(matrix(300, 280, 9)).cuda()
    for kw in ({"prec": "f32"}, {"k": 130}, {"d_mode": 1}):
        k = kw.get("k", 10)
        ell = k + 10
        t = torch.empty((ell, ell), dtype=torch.float32, device="cuda")
        rq = corutv.make_request(a, k, 10, 1, kw.get("prec", "bf16"), None, t, d_mode=kw.get("d_mode", 0))
        with pytest.raises(corutv.CorutvError) as ei:
            corutv.corutv_factor_batch(ctx.handle, [rq])
        assert ei.value.status == corutv.EINVAL
    a64 = torch.from_numpy(matrix(300, 280, 9).astype(np.float64)).cuda()
    t = torch.empty((20, 20), dtype=torch.float64, device="cuda")
    with pytest.raises(corutv.CorutvError):
        corutv.corutv_factor_batch(ctx.handle, [corutv.make_request(a64, 10, 10, 1, "bf16", None, t)])


def test_batch_of_many_small_problems(ctx):
    """64 problems at once (the grid's z extent, the records buffer and the
    stream-K partial storage of many problems): a sample of them equal their
    batch-of-one results bitwise, and every one meets the BF16 budget of the
    oracle's error on the same seeded test matrix."""
    rng = np.random.default_rng(11)
    shapes = []
    for i in range(64):
        m, n = (int(v) for v in rng.integers(256, 900, size=2))
        k = int(rng.integers(5, 40))
        shapes.append((m, n, k, 10, int(rng.integers(0, 3)), 200 + i))
    mats = [torch.from_numpy(matrix(m, n, s)).cuda() for (m, n, k, p, q, s) in shapes]
    res = run_batch(ctx, mats, shapes)
    for i in (0, 17, 63):
        alone = run_batch(ctx, [mats[i]], [shapes[i]])[0]
        assert np.array_equal(alone["T"], res[i]["T"]) and np.array_equal(alone["U"], res[i]["U"])
    for a, got, (m, n, k, p, q, s) in zip(mats, res, shapes):
        a64 = a.cpu().numpy().astype(np.float64)
        ell = k + p
        ref = oracle.corutv(a64, k, p, q, seed=s, stream=7)
        na = np.linalg.norm(a64)
        e_gpu = np.linalg.norm(a64 - got["U"] @ got["T"] @ got["V"].T) / na
        e_or = np.linalg.norm(a64 - ref["U"] @ ref["T"] @ ref["V"].T) / na
        budget = 4 * U_BF16 * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
        assert e_gpu <= e_or + budget, (m, n, k, q, e_gpu, e_or, budget)


def test_batched_serving_results_equal_the_grouped_path_alone(ctx):
    """Continuous batching (corutv_set_batching): requests submitted in two
    waves with a host pause between them are admitted as batches on the two
    lanes; every result is bitwise that of the request alone through
    corutv_factor_batch, and a request the grouped path does not take (FP64
    sketches) runs in a slot meanwhile and matches its corutv_factor call."""
    shapes = SHAPES + [(520, 610, 12, 10, 1, 7), (900, 300, 40, 10, 2, 8)]
    mats = [torch.from_numpy(matrix(m, n, s)).cuda() for (m, n, k, p, q, s) in shapes]
    alone = [run_batch(ctx, [a], [sh])[0] for a, sh in zip(mats, shapes)]
    a64 = torch.from_numpy(matrix(400, 350, 9).astype(np.float64)).cuda()
    ref64 = ctx.factor(a64, 10, 5, 1, "f64", seed=3)
    assert ctx.sync() == 0
    ref64 = {x: host(ref64[x]) for x in ("U", "T", "V")}
    with Context(0, max_slots=4) as sctx:
        corutv.corutv_set_batching(sctx.handle, 64)
        tickets, outs = [], []
        for i, (a, (m, n, k, p, q, seed)) in enumerate(zip(mats, shapes)):
            rq, out = request(a, k, p, q, seed)
            tickets.append(corutv.corutv_submit(sctx.handle, rq))
            outs.append(out)
            if i == 3:
                torch.cuda.synchronize()
        u = torch.empty((400, 15), dtype=torch.float64, device="cuda")
        t = torch.empty((15, 15), dtype=torch.float64, device="cuda")
        v = torch.empty((350, 15), dtype=torch.float64, device="cuda")
        t64 = corutv.corutv_submit(sctx.handle, corutv.make_request(a64, 10, 5, 1, "f64", u, t, v, seed=3))
        for tk in tickets + [t64]:
            st, _ = corutv.corutv_poll(sctx.handle, tk, timeout_us=120_000_000)
            assert st == corutv.OK
        for o, want in zip(outs, alone):
            for x in ("U", "T", "V", "perm"):
                assert np.array_equal(host(o[x]), want[x]), x
        for x, got in (("U", u), ("T", t), ("V", v)):
            assert np.array_equal(host(got), ref64[x]), x


def test_batch_at_the_widest_sketch(ctx):
    """ell = 128 (the widest tensor-core sketch) beside a narrow problem: the
    projection's B panel then needs two TMA boxes and two MMA N chunks, its
    ring the one-CTA-per-SM budget, and the Cholesky, QRCP and R^-1 their
    largest shared memory; both problems within the BF16 budget of the
    oracle and bitwise equal to their batches of one."""
    shapes = [(700, 650, 118, 10, 1, 31), (400, 380, 9, 10, 2, 32)]
    mats = [torch.from_numpy(matrix(m, n, s)).cuda() for (m, n, k, p, q, s) in shapes]
    res = run_batch(ctx, mats, shapes)
    for i, (a, got, (m, n, k, p, q, s)) in enumerate(zip(mats, res, shapes)):
        a64 = a.cpu().numpy().astype(np.float64)
        ell = k + p
        ref = oracle.corutv(a64, k, p, q, seed=s, stream=7)
        na = np.linalg.norm(a64)
        e_gpu = np.linalg.norm(a64 - got["U"] @ got["T"] @ got["V"].T) / na
        e_or = np.linalg.norm(a64 - ref["U"] @ ref["T"] @ ref["V"].T) / na
        budget = 4 * U_BF16 * np.sqrt(ell) * np.linalg.norm(a64, 2) / na
        assert e_gpu <= e_or + budget, (m, n, k, q, e_gpu, e_or, budget)
        alone = run_batch(ctx, [a], [shapes[i]])[0]
        for x in ("U", "T", "V", "perm"):
            assert np.array_equal(alone[x], got[x]), (i, x)


def test_set_batching_rejects_out_of_range(ctx):
    for bad in (-1, 4097):
        with pytest.raises(corutv.CorutvError) as ei:
            corutv.corutv_set_batching(ctx.handle, bad)
        assert ei.value.status == corutv.EINVAL
    corutv.corutv_set_batching(ctx.handle, 0)
