"""Ulp-level checks of the FP64 reciprocal square root and reciprocal used by
the small factorisations (they replace the FP64 divide / sqrt sequences with
the hardware's FP64 estimate and one third-order refinement step, and fall
back to the library operations outside 2^-999 .. 2^1001).

Through the C ABI: the thin QR of C = [diag(s); 0] has the Gram diag(s^2),
whose Cholesky factor is R = diag(|s|), computed on the device as
d * rsqrt(d) with d = s^2. For s spread over many binades (both paths) that
product must match |s| to a few ulp (the second CholeskyQR pass factors an identity Gram
and leaves R unchanged). The reciprocal is exercised by the QRCP of a
2 x 2 matrix, whose factors have closed forms.
"""

import numpy as np
import pytest
import torch

from paper_1906_04572_gb300 import Context, corutv

pytestmark = pytest.mark.gpu


def test_cholesky_diagonal_rsqrt_within_few_ulp():
    rng = np.random.default_rng(7)
    ell, rows = 96, 200
    with Context(0) as ctx:
        worst = 0.0
        for trial in range(8):
            # magnitudes 2^-510 .. 2^510 so that s^2 stays normal (the fast path
            # takes 2^-999 <= d < 2^1001, the ends the library fallback); random signs
            e = rng.uniform(-510, 510, ell)
            s = np.ldexp(rng.uniform(1.0, 2.0, ell), e.astype(int)) * rng.choice([-1.0, 1.0], ell)
            c = np.zeros((rows, ell))
            c[np.arange(ell), np.arange(ell)] = s
            C = torch.from_numpy(c).cuda()
            Q = torch.empty_like(C)
            R = torch.empty((ell, ell), dtype=torch.float64, device="cuda")
            corutv.corutv_orth(ctx.handle, C, Q, R)
            assert ctx.sync() == 0
            r = R.cpu().numpy()
            diag = np.abs(np.diag(r))
            ulps = np.abs(diag - np.abs(s)) / np.spacing(np.abs(s))
            worst = max(worst, float(ulps.max()))
            assert np.count_nonzero(np.triu(r, 1)) == 0
        assert worst <= 8.0, worst  # a second-order step from a 2^-20 estimate would show ~2^-40, i.e. thousands of ulp


def test_qrcp_2x2_closed_form():
    # D = [[a, b], [c, d]] with column 0 the larger: pivot stays, R[0,0] = |col 0|,
    # R[0,1] = col0 . col1 / |col 0|, |R[1,1]| = |det| / |col 0|
    rng = np.random.default_rng(3)
    with Context(0) as ctx:
        for _ in range(20):
            m = rng.standard_normal((2, 2)) * np.ldexp(1.0, int(rng.integers(-300, 300)))
            if np.linalg.norm(m[:, 1]) > np.linalg.norm(m[:, 0]):
                m = m[:, ::-1].copy()
            D = torch.from_numpy(m).cuda()
            Qt = torch.empty((2, 2), dtype=torch.float64, device="cuda")
            Rt = torch.empty_like(Qt)
            perm = torch.empty(2, dtype=torch.int32, device="cuda")
            corutv.corutv_qrcp(ctx.handle, D, Qt, Rt, perm)
            assert ctx.sync() == 0
            r, q, p = Rt.cpu().numpy(), Qt.cpu().numpy(), perm.cpu().numpy()
            assert list(p) == [0, 1]
            n0 = np.hypot(m[0, 0], m[1, 0])
            assert abs(r[0, 0] - n0) <= 8 * np.spacing(n0)
            r01 = (m[0, 0] * m[0, 1] + m[1, 0] * m[1, 1]) / n0
            assert abs(r[0, 1] - r01) <= 1e-14 * np.linalg.norm(m)
            det = abs(m[0, 0] * m[1, 1] - m[0, 1] * m[1, 0]) / n0
            assert abs(r[1, 1] - det) <= 1e-14 * np.linalg.norm(m)
            assert np.linalg.norm(q.T @ q - np.eye(2)) < 4e-15
            assert np.linalg.norm(q @ r - m) <= 4e-15 * np.linalg.norm(m)
