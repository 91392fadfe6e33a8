"""Seeded synthetic workloads for CoR-UTV and ALM-CoRUTV.

This module only draws inputs: test matrices with a prescribed spectrum, the
Gaussian test matrix Psi, robust-PCA problems M = L + S and serving request
streams. It holds no step of the method itself, so both the CPU oracle and the
CUDA path can be fed from it without sharing any of the method's arithmetic.
Everything is numpy, float64 unless a caller casts, and reproducible from an
integer seed.

Workload shapes follow the paper's experiments:
  * Sec. 5.1/5.2: A = U diag(sigma) V^T (+ noise), U, V Haar-distributed
    orthonormal factors, square order 1e3, decaying singular values.
  * Sec. 5.3: M = L + S with L = G1 G2^T (Gaussian factors) and a sparse S.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "haar",
    "spectrum_matrix",
    "gaussian_psi",
    "Factorisation",
    "exact_rank_case",
    "factor_c1",
    "factor_c2",
    "factor_c3",
    "rpca_problem",
    "rpca_c4",
    "rpca_table1",
    "serving_requests",
]


def haar(rng: np.random.Generator, rows: int, cols: int) -> np.ndarray:
    """Haar-distributed rows x cols matrix with orthonormal columns.

    QR of a standard Gaussian with the signs fixed so that diag(R) > 0
    (Mezzadri, Notices AMS 2007); that sign fix is what makes the distribution
    Haar rather than merely orthonormal.
    """
    g = rng.standard_normal((rows, cols))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s


def spectrum_matrix(m: int, n: int, sigma: np.ndarray, noise: float = 0.0,
                    seed: int = 0) -> np.ndarray:
    """A = U diag(sigma) V^T + noise * G, with U (m x r), V (n x r) Haar and
    G i.i.d. N(0, 1); r = len(sigma). Returns float64, C-contiguous."""
    rng = np.random.default_rng(seed)
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    u = haar(rng, m, r)
    v = haar(rng, n, r)
    a = (u * sigma) @ v.T
    if noise:
        a += noise * rng.standard_normal((m, n))
    return np.ascontiguousarray(a)


def spectrum_factors(m: int, n: int, sigma: np.ndarray, seed: int = 0) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(U, sigma, V) of spectrum_matrix(m, n, sigma, 0.0, seed): the same Haar
    factors (same generator, same draw order), so that a caller can form the
    product U diag(sigma) V^T on a device for large sizes."""
    rng = np.random.default_rng(seed)
    sigma = np.asarray(sigma, dtype=np.float64)
    r = sigma.shape[0]
    u = haar(rng, m, r)
    v = haar(rng, n, r)
    return u, sigma, v


def gaussian_psi(n: int, ell: int, seed: int = 0) -> np.ndarray:
    """Psi: n x ell with i.i.d. standard Gaussian entries (Sec. 3.1, Alg. 1
    step 1). Drawn here so that it can be injected into both implementations."""
    rng = np.random.default_rng(np.random.SeedSequence([seed, 0x505349]))
    return rng.standard_normal((n, ell))


@dataclasses.dataclass
class Factorisation:
    """One CoR-UTV problem instance."""
    name: str
    a: np.ndarray          # m x n, float64
    k: int
    p: int
    q: int
    sigma: np.ndarray      # singular values used to build a (before noise)
    noise: float

    @property
    def m(self) -> int:
        return self.a.shape[0]

    @property
    def n(self) -> int:
        return self.a.shape[1]

    @property
    def ell(self) -> int:
        return self.k + self.p


def exact_rank_case(m: int, n: int, rank: int, k: int, p: int, q: int,
                    seed: int = 0) -> Factorisation:
    """Exactly rank-`rank` matrix with singular values rank, rank-1, ..., 1."""
    sigma = np.arange(rank, 0, -1, dtype=np.float64)
    return Factorisation(f"exact_rank{rank}_{m}x{n}", spectrum_matrix(m, n, sigma, 0.0, seed),
                         k, p, q, sigma, 0.0)


def factor_c1(seed: int = 0, noise: float = 1e-6) -> Factorisation:
    """1000 x 1000, exact rank 10 with sigma = 10, 9, ..., 1 (linearly spaced),
    Haar factors, plus i.i.d. N(0, 1e-6^2) noise; k = 10, p = 5, q = 0."""
    sigma = np.linspace(10.0, 1.0, 10)
    return Factorisation("c1_1000x1000_l15_q0", spectrum_matrix(1000, 1000, sigma, noise, seed),
                         10, 5, 0, sigma, noise)


def _c2_sigma() -> np.ndarray:
    i = np.arange(1, 201, dtype=np.float64)
    return i ** -2.0


def factor_c2(q: int = 2, seed: int = 0, m: int = 8000, n: int = 6000) -> Factorisation:
    """8000 x 6000, sigma_i = i^-2 for i <= 200 (zero beyond), plus i.i.d.
    N(0, 1e-4^2) noise, Haar factors; k = 50, ell = 60, q in {1, 2}."""
    return Factorisation(f"c2_{m}x{n}_l60_q{q}", spectrum_matrix(m, n, _c2_sigma(), 1e-4, seed),
                         50, 10, q, _c2_sigma(), 1e-4)


def c3_sigma(n: int) -> np.ndarray:
    """sigma_i = exp(-i/20), kept while sigma_i >= 1e-18 sigma_1 (the rest is
    below double rounding of the product and is dropped)."""
    i = np.arange(1, n + 1, dtype=np.float64)
    s = np.exp(-i / 20.0)
    return s[s >= 1e-18 * s[0]]


def factor_c3(seed: int = 0, m: int = 20000, n: int = 20000, q: int = 2) -> Factorisation:
    """20000 x 20000 dense, sigma_i = exp(-i/20), Haar factors, k = 100,
    ell = 110, q = 2. No noise."""
    s = c3_sigma(min(m, n))
    return Factorisation(f"c3_{m}x{n}_l110_q{q}", spectrum_matrix(m, n, s, 0.0, seed),
                         100, 10, q, s, 0.0)


@dataclasses.dataclass
class RpcaProblem:
    name: str
    m_obs: np.ndarray      # M = L + S
    l_true: np.ndarray
    s_true: np.ndarray
    rank: int


def rpca_problem(m: int, n: int, rank: int, density: float, values: str,
                 seed: int = 0, amplitude: float = 50.0) -> RpcaProblem:
    """M = L + S with L = G1 G2^T (G1: m x rank, G2: n x rank, N(0, 1)) and S
    supported on round(density*m*n) positions drawn uniformly without
    replacement. values = "uniform" -> U[-amplitude, amplitude];
    values = "pm" -> +-amplitude with equal probability (Sec. 5.3 uses +-80)."""
    rng = np.random.default_rng(seed)
    g1 = rng.standard_normal((m, rank))
    g2 = rng.standard_normal((n, rank))
    low = g1 @ g2.T
    nnz = int(round(density * m * n))
    pos = rng.choice(m * n, size=nnz, replace=False)
    s = np.zeros(m * n)
    if values == "uniform":
        s[pos] = rng.uniform(-amplitude, amplitude, size=nnz)
    elif values == "pm":
        s[pos] = amplitude * rng.choice(np.array([-1.0, 1.0]), size=nnz)
    else:
        raise ValueError(values)
    s = s.reshape(m, n)
    return RpcaProblem(f"rpca_{m}x{n}_r{rank}", np.ascontiguousarray(low + s), low, s, rank)


def rpca_c4(seed: int = 0) -> RpcaProblem:
    """4800 x 1200, rank-5 Gaussian factors, 10 % support, U[-50, 50]."""
    return rpca_problem(4800, 1200, 5, 0.10, "uniform", seed, 50.0)


def rpca_table1(n: int, seed: int = 0) -> RpcaProblem:
    """Sec. 5.3 / Table 1 shape: n x n, rank 0.05 n, 0.05 n^2 entries of +-80."""
    return rpca_problem(n, n, int(round(0.05 * n)), 0.05, "pm", seed, 80.0)


@dataclasses.dataclass
class Request:
    idx: int
    arrival_s: float
    m: int
    n: int
    k: int
    p: int
    q: int
    seed: int


def serving_requests(count: int = 1024, rate_per_s: float = 2000.0, seed: int = 0,
                     lo: int = 256, hi: int = 4096) -> list[Request]:
    """A stream of independent CoR-UTV requests: Poisson arrivals at
    `rate_per_s`, m, n ~ U[lo, hi], k ~ U[5, 64], ell = k + 10, q ~ U{0,1,2}."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps) - gaps[0]
    out = []
    for i in range(count):
        m = int(rng.integers(lo, hi + 1))
        n = int(rng.integers(lo, hi + 1))
        k = int(rng.integers(5, 65))
        q = int(rng.integers(0, 3))
        out.append(Request(i, float(t[i]), m, n, k, 10, q, int(rng.integers(0, 2**31 - 1))))
    return out


def serving_matrix(req: Request, max_rank: int = 256) -> np.ndarray:
    """Matrix of one serving request: sigma_i = i^-1.5 on the first
    min(m, n, max_rank) singular directions, Haar factors, float64. The tail
    beyond max_rank (sigma < 256^-1.5 ~ 2.4e-4) is dropped to keep host-side
    generation of 1024 requests fast."""
    r = min(req.m, req.n, max_rank)
    i = np.arange(1, r + 1, dtype=np.float64)
    return spectrum_matrix(req.m, req.n, i ** -1.5, 0.0, req.seed)


def serving_factors(req: Request, max_rank: int = 256) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """(U, sigma, V) of serving_matrix(req, max_rank): the same Haar factors
    (same generator, same draw order), so U diag(sigma) V^T is that matrix.
    Lets a caller form the product on a device."""
    r = min(req.m, req.n, max_rank)
    sigma = np.arange(1, r + 1, dtype=np.float64) ** -1.5
    rng = np.random.default_rng(req.seed)
    u = haar(rng, req.m, r)
    v = haar(rng, req.n, r)
    return u, sigma, v


def frob(x: np.ndarray) -> float:
    return float(math.sqrt(float(np.sum(np.square(x, dtype=np.float64)))))
