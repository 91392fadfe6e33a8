"""ctypes front end of the FP64 CPU oracle (oracle/corutv_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and bench.py's
CPU-baseline / reference arm. The product path never imports this package.

`build()` compiles the C source with gcc (-O3, OpenMP, no FMA contraction so
that every product and sum rounds exactly as written).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "corutv_oracle.c")
_HDR = os.path.join(_HERE, "corutv_oracle.h")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so in-tree if missing or older than its sources."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile a (possibly edited) copy of the oracle source into out_path.
    Used by the planted-mistake tests, which mutate the text on the CPU."""
    d = os.path.dirname(out_path)
    src = os.path.join(d, "corutv_oracle.c")
    with open(src, "w") as f:
        f.write(src_text)
    with open(os.path.join(d, "corutv_oracle.h"), "w") as f:
        f.write(open(_HDR).read())
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", out_path, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _bind(path):
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    i64 = ctypes.c_int64
    lib.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
    lib.or_gauss_entry.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_uint32]
    lib.or_gauss_entry.restype = ctypes.c_double
    lib.or_gauss_matrix.argtypes = [ctypes.c_uint64, ctypes.c_uint32, i64, i64, dp]
    lib.or_gemm_ax.argtypes = [i64, i64, i64, dp, i64, dp, dp]
    lib.or_gemm_aty.argtypes = [i64, i64, i64, dp, i64, dp, dp]
    lib.or_qr.argtypes = [i64, i64, dp, i64, dp, dp]
    lib.or_qrcp.argtypes = [i64, dp, dp, dp, ip]
    lib.or_corutv.argtypes = [dp, i64, i64, i64, i64, i64, i64, dp, ctypes.c_uint64,
                              ctypes.c_uint32, ctypes.c_int, dp, dp, dp, ip, dp, dp, dp]
    lib.or_shrink.argtypes = [i64, dp, ctypes.c_double, dp]
    lib.or_norm2.argtypes = [dp, i64, i64, i64]
    lib.or_norm2.restype = ctypes.c_double
    lib.or_rpca.argtypes = [dp, i64, i64, i64, i64, ctypes.c_double, ctypes.c_double,
                            ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            ctypes.c_int, ctypes.c_uint64, dp, dp,
                            ctypes.POINTER(ctypes.c_int), dp,
                            ctypes.POINTER(ctypes.c_int), dp,
                            ctypes.POINTER(ctypes.c_int), dp]
    for f in ("or_qr", "or_qrcp", "or_corutv", "or_rpca"):
        getattr(lib, f).restype = ctypes.c_int
    return lib


_override = threading.local()


def _load():
    """The bound oracle library: the in-tree build, or the variant selected
    with `use_library` (planted-mistake tests)."""
    global _lib
    lib = getattr(_override, "lib", None)
    if lib is not None:
        return lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


class use_library:
    """Context manager: route this thread's oracle calls to another build."""

    def __init__(self, path):
        self.lib = _bind(path)

    def __enter__(self):
        self.prev = getattr(_override, "lib", None)
        _override.lib = self.lib
        return self

    def __exit__(self, *exc):
        _override.lib = self.prev
        return False


def _dp(x):
    if x is None:
        return None
    return x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(status, what):
    if status != 0:
        raise OracleError(f"{what} failed with status {status}")


def philox4x32_10(ctr, key):
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.or_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def gauss_entry(seed: int, stream: int, i: int, j: int) -> float:
    return float(_load().or_gauss_entry(seed, stream, i, j))


def gauss_matrix(seed: int, stream: int, n: int, ell: int) -> np.ndarray:
    out = np.empty((n, ell))
    _load().or_gauss_matrix(seed, stream, n, ell, _dp(out))
    return out


def gemm_ax(a: np.ndarray, x: np.ndarray) -> np.ndarray:
    """C = A X (eq. 4)."""
    a, x = _f64(a), _f64(x)
    m, n = a.shape
    out = np.empty((m, x.shape[1]))
    _load().or_gemm_ax(m, n, x.shape[1], _dp(a), n, _dp(x), _dp(out))
    return out


def gemm_aty(a: np.ndarray, y: np.ndarray) -> np.ndarray:
    """C = A^T Y (eq. 5)."""
    a, y = _f64(a), _f64(y)
    m, n = a.shape
    out = np.empty((n, y.shape[1]))
    _load().or_gemm_aty(m, n, y.shape[1], _dp(a), n, _dp(y), _dp(out))
    return out


def qr(c: np.ndarray):
    c = _f64(c)
    m, l = c.shape
    q = np.empty((m, l))
    r = np.empty((l, l))
    _check(_load().or_qr(m, l, _dp(c), l, _dp(q), _dp(r)), "or_qr")
    return q, r


def qrcp(d: np.ndarray):
    d = _f64(d)
    l = d.shape[0]
    qt = np.empty((l, l))
    rt = np.empty((l, l))
    perm = np.empty(l, dtype=np.int32)
    _check(_load().or_qrcp(l, _dp(d), _dp(qt), _dp(rt),
                           perm.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), "or_qrcp")
    return qt, rt, perm


def corutv(a: np.ndarray, k: int, p: int, q: int, psi: np.ndarray | None = None,
           seed: int = 0, stream: int = 0, literal: bool = False) -> dict:
    """CoR-UTV (Algorithm 1). Returns dict with U, T, V, perm, Q1, Q2, D."""
    a = _f64(a)
    m, n = a.shape
    l = k + p
    if psi is not None:
        psi = _f64(psi)
        assert psi.shape == (n, l)
    out = {
        "U": np.empty((m, l)), "T": np.empty((l, l)), "V": np.empty((n, l)),
        "perm": np.empty(l, dtype=np.int32), "Q1": np.empty((m, l)), "Q2": np.empty((n, l)),
        "D": np.empty((l, l)),
    }
    st = _load().or_corutv(_dp(a), m, n, n, k, p, q, _dp(psi), seed, stream, int(literal),
                           _dp(out["U"]), _dp(out["T"]), _dp(out["V"]),
                           out["perm"].ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           _dp(out["Q1"]), _dp(out["Q2"]), _dp(out["D"]))
    _check(st, "or_corutv")
    return out


def corutv_lower(a: np.ndarray, k: int, p: int, q: int, psi: np.ndarray | None = None,
                 seed: int = 0, stream: int = 0) -> dict:
    """CoR-UTV with a lower triangular middle factor, the variant Sec. 3 sets
    beside the m >= n form for m < n and calls a direct modification of it.
    Reading: Algorithm 1 applied to A^T. Its factorisation A^T ~ U' T' V'^T
    gives A ~ V' T'^T U'^T, so U = V' = Q2' P (m x ell), T = T'^T (lower
    triangular), V = U' = Q1' Qt (n x ell); perm is the column permutation of
    U. psi is the m x ell test matrix of A^T. Q1, Q2 and D are those of the
    run on A^T (Q1: n x ell, Q2: m x ell). Any shape is accepted."""
    a = _f64(a)
    o = corutv(np.ascontiguousarray(a.T), k, p, q, psi=psi, seed=seed, stream=stream)
    return {"U": o["V"], "T": np.ascontiguousarray(o["T"].T), "V": o["U"], "perm": o["perm"],
            "Q1": o["Q1"], "Q2": o["Q2"], "D": o["D"]}


def corutv_dapprox(a: np.ndarray, k: int, p: int, q: int, psi: np.ndarray) -> dict:
    """CoR-UTV with the single-pass core (Sec. 3.1, the paragraph after eq. 9;
    Algorithm 1, its "D_approx" alternative): D = Q1^T A Q2 (eq. 7) is replaced
    by D_approx = Q1^T C1 (Q2^T X)^+, where C1 = A X is the last product with A
    and X the matrix it was formed from -- Psi when q = 0, else the
    re-orthonormalised C2 of the round before (the text writes Psi, Algorithm 1
    the current C2; the text's reading, applied to the power method, is the
    matrix C1 was formed from). The loop is the oracle's own (the same steps as
    `corutv`); the pseudo-inverse of the ell x ell matrix Q2^T X is numpy's
    (SVD-based) pinv. Returns dict with U, T, V, perm, Q1, Q2, D."""
    a = _f64(a)
    x = _f64(psi).copy()
    n, l = x.shape
    assert l == k + p and a.shape[1] == n
    for it in range(q + 1):
        c1 = gemm_ax(a, x)                 # eq. 4
        q1, _ = qr(c1)
        c2 = gemm_aty(a, q1)               # eq. 5 with C1 -> Q1
        if it < q:
            x, _ = qr(c2)
    q2, _ = qr(c2)
    d = (q1.T @ c1) @ np.linalg.pinv(q2.T @ x)
    qt, rt, perm = qrcp(d)                 # eq. 8
    return {"U": q1 @ qt, "T": rt, "V": q2[:, perm], "perm": perm, "Q1": q1, "Q2": q2, "D": d}


def shrink(x: np.ndarray, delta: float) -> np.ndarray:
    x = _f64(x)
    out = np.empty_like(x)
    _load().or_shrink(x.size, _dp(x), float(delta), _dp(out))
    return out


def norm2(mat: np.ndarray) -> float:
    mat = _f64(mat)
    return float(_load().or_norm2(_dp(mat), mat.shape[0], mat.shape[1], mat.shape[1]))


def rpca_defaults(mat: np.ndarray, mu0: float | None = None) -> dict:
    """Parameter reading used when the caller gives none: lambda =
    1/sqrt(max(m, n)) (Candes et al. 2011), mu0 = 1.25/||M||_2, rho = 1.6,
    mu_bar = 1e7 mu0 (Lin, Chen & Ma 2010), tol = 1e-5 (Sec. 5.3)."""
    m, n = mat.shape
    if mu0 is None:
        mu0 = 1.25 / norm2(mat)
    return {"lam": 1.0 / np.sqrt(max(m, n)), "mu0": mu0, "mu_bar": 1e7 * mu0, "rho": 1.6,
            "tol": 1e-5}


def rpca(mat: np.ndarray, k: int, lam: float, mu0: float, mu_bar: float, rho: float,
         tol: float, max_iter: int, seed: int = 0) -> dict:
    """ALM-CoRUTV (Algorithm 2)."""
    mat = _f64(mat)
    m, n = mat.shape
    lo = np.empty((m, n))
    so = np.empty((m, n))
    iters = ctypes.c_int(0)
    rank = ctypes.c_int(0)
    zeta = ctypes.c_double(0.0)
    zh = np.zeros(max_iter)
    rh = np.zeros(max_iter, dtype=np.int32)
    mh = np.zeros(max_iter)
    st = _load().or_rpca(_dp(mat), m, n, n, k, lam, mu0, mu_bar, rho, tol, max_iter, seed,
                         _dp(lo), _dp(so), ctypes.byref(iters), ctypes.byref(zeta),
                         ctypes.byref(rank), _dp(zh),
                         rh.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dp(mh))
    _check(st, "or_rpca")
    it = iters.value
    return {"L": lo, "S": so, "iters": it, "zeta": zeta.value, "rank": rank.value,
            "zeta_hist": zh[:it], "rank_hist": rh[:it].astype(int), "mu_hist": mh[:it]}
