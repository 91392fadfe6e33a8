"""Python binding of libcorutv (include/corutv.h): argument marshalling only.

Every function named corutv_* calls the C entry point of the same name with
pointers taken from torch tensors (host or CUDA) or numpy arrays. Nothing here
computes any step of the method; if the shared library is missing the import
of the library raises, there is no fallback.
"""

from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcorutv.so")

OK, EINVAL, ENOMEM, ECUDA, EPENDING, ETIMEDOUT, ENOTCONV, EBREAKDOWN = range(8)
F64, F32 = 0, 1
P_F64, P_F32, P_TF32, P_BF16, P_BF16X3 = 0, 1, 2, 3, 4
PREC_NAMES = {"f64": P_F64, "f32": P_F32, "tf32": P_TF32, "bf16": P_BF16, "bf16x3": P_BF16X3}
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EPENDING", 5: "ETIMEDOUT",
                6: "ENOTCONV", 7: "EBREAKDOWN"}


class CorutvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int64), ("p", ctypes.c_int64), ("q", ctypes.c_int64),
                ("sketch_prec", ctypes.c_int32), ("d_mode", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_uint32), ("t_lower", ctypes.c_uint32),
                ("psi", ctypes.c_void_p), ("power_form", ctypes.c_uint32), ("bf16_last_round", ctypes.c_uint32)]


class Request(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int), ("A", ctypes.c_void_p), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("lda", ctypes.c_int64), ("opts", Opts),
                ("U", ctypes.c_void_p), ("T", ctypes.c_void_p), ("V", ctypes.c_void_p),
                ("ldu", ctypes.c_int64), ("ldv", ctypes.c_int64), ("perm", ctypes.c_void_p)]


# corutv_allreduce_fn: (buf, count, dtype, user) -> status
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p)

_lib = None
_lock = threading.Lock()

_SIGS = {
    "corutv_create": ([ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_size_t, ctypes.c_int], ctypes.c_int),
    "corutv_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "corutv_last_error": ([ctypes.c_void_p], ctypes.c_char_p),
    "corutv_set_stream": ([ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "corutv_sync": ([ctypes.c_void_p], ctypes.c_int),
    "corutv_factor": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                       ctypes.c_int64, ctypes.POINTER(Opts), ctypes.c_void_p, ctypes.c_int64,
                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "corutv_rpca": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                     ctypes.c_int64, ctypes.POINTER(Opts), ctypes.c_double, ctypes.c_double, ctypes.c_double,
                     ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                     ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "corutv_factor_rows": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                            ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(Opts), ALLREDUCE_FN, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                            ctypes.c_void_p], ctypes.c_int),
    "corutv_submit": ([ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
    "corutv_factor_batch": ([ctypes.c_void_p, ctypes.POINTER(Request), ctypes.c_int], ctypes.c_int),
    "corutv_set_batching": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "corutv_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)],
                    ctypes.c_int),
    "corutv_profile_enable": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "corutv_set_graphs": ([ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "corutv_set_autotune": ([ctypes.c_int], ctypes.c_int),
    "corutv_autotune_entry": ([ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
    "corutv_profile_read": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "corutv_gaussian": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int64,
                         ctypes.c_void_p, ctypes.c_int64], ctypes.c_int),
    "corutv_sketch": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                       ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64], ctypes.c_int),
    "corutv_orth": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                     ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p], ctypes.c_int),
    "corutv_qrcp": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                     ctypes.c_void_p], ctypes.c_int),
    "corutv_selftest_wait": ([ctypes.c_void_p, ctypes.c_int64], ctypes.c_int),
    "corutv_orth_noalloc": ([ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                             ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
}

EXPORTED = tuple(_SIGS)


def load(path: str | None = None):
    """Load libcorutv.so (built by paper_1906_04572_gb300.build). Raises if
    it is missing: the product path has no fallback."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise ImportError(f"{p} is missing; build it with paper_1906_04572_gb300.build.build()")
            lib = ctypes.CDLL(p)
            for name, (args, res) in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            _lib = lib
    return _lib


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _rowmajor_ld(x) -> int:
    if _is_torch(x):
        if x.dim() != 2 or x.stride(1) != 1:
            raise ValueError("matrices must be 2-D with unit column stride (row-major)")
        return int(x.stride(0))
    if x.ndim != 2 or x.strides[1] != x.itemsize:
        raise ValueError("matrices must be 2-D with unit column stride (row-major)")
    return x.strides[0] // x.itemsize


def _dtype_code(x) -> int:
    if _is_torch(x):
        import torch
        if x.dtype == torch.float64:
            return F64
        if x.dtype == torch.float32:
            return F32
    else:
        if x.dtype == np.float64:
            return F64
        if x.dtype == np.float32:
            return F32
    raise TypeError(f"A must be float64 or float32, got {x.dtype}")


def _check(ctx, status: int, allow=(OK,)):
    if status not in allow:
        msg = load().corutv_last_error(ctx)
        raise CorutvError(status, msg.decode() if msg else "")
    return status


def _opts(k, p, q, prec, seed=0, stream=0, psi=None, d_mode=0, t_lower=0, power_form=0,
          bf16_last_round=0) -> Opts:
    o = Opts()
    o.power_form = int(power_form)
    o.bf16_last_round = int(bf16_last_round)
    o.k, o.p, o.q = int(k), int(p), int(q)
    o.sketch_prec = PREC_NAMES[prec] if isinstance(prec, str) else int(prec)
    o.d_mode = int(d_mode)
    o.t_lower = int(t_lower)
    o.seed = int(seed)
    o.stream = int(stream)
    o.psi = _ptr(psi).value if psi is not None else None
    return o


def _use_torch_stream(ctx, x):
    if _is_torch(x) and x.is_cuda:
        import torch
        s = torch.cuda.current_stream(x.device).cuda_stream
        _check(ctx, load().corutv_set_stream(ctx, ctypes.c_void_p(s)))


# --------------------------------------------------------------------------
# the C entry points, one Python function each
# --------------------------------------------------------------------------

def corutv_create(device: int = 0, mem_budget_bytes: int = 0, max_slots: int = 0):
    h = ctypes.c_void_p()
    st = load().corutv_create(ctypes.byref(h), device, mem_budget_bytes, max_slots)
    if st != OK:
        raise CorutvError(st, load().corutv_last_error(None).decode())
    return h


def corutv_destroy(ctx) -> None:
    load().corutv_destroy(ctx)


def corutv_last_error(ctx=None) -> str:
    return load().corutv_last_error(ctx).decode()


def corutv_set_stream(ctx, stream_handle: int) -> None:
    _check(ctx, load().corutv_set_stream(ctx, ctypes.c_void_p(stream_handle)))


def corutv_sync(ctx) -> int:
    return _check(ctx, load().corutv_sync(ctx))


def corutv_factor(ctx, A, k: int, p: int, q: int, prec="f64", U=None, T=None, V=None, perm=None,
                  psi=None, seed: int = 0, stream: int = 0, d_mode: int = 0, t_lower: int = 0,
                  power_form: int = 0, bf16_last_round: int = 0) -> int:
    """Algorithm 1 into caller-provided U (m x ell), T (ell x ell), V (n x ell),
    perm (ell int32). Buffers must share A's device and dtype. t_lower = 1:
    the lower-triangular-T variant (Algorithm 1 on A^T; psi is then m x ell)."""
    m, n = A.shape
    o = _opts(k, p, q, prec, seed, stream, psi, d_mode, t_lower, power_form, bf16_last_round)
    _use_torch_stream(ctx, A)
    st = load().corutv_factor(ctx, _dtype_code(A), _ptr(A), m, n, _rowmajor_ld(A), ctypes.byref(o),
                              _ptr(U), _rowmajor_ld(U) if U is not None else 0, _ptr(T), _ptr(V),
                              _rowmajor_ld(V) if V is not None else 0, _ptr(perm))
    return _check(ctx, st)


def allreduce_callback(sum_fn):
    """A corutv_allreduce_fn from a Python function sum_fn(array) that
    replaces a 1-D numpy array (float64 or float32, a view of the library's
    host buffer) by its sum over the ranks. Keep the returned object alive
    for as long as the library may call it."""
    def cb(buf, count, dtype, user):
        try:
            ct = ctypes.c_double if dtype == F64 else ctypes.c_float
            arr = np.ctypeslib.as_array(ctypes.cast(buf, ctypes.POINTER(ct)), shape=(int(count),))
            sum_fn(arr)
            return OK
        except Exception:  # reported to the library as a failed exchange
            return ECUDA
    return ALLREDUCE_FN(cb)


def torch_distributed_sum(arr) -> None:
    """sum_fn for allreduce_callback over the default torch.distributed group
    (for example gloo): the array is summed in place."""
    import torch
    import torch.distributed as dist
    t = torch.from_numpy(arr)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)


def corutv_factor_rows(ctx, A_local, m_total: int, k: int, p: int, q: int, prec, allreduce, U=None, T=None,
                       V=None, perm=None, seed: int = 0, stream: int = 0) -> int:
    """The row-partitioned form: this rank's rows A_local (device), the rows of
    all ranks m_total; allreduce from allreduce_callback (the same on every
    rank). U: this rank's rows of U; T, V, perm replicated."""
    m, n = A_local.shape
    o = _opts(k, p, q, prec, seed, stream)
    _use_torch_stream(ctx, A_local)
    st = load().corutv_factor_rows(ctx, _dtype_code(A_local), _ptr(A_local), m, n, _rowmajor_ld(A_local),
                                   int(m_total), ctypes.byref(o), allreduce, None, _ptr(U),
                                   _rowmajor_ld(U) if U is not None else 0, _ptr(T), _ptr(V),
                                   _rowmajor_ld(V) if V is not None else 0, _ptr(perm))
    return _check(ctx, st)


def corutv_rpca(ctx, M, k: int, L, S, lam=0.0, mu0=0.0, mu_bar=0.0, rho=0.0, tol=0.0, max_iter=0,
                prec="f32", seed: int = 0, stream: int = 0, allow_notconv: bool = False) -> dict:
    """Algorithm 2 into caller-provided L and S (m x n, like M)."""
    m, n = M.shape
    o = _opts(k, k, 1, prec, seed, stream)
    it = ctypes.c_int(0)
    z = ctypes.c_double(0.0)
    r = ctypes.c_int(0)
    _use_torch_stream(ctx, M)
    st = load().corutv_rpca(ctx, _dtype_code(M), _ptr(M), m, n, _rowmajor_ld(M), ctypes.byref(o), lam, mu0,
                            mu_bar, rho, tol, int(max_iter), _ptr(L), _ptr(S), ctypes.byref(it),
                            ctypes.byref(z), ctypes.byref(r))
    _check(ctx, st, allow=(OK, ENOTCONV) if allow_notconv else (OK,))
    return {"status": st, "iters": it.value, "zeta": z.value, "rank": r.value}


def make_request(A, k, p, q, prec, U, T, V=None, perm=None, psi=None, seed=0, stream=0, d_mode=0,
                 t_lower=0, power_form=0, bf16_last_round=0) -> Request:
    """Request descriptor; for a CUDA tensor A it remembers the torch stream
    current now, which corutv_submit makes the context's stream so that the
    request waits for A's producer on it."""
    m, n = A.shape
    rq = Request()
    if _is_torch(A) and A.is_cuda:
        import torch
        rq._torch_stream = torch.cuda.current_stream(A.device).cuda_stream
    rq.dtype = _dtype_code(A)
    rq.A = _ptr(A).value
    rq.m, rq.n, rq.lda = m, n, _rowmajor_ld(A)
    rq.opts = _opts(k, p, q, prec, seed, stream, psi, d_mode, t_lower, power_form, bf16_last_round)
    rq.U = _ptr(U).value if U is not None else None
    rq.T = _ptr(T).value
    rq.V = _ptr(V).value if V is not None else None
    rq.ldu = _rowmajor_ld(U) if U is not None else 0
    rq.ldv = _rowmajor_ld(V) if V is not None else 0
    rq.perm = _ptr(perm).value if perm is not None else None
    return rq


def corutv_submit(ctx, req: Request) -> int:
    t = ctypes.c_uint64(0)
    s = getattr(req, "_torch_stream", None)
    if s is not None:
        _check(ctx, load().corutv_set_stream(ctx, ctypes.c_void_p(s)))
    _check(ctx, load().corutv_submit(ctx, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def corutv_factor_batch(ctx, reqs) -> int:
    """Grouped launches over the requests (make_request descriptors, device
    tensors), enqueued on the torch stream current for the first request's A."""
    arr = (Request * len(reqs))(*reqs)
    s = getattr(reqs[0], "_torch_stream", None) if reqs else None
    if s is not None:
        _check(ctx, load().corutv_set_stream(ctx, ctypes.c_void_p(s)))
    return _check(ctx, load().corutv_factor_batch(ctx, arr, len(reqs)))


def corutv_set_batching(ctx, max_batch: int) -> int:
    return _check(ctx, load().corutv_set_batching(ctx, int(max_batch)))


def corutv_poll(ctx, ticket: int, timeout_us: int = -1):
    """Returns (status, latency_s); status EPENDING / ETIMEDOUT when unfinished."""
    lat = ctypes.c_double(0.0)
    st = load().corutv_poll(ctx, ticket, timeout_us, ctypes.byref(lat))
    _check(ctx, st, allow=(OK, EPENDING, ETIMEDOUT))
    return st, lat.value


STAGE_SKETCH, STAGE_PROJECT, STAGE_ORTH, STAGE_QRCP, STAGE_FACTOR, STAGE_ALL = 0, 1, 2, 3, 4, -1


def corutv_set_autotune(enable: bool = True) -> None:
    """Tune the tensor-core products' stage shape on first use (process-wide)."""
    status = load().corutv_set_autotune(int(bool(enable)))
    if status != OK:
        raise CorutvError(status, "corutv_set_autotune failed")


def corutv_autotune_entries() -> list:
    """The tuned product shapes and their choices."""
    lib = load()
    out = []
    i = 0
    while True:
        mt, kt = ctypes.c_int64(), ctypes.c_int64()
        nb, tr, kg, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        us = ctypes.c_float()
        count = lib.corutv_autotune_entry(i, ctypes.byref(mt), ctypes.byref(kt), ctypes.byref(nb), ctypes.byref(tr),
                                          ctypes.byref(kg), ctypes.byref(st), ctypes.byref(us))
        if i >= count:
            return out
        out.append({"m": mt.value, "k": kt.value, "panel_cols": nb.value, "trans": tr.value,
                    "kgroup": kg.value, "stages": st.value, "us": us.value})
        i += 1


def corutv_set_graphs(ctx, enable: bool = True) -> None:
    """Replay repeated device-pointer factorisations from captured CUDA graphs."""
    _check(ctx, load().corutv_set_graphs(ctx, int(bool(enable))))


def corutv_profile_enable(ctx, enable: bool = True) -> None:
    _check(ctx, load().corutv_profile_enable(ctx, int(bool(enable))))


def corutv_profile_read(ctx, stage: int):
    """(total_ms, count) of a stage; for STAGE_ALL, (0.0, kernels launched)."""
    ms = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    _check(ctx, load().corutv_profile_read(ctx, int(stage), ctypes.byref(ms), ctypes.byref(cnt)))
    return ms.value, cnt.value


def corutv_gaussian(ctx, seed: int, stream: int, psi) -> None:
    n, ell = psi.shape
    _use_torch_stream(ctx, psi)
    _check(ctx, load().corutv_gaussian(ctx, seed, stream, n, ell, _ptr(psi), _rowmajor_ld(psi)))


def corutv_sketch(ctx, A, X, C, trans: int, prec="f64") -> None:
    m, n = A.shape
    ell = X.shape[1]
    _use_torch_stream(ctx, A)
    p = PREC_NAMES[prec] if isinstance(prec, str) else int(prec)
    _check(ctx, load().corutv_sketch(ctx, _dtype_code(A), p, int(trans), _ptr(A), m, n, _rowmajor_ld(A),
                                     _ptr(X), _rowmajor_ld(X), ell, _ptr(C), _rowmajor_ld(C)))


def corutv_orth(ctx, C, Q, R=None) -> None:
    rows, ell = C.shape
    _use_torch_stream(ctx, C)
    _check(ctx, load().corutv_orth(ctx, _ptr(C), rows, ell, _rowmajor_ld(C), _ptr(Q), _rowmajor_ld(Q), _ptr(R)))


def corutv_selftest_wait(ctx, limit_ns: int) -> None:
    """Enqueue the bounded-wait probe (see the header); corutv_sync then
    returns ETIMEDOUT."""
    _check(ctx, load().corutv_selftest_wait(ctx, int(limit_ns)))


def corutv_qrcp(ctx, D, Qt, Rt, perm) -> None:
    ell = D.shape[0]
    _use_torch_stream(ctx, D)
    _check(ctx, load().corutv_qrcp(ctx, _ptr(D), ell, _ptr(Qt), _ptr(Rt), _ptr(perm)))


def corutv_orth_noalloc(C, Q, R=None, info=None, stream_handle=None) -> None:
    """Thin QR like corutv_orth, for callers that cannot allocate device
    memory: no context, no allocation, temporaries in the library's fixed
    16 MiB device array. All tensors on the current CUDA device."""
    rows, ell = C.shape
    if stream_handle is None:
        import torch
        stream_handle = torch.cuda.current_stream(C.device).cuda_stream
    st = load().corutv_orth_noalloc(_ptr(C), rows, ell, _rowmajor_ld(C), _ptr(Q), _rowmajor_ld(Q), _ptr(R),
                                    _ptr(info), ctypes.c_void_p(stream_handle))
    if st != OK:
        raise CorutvError(st, load().corutv_last_error(None).decode())


# --------------------------------------------------------------------------
# convenience: allocate outputs like A and return them
# --------------------------------------------------------------------------

class Context:
    """Owns one corutv context; closes it on exit."""

    def __init__(self, device: int = 0, mem_budget_bytes: int = 0, max_slots: int = 0):
        self.handle = corutv_create(device, mem_budget_bytes, max_slots)

    def close(self):
        if self.handle is not None:
            corutv_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self, A, k, p, q, prec="f64", psi=None, seed=0, stream=0, want_uv=True, d_mode=0, t_lower=0,
               power_form=0, bf16_last_round=0):
        import torch
        m, n = A.shape
        ell = k + p
        kw = dict(device=A.device, dtype=A.dtype)
        U = torch.empty((m, ell), **kw) if want_uv else None
        V = torch.empty((n, ell), **kw) if want_uv else None
        T = torch.empty((ell, ell), **kw)
        perm = torch.empty(ell, dtype=torch.int32, device=A.device)
        corutv_factor(self.handle, A, k, p, q, prec, U, T, V, perm, psi, seed, stream, d_mode, t_lower,
                      power_form, bf16_last_round)
        return {"U": U, "T": T, "V": V, "perm": perm}

    def rpca(self, M, k, **kw):
        import torch
        L = torch.empty_like(M)
        S = torch.empty_like(M)
        out = corutv_rpca(self.handle, M, k, L, S, **kw)
        out.update({"L": L, "S": S})
        return out

    def sync(self):
        return corutv_sync(self.handle)
