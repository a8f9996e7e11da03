"""Thin ctypes binding of libevc (include/evc.h).

Argument marshalling only: every step of the estimator runs in the CUDA
library.  Functions keep the C names; ``Context`` is a small convenience
wrapper that owns an ``evc_ctx*`` and hands torch-allocated device scratch to
the library (PyTorch is used for device memory and streams only).

Importing this module does not load the library; the first call does, and it
raises ``RuntimeError`` if ``libevc.so`` is missing or cannot be loaded --
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libevc.so")
_lock = threading.Lock()
_lib = None

(EVC_OK, EVC_EINVAL, EVC_ENOMEM, EVC_ECUDA, EVC_ENUMERIC, EVC_ETIMEOUT, EVC_EUNSUPPORTED,
 EVC_EAGAIN) = range(8)
EVC_FP64, EVC_MIXED = 0, 1
EVC_PREC_IDENTITY, EVC_PREC_JACOBI, EVC_PREC_CHEB_KINETIC = 0, 1, 2
EVC_OPT_GRAPH, EVC_OPT_PROFILE, EVC_OPT_QUADRATURE, EVC_OPT_MIN_STEPS, EVC_OPT_PROBE_OFFSET = 1, 2, 3, 4, 5
EVC_OPT_CHEB_FORM = 6
EVC_OPT_BASIS_BF16 = 7
EVC_OPT_REORTH_ROWS, EVC_OPT_STENCIL_ZB, EVC_OPT_CSR_THREADS = 8, 9, 10
EVC_OPT_METHOD = 11
EVC_OPT_STENCIL_PATCH = 12
EVC_OPT_STENCIL_GROUPS = 13
EVC_OPT_SHARED_KRYLOV = 14
EVC_OPT_TINV_LANCZOS = 15
EVC_METHOD_LANCZOS, EVC_METHOD_ARNOLDI = 0, 1
EVC_CHEB_FACTORED, EVC_CHEB_CLENSHAW = 0, 1
EVC_QUAD_GAUSS, EVC_QUAD_GA = 0, 1
(EVC_K_INIT, EVC_K_JACOBI, EVC_K_STENCIL, EVC_K_CSR, EVC_K_DOTS, EVC_K_REDUCE, EVC_K_UPDATE,
 EVC_K_FINISH) = range(8)
KERNEL_NAMES = ["init", "jacobi", "stencil", "csr", "dots", "reduce", "update", "finish"]
EVC_MAX_STEPS = 256

# Symbols declared in include/evc.h, in declaration order.
EXPORTED = [
    "evc_create_csr", "evc_create_stencil", "evc_set_values", "evc_set_precond",
    "evc_workspace_bytes", "evc_set_workspace", "evc_count", "evc_count_slices",
    "evc_count_slices_async", "evc_sync", "evc_get_tridiag", "evc_get_quad_bound", "evc_set_option",
    "evc_get_profile", "evc_autotune", "evc_server_create", "evc_server_add_matrix", "evc_server_submit",
    "evc_server_poll", "evc_server_wait", "evc_server_stats", "evc_server_destroy",
    "evc_gauss_quadrature_static", "evc_wait_selftest", "evc_last_error", "evc_destroy",
    "evc_version", "evc_cheb_kinetic",
]


class EvcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"evc error {code}: {msg}")
        self.code = code


class evc_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p), ("val_is_fp32", C.c_int32),
                ("on_device", C.c_int32), ("check", C.c_int32), ("reserved", C.c_int32)]


class evc_prof_rec(C.Structure):
    _fields_ = [("kind", C.c_int32), ("step", C.c_int32), ("ms", C.c_double), ("bytes", C.c_double),
                ("span", C.c_int32), ("reserved", C.c_int32)]


class evc_tuning(C.Structure):
    _fields_ = [("stencil_zb", C.c_int), ("stencil_patch", C.c_int), ("stencil_groups", C.c_int),
                ("csr_threads", C.c_int),
                ("reorth_rows", C.c_int),
                ("steps", C.c_int), ("ms_before", C.c_double), ("ms_after", C.c_double)]


class evc_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("batch_size", C.c_int32), ("estimate", C.c_double),
                ("n_below", C.c_double * 2), ("steps", C.c_int32 * 2), ("t_submit", C.c_double),
                ("t_start", C.c_double), ("t_done", C.c_double)]


class evc_server_counters(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("used_bytes", C.c_uint64),
                ("peak_bytes", C.c_uint64), ("pending", C.c_int64), ("batches", C.c_int64),
                ("completed", C.c_int64), ("merged", C.c_int64)]


def lib_path() -> str:
    return _LIB_PATH


def load(path: str | None = None):
    """Load libevc.so (once) and declare the C signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or _LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libevc.so not built ({p}); run __graft_entry__.build()")
        lib = C.CDLL(p)
        vp, d, i32, i64, u64 = C.c_void_p, C.c_double, C.c_int, C.c_int64, C.c_uint64
        pp = C.POINTER(C.c_void_p)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        sig = {
            "evc_create_csr": (i32, [C.POINTER(evc_csr), i32, vp, pp]),
            "evc_create_stencil": (i32, [i32, d, i32, vp, i32, i32, i32, vp, pp]),
            "evc_set_values": (i32, [vp, vp, i32]),
            "evc_set_precond": (i32, [vp, i32, d, d]),
            "evc_workspace_bytes": (C.c_size_t, [vp, i32, i32, i32]),
            "evc_set_workspace": (i32, [vp, vp, C.c_size_t]),
            "evc_count": (i32, [vp, d, d, i32, i32, d, u64, dp, dp, ip]),
            "evc_count_slices": (i32, [vp, dp, i32, i32, i32, d, u64, dp, dp, ip]),
            "evc_count_slices_async": (i32, [vp, dp, i32, i32, i32, d, u64, vp, vp, vp]),
            "evc_sync": (i32, [vp]),
            "evc_get_tridiag": (i32, [vp, dp, dp, ip]),
            "evc_get_quad_bound": (i32, [vp, dp]),
            "evc_autotune": (i32, [vp, i32, i32, i32, C.POINTER(evc_tuning)]),
            "evc_wait_selftest": (i32, [d, C.POINTER(C.c_int)]),
            "evc_set_option": (i32, [vp, i32, i64]),
            "evc_get_profile": (i32, [vp, C.POINTER(evc_prof_rec), i32, ip]),
            "evc_server_create": (i32, [C.c_size_t, i32, i32, pp]),
            "evc_server_add_matrix": (i32, [vp, vp, ip]),
            "evc_server_submit": (i32, [vp, i32, d, d, i32, i32, d, u64, vp,
                                        C.POINTER(C.c_int64)]),
            "evc_server_poll": (i32, [vp, C.c_int64, C.POINTER(evc_result)]),
            "evc_server_wait": (i32, [vp, C.c_int64, d, C.POINTER(evc_result)]),
            "evc_server_stats": (i32, [vp, C.POINTER(evc_server_counters)]),
            "evc_server_destroy": (None, [vp]),
            "evc_gauss_quadrature_static": (i32, [vp, vp, vp, i32, i32, d, vp, vp, vp,
                                                  C.c_char_p, C.c_size_t]),
            "evc_last_error": (C.c_char_p, [vp]),
            "evc_destroy": (None, [vp]),
            "evc_version": (i32, []),
            "evc_cheb_kinetic": (i32, [i32, d, i32, d, i32, C.POINTER(C.c_double),
                                       C.POINTER(C.c_double), C.POINTER(C.c_double), ip]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int))


def _check(ctx, rc):
    if rc != EVC_OK:
        msg = load().evc_last_error(ctx).decode() if ctx else ""
        raise EvcError(rc, msg)


# ----------------------------------------------------------- C-named calls

def evc_create_csr(row_ptr, col, val, precision=EVC_FP64, stream=None, check=True, on_device=False):
    """row_ptr/col/val: numpy arrays (host) or torch CUDA tensors (on_device=True)."""
    lib = load()
    keep = []
    if on_device:
        n = int(row_ptr.numel()) - 1
        nnz = int(col.numel())
        a = evc_csr(n, nnz, row_ptr.data_ptr(), col.data_ptr(), val.data_ptr(),
                    1 if str(val.dtype) == "torch.float32" else 0, 1, 0, 0)
    else:
        rp = np.ascontiguousarray(row_ptr, dtype=np.int64)
        ci = np.ascontiguousarray(col, dtype=np.int32)
        fp32 = np.asarray(val).dtype == np.float32
        va = np.ascontiguousarray(val, dtype=np.float32 if fp32 else np.float64)
        keep += [rp, ci, va]
        a = evc_csr(len(rp) - 1, len(ci), rp.ctypes.data, ci.ctypes.data, va.ctypes.data,
                    1 if fp32 else 0, 0, 1 if check else 0, 0)
    out = C.c_void_p()
    rc = lib.evc_create_csr(C.byref(a), precision, stream, C.byref(out))
    if rc != EVC_OK:
        raise EvcError(rc, "evc_create_csr failed")
    return out.value


def evc_create_stencil(N, h, order, V, precision=EVC_FP64, stream=None, on_device=False):
    lib = load()
    if on_device:
        ptr, fp32 = V.data_ptr(), 1 if str(V.dtype) == "torch.float32" else 0
    else:
        fp32 = 1 if np.asarray(V).dtype == np.float32 else 0
        Va = np.ascontiguousarray(V, dtype=np.float32 if fp32 else np.float64)
        ptr = Va.ctypes.data
    out = C.c_void_p()
    rc = lib.evc_create_stencil(int(N), float(h), int(order), ptr, fp32, 1 if on_device else 0,
                                precision, stream, C.byref(out))
    if rc != EVC_OK:
        raise EvcError(rc, "evc_create_stencil failed")
    return out.value


def evc_set_values(ctx, values_ptr, on_device):
    _check(ctx, load().evc_set_values(ctx, values_ptr, 1 if on_device else 0))


def evc_set_precond(ctx, kind, p0=0.0, p1=0.0):
    _check(ctx, load().evc_set_precond(ctx, kind, float(p0), float(p1)))


def evc_workspace_bytes(ctx, nshift, nprobe, maxsteps):
    return int(load().evc_workspace_bytes(ctx, nshift, nprobe, maxsteps))


def evc_set_workspace(ctx, dptr, nbytes):
    _check(ctx, load().evc_set_workspace(ctx, dptr, nbytes))


def evc_count(ctx, xi, eta, nprobe, maxsteps, tol=0.0, seed=0):
    est = np.zeros(1)
    quad = np.zeros(2 * nprobe)
    steps = np.zeros(2, dtype=np.int32)
    _check(ctx, load().evc_count(ctx, xi, eta, nprobe, maxsteps, tol, C.c_uint64(seed),
                                 _dp(est), _dp(quad), _ip(steps)))
    return float(est[0]), quad.reshape(2, nprobe), steps


def evc_count_slices(ctx, shifts, nprobe, maxsteps, tol=0.0, seed=0):
    sh = np.ascontiguousarray(shifts, dtype=np.float64)
    S = sh.size
    L = np.zeros(S)
    quad = np.zeros(S * nprobe)
    steps = np.zeros(S, dtype=np.int32)
    _check(ctx, load().evc_count_slices(ctx, _dp(sh), S, nprobe, maxsteps, tol, C.c_uint64(seed),
                                        _dp(L), _dp(quad), _ip(steps)))
    return L, quad.reshape(S, nprobe), steps


def evc_count_slices_async(ctx, shifts, nprobe, maxsteps, tol, seed, d_n_below, d_quad, d_steps):
    sh = np.ascontiguousarray(shifts, dtype=np.float64)
    _check(ctx, load().evc_count_slices_async(ctx, _dp(sh), sh.size, nprobe, maxsteps, tol,
                                              C.c_uint64(seed), d_n_below, d_quad, d_steps))


def evc_sync(ctx):
    _check(ctx, load().evc_sync(ctx))


def evc_get_tridiag(ctx, ncol, maxsteps):
    a = np.zeros(ncol * maxsteps)
    b = np.zeros(ncol * (maxsteps + 1))
    kd = np.zeros(ncol, dtype=np.int32)
    _check(ctx, load().evc_get_tridiag(ctx, _dp(a), _dp(b), _ip(kd)))
    return a.reshape(ncol, maxsteps), b.reshape(ncol, maxsteps + 1), kd


def evc_get_quad_bound(ctx, ncol):
    out = np.zeros(ncol)
    _check(ctx, load().evc_get_quad_bound(ctx, _dp(out)))
    return out


def evc_set_option(ctx, option, value):
    _check(ctx, load().evc_set_option(ctx, option, int(value)))


def evc_autotune(ctx, nshift, nprobe, maxsteps):
    """Pick the kernels' tile shapes for this launch shape; returns the choice."""
    t = evc_tuning()
    _check(ctx, load().evc_autotune(ctx, nshift, nprobe, maxsteps, C.byref(t)))
    return {f: getattr(t, f) for f, _ in evc_tuning._fields_}


def evc_wait_selftest(limit_ms):
    """Run a wait that can never complete under a limit of limit_ms; returns the
    status the bounded wait produced (EVC_ETIMEOUT when it gave up as designed)."""
    st = C.c_int(-1)
    _check(None, load().evc_wait_selftest(float(limit_ms), C.byref(st)))
    return st.value


def evc_get_profile(ctx):
    """Launch list of the last call: list of (kind, step, ms, bytes, span);
    span = 1 marks the record that times a concurrent chunk-group segment."""
    lib = load()
    n = C.c_int(0)
    _check(ctx, lib.evc_get_profile(ctx, None, 0, C.byref(n)))
    recs = (evc_prof_rec * max(1, n.value))()
    _check(ctx, lib.evc_get_profile(ctx, recs, n.value, C.byref(n)))
    return [(r.kind, r.step, r.ms, r.bytes, r.span) for r in recs[:n.value]]


EVC_STATIC_QUAD_MAX = 262144


# ------------------------------------------------------------------ server

def _result_dict(r):
    return {"status": r.status, "batch_size": r.batch_size, "estimate": r.estimate,
            "n_below": [r.n_below[0], r.n_below[1]], "steps": [r.steps[0], r.steps[1]],
            "t_submit": r.t_submit, "t_start": r.t_start, "t_done": r.t_done}


def evc_server_create(budget_bytes, slots=4, max_batch=16):
    out = C.c_void_p()
    rc = load().evc_server_create(int(budget_bytes), slots, max_batch, C.byref(out))
    if rc != EVC_OK:
        raise EvcError(rc, "evc_server_create failed")
    return out.value


def evc_server_add_matrix(srv, ctx):
    mid = C.c_int(0)
    rc = load().evc_server_add_matrix(srv, ctx, C.byref(mid))
    if rc != EVC_OK:
        raise EvcError(rc, "evc_server_add_matrix failed")
    return mid.value


def evc_server_submit(srv, matrix_id, xi, eta, nprobe, maxsteps, tol=0.0, seed=0, quad_buf=None):
    """quad_buf: optional float64 numpy array of 2*nprobe, filled on completion."""
    t = C.c_int64(0)
    ptr = quad_buf.ctypes.data if quad_buf is not None else None
    rc = load().evc_server_submit(srv, matrix_id, xi, eta, nprobe, maxsteps, tol, C.c_uint64(seed),
                                  ptr, C.byref(t))
    if rc != EVC_OK:
        raise EvcError(rc, "evc_server_submit failed")
    return t.value


def evc_server_wait(srv, ticket, timeout_s=-1.0):
    r = evc_result()
    rc = load().evc_server_wait(srv, ticket, timeout_s, C.byref(r))
    return rc, _result_dict(r)


def evc_server_poll(srv, ticket):
    r = evc_result()
    rc = load().evc_server_poll(srv, ticket, C.byref(r))
    return rc, _result_dict(r)


def evc_server_stats(srv):
    st = evc_server_counters()
    rc = load().evc_server_stats(srv, C.byref(st))
    if rc != EVC_OK:
        raise EvcError(rc, "evc_server_stats failed")
    return {k: getattr(st, k) for k, _ in st._fields_}


def evc_server_destroy(srv):
    if srv:
        load().evc_server_destroy(srv)


def evc_gauss_quadrature_static(d_alpha, d_beta, d_kcol, k, ncol, vnorm2, d_quad, d_status=None,
                                stream=None):
    """Allocation-free quadrature (device pointers in and out; d_status an
    optional device int32 that receives the kernel's status); returns
    (status of the call, message)."""
    buf = C.create_string_buffer(256)
    rc = load().evc_gauss_quadrature_static(d_alpha, d_beta, d_kcol, int(k), int(ncol),
                                            float(vnorm2), d_quad, d_status, stream, buf, 256)
    return rc, buf.value.decode()


def evc_last_error(ctx):
    return load().evc_last_error(ctx).decode()


def evc_destroy(ctx):
    if ctx:
        load().evc_destroy(ctx)


def evc_version():
    return int(load().evc_version())


def evc_cheb_kinetic(order, h, degree, c=1.0, N=0):
    """The kinetic Chebyshev preconditioner the library builds (host only):
    dict with a, b, pmin (over the N^3 grid's spectrum; 0.0 for N = 0), g,
    sign, coef[d+1] and factors [(re, im, is_pair)]."""
    lib = load()
    info = (C.c_double * 5)()
    coef = (C.c_double * (max(degree, 0) + 1))()
    fac = (C.c_double * (3 * max(degree, 1)))()
    nf = C.c_int(0)
    rc = lib.evc_cheb_kinetic(order, h, degree, c, N, info, coef, fac, C.byref(nf))
    if rc != EVC_OK:
        raise EvcError(rc, "evc_cheb_kinetic: invalid arguments")
    return {"a": info[0], "b": info[1], "pmin": info[2], "g": info[3], "sign": info[4],
            "coef": np.array(coef[:degree + 1]),
            "factors": [(fac[3 * f], fac[3 * f + 1], fac[3 * f + 2] != 0.0) for f in range(nf.value)]}


# ------------------------------------------------------------- convenience

class Context:
    """Owns an evc_ctx*; optionally backs its scratch with a torch CUDA buffer."""

    def __init__(self, handle, torch_workspace=True):
        self.h = handle
        self._ws = None
        self._torch_ws = torch_workspace

    @classmethod
    def csr(cls, csr, precision=EVC_FP64, stream=None, **kw):
        return cls(evc_create_csr(*csr, precision=precision, stream=stream), **kw)

    @classmethod
    def stencil(cls, N, h, order, V, precision=EVC_FP64, stream=None, **kw):
        return cls(evc_create_stencil(N, h, order, V, precision=precision, stream=stream), **kw)

    def set_precond(self, kind, p0=0.0, p1=0.0):
        evc_set_precond(self.h, kind, p0, p1)
        return self

    def set_option(self, option, value):
        evc_set_option(self.h, option, value)
        return self

    def autotune(self, nshift, nprobe, maxsteps):
        return evc_autotune(self.h, nshift, nprobe, maxsteps)

    def reserve(self, nshift, nprobe, maxsteps):
        """Allocate the library's scratch from the torch caching allocator."""
        need = evc_workspace_bytes(self.h, nshift, nprobe, maxsteps)
        if self._torch_ws and (self._ws is None or self._ws.numel() < need):
            import torch
            self._ws = None
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
            ptr = self._ws.data_ptr()
            aligned = (ptr + 255) & ~255
            evc_set_workspace(self.h, aligned, need + 256 - (aligned - ptr))

    def count(self, xi, eta, nprobe, maxsteps, tol=0.0, seed=0):
        self.reserve(2, nprobe, maxsteps)
        return evc_count(self.h, xi, eta, nprobe, maxsteps, tol, seed)

    def count_slices(self, shifts, nprobe, maxsteps, tol=0.0, seed=0):
        self.reserve(len(shifts), nprobe, maxsteps)
        return evc_count_slices(self.h, shifts, nprobe, maxsteps, tol, seed)

    def tridiag(self, ncol, maxsteps):
        return evc_get_tridiag(self.h, ncol, maxsteps)

    def quad_bound(self, ncol):
        return evc_get_quad_bound(self.h, ncol)

    def close(self):
        if self.h:
            evc_destroy(self.h)
            self.h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
