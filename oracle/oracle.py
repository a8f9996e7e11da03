"""ctypes binding of the FP64 oracle (oracle/evc_oracle.c).

TEST INFRASTRUCTURE ONLY -- see the package docstring. The shared object is
compiled with plain gcc (-O2, OpenMP) on first use if it is missing.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evc_oracle.c")
_LIB = os.path.join(_HERE, "libevc_oracle.so")
_lock = threading.Lock()
_lib = None

OP_DENSE, OP_CSR, OP_STENCIL = 0, 1, 2
PREC_NONE, PREC_JACOBI, PREC_CHEB, PREC_DENSE = 0, 1, 2, 3

# Breakdown threshold of the FP64 oracle: beta_{i+1} <= 1e-12 * max(|alpha|, beta).
BREAKDOWN_REL = 1e-12


def build(force: bool = False) -> str:
    """Compile the oracle shared object (gcc, -O2, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("n", C.c_int64),
        ("op_kind", C.c_int32),
        ("prec_kind", C.c_int32),
        ("dense", C.c_void_p),
        ("row_ptr", C.c_void_p),
        ("col", C.c_void_p),
        ("val", C.c_void_p),
        ("N", C.c_int32),
        ("order", C.c_int32),
        ("h", C.c_double),
        ("V", C.c_void_p),
        ("jac_eps", C.c_double),
        ("cheb_degree", C.c_int32),
        ("reserved", C.c_int32),
        ("cheb_c", C.c_double),
        ("denseM", C.c_void_p),
    ]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            P = C.POINTER(_Problem)
            d = C.POINTER(C.c_double)
            lib.evo_mix64.restype = C.c_uint64
            lib.evo_mix64.argtypes = [C.c_uint64]
            lib.evo_probe_entry.restype = C.c_double
            lib.evo_probe_entry.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
            lib.evo_probe_vector.argtypes = [C.c_uint64, C.c_uint64, C.c_int64, d]
            for name in ("evo_apply_A",):
                getattr(lib, name).argtypes = [P, d, d]
            for name in ("evo_apply_M", "evo_apply_C"):
                getattr(lib, name).argtypes = [P, C.c_double, d, d]
            lib.evo_cheb_coeffs.argtypes = [C.c_int, C.c_double, C.c_double, d]
            lib.evo_kinetic_interval.argtypes = [P, d, d]
            lib.evo_lanczos.argtypes = [P, C.c_double, d, C.c_int, C.c_double, d, d, d,
                                        C.POINTER(C.c_int)]
            lib.evo_tridiag_eig.argtypes = [C.c_int, d, d, d, d]
            lib.evo_gauss_quad.restype = C.c_double
            lib.evo_gauss_quad.argtypes = [C.c_int, d, d, C.c_double]
            lib.evo_count.argtypes = [P, d, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_double,
                                      C.c_uint64, C.c_double, C.c_int, d,
                                      C.POINTER(C.c_int), d]
            lib.evo_count_rule.argtypes = [P, d, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                           C.c_double, C.c_uint64, C.c_double, C.c_int, C.c_int,
                                           C.c_int, d, C.POINTER(C.c_int), d]
            lib.evo_ga_quad.restype = C.c_double
            lib.evo_ga_quad.argtypes = [C.c_int, d, d, C.c_double]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Problem:
    """A (matrix, preconditioner) pair in the oracle's terms; keeps its arrays alive."""

    def __init__(self, n, op_kind, prec_kind=PREC_NONE, *, dense=None, csr=None, N=0, h=0.0,
                 order=2, V=None, jac_eps=1e-3, cheb_degree=8, cheb_c=1.0, denseM=None):
        self._keep = []
        s = _Problem()
        s.n = int(n)
        s.op_kind = op_kind
        s.prec_kind = prec_kind

        def keep(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a.ctypes.data

        s.dense = keep(dense, np.float64)
        if csr is not None:
            s.row_ptr = keep(csr[0], np.int64)
            s.col = keep(csr[1], np.int32)
            s.val = keep(csr[2], np.float64)
        s.N, s.order, s.h = int(N), int(order), float(h)
        s.V = keep(V, np.float64)
        s.jac_eps, s.cheb_degree, s.cheb_c = float(jac_eps), int(cheb_degree), float(cheb_c)
        s.denseM = keep(denseM, np.float64)
        self.s = s
        self.n = int(n)

    @classmethod
    def dense_matrix(cls, A, prec_kind=PREC_NONE, **kw):
        return cls(A.shape[0], OP_DENSE, prec_kind, dense=A, **kw)

    @classmethod
    def csr_matrix(cls, csr, prec_kind=PREC_NONE, **kw):
        return cls(len(csr[0]) - 1, OP_CSR, prec_kind, csr=csr, **kw)

    @classmethod
    def stencil(cls, N, h, order, V, prec_kind=PREC_NONE, **kw):
        return cls(N ** 3, OP_STENCIL, prec_kind, N=N, h=h, order=order, V=V, **kw)

    @property
    def ref(self):
        return C.byref(self.s)


def mix64(z: int) -> int:
    return int(_load().evo_mix64(C.c_uint64(z & 0xFFFFFFFFFFFFFFFF)))


def probe_vector(seed: int, j: int, n: int) -> np.ndarray:
    v = np.empty(n, dtype=np.float64)
    _load().evo_probe_vector(seed, j, n, _dp(v))
    return v


def apply_A(P: Problem, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(P.n)
    assert _load().evo_apply_A(P.ref, _dp(x), _dp(y)) == 0
    return y


def apply_M(P: Problem, tau, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(P.n)
    assert _load().evo_apply_M(P.ref, tau, _dp(x), _dp(y)) == 0
    return y


def apply_C(P: Problem, tau, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(P.n)
    assert _load().evo_apply_C(P.ref, tau, _dp(x), _dp(y)) == 0
    return y


def cheb_coeffs(degree, a, b):
    c = np.empty(degree + 1)
    assert _load().evo_cheb_coeffs(degree, a, b, _dp(c)) == 0
    return c


def kinetic_interval(P: Problem):
    a, b = C.c_double(), C.c_double()
    assert _load().evo_kinetic_interval(P.ref, C.byref(a), C.byref(b)) == 0
    return a.value, b.value


def lanczos(P: Problem, tau, v, k, breakdown_rel=BREAKDOWN_REL, want_Q=False):
    """Algorithm 1: returns (alpha[k_done], beta[k_done+1], Q or None, k_done)."""
    v = np.ascontiguousarray(v, dtype=np.float64)
    alpha = np.zeros(k)
    beta = np.zeros(k + 1)
    Q = np.zeros((k + 1, P.n)) if want_Q else None
    kd = C.c_int(0)
    rc = _load().evo_lanczos(P.ref, tau, _dp(v), k, breakdown_rel, _dp(alpha), _dp(beta),
                             _dp(Q) if want_Q else None, C.byref(kd))
    assert rc == 0, rc
    kd = kd.value
    return alpha[:kd], beta[:kd + 1], (Q[:kd + 1] if want_Q else None), kd


def tridiag_eig(alpha, beta):
    """Eigenvalues (ascending) and eigenvector first components of J_k."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    k = alpha.size
    if beta.size < k:
        beta = np.concatenate([beta, np.zeros(k - beta.size)])
    th = np.empty(k)
    z1 = np.empty(k)
    assert _load().evo_tridiag_eig(k, _dp(alpha), _dp(beta), _dp(th), _dp(z1)) == 0
    return th, z1


def gauss_quad(alpha, beta, vnorm2):
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    k = alpha.size
    if beta.size < k:
        beta = np.concatenate([beta, np.zeros(k - beta.size)])
    return float(_load().evo_gauss_quad(k, _dp(alpha), _dp(beta), vnorm2))


def ga_quad(alpha, beta, vnorm2):
    """Generalized averaged Gauss quadrature from alpha[k], beta[k+1]."""
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    assert beta.size >= alpha.size + 1
    return float(_load().evo_ga_quad(alpha.size, _dp(alpha), _dp(beta), vnorm2))


def quad_bound_log10(beta, k, vnorm2):
    """log10 of the computable factor of the Gauss quadrature error bound
    (Sec. 3, Eq. qbound): after k Lanczos steps from v/||v||,
        |eps_k| <= N_k * ||v||^2 * beta_2^2 ... beta_{k+1}^2 / (2k)!
    where N_k bounds |f^(2k)| on an interval holding the spectrum; this
    returns log10(||v||^2 beta_2^2 ... beta_{k+1}^2 / (2k)!).  beta[i] is
    beta_{i+1} (beta[0] = beta_1 = 0).  A zero beta_j (j = 2..k+1: the process
    broke down) makes the rule exact (Proposition 1): -inf."""
    beta = np.asarray(beta, dtype=np.float64)
    assert k >= 1 and beta.size >= k + 1
    s = np.log10(vnorm2)
    for j in range(2, k + 2):
        b = beta[j - 1]
        if not b > 0.0:
            return -np.inf
        s += 2.0 * np.log10(b)
    for i in range(1, 2 * k + 1):        # (2k)!
        s -= np.log10(i)
    return float(s)


def count(P: Problem, shifts, m, kmax, tol=0.0, seed=0, probe_ids=None,
          breakdown_rel=BREAKDOWN_REL, nthreads=0, rule=0, min_steps=3):
    """Algorithm 2 for every shift: returns (quad[S, m], steps[S], L[S]).

    rule 0: Gauss quadrature (Eq. gauss_quad); 1: generalized averaged Gauss
    (Sec. 3.4)."""
    shifts = np.ascontiguousarray(shifts, dtype=np.float64)
    S = shifts.size
    quad = np.zeros(S * m)
    steps = np.zeros(S, dtype=np.int32)
    L = np.zeros(S)
    pid = None
    if probe_ids is not None:
        pid = np.ascontiguousarray(probe_ids, dtype=np.int64)
        assert pid.size == m
    rc = _load().evo_count_rule(P.ref, _dp(shifts), S, m,
                                pid.ctypes.data if pid is not None else None, kmax, tol,
                                C.c_uint64(seed), breakdown_rel, nthreads, int(rule),
                                int(min_steps), _dp(quad),
                                steps.ctypes.data_as(C.POINTER(C.c_int)), _dp(L))
    assert rc == 0, rc
    return quad.reshape(S, m), steps, L
