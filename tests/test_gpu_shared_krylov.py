"""Shared Krylov runs under the identity preconditioner.

Without a preconditioner, Algorithm 1 on A - tau I produces J_k(A) - tau I from
the same Krylov space for every tau, so one Lanczos run per probe serves all
shifts of a call: shift tau's Gauss quadrature (Eq. gauss_quad) sums the
weights of the Ritz values of J_k(A) below tau.  These tests compare the
shared run with per-shift runs (EVC_OPT_SHARED_KRYLOV = 0) and with the FP64
oracle, which runs Algorithm 1 on A - tau I for each shift separately:
per-probe quadrature within 1e-8 in FP64, stop steps equal, tridiagonals
within rounding; the estimate within 0.5 in mixed precision.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1602_02306_gb300 import evc
from paper_1602_02306_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02306_gb300 import build
    build.build()
    evc.load()


def _indefinite(n=300, seed=7):
    A = I.random_symmetric_dense(n, seed=seed)
    A[np.abs(A) < 1.2] = 0.0
    A = 0.5 * (A + A.T) + np.diag(np.linspace(-3, 3, n))
    return I.dense_to_csr(A)


@pytest.mark.parametrize("tol", [0.0, 0.25])
def test_shared_run_matches_oracle_per_shift_fp64(tol):
    csr = _indefinite()
    shifts, m, k = [-1.0, 0.25, 2.0], 37, 25
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_IDENTITY)
        L, q, st = ctx.count_slices(shifts, m, k, tol=tol, seed=0)
        a, b, kd = ctx.tridiag(len(shifts) * m, k)
        ctx.set_option(evc.EVC_OPT_SHARED_KRYLOV, 0)
        L0, q0, st0 = ctx.count_slices(shifts, m, k, tol=tol, seed=0)
    P = O.Problem.csr_matrix(csr, O.PREC_NONE)
    qr, sr, Lr = O.count(P, shifts, m, k, tol=tol, seed=0)
    assert list(st) == list(sr) == list(st0)
    assert np.max(np.abs(q - qr)) < FP64_TOL
    assert np.max(np.abs(q - q0)) < FP64_TOL
    np.testing.assert_allclose(L, Lr, rtol=0, atol=1e-9)
    # the reported tridiagonal of (shift s, probe j) is J_k(A) - tau_s I
    for c in (0, 36, 37, 110):
        s, j = divmod(c, m)
        v = O.probe_vector(0, j, 300)
        al, be, _, kdo = O.lanczos(P, shifts[s], v, int(st[s]))
        assert kd[c] == kdo
        np.testing.assert_allclose(a[c, :kdo], al, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(b[c, :kdo + 1], be, rtol=1e-10, atol=1e-10)


def test_shared_run_stencil_and_ga_rule():
    # a stencil Hamiltonian, both quadrature rules, 5 shifts
    N, h = 10, 0.3
    V = I.gaussian_wells(N, h, nwells=4, seed=1)
    shifts, m, k = [-3.0, -2.0, -1.2, -0.5, 0.3], 32, 16
    P = O.Problem.stencil(N, h, 2, V, O.PREC_NONE)
    for rule in (evc.EVC_QUAD_GAUSS, evc.EVC_QUAD_GA):
        with evc.Context.stencil(N, h, 2, V, precision=evc.EVC_FP64) as ctx:
            ctx.set_precond(evc.EVC_PREC_IDENTITY)
            ctx.set_option(evc.EVC_OPT_QUADRATURE, rule)
            L, q, st = ctx.count_slices(shifts, m, k, seed=3)
        qr, sr, Lr = O.count(P, shifts, m, k, seed=3, rule=rule)
        assert np.max(np.abs(q - qr)) < FP64_TOL


def test_shared_run_mixed_estimate():
    csr = I.powerlaw_symmetric(20000, seed=2)
    shifts, m, k = [-0.5, 0.5], 64, 40
    with evc.Context.csr(csr, precision=evc.EVC_MIXED) as ctx:
        ctx.set_precond(evc.EVC_PREC_IDENTITY)
        L, q, st = ctx.count_slices(shifts, m, k, seed=0)
    P = O.Problem.csr_matrix(csr, O.PREC_NONE)
    qr, sr, Lr = O.count(P, shifts, m, k, seed=0)
    assert abs((L[1] - L[0]) - (Lr[1] - Lr[0])) < 0.5
    assert np.max(np.abs(L - Lr)) < 0.5


def test_shared_run_async_outputs():
    # the asynchronous entry leaves every (shift, probe) quadrature on the
    # device, as the synchronous one returns them
    import torch
    csr = _indefinite(200, seed=9)
    shifts, m, k = [-0.7, 0.1, 0.9, 1.6], 40, 20
    with evc.Context.csr(csr, precision=evc.EVC_MIXED) as ctx:
        ctx.set_precond(evc.EVC_PREC_IDENTITY)
        L, q, st = ctx.count_slices(shifts, m, k, tol=0.3, seed=2)
        dq = torch.empty(len(shifts) * m, dtype=torch.float64, device="cuda")
        dL = torch.empty(len(shifts), dtype=torch.float64, device="cuda")
        ds = torch.empty(len(shifts), dtype=torch.int32, device="cuda")
        evc.evc_count_slices_async(ctx.h, shifts, m, k, 0.3, 2, dL.data_ptr(), dq.data_ptr(),
                                   ds.data_ptr())
        evc.evc_sync(ctx.h)
    np.testing.assert_array_equal(dq.cpu().numpy().reshape(len(shifts), m), q)
    np.testing.assert_array_equal(dL.cpu().numpy(), L)
    np.testing.assert_array_equal(ds.cpu().numpy(), st)
