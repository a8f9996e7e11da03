"""GPU parity of the preconditioned Arnoldi-type estimator (Sec. 4) against
its FP64 oracle (oracle/arnoldi.py): same hashed probes, per-probe quadrature
within 1e-8 in FP64, estimate within 0.5 in mixed precision.  The GPU
orthogonalises with the Gram-corrected classical sweep where Algorithm 3
uses modified Gram-Schmidt, and takes e_1^T h(H_k) e_1 from the matrix sign
function where the paper uses Z and Z^{-1}: equal up to rounding."""
import numpy as np
import pytest

from oracle import arnoldi as AR
from oracle import oracle as O
from paper_1602_02306_gb300 import evc
from paper_1602_02306_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02306_gb300 import build
    build.build()
    evc.load()


def _stencil(N, order, V, prec, pk, shifts, m, k, tol=0.0, method=evc.EVC_METHOD_ARNOLDI):
    with evc.Context.stencil(N, 0.3, order, V, precision=prec) as ctx:
        if pk == "cheb":
            ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
        elif pk == "jacobi":
            ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        ctx.set_option(evc.EVC_OPT_METHOD, method)
        return ctx.count_slices(shifts, m, k, tol=tol, seed=0)


_OPK = {"cheb": O.PREC_CHEB, "jacobi": O.PREC_JACOBI, "identity": O.PREC_NONE}


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("pk", ["cheb", "jacobi", "identity"])
def test_stencil_arnoldi_fp64_per_probe(order, pk):
    N, shifts, m, k = 10, [-2.5, 0.5], 36, 12
    V = I.gaussian_wells(N, 0.3, nwells=4, seed=1)
    L, q, st = _stencil(N, order, V, evc.EVC_FP64, pk, shifts, m, k)
    P = O.Problem.stencil(N, 0.3, order, V, _OPK[pk], cheb_degree=8, cheb_c=1.0, jac_eps=1e-3)
    qr, sr, Lr = AR.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(q - qr)) < 1e-8
    np.testing.assert_allclose(L, Lr, rtol=0, atol=1e-9)


@pytest.mark.parametrize("pk", ["jacobi", "identity"])
def test_csr_arnoldi_fp64_per_probe(pk):
    A = I.random_symmetric_dense(300, seed=7)
    A[np.abs(A) < 1.2] = 0.0
    A = 0.5 * (A + A.T) + np.diag(np.linspace(-3, 3, 300))
    csr = I.dense_to_csr(A)
    shifts, m, k = [-1.0, 0.25, 2.0], 37, 20
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        if pk == "jacobi":
            ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        ctx.set_option(evc.EVC_OPT_METHOD, evc.EVC_METHOD_ARNOLDI)
        L, q, st = ctx.count_slices(shifts, m, k, seed=0)
    P = O.Problem.csr_matrix(csr, _OPK[pk], jac_eps=1e-3)
    qr, sr, Lr = AR.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(q - qr)) < 1e-8


def test_arnoldi_identity_equals_lanczos_on_gpu():
    # T = I, symmetric A: the Arnoldi quadrature is the Gauss quadrature
    N, shifts, m, k = 9, [-1.5, 0.8], 32, 10
    V = I.gaussian_wells(N, 0.3, nwells=3, seed=1)
    La, qa, _ = _stencil(N, 2, V, evc.EVC_FP64, "identity", shifts, m, k)
    Ll, ql, _ = _stencil(N, 2, V, evc.EVC_FP64, "identity", shifts, m, k,
                         method=evc.EVC_METHOD_LANCZOS)
    assert np.max(np.abs(qa - ql)) < 1e-8


def test_arnoldi_mixed_estimate_within_half():
    N, shifts, m, k = 16, [-3.0, 1.0], 64, 20
    V = I.gaussian_wells(N, 0.3, nwells=6, seed=1)
    L, q, st = _stencil(N, 2, V, evc.EVC_MIXED, "cheb", shifts, m, k)
    P = O.Problem.stencil(N, 0.3, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, sr, Lr = AR.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(L - Lr)) < 0.5
    assert abs((L[1] - L[0]) - (Lr[1] - Lr[0])) < 0.5


def test_arnoldi_adaptive_stop_matches_oracle():
    N, shifts = 8, list(np.linspace(-4.0, 2.0, 5))
    V = I.gaussian_wells(N, 0.3, nwells=3, seed=1)
    L, q, st = _stencil(N, 2, V, evc.EVC_FP64, "cheb", shifts, 12, 30, tol=0.25)
    P = O.Problem.stencil(N, 0.3, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, sr, Lr = AR.count(P, shifts, 12, 30, tol=0.25, seed=0)
    assert list(st) == list(sr)
    assert np.max(np.abs(q - qr)) < 1e-8


def test_arnoldi_limits():
    V = I.gaussian_wells(8, 0.3, nwells=2, seed=1)
    with evc.Context.stencil(8, 0.3, 2, V, precision=evc.EVC_FP64) as ctx:
        ctx.set_option(evc.EVC_OPT_METHOD, evc.EVC_METHOD_ARNOLDI)
        with pytest.raises(evc.EvcError):
            ctx.count_slices([0.0], 8, 91)
        ctx.set_option(evc.EVC_OPT_QUADRATURE, evc.EVC_QUAD_GA)
        with pytest.raises(evc.EvcError):
            ctx.count_slices([0.0], 8, 10)
        ctx.set_option(evc.EVC_OPT_QUADRATURE, evc.EVC_QUAD_GAUSS)
        ctx.count_slices([0.0], 8, 10)
        with pytest.raises(evc.EvcError):
            ctx.tridiag(8, 10)
        with pytest.raises(evc.EvcError):
            ctx.set_option(evc.EVC_OPT_METHOD, 2)


def test_arnoldi_long_run_matches_oracle():
    # 80 steps: H_80 in the quadrature kernel's shared memory
    N, shifts, m, k = 10, [-1.0, 0.5], 8, 80
    V = I.gaussian_wells(N, 0.3, nwells=4, seed=1)
    L, q, st = _stencil(N, 2, V, evc.EVC_FP64, "identity", shifts, m, k)
    P = O.Problem.stencil(N, 0.3, 2, V, O.PREC_NONE)
    qr, sr, Lr = AR.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(q - qr)) < 1e-7


def test_arnoldi_breakdown_at_p_distinct_eigenvalues():
    # T = I and p distinct eigenvalues: the Arnoldi process stops at step p
    # (h_{p+1,p} = 0) and the quadrature is exact, in both precisions
    distinct = [-2.0, -0.5, 0.7, 1.5, 3.0]
    A = I.random_symmetric_dense(64, seed=4, distinct=distinct)
    csr = I.dense_to_csr(A)
    w, U = np.linalg.eigh(A)
    for prec in (evc.EVC_FP64, evc.EVC_MIXED):
        with evc.Context.csr(csr, precision=prec) as ctx:
            ctx.set_option(evc.EVC_OPT_METHOD, evc.EVC_METHOD_ARNOLDI)
            L, q, st = ctx.count_slices([0.0], 4, 12, seed=0)
        for j in range(4):
            v = O.probe_vector(0, j, 64)
            exact = float(np.sum((U[:, w < 0].T @ v) ** 2))
            assert abs(q[0, j] - exact) < (1e-8 if prec == evc.EVC_FP64 else 1e-3)
