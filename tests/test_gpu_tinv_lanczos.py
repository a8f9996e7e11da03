"""T^{-1}-inner-product Lanczos (Sec. 4, Eq. lanT1) on the GPU.

EVC_OPT_TINV_LANCZOS = 1 runs T (A - tau I) Y_k = Y_{k+1} J_{k+1,k} with
Y^T T^{-1} Y = I from y_1 = M q_1, for the Jacobi T = M^2.  The FP64 oracle of
the process (oracle/lanczos_tinv.py, carrying Z = T^{-1} Y through the
recurrence) gives the tridiagonal and, by Eq. gauss_quad, the per-probe
quadrature of every (shift, probe) column: FP64 within 1e-8, the tridiagonal
within 1e-10; the same numbers as Algorithm 1 (EVC_OPT_TINV_LANCZOS = 0)
within rounding; mixed-precision estimates within 0.5 of FP64.
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.lanczos_tinv import lanczos_tinv
from paper_1602_02306_gb300 import evc
from paper_1602_02306_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-8
EPS = 1e-3


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


def _oracle_tinv(P, shifts, m, k, seed=0, rule=evc.EVC_QUAD_GAUSS, steps=None):
    """Per-probe quadratures of Eq. lanT1 with the oracle's Jacobi M."""
    n = P.n
    q = np.zeros((len(shifts), m))
    tri = {}
    for s, tau in enumerate(shifts):
        mdiag = O.apply_M(P, tau, np.ones(n))
        ks = k if steps is None else int(steps[s])
        for j in range(m):
            v = O.probe_vector(seed, j, n)
            q1 = v / np.linalg.norm(v)
            # one step more than the rule needs: the GA rule reads beta_{k+1}
            al, be, kd = lanczos_tinv(lambda x: O.apply_A(P, x) - tau * x,
                                      lambda x: mdiag ** 2 * x, mdiag * q1, q1 / mdiag, ks)
            tri[(s, j)] = (al, be, kd)
            q[s, j] = (O.gauss_quad(al, be, n) if rule == evc.EVC_QUAD_GAUSS
                       else O.ga_quad(al, be, n))
    return q, tri


def test_csr_fp64_against_the_oracle_and_algorithm1():
    # 3 shifts x 37 probes: chunks mix shifts (the per-column weight path)
    csr = _indefinite()
    shifts, m, k = [-1.0, 0.25, 2.0], 37, 25
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, EPS)
        ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
        L, q, st = ctx.count_slices(shifts, m, k, seed=0)
        a, b, kd = ctx.tridiag(len(shifts) * m, k)
        ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 0)
        L1, q1, st1 = ctx.count_slices(shifts, m, k, seed=0)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI, jac_eps=EPS)
    qr, tri = _oracle_tinv(P, shifts, m, k)
    assert np.max(np.abs(q - qr)) < FP64_TOL
    assert np.max(np.abs(q - q1)) < FP64_TOL
    np.testing.assert_allclose(L, L1, rtol=0, atol=1e-9)
    assert list(st) == list(st1) == [k] * 3
    for c in (0, 36, 37, 74, 110):
        s, j = divmod(c, m)
        al, be, kdo = tri[(s, j)]
        assert kd[c] == kdo
        np.testing.assert_allclose(a[c, :kdo], al, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(b[c, :kdo + 1], be, rtol=1e-10, atol=1e-10)


def test_csr_fp64_adaptive_stop_and_ga_rule():
    # under a tolerance the stop steps equal Algorithm 1's; the GA rule too
    csr = _indefinite(257, seed=4)
    shifts, m, k = [-0.8, 0.6], 64, 30
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI, jac_eps=EPS)
    for rule in (evc.EVC_QUAD_GAUSS, evc.EVC_QUAD_GA):
        with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
            ctx.set_precond(evc.EVC_PREC_JACOBI, EPS)
            ctx.set_option(evc.EVC_OPT_QUADRATURE, rule)
            ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
            L, q, st = ctx.count_slices(shifts, m, k, tol=0.3, seed=5)
        qa, sa, La = O.count(P, shifts, m, k, tol=0.3, seed=5, rule=rule)
        assert list(st) == list(sa)
        assert np.max(np.abs(q - qa)) < FP64_TOL
        qr, _ = _oracle_tinv(P, shifts, m, k, seed=5, rule=rule, steps=st)
        assert np.max(np.abs(q - qr)) < FP64_TOL


@pytest.mark.parametrize("order,patch", [(2, 1), (4, 1), (2, 2), (4, 2)])
def test_stencil_fp64_against_the_oracle(order, patch):
    # per-thread pass and 2 x 2 patch pass (both scale output rows by T)
    N, h = 10, 0.3
    V = I.gaussian_wells(N, h, nwells=4, seed=1)
    shifts, m, k = [-2.0, -0.7], 40, 18
    with evc.Context.stencil(N, h, order, V, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, EPS)
        ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
        ctx.set_option(evc.EVC_OPT_STENCIL_PATCH, patch)
        L, q, st = ctx.count_slices(shifts, m, k, seed=2)
    P = O.Problem.stencil(N, h, order, V, O.PREC_JACOBI, jac_eps=EPS)
    qr, _ = _oracle_tinv(P, shifts, m, k, seed=2)
    assert np.max(np.abs(q - qr)) < FP64_TOL
    qa, sa, La = O.count(P, shifts, m, k, seed=2)
    assert np.max(np.abs(q - qa)) < FP64_TOL


def test_breakdown_on_a_small_matrix():
    # n = 20 < k: the process stops at the invariant subspace like Algorithm 1
    csr = _indefinite(20, seed=3)
    shifts, m, k = [0.1], 8, 30
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, EPS)
        ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
        L, q, st = ctx.count_slices(shifts, m, k, seed=1)
        a, b, kd = ctx.tridiag(m, 20)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI, jac_eps=EPS)
    qa, sa, La = O.count(P, shifts, m, k, seed=1)
    assert np.max(np.abs(q - qa)) < FP64_TOL
    assert all(1 <= int(x) <= 20 for x in kd[:m])


def test_mixed_estimate_within_half_of_fp64():
    csr = I.powerlaw_symmetric(20000, seed=2)
    shifts, m, k = [-0.5, 0.5], 64, 40
    out = {}
    for prec in (evc.EVC_FP64, evc.EVC_MIXED):
        with evc.Context.csr(csr, precision=prec) as ctx:
            ctx.set_precond(evc.EVC_PREC_JACOBI, EPS)
            ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
            out[prec] = ctx.count_slices(shifts, m, k, seed=0)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI, jac_eps=EPS)
    qr, sr, Lr = O.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(out[evc.EVC_FP64][1] - qr)) < FP64_TOL
    # the count of the interval, and each shift's n_below, in mixed precision
    Lm, Lf = out[evc.EVC_MIXED][0], out[evc.EVC_FP64][0]
    assert abs((Lm[1] - Lm[0]) - (Lf[1] - Lf[0])) < 0.5


def test_mixed_fp32_ragged_columns_against_fp64():
    # FP32 vectors with chunks that mix shifts (m = 45): the per-column T and
    # T^{-1} arrays of the operator and the reorthogonalisation
    csr = _indefinite(999, seed=12)
    shifts, m, k = [-1.5, 0.0, 1.5], 45, 30
    res = {}
    for prec in (evc.EVC_FP64, evc.EVC_MIXED):
        with evc.Context.csr(csr, precision=prec) as ctx:
            ctx.set_precond(evc.EVC_PREC_JACOBI, EPS)
            ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
            res[prec] = ctx.count_slices(shifts, m, k, seed=4)
    np.testing.assert_allclose(res[evc.EVC_MIXED][0], res[evc.EVC_FP64][0], rtol=0, atol=0.5)


def test_identity_is_algorithm1_and_unsupported_forms_fail():
    csr = _indefinite(200, seed=8)
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_IDENTITY)
        L0, q0, _ = ctx.count_slices([0.3], 32, 12, seed=0)
        ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
        L1, q1, _ = ctx.count_slices([0.3], 32, 12, seed=0)
        np.testing.assert_array_equal(q0, q1)     # T = I: the same process
        ctx.set_precond(evc.EVC_PREC_JACOBI, EPS)
        ctx.set_option(evc.EVC_OPT_METHOD, evc.EVC_METHOD_ARNOLDI)
        with pytest.raises(evc.EvcError) as e:
            ctx.count_slices([0.3], 32, 12, seed=0)
        assert e.value.code == evc.EVC_EUNSUPPORTED
        with pytest.raises(evc.EvcError):
            ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 2)
    V = I.gaussian_wells(8, 0.3, nwells=2, seed=1)
    with evc.Context.stencil(8, 0.3, 2, V, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
        ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
        with pytest.raises(evc.EvcError) as e:
            ctx.count_slices([-1.0], 32, 10, seed=0)
        assert e.value.code == evc.EVC_EUNSUPPORTED
        ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 0)
        ctx.count_slices([-1.0], 32, 10, seed=0)  # the context stays usable


@pytest.mark.parametrize("order", [2, 4])
def test_stencil_patch_pass_is_bitwise_the_per_thread_pass(order):
    # mixed precision, chunks that mix shifts (m = 24): the patch kernel's
    # T-scaled rows equal the per-thread kernel's bit for bit
    N, h = 12, 0.3
    V = I.gaussian_wells(N, h, nwells=4, seed=3)
    shifts, m, k = [-2.2, -1.0, 0.1], 24, 15
    res = []
    for patch in (1, 2):
        with evc.Context.stencil(N, h, order, V, precision=evc.EVC_MIXED) as ctx:
            ctx.set_precond(evc.EVC_PREC_JACOBI, EPS)
            ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, 1)
            ctx.set_option(evc.EVC_OPT_STENCIL_PATCH, patch)
            res.append(ctx.count_slices(shifts, m, k, seed=6))
    np.testing.assert_array_equal(res[0][1], res[1][1])
    np.testing.assert_array_equal(res[0][0], res[1][0])
