"""The Chebyshev preconditioner M = p_d(K) applied in factored form (roots of
p_d, quadratic factors for conjugate pairs) and by Clenshaw's recurrence: the
same operator up to rounding, so per-probe quadratures agree with each other
and with the FP64 oracle (which sums the series by the T_j recurrence)."""
import numpy as np
import pytest

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


def _count(N, order, prec, form, degree, shifts, m, k, h=0.3, tol=0.0, patch=1):
    V = I.gaussian_wells(N, h, nwells=5, seed=1)
    with evc.Context.stencil(N, h, order, V, precision=prec) as ctx:
        ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, degree, 1.0)
        ctx.set_option(evc.EVC_OPT_CHEB_FORM, form)
        ctx.set_option(evc.EVC_OPT_STENCIL_PATCH, patch)
        L, q, st = ctx.count_slices(shifts, m, k, tol=tol, seed=0)
    return V, L, q, st


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("degree", [1, 3, 8, 12])
def test_factored_equals_clenshaw_and_oracle_fp64(order, degree):
    # odd degrees have a real root: the single-factor pass is exercised too
    N, shifts, m, k = 11, [-2.5, 0.5], 36, 10
    V, L1, q1, _ = _count(N, order, evc.EVC_FP64, evc.EVC_CHEB_FACTORED, degree, shifts, m, k)
    _, L2, q2, _ = _count(N, order, evc.EVC_FP64, evc.EVC_CHEB_CLENSHAW, degree, shifts, m, k)
    assert np.max(np.abs(q1 - q2)) < 1e-8
    P = O.Problem.stencil(N, 0.3, order, V, O.PREC_CHEB, cheb_degree=degree, cheb_c=1.0)
    qr, sr, Lr = O.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(q1 - qr)) < 1e-8


def test_factored_mixed_within_half_of_oracle():
    N, shifts, m, k = 16, [-3.0, 1.0], 64, 20
    V, L, q, _ = _count(N, 2, evc.EVC_MIXED, evc.EVC_CHEB_FACTORED, 8, shifts, m, k)
    _, Lc, qc, _ = _count(N, 2, evc.EVC_MIXED, evc.EVC_CHEB_CLENSHAW, 8, shifts, m, k)
    P = O.Problem.stencil(N, 0.3, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, sr, Lr = O.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(L - Lr)) < 0.5
    assert abs((L[1] - L[0]) - (Lr[1] - Lr[0])) < 0.5
    # rounding only: the two forms agree far inside the count tolerance
    assert np.max(np.abs(L - Lc)) < 0.05


@pytest.mark.parametrize("patch", [1, 2])
def test_factored_adaptive_stop_matches_oracle(patch):
    # chunks stop at different steps and leave the stencil grid on the device
    N, shifts = 10, list(np.linspace(-4.0, 2.0, 7))
    V, L, q, st = _count(N, 2, evc.EVC_FP64, evc.EVC_CHEB_FACTORED, 8, shifts, 16, 30, tol=0.25,
                         patch=patch)
    assert len(set(st)) > 1
    P = O.Problem.stencil(N, 0.3, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, sr, Lr = O.count(P, shifts, 16, 30, tol=0.25, seed=0)
    assert list(st) == list(sr)
    assert np.max(np.abs(q - qr)) < 1e-8


def test_cheb_form_option_validates():
    V = I.gaussian_wells(8, 0.3, nwells=2, seed=1)
    with evc.Context.stencil(8, 0.3, 2, V, precision=evc.EVC_FP64) as ctx:
        with pytest.raises(evc.EvcError):
            ctx.set_option(evc.EVC_OPT_CHEB_FORM, 2)


def test_bf16_basis_option():
    # accuracy trial: a BF16-rounded basis changes the estimate by far less
    # than the Hutchinson error but is not the FP32 result; FP64 contexts refuse it
    N, shifts, m, k = 16, [-3.0, 1.0], 64, 20
    V = I.gaussian_wells(N, 0.3, nwells=5, seed=1)
    with evc.Context.stencil(N, 0.3, 2, V, precision=evc.EVC_MIXED) as ctx:
        ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
        L32, q32, _ = ctx.count_slices(shifts, m, k, seed=0)
        ctx.set_option(evc.EVC_OPT_BASIS_BF16, 1)
        L16, q16, _ = ctx.count_slices(shifts, m, k, seed=0)
        ctx.set_option(evc.EVC_OPT_BASIS_BF16, 0)
        L32b, _, _ = ctx.count_slices(shifts, m, k, seed=0)
    np.testing.assert_array_equal(L32, L32b)
    assert not np.array_equal(q32, q16)
    assert np.all(np.isfinite(q16))
    assert np.max(np.abs(L16 - L32)) < 2.0
    with evc.Context.stencil(8, 0.3, 2, I.gaussian_wells(8, 0.3, nwells=2, seed=1),
                             precision=evc.EVC_FP64) as ctx:
        with pytest.raises(evc.EvcError):
            ctx.set_option(evc.EVC_OPT_BASIS_BF16, 1)
