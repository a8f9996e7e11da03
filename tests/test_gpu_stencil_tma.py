"""The stencil pass on tensor-copied block tiles (EVC_OPT_STENCIL_PATCH = 3):
the same points, operands and arithmetic as the 2 x 2 patch pass, so every
count is bitwise the patch pass's -- for both stencil orders and precisions,
every operand set the library issues (Chebyshev factors and Clenshaw steps,
the shifted Hamiltonian with -beta q_(i-1), the T-scaled rows of the
T^-1-inner-product process), short z segments that leave the copy pipeline
partly filled, concurrent chunk groups and adaptive stops -- and FP64 stays on
the oracle.  Grids that are not a whole number of tiles fall back to the patch
pass."""
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


def _run(N, order, prec, precond, patch, zb=32, groups=1, form=evc.EVC_CHEB_FACTORED, tinv=0,
         shifts=(-2.0, 0.5), m=40, k=8, tol=0.0, graph=True):
    V = I.gaussian_wells(N, 0.3, nwells=4, seed=1)
    with evc.Context.stencil(N, 0.3, order, V, precision=prec) as ctx:
        if precond == "cheb":
            ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
            ctx.set_option(evc.EVC_OPT_CHEB_FORM, form)
        elif precond == "jacobi":
            ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3, 0.0)
            ctx.set_option(evc.EVC_OPT_TINV_LANCZOS, tinv)
        ctx.set_option(evc.EVC_OPT_STENCIL_PATCH, patch)
        ctx.set_option(evc.EVC_OPT_STENCIL_ZB, zb)
        ctx.set_option(evc.EVC_OPT_STENCIL_GROUPS, groups)
        if not graph:
            ctx.set_option(evc.EVC_OPT_GRAPH, 0)
        L, q, st = ctx.count_slices(list(shifts), m, k, tol=tol, seed=0)
    return V, L, q, st


def _same(a, b):
    for x, y in zip(a[1:], b[1:]):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("prec", [evc.EVC_MIXED, evc.EVC_FP64])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("N", [8, 16, 24])
def test_tiles_equal_patch_chebyshev(N, order, prec):
    # 2 shifts x 40 probes = 3 chunks, one of them mixing shifts; N = 8 is a
    # single tile whose arms wrap on both sides
    for zb in (1, 5, 32):
        _same(_run(N, order, prec, "cheb", 2, zb=zb), _run(N, order, prec, "cheb", 3, zb=zb))


@pytest.mark.parametrize("prec", [evc.EVC_MIXED, evc.EVC_FP64])
@pytest.mark.parametrize("order", [2, 4])
def test_tiles_equal_patch_other_operand_sets(order, prec):
    # Clenshaw steps (x, prev and pp operands), the unpreconditioned shifted
    # Hamiltonian (V, shift and pp), and the T-scaled rows of the T^-1 process
    N = 16
    for kw in (dict(precond="cheb", form=evc.EVC_CHEB_CLENSHAW),
               dict(precond="none"),
               dict(precond="jacobi", tinv=1)):
        for zb in (3, 16):
            _same(_run(N, order, prec, patch=2, zb=zb, **kw), _run(N, order, prec, patch=3, zb=zb, **kw))


@pytest.mark.parametrize("prec", [evc.EVC_MIXED, evc.EVC_FP64])
def test_tiles_groups_stop_and_no_graph(prec):
    # concurrent chunk groups, an adaptive stop that switches chunks off, and
    # launches outside a graph
    args = dict(N=24, order=4, prec=prec, precond="cheb", shifts=(-3.0, -1.0, 0.5), m=64, k=20,
                tol=0.3)
    ref = _run(patch=2, **args)
    _same(ref, _run(patch=3, groups=3, **args))
    _same(ref, _run(patch=3, graph=False, **args))


@pytest.mark.parametrize("order", [2, 4])
def test_tiles_fp64_on_the_oracle(order):
    N, shifts, m, k = 16, [-2.5, 0.5], 36, 12
    V, L, q, st = _run(N, order, evc.EVC_FP64, "cheb", 3, zb=7, shifts=shifts, m=m, k=k)
    P = O.Problem.stencil(N, 0.3, order, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, _, _ = O.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(q - qr)) < 1e-8


@pytest.mark.parametrize("prec", [evc.EVC_MIXED, evc.EVC_FP64])
def test_partial_tiles_fall_back_to_patch(prec):
    # 12 is not a multiple of the 8-point tile: the patch pass runs
    _same(_run(12, 4, prec, "cheb", 2), _run(12, 4, prec, "cheb", 3))
