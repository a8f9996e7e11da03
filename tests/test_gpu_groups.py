"""Concurrent chunk groups of the stencil operator (EVC_OPT_STENCIL_GROUPS).

The column chunks of a step are independent until the reorthogonalisation
(Algorithm 1: every probe runs its own Lanczos process), so the stencil
passes of one operator application may run as several groups of chunks on
concurrent streams.  Each chunk is computed by the same kernels with the same
arguments as with one stream, so every per-probe quadrature, step count and
estimate must be bitwise equal to the one-stream run, which the other tests
compare with the FP64 oracle."""
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


def _run(N, order, prec, precond, shifts, m, k, groups, tol=0.0, patch=2,
         method=evc.EVC_METHOD_LANCZOS, graph=True, profile=False):
    V = I.gaussian_wells(N, 0.3, nwells=5, seed=1)
    with evc.Context.stencil(N, 0.3, order, V, precision=prec) as ctx:
        if precond == "cheb":
            ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
        elif precond == "jacobi":
            ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3, 0.0)
        ctx.set_option(evc.EVC_OPT_STENCIL_PATCH, patch)
        ctx.set_option(evc.EVC_OPT_METHOD, method)
        ctx.set_option(evc.EVC_OPT_STENCIL_GROUPS, groups)
        if not graph:
            ctx.set_option(evc.EVC_OPT_GRAPH, 0)
        if profile:
            ctx.set_option(evc.EVC_OPT_PROFILE, 1)
        L, q, st = ctx.count_slices(shifts, m, k, tol=tol, seed=0)
        recs = evc.evc_get_profile(ctx.h) if profile else None
    return V, L, q, st, recs


def _same(a, b):
    for x, y in zip(a[1:4], b[1:4]):
        assert np.array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("prec", [evc.EVC_MIXED, evc.EVC_FP64])
@pytest.mark.parametrize("groups", [2, 3, 4])
def test_lanczos_chebyshev_groups_bitwise(prec, groups):
    # 2 shifts x 64 probes = 4 chunks; 3 groups split them unevenly (1, 1, 2)
    args = (16, 2, prec, "cheb", [-3.0, 1.0], 64, 12)
    _same(_run(*args, groups=1), _run(*args, groups=groups))


def test_groups_fp64_parity_with_oracle():
    V, L, q, st, _ = _run(12, 2, evc.EVC_FP64, "cheb", [-2.5, 0.5], 48, 10, groups=2)
    P = O.Problem.stencil(12, 0.3, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, _, _ = O.count(P, [-2.5, 0.5], 48, 10, seed=0)
    assert np.max(np.abs(q - qr)) < 1e-8


def test_groups_adaptive_stop_bitwise():
    # chunks leave the grid at different steps; 7 shifts x 16 probes = 4 chunks
    args = (10, 2, evc.EVC_FP64, "cheb", list(np.linspace(-4.0, 2.0, 7)), 16, 30)
    a, b = _run(*args, groups=1, tol=0.25), _run(*args, groups=2, tol=0.25)
    assert len(set(a[3])) > 1
    _same(a, b)


@pytest.mark.parametrize("patch", [1, 2])
def test_groups_13_point_bitwise(patch):
    args = (12, 4, evc.EVC_MIXED, "cheb", [-2.0, 0.5], 64, 10)
    _same(_run(*args, groups=1, patch=patch), _run(*args, groups=2, patch=patch))


def test_groups_jacobi_and_identity_bitwise():
    # one grouped pass per step (the Jacobi-scaled pass kernel, and the plain one)
    for precond in ("jacobi", "identity"):
        args = (14, 2, evc.EVC_FP64, precond, [-1.0, 2.0], 64, 12)
        _same(_run(*args, groups=1), _run(*args, groups=2))


def test_groups_arnoldi_bitwise():
    args = (12, 2, evc.EVC_FP64, "cheb", [-2.0, 0.5], 64, 10)
    kw = dict(method=evc.EVC_METHOD_ARNOLDI)
    _same(_run(*args, groups=1, **kw), _run(*args, groups=2, **kw))


def test_groups_without_graph_bitwise():
    args = (12, 2, evc.EVC_MIXED, "cheb", [-2.0, 0.5], 64, 8)
    _same(_run(*args, groups=1, graph=False), _run(*args, groups=4, graph=False))


def test_more_groups_than_chunks():
    # 20 columns are one chunk: the segment is not split
    args = (10, 2, evc.EVC_FP64, "cheb", [-1.0, 1.0], 10, 8)
    _same(_run(*args, groups=1), _run(*args, groups=4))


def test_group_span_records():
    k = 6
    args = (12, 2, evc.EVC_MIXED, "cheb", [-2.0, 0.5], 64, k)
    one = _run(*args, groups=1, profile=True)[4]
    two = _run(*args, groups=2, profile=True)[4]
    st1 = [r for r in one if r[0] == evc.EVC_K_STENCIL]
    assert all(r[4] == 0 and r[2] > 0 for r in st1)
    spans = [r for r in two if r[4] == 1]
    launches = [r for r in two if r[0] == evc.EVC_K_STENCIL and r[4] == 0]
    # one span per step; every launch of the segment twice (two groups), untimed
    assert [r[1] for r in spans] == list(range(1, k + 1))
    assert all(r[0] == evc.EVC_K_STENCIL and r[2] > 0 for r in spans)
    assert len(launches) == 2 * len(st1) and all(r[2] < 0 for r in launches)
    for i in range(1, k + 1):
        b1 = sum(r[3] for r in st1 if r[1] == i)
        assert [r[3] for r in spans if r[1] == i][0] == pytest.approx(b1, rel=1e-12)
        assert sum(r[3] for r in launches if r[1] == i) == pytest.approx(b1, rel=1e-12)
    # the other kernel classes are unchanged
    other = lambda recs: [(r[0], r[1]) for r in recs if r[0] != evc.EVC_K_STENCIL]
    assert other(one) == other(two)


def test_groups_option_validates():
    V = I.gaussian_wells(8, 0.3, nwells=2, seed=1)
    with evc.Context.stencil(8, 0.3, 2, V, precision=evc.EVC_FP64) as ctx:
        for bad in (0, 5, -1):
            with pytest.raises(evc.EvcError):
                ctx.set_option(evc.EVC_OPT_STENCIL_GROUPS, bad)
    csr = I.laplace2d_dirichlet(8)
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        with pytest.raises(evc.EvcError):
            ctx.set_option(evc.EVC_OPT_STENCIL_GROUPS, 2)
