"""The tile-shape parameters and the autotuner that picks them: shapes that
do not touch the arithmetic leave results bitwise unchanged, the rows per
block of the reorthogonalisation only reorders sums, and a tuned context
still matches the FP64 oracle."""
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


def _stencil_ctx(N, prec=evc.EVC_FP64):
    V = I.gaussian_wells(N, 0.3, nwells=5, seed=1)
    ctx = evc.Context.stencil(N, 0.3, 2, V, precision=prec)
    ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
    return V, ctx


def test_stencil_zb_leaves_results_unchanged():
    shifts, m, k = [-2.0, 0.5], 40, 8
    V, ctx = _stencil_ctx(37)
    with ctx:
        ref = ctx.count_slices(shifts, m, k)[1]
        for zb in (1, 5, 16, 64, 100):
            ctx.set_option(evc.EVC_OPT_STENCIL_ZB, zb)
            np.testing.assert_array_equal(ctx.count_slices(shifts, m, k)[1], ref)


def test_csr_threads_leave_results_unchanged():
    csr = I.powerlaw_symmetric(20000, cap=300, seed=2)
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        ref = ctx.count_slices([-0.5, 0.5], 33, 10)[1]
        for nt in (128, 512, 256):
            ctx.set_option(evc.EVC_OPT_CSR_THREADS, nt)
            np.testing.assert_array_equal(ctx.count_slices([-0.5, 0.5], 33, 10)[1], ref)


@pytest.mark.parametrize("prec", [evc.EVC_FP64, evc.EVC_MIXED])
def test_csr_uniform_shift_chunks_match_mixed_chunks(prec):
    # chunks whose 32 columns share a shift run a specialised CSR pass (one
    # Jacobi scale per gathered entry); a column batched so that its chunk
    # mixes shifts runs the general pass: the rows are bitwise the same
    csr = I.powerlaw_symmetric(20011, cap=300, seed=2)
    with evc.Context.csr(csr, precision=prec) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        alone = ctx.count_slices([0.5], 33, 10)[1]           # one shift: uniform chunks
        mixed = ctx.count_slices([-0.5, 0.5], 33, 10)[1]     # 66 columns: chunk 1 mixes
        np.testing.assert_array_equal(mixed[1], alone[0])
        for nt in (128, 512):
            ctx.set_option(evc.EVC_OPT_CSR_THREADS, nt)
            np.testing.assert_array_equal(ctx.count_slices([-0.5, 0.5], 33, 10)[1], mixed)


def test_reorth_rows_reorder_sums_only():
    shifts, m, k = [-2.5, 0.5], 36, 12
    V, ctx = _stencil_ctx(25)
    P = O.Problem.stencil(25, 0.3, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, _, _ = O.count(P, shifts, m, k, seed=0)
    with ctx:
        for rows in (64, 1728, 3456, 6912, 100000):
            ctx.set_option(evc.EVC_OPT_REORTH_ROWS, rows)
            q = ctx.count_slices(shifts, m, k)[1]
            assert np.max(np.abs(q - qr)) < 1e-8


def test_autotune_choices_and_parity():
    shifts, m, k = [-2.5, 0.5], 40, 10
    V, ctx = _stencil_ctx(30)
    with ctx:
        t = ctx.autotune(len(shifts), m, k)
        assert t["stencil_zb"] in (16, 30) and t["csr_threads"] == 0
        assert t["stencil_patch"] in (1, 2)
        assert t["stencil_groups"] in (1, 2, 4)     # 80 columns: 3 chunks, so at most 2 groups
        assert t["stencil_groups"] <= 3
        assert t["reorth_rows"] in (64, 128, 256, 512, 1024, 1728, 3456, 6912, 13824)
        assert t["ms_before"] > 0 and t["ms_after"] > 0 and t["steps"] == 6
        q = ctx.count_slices(shifts, m, k)[1]
    P = O.Problem.stencil(30, 0.3, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, _, _ = O.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(q - qr)) < 1e-8


def test_autotune_csr_and_batch_independence():
    csr = I.powerlaw_symmetric(30000, cap=300, seed=2)
    with evc.Context.csr(csr, precision=evc.EVC_MIXED) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        t = ctx.autotune(3, 32, 12)
        assert t["csr_threads"] in (128, 256, 512) and t["stencil_zb"] == 0
        # a column's result is the same alone and batched, with the tuned shapes
        q1 = ctx.count_slices([0.1], 32, 12)[1]
        q3 = ctx.count_slices([-0.4, 0.1, 0.3], 32, 12)[1]
    np.testing.assert_array_equal(q1[0], q3[1])


def test_tuning_options_validate():
    V, ctx = _stencil_ctx(8)
    with ctx:
        for opt, bad in ((evc.EVC_OPT_REORTH_ROWS, 32), (evc.EVC_OPT_STENCIL_ZB, -1),
                         (evc.EVC_OPT_CSR_THREADS, 256)):
            with pytest.raises(evc.EvcError):
                ctx.set_option(opt, bad)
        with pytest.raises(evc.EvcError):
            ctx.autotune(0, 8, 4)


@pytest.mark.parametrize("N,order", [(10, 2), (16, 4), (12, 2), (9, 2)])
@pytest.mark.parametrize("prec", [evc.EVC_FP64, evc.EVC_MIXED])
def test_stencil_patch_agrees_with_single_points(N, order, prec):
    # 2 x 2 patches (odd N falls back to one point per thread)
    V = I.gaussian_wells(N, 0.3, nwells=4, seed=1)
    shifts, m, k = [-2.0, 0.5], 40, 10
    res = []
    for patch in (1, 2):
        with evc.Context.stencil(N, 0.3, order, V, precision=prec) as ctx:
            ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
            ctx.set_option(evc.EVC_OPT_STENCIL_PATCH, patch)
            res.append(ctx.count_slices(shifts, m, k, seed=0))
    if prec == evc.EVC_FP64:
        assert np.max(np.abs(res[0][1] - res[1][1])) < 1e-10
        P = O.Problem.stencil(N, 0.3, order, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
        qr, _, _ = O.count(P, shifts, m, k, seed=0)
        assert np.max(np.abs(res[1][1] - qr)) < 1e-8
    else:
        assert np.max(np.abs(res[0][0] - res[1][0])) < 0.05


def test_stencil_patch_unpreconditioned_and_zb():
    # the shifted-Hamiltonian pass with -beta q_(i-1) (operand sets V and V+pp)
    V = I.gaussian_wells(14, 0.3, nwells=4, seed=1)
    P = O.Problem.stencil(14, 0.3, 2, V, O.PREC_NONE)
    qr, _, _ = O.count(P, [-1.0, 0.7], 33, 12, seed=0)
    with evc.Context.stencil(14, 0.3, 2, V, precision=evc.EVC_FP64) as ctx:
        ctx.set_option(evc.EVC_OPT_STENCIL_PATCH, 2)
        for zb in (3, 32):
            ctx.set_option(evc.EVC_OPT_STENCIL_ZB, zb)
            q = ctx.count_slices([-1.0, 0.7], 33, 12, seed=0)[1]
            assert np.max(np.abs(q - qr)) < 1e-8


def test_small_problem_splits_rows():
    # n = 1024: the tuner may split the reorthogonalisation into 64-row blocks;
    # FP64 results stay on the oracle
    csr = I.laplace2d_dirichlet(32)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI, jac_eps=1e-3)
    qr, _, _ = O.count(P, [1.0, 2.0], 16, 40, seed=0)
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        for rows in (64, 256):
            ctx.set_option(evc.EVC_OPT_REORTH_ROWS, rows)
            q = ctx.count_slices([1.0, 2.0], 16, 40, seed=0)[1]
            assert np.max(np.abs(q - qr)) < 1e-8
        t = ctx.autotune(2, 16, 40)
        q = ctx.count_slices([1.0, 2.0], 16, 40, seed=0)[1]
        assert np.max(np.abs(q - qr)) < 1e-8
        with pytest.raises(evc.EvcError):
            ctx.set_option(evc.EVC_OPT_REORTH_ROWS, 1)
