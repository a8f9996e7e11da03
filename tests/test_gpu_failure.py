"""Failure detection on the GPU without a fault: a device wait that can never
complete gives up after its bounded limit, the host reads EVC_ETIMEOUT, and
the context goes on working."""
import time

import numpy as np
import pytest

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


def test_bounded_wait_reports_timeout_and_the_device_stays_usable():
    t0 = time.perf_counter()
    st = evc.evc_wait_selftest(20.0)
    dt = time.perf_counter() - t0
    assert st == evc.EVC_ETIMEOUT
    assert dt >= 0.015                      # it did wait about the limit ...
    assert dt < 5.0                         # ... and did not hang
    # a count on the same device right after
    csr = I.laplace2d_dirichlet(12)
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        L, q, st2 = ctx.count_slices([1.0, 2.0], 8, 10)
    assert np.all(np.isfinite(q))


def test_wait_selftest_rejects_bad_limits():
    for bad in (0.0, -1.0, 1e6):
        with pytest.raises(evc.EvcError):
            evc.evc_wait_selftest(bad)


# ----------------------------------------------- faults made on the host side

def test_nan_in_csr_values_reports_numeric_and_context_recovers():
    # a NaN among the matrix values (set after creation, so the host-side
    # validation does not catch it) poisons alpha/beta: the count returns
    # EVC_ENUMERIC; good values afterwards give the same result as a fresh
    # context
    rp, col, val = I.laplace2d_dirichlet(16)
    with evc.Context.csr((rp, col, val), precision=evc.EVC_MIXED) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        L0, q0, _ = ctx.count_slices([1.0, 2.0], 8, 12)
        bad = val.copy()
        bad[37] = np.nan
        evc.evc_set_values(ctx.h, bad.ctypes.data, False)
        with pytest.raises(evc.EvcError) as ei:
            ctx.count_slices([1.0, 2.0], 8, 12)
        assert ei.value.code == evc.EVC_ENUMERIC
        good = np.ascontiguousarray(val)
        evc.evc_set_values(ctx.h, good.ctypes.data, False)
        L1, q1, _ = ctx.count_slices([1.0, 2.0], 8, 12)
    np.testing.assert_array_equal(q0, q1)


def test_nan_in_potential_reports_numeric_and_context_recovers():
    N, h = 8, 0.3
    V = I.gaussian_wells(N, h, nwells=3, seed=1)
    for prec in (evc.EVC_FP64, evc.EVC_MIXED):
        with evc.Context.stencil(N, h, 2, V, precision=prec) as ctx:
            ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
            L0, q0, _ = ctx.count_slices([-2.0], 32, 10)
            Vb = V.copy()
            Vb[100] = np.inf
            evc.evc_set_values(ctx.h, Vb.ctypes.data, False)
            with pytest.raises(evc.EvcError) as ei:
                ctx.count_slices([-2.0], 32, 10)
            assert ei.value.code == evc.EVC_ENUMERIC
            Vg = np.ascontiguousarray(V)
            evc.evc_set_values(ctx.h, Vg.ctypes.data, False)
            L1, q1, _ = ctx.count_slices([-2.0], 32, 10)
        np.testing.assert_array_equal(q0, q1)


def test_workspace_too_small_reports_enomem_and_context_recovers():
    import torch
    csr = I.laplace2d_dirichlet(12)
    ctx = evc.Context.csr(csr, precision=evc.EVC_FP64, torch_workspace=False)
    try:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        need = evc.evc_workspace_bytes(ctx.h, 2, 8, 10)
        small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
        evc.evc_set_workspace(ctx.h, small.data_ptr(), small.numel())
        with pytest.raises(evc.EvcError) as ei:
            evc.evc_count_slices(ctx.h, [1.0, 2.0], 8, 10)
        assert ei.value.code == evc.EVC_ENOMEM
        assert "workspace too small" in evc.evc_last_error(ctx.h)
        big = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        aligned = (big.data_ptr() + 255) & ~255
        evc.evc_set_workspace(ctx.h, aligned, need)
        L, q, st = evc.evc_count_slices(ctx.h, [1.0, 2.0], 8, 10)
        assert np.all(np.isfinite(q)) and list(st) == [10, 10]
    finally:
        ctx.close()
