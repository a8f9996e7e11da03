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
