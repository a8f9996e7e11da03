"""The allocation-free quadrature entry point against the estimator.

evc_gauss_quadrature_static serves callers that cannot allocate device
memory when they call it (inside another framework's graph capture, under
an allocation-forbidding memory pool, or without a device allocator); its
eigensolver scratch is a fixed array compiled into the library.  This file
checks it through the C ABI against the per-probe quadratures that
evc_count_slices returns for the same tridiagonals, on two calls in a row
(the second call reuses the scratch the first one left behind).  It is
named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1602_02306_gb300 import evc
from paper_1602_02306_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-8   # the FP64 per-probe tolerance of the parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02306_gb300 import build
    build.build()
    evc.load()


def test_static_quadrature_matches_count_slices_twice():
    import torch
    csr = I.laplace2d_dirichlet(24)
    n = 24 * 24
    shifts, m, k = [0.8, 1.9, 3.1], 20, 30
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        L, q, st = ctx.count_slices(shifts, m, k, seed=5)
        a, b, kd = ctx.tridiag(len(shifts) * m, k)
    ncol = len(shifts) * m
    # the estimator's device layout: [step][column]
    d_alpha = torch.tensor(np.ascontiguousarray(a.T), dtype=torch.float64, device="cuda")
    d_beta = torch.tensor(np.ascontiguousarray(b.T), dtype=torch.float64, device="cuda")
    d_k = torch.tensor(kd, dtype=torch.int32, device="cuda")
    outs = []
    for _ in range(2):
        d_q = torch.full((ncol,), -7.0, dtype=torch.float64, device="cuda")
        rc, msg = evc.evc_gauss_quadrature_static(d_alpha.data_ptr(), d_beta.data_ptr(),
                                                  d_k.data_ptr(), k, ncol, float(n),
                                                  d_q.data_ptr())
        assert rc == evc.EVC_OK, msg
        torch.cuda.synchronize()
        outs.append(d_q.cpu().numpy())
    ref = q.reshape(-1)
    for got in outs:
        assert np.max(np.abs(got - ref)) < TOL
    np.testing.assert_array_equal(outs[0], outs[1])


def test_static_quadrature_rejects_oversize():
    import torch
    k = 64
    ncol = evc.EVC_STATIC_QUAD_MAX // k + 1
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc, msg = evc.evc_gauss_quadrature_static(d.data_ptr(), d.data_ptr(), None, k, ncol, 1.0,
                                              d.data_ptr())
    assert rc == evc.EVC_EINVAL
    assert "EVC_STATIC_QUAD_MAX" in msg
