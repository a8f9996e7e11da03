"""The allocation-free quadrature entry point against the estimator and the oracle.

evc_gauss_quadrature_static serves callers that cannot allocate device
memory when they call it (inside another framework's graph capture, under
an allocation-forbidding memory pool, or without a device allocator); its
eigensolver scratch is a fixed array compiled into the library.  This file
checks it through the C ABI on two calls in a row (the second call reuses
the scratch the first one left behind):
  * against the per-probe quadratures that evc_count_slices returns for the
    same tridiagonals, and against the FP64 oracle's Gauss quadrature
    (Eq. gauss_quad) of each tridiagonal;
  * on random tridiagonals with per-column sizes, against the oracle;
  * its status word: out-of-range sizes and non-finite input are reported,
    not clamped or hidden.
It is named so that pytest collects it last.
"""
import numpy as np
import pytest

from oracle import oracle as O
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


def _call(d_alpha, d_beta, d_k, k, ncol, vnorm2):
    import torch
    d_q = torch.full((ncol,), -7.0, dtype=torch.float64, device="cuda")
    d_st = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    rc, msg = evc.evc_gauss_quadrature_static(d_alpha.data_ptr(), d_beta.data_ptr(),
                                              None if d_k is None else d_k.data_ptr(), k, ncol,
                                              float(vnorm2), d_q.data_ptr(), d_st.data_ptr())
    assert rc == evc.EVC_OK, msg
    torch.cuda.synchronize()
    return d_q.cpu().numpy(), int(d_st.item())


def test_static_quadrature_matches_count_slices_and_oracle_twice():
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
    outs = [_call(d_alpha, d_beta, d_k, k, ncol, n) for _ in range(2)]
    ref = q.reshape(-1)
    orc = np.array([O.gauss_quad(a[c, :kd[c]], b[c, :kd[c] + 1], n) for c in range(ncol)])
    for got, status in outs:
        assert status == evc.EVC_OK
        assert np.max(np.abs(got - ref)) < TOL
        assert np.max(np.abs(got - orc)) < TOL
    np.testing.assert_array_equal(outs[0][0], outs[1][0])


def test_static_quadrature_random_tridiagonals_against_oracle():
    import torch
    rng = np.random.default_rng(11)
    k, ncol, vn = 40, 300, 1000.0
    alpha = rng.standard_normal((ncol, k)) * 2.0
    beta = np.abs(rng.standard_normal((ncol, k + 1))) + 0.05
    beta[:, 0] = 0.0
    kcol = rng.integers(1, k + 1, size=ncol).astype(np.int32)
    d_alpha = torch.tensor(np.ascontiguousarray(alpha.T), device="cuda")
    d_beta = torch.tensor(np.ascontiguousarray(beta.T), device="cuda")
    d_k = torch.tensor(kcol, device="cuda")
    want = np.array([O.gauss_quad(alpha[c, :kcol[c]], beta[c, :kcol[c] + 1], vn)
                     for c in range(ncol)])
    for _ in range(2):
        got, status = _call(d_alpha, d_beta, d_k, k, ncol, vn)
        assert status == evc.EVC_OK
        np.testing.assert_allclose(got, want, rtol=0, atol=TOL * vn)


def test_static_quadrature_reports_bad_sizes_and_nonfinite_input():
    import torch
    rng = np.random.default_rng(12)
    k, ncol = 12, 64
    alpha = rng.standard_normal((ncol, k))
    beta = np.abs(rng.standard_normal((ncol, k + 1))) + 0.1
    kcol = np.full(ncol, k, dtype=np.int32)
    kcol[5] = k + 1          # outside [1, k]: rejected, not clamped
    kcol[9] = 0
    d_alpha = torch.tensor(np.ascontiguousarray(alpha.T), device="cuda")
    d_beta = torch.tensor(np.ascontiguousarray(beta.T), device="cuda")
    got, status = _call(d_alpha, d_beta, torch.tensor(kcol, device="cuda"), k, ncol, 1.0)
    assert status == evc.EVC_EINVAL
    assert np.isnan(got[5]) and np.isnan(got[9])
    good = [c for c in range(ncol) if c not in (5, 9)]
    want = np.array([O.gauss_quad(alpha[c], beta[c, :k + 1], 1.0) for c in good])
    np.testing.assert_allclose(got[good], want, rtol=0, atol=TOL)
    # a NaN coefficient: the eigensolve cannot converge -> EVC_ENUMERIC, NaN out
    alpha[3, 4] = np.nan
    d_alpha = torch.tensor(np.ascontiguousarray(alpha.T), device="cuda")
    got, status = _call(d_alpha, d_beta, None, k, ncol, 1.0)
    assert status == evc.EVC_ENUMERIC
    assert np.isnan(got[3]) and np.all(np.isfinite(np.delete(got, 3)))


def test_static_quadrature_rejects_oversize():
    import torch
    k = 64
    ncol = evc.EVC_STATIC_QUAD_MAX // k + 1
    d = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc, msg = evc.evc_gauss_quadrature_static(d.data_ptr(), d.data_ptr(), None, k, ncol, 1.0,
                                              d.data_ptr())
    assert rc == evc.EVC_EINVAL
    assert "EVC_STATIC_QUAD_MAX" in msg
