"""Parity at the benchmark's full sizes, on sampled probes.

The GPU runs the whole workload exactly as bench.py does (all shifts and
probes in one batched launch, in the tile shapes its autotuner picks on a
GB300); the FP64 oracle recomputes a sample of probe
columns one by one at full size, on all host cores.  FP64 mode: per-probe
quadrature within 1e-8.  Mixed mode: per-probe quadrature within 0.5 and the
sampled mean within 0.5 (the estimate tolerance).  With a tolerance-driven
stop, the oracle reproduces each sampled probe at the step its shift stopped
on the GPU (the stop rule itself is checked against the oracle on smaller
problems in test_gpu_parity.py).
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1602_02306_gb300 import evc, workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FP64_TOL = 1e-8
MIXED_TOL = 0.5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02306_gb300 import build
    build.build()
    evc.load()


# The tile shapes the library's autotuner picks for these workloads on a GB300
# (the benchmark's launch configuration): tensor-copied 7-point tiles with four
# chunk groups on 64^3, 13-point register patches on 96^3, 128-thread CSR blocks.
BENCH_SHAPES = {
    "fd64": {evc.EVC_OPT_STENCIL_PATCH: 3, evc.EVC_OPT_STENCIL_ZB: 32, evc.EVC_OPT_STENCIL_GROUPS: 4},
    "slicing96": {evc.EVC_OPT_STENCIL_PATCH: 2, evc.EVC_OPT_STENCIL_ZB: 64,
                  evc.EVC_OPT_STENCIL_GROUPS: 1},
    "powerlaw2m": {evc.EVC_OPT_CSR_THREADS: 128},
}


def _gpu(W, precision, method=evc.EVC_METHOD_LANCZOS, tinv=0, shapes=None):
    import torch
    if W.kind == "stencil":
        ctx = evc.Context.stencil(W.N, W.h, W.order, W.potential(), precision=precision)
    else:
        ctx = evc.Context.csr(W.csr(), precision=precision)
    kind = {"identity": evc.EVC_PREC_IDENTITY, "jacobi": evc.EVC_PREC_JACOBI,
            "cheb": evc.EVC_PREC_CHEB_KINETIC}[W.precond]
    with ctx:
        need = evc.evc_workspace_bytes(ctx.h, len(W.shifts), W.nprobe, W.maxsteps)
        free, _ = torch.cuda.mem_get_info()
        if need > 0.9 * free:
            pytest.skip(f"workspace {need / 1e9:.0f} GB does not fit")
        ctx.set_precond(kind, *W.prec_params)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_MIN_STEPS, W.min_steps)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_METHOD, method)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_TINV_LANCZOS, tinv)
        for opt, val in (shapes or {}).items():
            evc.evc_set_option(ctx.h, opt, val)
        out = ctx.count_slices(W.shifts, W.nprobe, W.maxsteps, tol=W.tol, seed=0)
    torch.cuda.empty_cache()
    return out


def _oracle_problem(W):
    if W.kind == "stencil":
        pk = {"identity": O.PREC_NONE, "jacobi": O.PREC_JACOBI, "cheb": O.PREC_CHEB}[W.precond]
        return O.Problem.stencil(W.N, W.h, W.order, W.potential(), pk,
                                 cheb_degree=int(W.prec_params[0]), cheb_c=float(W.prec_params[1]),
                                 jac_eps=float(W.prec_params[0]))
    pk = {"identity": O.PREC_NONE, "jacobi": O.PREC_JACOBI}[W.precond]
    return O.Problem.csr_matrix(W.csr(), pk, jac_eps=float(W.prec_params[0]))


def _sample_oracle(W, P, shift_idx, probe_ids, steps):
    """Oracle quadratures of the sampled (shift, probe) columns at the GPU's stop steps."""
    out = {}
    for s in shift_idx:
        q, _, _ = O.count(P, [W.shifts[s]], len(probe_ids), int(steps[s]), tol=0.0, seed=0,
                          probe_ids=probe_ids, nthreads=os.cpu_count() or 1)
        out[s] = q[0]
    return out


def test_fd_hamiltonian_64_fullsize():
    W = workloads.fd_hamiltonian_64()
    L64, q64, st64 = _gpu(W, evc.EVC_FP64, shapes=BENCH_SHAPES["fd64"])
    Lmx, qmx, stmx = _gpu(W, evc.EVC_MIXED, shapes=BENCH_SHAPES["fd64"])
    assert list(st64) == list(stmx) == [W.maxsteps] * len(W.shifts)
    P = _oracle_problem(W)
    ids = [0, 13, 31, 40, 63]
    ref = _sample_oracle(W, P, range(len(W.shifts)), ids, st64)
    for s in range(len(W.shifts)):
        np.testing.assert_allclose(q64[s, ids], ref[s], rtol=0, atol=FP64_TOL)
        assert np.max(np.abs(qmx[s, ids] - ref[s])) < MIXED_TOL
    # all probes: mixed against the (oracle-checked) FP64 path
    assert abs((Lmx[-1] - Lmx[0]) - (L64[-1] - L64[0])) < MIXED_TOL


@pytest.fixture(scope="module")
def powerlaw_2m_runs():
    W = workloads.powerlaw_2m()
    L64, q64, st64 = _gpu(W, evc.EVC_FP64, shapes=BENCH_SHAPES["powerlaw2m"])
    Lmx, qmx, stmx = _gpu(W, evc.EVC_MIXED, shapes=BENCH_SHAPES["powerlaw2m"])
    return W, (L64, q64, st64), (Lmx, qmx, stmx)


def test_powerlaw_2m_fullsize(powerlaw_2m_runs):
    # n = 2,000,000: per-probe quadratures near 1e6, far from converged at
    # k = 50.  FP64 matches the oracle per probe to 1e-12 relative.  The mixed
    # path forms its Jacobi scales from the FP64 diagonal; its per-probe values
    # stay within 1e-3 relative of the oracle and each n_below within 5e-5
    # relative of FP64 (measured up to 1.3e-5: FP32 rounding moves the
    # unconverged Ritz values, and the odd one crossing the shift moves its
    # probe's quadrature by a Gauss weight of ~n/k; see the next test).
    W, (L64, q64, st64), (Lmx, qmx, stmx) = powerlaw_2m_runs
    P = _oracle_problem(W)
    ids = [0, 77, 127]
    ref = _sample_oracle(W, P, range(len(W.shifts)), ids, st64)
    for s in range(len(W.shifts)):
        np.testing.assert_allclose(q64[s, ids], ref[s], rtol=1e-12, atol=FP64_TOL)
        np.testing.assert_allclose(qmx[s, ids], ref[s], rtol=1e-3)
    np.testing.assert_allclose(Lmx, L64, rtol=5e-5)


@pytest.mark.xfail(strict=True, reason="FP32-mixed count on the 2M-row power-law workload is "
                   "about 10 away from FP64 (measured +11.07 and -3.92 on an estimate of 77,414 "
                   "with two roundings of the CSR sums): FP32 vectors leave ~1e-5 relative per "
                   "unconverged probe, and a Ritz value crossing a shift moves a probe by ~n/k")
def test_powerlaw_2m_mixed_estimate_within_half(powerlaw_2m_runs):
    # the stated target: the FP32-mixed estimate within 0.5 of FP64's
    W, (L64, _, _), (Lmx, _, _) = powerlaw_2m_runs
    assert abs((Lmx[-1] - Lmx[0]) - (L64[-1] - L64[0])) < MIXED_TOL


def test_powerlaw_2m_tinv_lanczos_fullsize(powerlaw_2m_runs):
    # the T^{-1}-inner-product process (Sec. 4, Eq. lanT1) on the same
    # workload: FP64 per probe equal to Algorithm 1's (measured 8.5e-7 on
    # values near 7e5, 1.2e-12 relative), mixed n_below within 5e-5 relative
    W, (L64, q64, st64), _ = powerlaw_2m_runs
    Lt, qt, stt = _gpu(W, evc.EVC_FP64, tinv=1)
    assert list(stt) == list(st64)
    np.testing.assert_allclose(qt, q64, rtol=1e-11, atol=FP64_TOL)
    Ltm, qtm, _ = _gpu(W, evc.EVC_MIXED, tinv=1)
    np.testing.assert_allclose(Ltm, L64, rtol=5e-5)
    ids = [0, 77, 127]
    ref = _sample_oracle(W, _oracle_problem(W), range(len(W.shifts)), ids, st64)
    for s in range(len(W.shifts)):
        np.testing.assert_allclose(qtm[s, ids], ref[s], rtol=1e-3)


def test_slicing_96_fullsize():
    W = workloads.batched_slicing_96()
    Lmx, qmx, stmx = _gpu(W, evc.EVC_MIXED, shapes=BENCH_SHAPES["slicing96"])
    assert all(W.min_steps <= s <= W.maxsteps for s in stmx)
    P = _oracle_problem(W)
    ids = [5, 50]
    shifts = [0, 15, 31]
    ref = _sample_oracle(W, P, shifts, ids, stmx)
    for s in shifts:
        assert np.max(np.abs(qmx[s, ids] - ref[s])) < MIXED_TOL
    # slice counts are differences of n_below; n_below is non-decreasing up to noise
    assert np.all(np.diff(Lmx) > -2.0)
    # FP64 on three of the shifts (the FP64 basis of all 32 does not fit): each
    # shift's columns and stop rule are independent of the others, so each is
    # compared with the same shift of the mixed run
    import dataclasses
    Wf = dataclasses.replace(W, shifts=[W.shifts[s] for s in shifts])
    Lf, qf, stf = _gpu(Wf, evc.EVC_FP64, shapes=BENCH_SHAPES["slicing96"])
    assert list(stf) == [int(stmx[s]) for s in shifts]
    for j, s in enumerate(shifts):
        assert abs(Lmx[s] - Lf[j]) < MIXED_TOL
        np.testing.assert_allclose(qf[j, ids], ref[s], rtol=0, atol=FP64_TOL)


def test_fd_hamiltonian_64_arnoldi_fullsize():
    # the Arnoldi-type estimator (Sec. 4) on the benchmark workload: FP64 and
    # mixed GPU counts against the numpy Arnoldi oracle on two sampled probes
    from oracle import arnoldi as AR
    W = workloads.fd_hamiltonian_64()
    L64, q64, _ = _gpu(W, evc.EVC_FP64, evc.EVC_METHOD_ARNOLDI)
    Lmx, qmx, _ = _gpu(W, evc.EVC_MIXED, evc.EVC_METHOD_ARNOLDI)
    P = _oracle_problem(W)
    pids = [5, 41]
    for s in range(len(W.shifts)):
        qr, _, _ = AR.count(P, [W.shifts[s]], len(pids), W.maxsteps, seed=0, probe_ids=pids)
        for j, pid in enumerate(pids):
            assert abs(q64[s, pid] - qr[0, j]) < FP64_TOL
            assert abs(qmx[s, pid] - qr[0, j]) < MIXED_TOL
    assert abs((Lmx[-1] - Lmx[0]) - (L64[-1] - L64[0])) < MIXED_TOL


def test_fd_hamiltonian_64_exact_count_statistical():
    # [lambda_min - 1, eta] holds exactly 300 eigenvalues (Sylvester inertia,
    # workloads.FD64_ETA).  At 50 steps both estimators are within 4 sample
    # standard errors of it (at the workload's 30 steps the quadrature is not
    # yet converged: ~249).
    W = workloads.fd_hamiltonian_64()
    for method in (evc.EVC_METHOD_LANCZOS, evc.EVC_METHOD_ARNOLDI):
        with evc.Context.stencil(W.N, W.h, W.order, W.potential(), precision=evc.EVC_MIXED) as ctx:
            ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, *W.prec_params)
            ctx.set_option(evc.EVC_OPT_METHOD, method)
            L, q, st = ctx.count_slices(W.shifts, W.nprobe, 50, seed=0)
        d = q[1] - q[0]
        se = d.std(ddof=1) / np.sqrt(d.size)
        assert abs((L[1] - L[0]) - 300.0) < 4.0 * se
