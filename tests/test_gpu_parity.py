"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Same seeded inputs and the same counter-hashed probes on both sides.
Tolerances: FP64 mode, per-probe quadrature within 1e-8 absolute; mixed
mode (FP32 vectors, FP64 recurrence scalars), estimate within 0.5 of the
oracle's.  Sizes span several tiles and ragged tails.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1602_02306_gb300 import evc
from paper_1602_02306_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-8
MIXED_EST_TOL = 0.5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1602_02306_gb300 import build
    build.build()
    evc.load()


def _gpu_csr(csr, prec, pkind, p0, shifts, m, k, tol=0.0, seed=0):
    with evc.Context.csr(csr, precision=prec) as ctx:
        ctx.set_precond(pkind, p0)
        L, q, st = ctx.count_slices(shifts, m, k, tol=tol, seed=seed)
        a, b, kd = ctx.tridiag(len(shifts) * m, min(k, len(csr[0]) - 1))
    return L, q, st, (a, b, kd)


def _gpu_stencil(N, h, order, V, prec, pkind, p0, p1, shifts, m, k, tol=0.0, seed=0):
    with evc.Context.stencil(N, h, order, V, precision=prec) as ctx:
        ctx.set_precond(pkind, p0, p1)
        L, q, st = ctx.count_slices(shifts, m, k, tol=tol, seed=seed)
    return L, q, st


# ------------------------------------------------------------ CSR, FP64

def test_plain_fp64_laplace32_per_probe():
    # 2D Dirichlet Laplacian 32x32, [1, 2], Jacobi, 16 probes, 40 steps
    csr = I.laplace2d_dirichlet(32)
    L, q, st, _ = _gpu_csr(csr, evc.EVC_FP64, evc.EVC_PREC_JACOBI, 1e-3, [1.0, 2.0], 16, 40)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI, jac_eps=1e-3)
    qr, sr, Lr = O.count(P, [1.0, 2.0], 16, 40, seed=0)
    assert np.max(np.abs(q - qr)) < FP64_TOL
    assert list(st) == list(sr) == [40, 40]
    assert abs((L[1] - L[0]) - (Lr[1] - Lr[0])) < 1e-9


def test_evc_count_estimate_matches_oracle():
    csr = I.laplace2d_dirichlet(32)
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        est, q, st = ctx.count(1.0, 2.0, 16, 40, seed=0)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI, jac_eps=1e-3)
    qr, _, Lr = O.count(P, [1.0, 2.0], 16, 40, seed=0)
    assert abs(est - (Lr[1] - Lr[0])) < 1e-9
    np.testing.assert_allclose(q, qr, rtol=0, atol=FP64_TOL)


@pytest.mark.parametrize("prec_kind", [evc.EVC_PREC_IDENTITY, evc.EVC_PREC_JACOBI])
def test_csr_random_indefinite_fp64_tridiag(prec_kind):
    # ragged: 37 probes -> 3 chunks with a padded tail, n = 300
    A = I.random_symmetric_dense(300, seed=7)
    A[np.abs(A) < 1.2] = 0.0
    A = 0.5 * (A + A.T) + np.diag(np.linspace(-3, 3, 300))
    csr = I.dense_to_csr(A)
    shifts = [-1.0, 0.25, 2.0]
    m, k = 37, 25
    L, q, st, (a, b, kd) = _gpu_csr(csr, evc.EVC_FP64, prec_kind, 1e-3, shifts, m, k)
    opk = O.PREC_NONE if prec_kind == evc.EVC_PREC_IDENTITY else O.PREC_JACOBI
    P = O.Problem.csr_matrix(csr, opk)
    qr, sr, Lr = O.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(q - qr)) < FP64_TOL
    np.testing.assert_allclose(L, Lr, rtol=0, atol=1e-9)
    # tridiagonals of a few columns against Algorithm 1 directly
    for c in (0, 36, 37, 110):
        s, j = divmod(c, m)
        v = O.probe_vector(0, j, 300)
        al, be, _, kdo = O.lanczos(P, shifts[s], v, k)
        assert kd[c] == kdo
        np.testing.assert_allclose(a[c, :kdo], al, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(b[c, :kdo + 1], be, rtol=1e-10, atol=1e-10)


def test_csr_adaptive_stop_rule_matches_oracle():
    csr = I.laplace2d_dirichlet(20)
    shifts = [0.5, 1.5, 3.0]
    L, q, st, _ = _gpu_csr(csr, evc.EVC_FP64, evc.EVC_PREC_JACOBI, 1e-3, shifts, 12, 40, tol=0.25)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    qr, sr, Lr = O.count(P, shifts, 12, 40, tol=0.25, seed=0)
    assert list(st) == list(sr)
    assert np.max(np.abs(q - qr)) < FP64_TOL
    assert all(2 <= s <= 40 for s in st) and min(st) < 40


def test_breakdown_at_p_distinct_eigenvalues():
    # Proposition 1: with p distinct eigenvalues Lanczos stops at step p, exactly
    distinct = [-2.0, -0.5, 0.7, 1.5, 3.0]
    A = I.random_symmetric_dense(64, seed=4, distinct=distinct)
    csr = I.dense_to_csr(A)
    for prec in (evc.EVC_FP64, evc.EVC_MIXED):
        L, q, st, (a, b, kd) = _gpu_csr(csr, prec, evc.EVC_PREC_IDENTITY, 0, [0.0], 4, 12)
        if prec == evc.EVC_FP64:
            assert list(kd) == [5, 5, 5, 5]
        w, U = np.linalg.eigh(A)
        for j in range(4):
            v = O.probe_vector(0, j, 64)
            exact = float(np.sum((U[:, w < 0].T @ v) ** 2))
            assert abs(q[0, j] - exact) < (1e-8 if prec == evc.EVC_FP64 else 1e-3)


@pytest.mark.parametrize("prec_kind", [evc.EVC_PREC_IDENTITY, evc.EVC_PREC_JACOBI])
def test_quad_bound_diagnostic_matches_oracle(prec_kind):
    # Sec. 3, Eq. qbound: the library's per-column log10(||v||^2 beta_2^2 ...
    # beta_{k+1}^2 / (2k)!) against the oracle's factor on Algorithm 1's own
    # tridiagonals (FP64), including columns cut short by the stop rule
    A = I.random_symmetric_dense(300, seed=7)
    A[np.abs(A) < 1.2] = 0.0
    A = 0.5 * (A + A.T) + np.diag(np.linspace(-3, 3, 300))
    csr = I.dense_to_csr(A)
    shifts, m, k = [-1.0, 0.25], 37, 20
    opk = O.PREC_NONE if prec_kind == evc.EVC_PREC_IDENTITY else O.PREC_JACOBI
    P = O.Problem.csr_matrix(csr, opk)
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(prec_kind, 1e-3)
        for tol in (0.0, 0.5):
            ctx.count_slices(shifts, m, k, tol=tol, seed=0)
            got = ctx.quad_bound(len(shifts) * m)
            _, _, kd = ctx.tridiag(len(shifts) * m, k)
            for c in (0, 5, 36, 37, 73):
                s, j = divmod(c, m)
                v = O.probe_vector(0, j, 300)
                _, be, _, _ = O.lanczos(P, shifts[s], v, int(kd[c]))
                assert got[c] == pytest.approx(O.quad_bound_log10(be, int(kd[c]), v @ v), abs=1e-8)
            assert np.all(np.isfinite(got))
    # p distinct eigenvalues: the process breaks down and the bound collapses
    distinct = [-2.0, -0.5, 0.7, 1.5, 3.0]
    D = I.random_symmetric_dense(64, seed=4, distinct=distinct)
    with evc.Context.csr(I.dense_to_csr(D), precision=evc.EVC_FP64) as ctx:
        ctx.count_slices([0.0], 4, 12, seed=0)
        got = ctx.quad_bound(4)
    assert np.all(got < -20.0)


def test_edge_sizes():
    csr = I.laplace2d_dirichlet(5)          # n = 25
    P = O.Problem.csr_matrix(csr, O.PREC_NONE)
    # m = 1, k = 1
    L, q, st, _ = _gpu_csr(csr, evc.EVC_FP64, evc.EVC_PREC_IDENTITY, 0, [3.9], 1, 1)
    qr, sr, Lr = O.count(P, [3.9], 1, 1, seed=0)
    assert abs(q[0, 0] - qr[0, 0]) < FP64_TOL and list(st) == [1]
    # maxsteps > n is clamped to n; the exhaustive Krylov space is exact
    L, q, st, _ = _gpu_csr(csr, evc.EVC_FP64, evc.EVC_PREC_IDENTITY, 0, [3.9], 3, 60)
    qr, sr, Lr = O.count(P, [3.9], 3, 60, seed=0)
    assert np.max(np.abs(q - qr)) < FP64_TOL


def test_one_by_one_and_two_by_two_matrices():
    # n = 1: J_1 = [a - tau], so the count of one probe is 1 iff a < tau (the
    # probe has ||v||^2 = 1); n = 2 with k clamped to 2 is exact (Proposition 1)
    one = (np.array([0, 1]), np.array([0], dtype=np.int32), np.array([0.7]))
    for prec in (evc.EVC_FP64, evc.EVC_MIXED):
        L, q, st, _ = _gpu_csr(one, prec, evc.EVC_PREC_IDENTITY, 0, [0.5, 0.9], 3, 5)
        np.testing.assert_array_equal(q, [[0.0] * 3, [1.0] * 3])
        assert list(st) == [1, 1]
    A = np.array([[1.0, 2.0], [2.0, -1.0]])            # eigenvalues +-sqrt(5)
    csr = I.dense_to_csr(A)
    P = O.Problem.csr_matrix(csr, O.PREC_NONE)
    L, q, st, _ = _gpu_csr(csr, evc.EVC_FP64, evc.EVC_PREC_IDENTITY, 0, [-3.0, 0.0, 3.0], 4, 9)
    qr, sr, Lr = O.count(P, [-3.0, 0.0, 3.0], 4, 9, seed=0)
    assert np.max(np.abs(q - qr)) < FP64_TOL
    # each probe's quadrature is exact: v^T h(A - tau I) v from the eigenvectors
    w, U = np.linalg.eigh(A)
    for s, tau in enumerate([-3.0, 0.0, 3.0]):
        for j in range(4):
            v = O.probe_vector(0, j, 2)
            exact = float(np.sum((U[:, w < tau].T @ v) ** 2))
            assert abs(q[s, j] - exact) < 1e-12


def test_maximum_steps_both_rules():
    # k = EVC_MAX_STEPS (256) on a random sparse indefinite n = 300 (no early
    # breakdown): the Gauss rule on J_256 against the oracle; the averaged rule
    # at k = 128 (a 255 x 255 extension; the oracle's cyclic Jacobi on the
    # 511 x 511 extension of k = 256 takes about a minute per probe)
    A = I.random_symmetric_dense(300, seed=17)
    A[np.abs(A) < 1.0] = 0.0
    A = 0.5 * (A + A.T) + np.diag(np.linspace(-2, 2, 300))
    csr = I.dense_to_csr(A)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    for rule, k in ((evc.EVC_QUAD_GAUSS, evc.EVC_MAX_STEPS), (evc.EVC_QUAD_GA, 128)):
        with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
            ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
            ctx.set_option(evc.EVC_OPT_QUADRATURE, rule)
            L, q, st = ctx.count_slices([0.3], 3, k, seed=1)
        qr, sr, Lr = O.count(P, [0.3], 3, k, seed=1, rule=rule)
        assert list(st) == list(sr)
        assert np.max(np.abs(q - qr)) < FP64_TOL


# --------------------------------------------------------- CSR, mixed

def test_csr_mixed_estimate_within_half():
    # generic sparse symmetric indefinite (power-law rows, Jacobi), 50 steps
    csr = I.powerlaw_symmetric(3000, seed=2)
    shifts = [-0.5, 0.5]
    L, q, st, _ = _gpu_csr(csr, evc.EVC_MIXED, evc.EVC_PREC_JACOBI, 1e-3, shifts, 64, 50)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    qr, sr, Lr = O.count(P, shifts, 64, 50, seed=0)
    assert abs((L[1] - L[0]) - (Lr[1] - Lr[0])) < MIXED_EST_TOL
    assert np.max(np.abs(L - Lr)) < MIXED_EST_TOL


def test_csr_mixed_estimate_within_half_large_count():
    # n = 20,000: n_- estimates near 1e4 per shift, Jacobi with eps = 1e-3 (so
    # m_r^2 reaches 1e3 on rows with a_rr near the shift).  The mixed path forms
    # the Jacobi scales and the shifted diagonal from the FP64 diagonal; the
    # estimate and each n_below stay within 0.5 of the FP64 oracle.
    csr = I.powerlaw_symmetric(20000, seed=2)
    shifts = [-0.5, 0.5]
    L, q, st, _ = _gpu_csr(csr, evc.EVC_MIXED, evc.EVC_PREC_JACOBI, 1e-3, shifts, 64, 50)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    qr, sr, Lr = O.count(P, shifts, 64, 50, seed=0)
    assert abs((L[1] - L[0]) - (Lr[1] - Lr[0])) < MIXED_EST_TOL
    assert np.max(np.abs(L - Lr)) < MIXED_EST_TOL


def test_csr_mixed_fp32_input_values_same_diagonal():
    # float32 values given to an FP64 and a mixed context describe the same
    # matrix, so both form the same FP64 diagonal; a context fed float64
    # values forms it from those.  The three estimates agree within 0.5.
    rp, col, val = I.powerlaw_symmetric(20000, seed=2)
    v32 = val.astype(np.float32)
    shifts = [-0.5, 0.5]
    out = []
    for prec, vals in ((evc.EVC_FP64, v32), (evc.EVC_MIXED, v32), (evc.EVC_MIXED, val)):
        with evc.Context.csr((rp, col, vals), precision=prec) as ctx:
            ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
            L, q, st = ctx.count_slices(shifts, 64, 50, seed=0)
        out.append(L)
    assert np.max(np.abs(out[0] - out[1])) < MIXED_EST_TOL
    P = O.Problem.csr_matrix((rp, col, val), O.PREC_JACOBI)
    _, _, Lr = O.count(P, shifts, 64, 50, seed=0)
    assert np.max(np.abs(out[2] - Lr)) < MIXED_EST_TOL


def test_csr_mixed_far_from_quadrature_convergence():
    # 2D Laplacian 40x40, scalar Jacobi, k = 40: far from quadrature
    # convergence, where a single classical Gram-Schmidt sweep over an FP32
    # basis loses orthogonality and biases the estimate.  The Gram-corrected
    # sweep keeps the mixed estimate within the FP64 tolerance.
    csr = I.laplace2d_dirichlet(40)
    out = {}
    for prec in (evc.EVC_FP64, evc.EVC_MIXED):
        L, q, st, _ = _gpu_csr(csr, prec, evc.EVC_PREC_JACOBI, 1e-3, [1.0, 2.0], 64, 40)
        out[prec] = (L, q)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    qr, _, Lr = O.count(P, [1.0, 2.0], 64, 40, seed=0)
    np.testing.assert_allclose(out[evc.EVC_FP64][0], Lr, rtol=0, atol=1e-9)
    assert np.max(np.abs(out[evc.EVC_FP64][1] - qr)) < FP64_TOL
    assert np.max(np.abs(out[evc.EVC_MIXED][0] - Lr)) < MIXED_EST_TOL


# ------------------------------------------------------------ stencil

@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("pk", ["cheb", "jacobi", "identity"])
def test_stencil_fp64_per_probe(order, pk):
    # N = 12: ragged x/y tiles; 40 probes x 2 shifts = 3 chunks (padded)
    N, h = 12, 0.3
    V = I.gaussian_wells(N, h, nwells=6, seed=1)
    shifts = [-2.5, 0.5]
    m, k = 40, 14
    kind = {"cheb": evc.EVC_PREC_CHEB_KINETIC, "jacobi": evc.EVC_PREC_JACOBI,
            "identity": evc.EVC_PREC_IDENTITY}[pk]
    p0, p1 = {"cheb": (8, 1.0), "jacobi": (1e-3, 0), "identity": (0, 0)}[pk]
    L, q, st = _gpu_stencil(N, h, order, V, evc.EVC_FP64, kind, p0, p1, shifts, m, k)
    opk = {"cheb": O.PREC_CHEB, "jacobi": O.PREC_JACOBI, "identity": O.PREC_NONE}[pk]
    P = O.Problem.stencil(N, h, order, V, opk, cheb_degree=8, cheb_c=1.0, jac_eps=1e-3)
    qr, sr, Lr = O.count(P, shifts, m, k, seed=0)
    assert np.max(np.abs(q - qr)) < FP64_TOL
    np.testing.assert_allclose(L, Lr, rtol=0, atol=1e-9)


@pytest.mark.parametrize("order", [2, 4])
def test_stencil_mixed_estimate(order):
    N, h = 16, 0.3
    V = I.gaussian_wells(N, h, nwells=8, seed=1)
    shifts = [-3.0, 1.0]
    m, k = 64, 20
    L, q, st = _gpu_stencil(N, h, order, V, evc.EVC_MIXED, evc.EVC_PREC_CHEB_KINETIC, 8, 1.0,
                            shifts, m, k)
    P = O.Problem.stencil(N, h, order, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, sr, Lr = O.count(P, shifts, m, k, seed=0)
    assert abs((L[1] - L[0]) - (Lr[1] - Lr[0])) < MIXED_EST_TOL
    assert np.max(np.abs(L - Lr)) < MIXED_EST_TOL


def test_stencil_adaptive_slices_fp64():
    N, h = 10, 0.3
    V = I.gaussian_wells(N, h, nwells=4, seed=1)
    shifts = list(np.linspace(-4.0, 2.0, 7))
    L, q, st = _gpu_stencil(N, h, 2, V, evc.EVC_FP64, evc.EVC_PREC_CHEB_KINETIC, 8, 1.0,
                            shifts, 16, 30, tol=0.25)
    P = O.Problem.stencil(N, h, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, sr, Lr = O.count(P, shifts, 16, 30, tol=0.25, seed=0)
    assert list(st) == list(sr)
    assert np.max(np.abs(q - qr)) < FP64_TOL


def test_results_independent_of_batch_mix():
    # a column's result is the same alone and batched with other shifts
    N, h = 10, 0.3
    V = I.gaussian_wells(N, h, nwells=4, seed=1)
    with evc.Context.stencil(N, h, 2, V, precision=evc.EVC_MIXED) as ctx:
        ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
        L1, q1, _ = ctx.count_slices([-1.0], 32, 15)
        L3, q3, _ = ctx.count_slices([-3.0, -1.0, 0.5], 32, 15)
    np.testing.assert_array_equal(q1[0], q3[1])


def test_graph_replay_and_eager_agree():
    csr = I.laplace2d_dirichlet(16)
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        a = ctx.count_slices([1.0, 2.0], 8, 20, seed=3)
        b = ctx.count_slices([1.0, 2.0], 8, 20, seed=3)      # replay of the cached graph
        c = ctx.count_slices([1.5, 2.5], 8, 20, seed=4)      # new shifts / seed, same graph
        evc.evc_set_option(ctx.h, evc.EVC_OPT_GRAPH, 0)
        d = ctx.count_slices([1.5, 2.5], 8, 20, seed=4)
    np.testing.assert_array_equal(a[1], b[1])
    np.testing.assert_array_equal(c[1], d[1])
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    qr, _, _ = O.count(P, [1.5, 2.5], 8, 20, seed=4)
    assert np.max(np.abs(c[1] - qr)) < FP64_TOL


# -------------------------------------------------------------- errors

def test_invalid_arguments_return_status():
    csr = I.laplace2d_dirichlet(4)
    with evc.Context.csr(csr) as ctx:
        for bad in [dict(nprobe=0, maxsteps=4), dict(nprobe=2, maxsteps=0),
                    dict(nprobe=2, maxsteps=evc.EVC_MAX_STEPS + 1)]:
            with pytest.raises(evc.EvcError) as e:
                evc.evc_count_slices(ctx.h, [1.0], bad["nprobe"], bad["maxsteps"])
            assert e.value.code == evc.EVC_EINVAL
        with pytest.raises(evc.EvcError) as e:
            evc.evc_count(ctx.h, 2.0, 1.0, 4, 4)
        assert e.value.code == evc.EVC_EINVAL
        with pytest.raises(evc.EvcError) as e:
            evc.evc_set_precond(ctx.h, evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
        assert e.value.code == evc.EVC_EUNSUPPORTED
    # asymmetric matrix is rejected by the host check
    rp, ci, va = I.laplace2d_dirichlet(4)
    va = va.copy()
    va[1] += 0.5
    with pytest.raises(evc.EvcError) as e:
        evc.evc_create_csr(rp, ci, va)
    assert e.value.code == evc.EVC_EINVAL
    # out-of-range column
    ci2 = ci.copy()
    ci2[3] = 99
    with pytest.raises(evc.EvcError):
        evc.evc_create_csr(rp, ci2, va)


# ------------------------------------------- generalized averaged quadrature

@pytest.mark.parametrize("prec", [evc.EVC_FP64, evc.EVC_MIXED])
def test_ga_quadrature_matches_oracle(prec):
    # Sec. 3.4: the same Lanczos steps, step 5 of Algorithm 2 on the extended
    # tridiagonal of Eq. GA_Tk.
    N, h = 12, 0.3
    V = I.gaussian_wells(N, h, nwells=6, seed=1)
    shifts = [-2.5, 0.5]
    m, k = 40, 10
    with evc.Context.stencil(N, h, 2, V, precision=prec) as ctx:
        ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_QUADRATURE, evc.EVC_QUAD_GA)
        L, q, st = ctx.count_slices(shifts, m, k)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_QUADRATURE, evc.EVC_QUAD_GAUSS)
        Lg, qg, _ = ctx.count_slices(shifts, m, k)
    P = O.Problem.stencil(N, h, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    qr, sr, Lr = O.count(P, shifts, m, k, seed=0, rule=1)
    qgr, _, _ = O.count(P, shifts, m, k, seed=0, rule=0)
    if prec == evc.EVC_FP64:
        assert np.max(np.abs(q - qr)) < FP64_TOL
        assert np.max(np.abs(qg - qgr)) < FP64_TOL
    assert np.max(np.abs(L - Lr)) < MIXED_EST_TOL
    assert np.max(np.abs(q - qg)) > 1e-6      # the two rules differ at k = 10


def test_ga_adaptive_csr_fp64():
    csr = I.laplace2d_dirichlet(20)
    shifts = [0.5, 1.5, 3.0]
    with evc.Context.csr(csr, precision=evc.EVC_FP64) as ctx:
        ctx.set_precond(evc.EVC_PREC_JACOBI, 1e-3)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_QUADRATURE, evc.EVC_QUAD_GA)
        L, q, st = ctx.count_slices(shifts, 12, 40, tol=0.25)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    qr, sr, Lr = O.count(P, shifts, 12, 40, tol=0.25, seed=0, rule=1)
    assert list(st) == list(sr)
    assert np.max(np.abs(q - qr)) < FP64_TOL


def test_probe_offset_shards_concatenate_to_the_unsharded_count():
    # sharding one count by probes (one GPU per shard) gives the same columns
    N, h = 12, 0.3
    V = I.gaussian_wells(N, h, nwells=6, seed=1)
    with evc.Context.stencil(N, h, 2, V, precision=evc.EVC_MIXED) as ctx:
        ctx.set_precond(evc.EVC_PREC_CHEB_KINETIC, 8, 1.0)
        L, q, _ = ctx.count_slices([-2.0, 0.5], 40, 12, seed=5)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_PROBE_OFFSET, 0)
        _, qa, _ = ctx.count_slices([-2.0, 0.5], 25, 12, seed=5)
        evc.evc_set_option(ctx.h, evc.EVC_OPT_PROBE_OFFSET, 25)
        _, qb, _ = ctx.count_slices([-2.0, 0.5], 15, 12, seed=5)
    np.testing.assert_array_equal(np.concatenate([qa, qb], axis=1), q)
