"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares the oracle with a
closed form, an independent library routine (numpy / scipy), an invariant, or
a printed value of the paper, chosen so that a dropped term, a wrong sign or
index, or a transposed operand in the oracle fails at least one of them.
"""
import json
import os

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import oracle as O
from paper_1602_02306_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _dense_C(P, tau):
    n = P.n
    return np.stack([O.apply_C(P, tau, e) for e in np.eye(n)], axis=1)


# ----------------------------------------------------------------- probes

def _mix64_py(z):
    M = (1 << 64) - 1
    z &= M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_mix64_matches_published_definition():
    # SplitMix64 finaliser (Steele, Lea & Flood 2014), big-int restatement.
    for z in [0, 1, 2, 0x9E3779B97F4A7C15, 12345678901234567, (1 << 64) - 1]:
        assert O.mix64(z) == _mix64_py(z)


def test_probe_entries_are_signs_of_the_hash():
    n = 257
    for seed, j in [(0, 0), (0, 5), (7, 3), (2**40 + 3, 1000)]:
        v = O.probe_vector(seed, j, n)
        want = np.array([-1.0 if (_mix64_py(seed ^ _mix64_py((j << 32) | i)) >> 63) else 1.0
                         for i in range(n)])
        np.testing.assert_array_equal(v, want)
    # zero mean / unit variance in the sample (Sec. 2, Eq. trace)
    v = O.probe_vector(0, 1, 200000)
    assert abs(v.mean()) < 0.01 and np.all(v * v == 1.0)


# -------------------------------------------------------------- operators

def test_csr_apply_matches_dense_matvec():
    csr = I.laplace2d_dirichlet(9)
    P = O.Problem.csr_matrix(csr)
    rp, ci, va = csr
    n = len(rp) - 1
    A = np.zeros((n, n))
    for r in range(n):
        for k in range(rp[r], rp[r + 1]):
            A[r, ci[k]] += va[k]
    x = np.random.default_rng(0).standard_normal(n)
    np.testing.assert_allclose(O.apply_A(P, x), A @ x, rtol=0, atol=1e-12)


def test_laplace2d_spectrum_closed_form():
    # the generator's matrix has the textbook Dirichlet spectrum
    N = 12
    rp, ci, va = I.laplace2d_dirichlet(N)
    n = N * N
    A = np.zeros((n, n))
    for r in range(n):
        A[r, ci[rp[r]:rp[r + 1]]] = va[rp[r]:rp[r + 1]]
    i = np.arange(1, N + 1)
    s = 4 * np.sin(i * np.pi / (2 * (N + 1))) ** 2
    lam = np.sort((s[:, None] + s[None, :]).ravel())
    np.testing.assert_allclose(np.linalg.eigvalsh(A), lam, atol=1e-12)


@pytest.mark.parametrize("order", [2, 4])
def test_stencil_plane_wave_symbol(order):
    # Plane waves are eigenvectors of the periodic FD Laplacian; the eigenvalue
    # of -1/2 Lap_h is the stencil symbol (textbook Fourier analysis).
    N, h = 6, 0.3
    P = O.Problem.stencil(N, h, order, np.zeros(N ** 3))
    g = np.arange(N)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    for kx, ky, kz in [(1, 0, 0), (0, 2, 1), (3, 3, 3), (2, 5, 1)]:
        th = 2 * np.pi * np.array([kx, ky, kz]) / N
        wave = np.cos(th[0] * x + th[1] * y + th[2] * z).ravel()
        if order == 2:
            sym = sum((1 - np.cos(t)) for t in th) / h ** 2
        else:
            sym = sum((30 - 32 * np.cos(t) + 2 * np.cos(2 * t)) for t in th) / (24 * h ** 2)
        np.testing.assert_allclose(O.apply_A(P, wave), sym * wave, atol=1e-10)


def test_stencil_potential_is_diagonal():
    N = 5
    V = np.random.default_rng(3).standard_normal(N ** 3)
    P = O.Problem.stencil(N, 0.4, 2, V)
    P0 = O.Problem.stencil(N, 0.4, 2, np.zeros(N ** 3))
    x = np.random.default_rng(4).standard_normal(N ** 3)
    np.testing.assert_allclose(O.apply_A(P, x) - O.apply_A(P0, x), V * x, atol=1e-12)


def test_stencil_symmetric():
    N = 5
    V = I.gaussian_wells(N, 0.3, nwells=3, seed=1)
    for order in (2, 4):
        P = O.Problem.stencil(N, 0.3, order, V)
        A = np.stack([O.apply_A(P, e) for e in np.eye(N ** 3)], axis=1)
        np.testing.assert_allclose(A, A.T, atol=1e-12)


def test_jacobi_preconditioner_definition():
    A = I.random_symmetric_dense(10, seed=5)
    P = O.Problem.dense_matrix(A, O.PREC_JACOBI, jac_eps=1e-3)
    tau = 0.3
    x = np.arange(10.0) - 4.0
    want = x / np.sqrt(np.abs(np.diag(A) - tau) + 1e-3)
    np.testing.assert_allclose(O.apply_M(P, tau, x), want, rtol=1e-15)


@pytest.mark.parametrize("order", [2, 4])
def test_stencil_jacobi_uses_the_operator_diagonal(order):
    # The Jacobi scaling of a stencil operator must use the diagonal of the
    # operator itself: a_rr = e_r^T A e_r, assembled here through apply_A on
    # unit vectors (apply_A is pinned to the plane-wave symbols above), so a
    # wrong kinetic diagonal in the Jacobi set-up (a 7-point value for the
    # 13-point stencil, a missing V, a wrong 1/h^2) fails.  M is diagonal.
    N, h, tau, eps = 5, 0.3, -1.25, 1e-3
    V = I.gaussian_wells(N, h, nwells=3, seed=1)
    P = O.Problem.stencil(N, h, order, V, O.PREC_JACOBI, jac_eps=eps)
    n = N ** 3
    for r in (0, 7, 62, n - 1):
        e = np.zeros(n)
        e[r] = 1.0
        a_rr = O.apply_A(P, e)[r]
        Me = O.apply_M(P, tau, e)
        want = 1.0 / np.sqrt(abs(a_rr - tau) + eps)
        assert abs(Me[r] - want) <= 1e-14 * want
        assert np.count_nonzero(Me) == 1


@pytest.mark.parametrize("order", [2, 4])
def test_chebyshev_coefficients_match_numpy_interpolant(order):
    # numpy's Chebyshev.interpolate uses first-kind Chebyshev points: the same
    # interpolant of x^-1/2, computed by an independent library.
    P = O.Problem.stencil(4, 0.3, order, np.zeros(64), O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    a, b = O.kinetic_interval(P)
    assert a == 1.0 and b == pytest.approx(1.0 + (6.0 if order == 2 else 8.0) / 0.09)
    ref = np.polynomial.Chebyshev.interpolate(lambda x: x ** -0.5, 8, domain=[a, b])
    np.testing.assert_allclose(O.cheb_coeffs(8, a, b), ref.coef, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("order", [2, 4])
def test_chebyshev_preconditioner_on_plane_waves(order):
    N, h, c = 6, 0.3, 1.0
    P = O.Problem.stencil(N, h, order, np.zeros(N ** 3), O.PREC_CHEB, cheb_degree=8, cheb_c=c)
    a, b = O.kinetic_interval(P)
    p = np.polynomial.Chebyshev.interpolate(lambda x: x ** -0.5, 8, domain=[a, b])
    g = np.arange(N)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    for kv in [(0, 0, 0), (1, 0, 0), (3, 3, 3), (1, 2, 3)]:
        th = 2 * np.pi * np.array(kv) / N
        wave = np.cos(th[0] * x + th[1] * y + th[2] * z).ravel()
        if order == 2:
            lamK = c + sum((1 - np.cos(t)) for t in th) / h ** 2
        else:
            lamK = c + sum((30 - 32 * np.cos(t) + 2 * np.cos(2 * t)) for t in th) / (24 * h ** 2)
        got = O.apply_M(P, 0.0, wave)
        np.testing.assert_allclose(got, p(lamK) * wave, atol=1e-11)
        # M approximates K^{-1/2} and is positive on spec(K) (T = M^2 HPD, Sec. 6)
        assert p(lamK) > 0
        assert abs(p(lamK) * np.sqrt(lamK) - 1) < 0.15


def test_congruence_preserves_inertia():
    # Sec. 2, Eq. (negi_T): C = M (A - tau I) M has the inertia of A - tau I.
    A = I.random_symmetric_dense(20, seed=11)
    tau = 0.1
    want = int((np.linalg.eigvalsh(A) < tau).sum())
    for prec in (O.PREC_NONE, O.PREC_JACOBI):
        P = O.Problem.dense_matrix(A, prec)
        assert int((np.linalg.eigvalsh(_dense_C(P, tau)) < 0).sum()) == want
    N = 4
    V = I.gaussian_wells(N, 0.3, nwells=2, seed=1)
    P = O.Problem.stencil(N, 0.3, 2, V, O.PREC_CHEB)
    H = np.stack([O.apply_A(O.Problem.stencil(N, 0.3, 2, V), e) for e in np.eye(N ** 3)], 1)
    tau = float(np.sort(np.linalg.eigvalsh(H))[10] + 1e-3)
    want = int((np.linalg.eigvalsh(H) < tau).sum())
    Cm = _dense_C(P, tau)
    np.testing.assert_allclose(Cm, Cm.T, atol=1e-10)
    assert int((np.linalg.eigvalsh(Cm) < 0).sum()) == want


# ---------------------------------------------------------------- Lanczos

def test_lanczos_relation_and_orthonormality():
    # Sec. 3, Eq. (lan): C Q_k = Q_{k+1} J_{k+1,k}, Q_{k+1}^T Q_{k+1} = I
    A = I.random_symmetric_dense(30, seed=1)
    P = O.Problem.dense_matrix(A, O.PREC_JACOBI)
    tau = 0.2
    v = O.probe_vector(0, 3, 30)
    k = 8
    al, be, Q, kd = O.lanczos(P, tau, v, k, want_Q=True)
    assert kd == k
    Qm = Q.T                                  # n x (k+1)
    Cm = _dense_C(P, tau)
    J = np.zeros((k + 1, k))
    for i in range(k):
        J[i, i] = al[i]
        J[i + 1, i] = be[i + 1]
        if i + 1 < k:
            J[i, i + 1] = be[i + 1]
    np.testing.assert_allclose(Cm @ Qm[:, :k], Qm @ J, atol=1e-12)
    np.testing.assert_allclose(Qm.T @ Qm, np.eye(k + 1), atol=1e-13)
    np.testing.assert_allclose(Qm[:, 0], v / np.linalg.norm(v), atol=1e-15)
    assert be[0] == 0.0 and np.all(be[1:] > 0)


def test_tridiag_eig_matches_scipy():
    rng = np.random.default_rng(2)
    for k in (1, 2, 5, 17, 50):
        al = rng.standard_normal(k)
        be = np.concatenate([[0.0], np.abs(rng.standard_normal(k))])
        th, z1 = O.tridiag_eig(al, be)
        w, Z = sla.eigh_tridiagonal(al, be[1:k])
        np.testing.assert_allclose(th, w, atol=1e-12)
        np.testing.assert_allclose(np.abs(z1), np.abs(Z[0]), atol=1e-10)


def test_weights_sum_to_norm_squared():
    # Sec. 3, Eq. (gauss_quad): sum_i w_i = ||v||^2 e_1^T e_1 = ||v||^2
    A = I.random_symmetric_dense(40, seed=3)
    P = O.Problem.dense_matrix(A)
    v = O.probe_vector(5, 0, 40)
    al, be, _, kd = O.lanczos(P, 0.0, v, 12)
    th, z1 = O.tridiag_eig(al, be)
    assert np.sum(40 * z1 ** 2) == pytest.approx(40.0, rel=1e-13)
    # shifting tau past every eigenvalue makes h(C) = I  ->  quadrature = ||v||^2
    lam = np.linalg.eigvalsh(A)
    al, be, _, _ = O.lanczos(P, lam[-1] + 1.0, v, 6)
    assert O.gauss_quad(al, be, 40.0) == pytest.approx(40.0, rel=1e-12)
    al, be, _, _ = O.lanczos(P, lam[0] - 1.0, v, 6)
    assert O.gauss_quad(al, be, 40.0) == 0.0


def test_moments_exact_to_degree_2k_minus_1():
    # Gauss quadrature is exact for polynomials of degree <= 2k-1 (Sec. 3.4):
    # ||v||^2 e_1^T J_k^j e_1 = v^T C^j v for j <= 2k-1.
    A = I.random_symmetric_dense(25, seed=8)
    P = O.Problem.dense_matrix(A, O.PREC_JACOBI)
    tau = -0.1
    v = O.probe_vector(1, 2, 25)
    Cm = _dense_C(P, tau)
    k = 5
    al, be, _, _ = O.lanczos(P, tau, v, k)
    J = np.diag(al) + np.diag(be[1:k], 1) + np.diag(be[1:k], -1)
    for j in range(0, 2 * k):
        lhs = 25.0 * np.linalg.matrix_power(J, j)[0, 0]
        rhs = v @ np.linalg.matrix_power(Cm, j) @ v
        assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-9)
    lhs = 25.0 * np.linalg.matrix_power(J, 2 * k)[0, 0]
    rhs = v @ np.linalg.matrix_power(Cm, 2 * k) @ v
    assert abs(lhs - rhs) > 1e-6 * abs(rhs)       # degree 2k is not exact in general


@pytest.mark.parametrize("k", [1, 3, 6])
def test_quad_bound_is_the_error_for_degree_2k(k):
    # Sec. 3, Eq. qbound: |eps_k| <= N_k ||v||^2 beta_2^2...beta_{k+1}^2 / (2k)!
    # with N_k >= |f^(2k)|.  For f(x) = x^(2k), f^(2k) = (2k)! and the bound is
    # attained: the Gauss error is ||v||^2 times the squared norm of the monic
    # degree-k orthogonal polynomial (it vanishes at the nodes).  So the
    # oracle's factor times (2k)! must equal v^T C^(2k) v - ||v||^2 e1^T J^(2k) e1.
    A = I.random_symmetric_dense(25, seed=8)
    P = O.Problem.dense_matrix(A, O.PREC_JACOBI)
    tau = -0.1
    v = O.probe_vector(1, 2, 25)
    Cm = _dense_C(P, tau)
    al, be, _, kd = O.lanczos(P, tau, v, k)
    assert kd == k
    J = np.diag(al) + np.diag(be[1:k], 1) + np.diag(be[1:k], -1)
    err = v @ np.linalg.matrix_power(Cm, 2 * k) @ v - 25.0 * np.linalg.matrix_power(J, 2 * k)[0, 0]
    import math
    bound = 10.0 ** O.quad_bound_log10(be, k, v @ v) * math.factorial(2 * k)
    assert err > 0 and bound == pytest.approx(err, rel=1e-7)


def test_quad_bound_holds_for_exp_and_is_exact_after_breakdown():
    # f = exp on C / ||C||: N_k = max e^x on the spectrum; the Gauss error of
    # v^T e^C v stays below the bound and above a small fraction of it.  After a
    # breakdown (p distinct eigenvalues, Proposition 1) the factor is -inf.
    A = I.random_symmetric_dense(30, seed=5)
    A = A / np.linalg.norm(A, 2)
    P = O.Problem.dense_matrix(A)
    v = O.probe_vector(2, 3, 30)
    w, U = np.linalg.eigh(A)
    exact = float(v @ (U * np.exp(w)) @ U.T @ v)
    for k in (2, 3, 4):
        al, be, _, _ = O.lanczos(P, 0.0, v, k)
        th, z1 = np.linalg.eigh(np.diag(al) + np.diag(be[1:k], 1) + np.diag(be[1:k], -1))
        quad = 30.0 * float(np.sum(np.exp(th) * z1[0] ** 2))
        bound = np.exp(w.max()) * 10.0 ** O.quad_bound_log10(be, k, v @ v)
        assert abs(exact - quad) <= bound
        assert abs(exact - quad) >= 1e-3 * bound
    D = I.random_symmetric_dense(30, seed=4, distinct=[-2.0, -0.5, 0.7, 1.5, 3.0])
    al, be, _, kd = O.lanczos(O.Problem.dense_matrix(D), 0.0, v, 12)
    assert kd == 5
    # beta_{p+1} is at rounding level: the bound collapses ...
    assert O.quad_bound_log10(be, kd, v @ v) < -25.0
    # ... and an exact zero makes the rule exact
    be = be.copy()
    be[kd] = 0.0
    assert O.quad_bound_log10(be, kd, v @ v) == -np.inf


def test_proposition1_exact_at_p_distinct_eigenvalues():
    # Sec. 3, Proposition 1: with p distinct eigenvalues of C, k = p is exact,
    # and the Lanczos process breaks down at step p.
    distinct = [-2.0, -0.5, 0.7, 1.5, 3.0]
    A = I.random_symmetric_dense(30, seed=4, distinct=distinct)
    P = O.Problem.dense_matrix(A)
    v = O.probe_vector(9, 1, 30)
    w, U = np.linalg.eigh(A)
    exact = float(np.sum((U[:, w < 0].T @ v) ** 2))           # Eq. (wsum)
    al, be, _, kd = O.lanczos(P, 0.0, v, 12)
    assert kd == len(distinct)
    assert O.gauss_quad(al, be, v @ v) == pytest.approx(exact, abs=1e-10)
    al3, be3, _, _ = O.lanczos(P, 0.0, v, 3)
    assert abs(O.gauss_quad(al3, be3, v @ v) - exact) > 1e-6


def test_ideal_preconditioner_exact_in_two_steps():
    # Sec. 6: T = |A - tau I|^-1 gives C with eigenvalues +-1, exact at k = 2.
    A = I.random_symmetric_dense(24, seed=6)
    tau = 0.05
    w, U = np.linalg.eigh(A - tau * np.eye(24))
    M = (U * np.abs(w) ** -0.5) @ U.T
    P = O.Problem.dense_matrix(A, O.PREC_DENSE, denseM=0.5 * (M + M.T))
    v = O.probe_vector(3, 7, 24)
    exact = float(np.sum((U[:, w < 0].T @ v) ** 2))
    al, be, _, kd = O.lanczos(P, tau, v, 6)
    assert kd == 2
    assert O.gauss_quad(al, be, v @ v) == pytest.approx(exact, abs=1e-10)


def test_theorem1_polynomial_identity():
    # Sec. 5, Theorem 1: ||v|| Q_k f(J_k) e_1 = f(C) v for polynomials f of
    # degree <= k-1.
    A = I.random_symmetric_dense(20, seed=12)
    P = O.Problem.dense_matrix(A, O.PREC_JACOBI)
    tau = 0.3
    v = O.probe_vector(2, 2, 20)
    k = 5
    al, be, Q, _ = O.lanczos(P, tau, v, k, want_Q=True)
    Qk = Q[:k].T
    J = np.diag(al) + np.diag(be[1:k], 1) + np.diag(be[1:k], -1)
    Cm = _dense_C(P, tau)
    e1 = np.eye(k)[0]
    for f in (lambda X: X @ X, lambda X: X @ X @ X - 2 * X):
        lhs = np.linalg.norm(v) * Qk @ (f(J) @ e1)
        np.testing.assert_allclose(lhs, f(Cm) @ v, atol=1e-10)


# --------------------------------------------------------------- estimator

def _hadamard(n):
    return sla.hadamard(n).astype(np.float64)


def _exhaustive_estimate(P, tau, n):
    # Full Sylvester-Hadamard probe set (H H^T = n I) and k = n: the
    # estimator equals trace h(C) = n_-(A - tau I) exactly (Eq. traceT).
    Hm = _hadamard(n)
    tot = 0.0
    for j in range(n):
        v = Hm[j]
        al, be, _, kd = O.lanczos(P, tau, v, n)
        tot += O.gauss_quad(al, be, v @ v)
    return tot / n


@pytest.mark.parametrize("prec", [O.PREC_NONE, O.PREC_JACOBI])
def test_exhaustive_hadamard_equals_inertia(prec):
    A = I.random_symmetric_dense(16, seed=21)
    lam = np.linalg.eigvalsh(A)
    xi, eta = -0.7, 0.9
    P = O.Problem.dense_matrix(A, prec)
    got = _exhaustive_estimate(P, eta, 16) - _exhaustive_estimate(P, xi, 16)
    want = int(((lam > xi) & (lam < eta)).sum())
    assert got == pytest.approx(want, abs=1e-8)


def test_exhaustive_on_laplace_grid():
    # 8x8 Dirichlet Laplacian: closed-form count below tau = 2.5
    csr = I.laplace2d_dirichlet(8)
    i = np.arange(1, 9)
    s = 4 * np.sin(i * np.pi / 18) ** 2
    want = int(((s[:, None] + s[None, :]) < 2.5).sum())
    for prec in (O.PREC_NONE, O.PREC_JACOBI):
        P = O.Problem.csr_matrix(csr, prec)
        assert _exhaustive_estimate(P, 2.5, 64) == pytest.approx(want, abs=1e-7)


def test_count_stop_rule_and_means():
    csr = I.laplace2d_dirichlet(10)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    shifts = [1.0, 2.3]
    quad, steps, L = O.count(P, shifts, 6, 20, tol=0.3, seed=4)
    np.testing.assert_allclose(L, quad.mean(axis=1), rtol=1e-15)
    for s, tau in enumerate(shifts):
        ks = steps[s]
        assert 3 <= ks <= 20
        # the fixed-k run with k = ks reproduces the stopped run
        q2, _, _ = O.count(P, [tau], 6, int(ks), tol=0.0, seed=4)
        np.testing.assert_allclose(q2[0], quad[s], rtol=0, atol=1e-9)
        # the rule: two consecutive changes within tol at ks, and not at any earlier step >= 3
        Ls = [O.count(P, [tau], 6, i, seed=4)[2][0] for i in range(1, int(ks) + 1)]
        small = [abs(Ls[i] - Ls[i - 1]) <= 0.3 for i in range(1, len(Ls))]   # small[i-1]: step i+1
        if ks < 20:                            # stopped by the rule, not by the cap
            assert small[ks - 2] and small[ks - 3]
        for i in range(3, ks):
            assert not (small[i - 2] and small[i - 3])
    # a minimum step count delays the stop
    _, steps5, _ = O.count(P, shifts, 6, 20, tol=0.3, seed=4, min_steps=8)
    assert all(s >= 8 for s in steps5)


def test_count_columns_independent_of_batch():
    csr = I.laplace2d_dirichlet(10)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    q_all, _, _ = O.count(P, [1.0, 2.0], 5, 15, seed=9)
    q_one, _, _ = O.count(P, [2.0], 2, 15, seed=9, probe_ids=[3, 1])
    np.testing.assert_array_equal(q_one[0], q_all[1, [3, 1]])


def test_plain_fp64_laplace32_statistical():
    # 32x32 Dirichlet Laplacian, [1, 2], Jacobi, 16 probes, 40 steps:
    # exact count 103 (closed form); the 16-probe Hutchinson estimate must be
    # within 4 standard errors of it.
    gold = json.load(open(os.path.join(GOLD, "laplace32_counts.json")))
    i = np.arange(1, 33)
    s = 4 * np.sin(i * np.pi / 66) ** 2
    lam = (s[:, None] + s[None, :]).ravel()
    assert int((lam < 1.0).sum()) == gold["n_below_1"]
    assert int((lam < 2.0 - 1e-12).sum()) == gold["n_below_2_strict"]
    P = O.Problem.csr_matrix(I.laplace2d_dirichlet(32), O.PREC_JACOBI)
    quad, steps, L = O.count(P, [1.0, 2.0], 16, 40, seed=0)
    d = quad[1] - quad[0]
    se = d.std(ddof=1) / np.sqrt(16)
    assert abs(d.mean() - gold["count_1_2_halfopen"]) < 4 * se + 1.0


@pytest.mark.slow
def test_paper_table1_laplace_unpreconditioned():
    # Sec. 7, Table 1: Laplace h = 2^-7, tau = 3000, exact 226; no
    # preconditioner, k = 134, m = 50, estimate within ~5% of the truth.
    g = json.load(open(os.path.join(GOLD, "paper_table1_laplace.json")))
    N = int(round(1 / g["h"])) - 1
    assert N * N == g["n"]
    i = np.arange(1, N + 1)
    s = 4 * np.sin(i * np.pi * g["h"] / 2) ** 2 / g["h"] ** 2
    assert int(((s[:, None] + s[None, :]) < g["tau"]).sum()) == g["exact_negative_inertia"]
    csr = I.laplace2d_dirichlet(N, scale=1.0 / g["h"] ** 2)
    P = O.Problem.csr_matrix(csr, O.PREC_NONE)
    quad, _, L = O.count(P, [g["tau"]], g["m"], g["no_prec_k"], seed=0)
    se = quad[0].std(ddof=1) / np.sqrt(g["m"])
    err = abs(L[0] - g["exact_negative_inertia"])
    assert err < max(4 * se, g["relative_error_reported"] * g["exact_negative_inertia"]) + 4 * se


# --------------------------------------------------- generalized averaged

def test_ga_quadrature_exact_to_degree_2k():
    # Sec. 3.4: the generalized averaged rule from k Lanczos steps is exact for
    # polynomials of degree 2k (Gauss: 2k-1).  The moments of the extended
    # (2k-1)-order tridiagonal match v^T C^j v up to j = 2k.
    A = I.random_symmetric_dense(25, seed=8)
    P = O.Problem.dense_matrix(A, O.PREC_JACOBI)
    tau = -0.1
    v = O.probe_vector(1, 2, 25)
    Cm = _dense_C(P, tau)
    for k in (2, 3, 5):
        al, be, _, _ = O.lanczos(P, tau, v, k + 1)
        al, be = al[:k], be[:k + 1]
        d = np.concatenate([al, al[:-1][::-1]])
        off = np.concatenate([be[1:k], [be[k]], be[1:k - 1][::-1]])
        J = np.diag(d) + np.diag(off, 1) + np.diag(off, -1)
        for j in range(0, 2 * k + 1):
            lhs = 25.0 * np.linalg.matrix_power(J, j)[0, 0]
            rhs = v @ np.linalg.matrix_power(Cm, j) @ v
            assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-9)
        lhs = 25.0 * np.linalg.matrix_power(J, 2 * k + 1)[0, 0]
        rhs = v @ np.linalg.matrix_power(Cm, 2 * k + 1) @ v
        assert abs(lhs - rhs) > 1e-6 * abs(rhs)
        # the oracle's GA quadrature is the step-function rule of exactly this matrix
        w, Z = np.linalg.eigh(J)
        assert O.ga_quad(al, be, 25.0) == pytest.approx(25.0 * np.sum(Z[0, w < 0] ** 2), abs=1e-10)


def test_ga_equals_gauss_after_breakdown_and_at_k1():
    distinct = [-2.0, -0.5, 0.7, 1.5, 3.0]
    A = I.random_symmetric_dense(30, seed=4, distinct=distinct)
    P = O.Problem.dense_matrix(A)
    v = O.probe_vector(9, 1, 30)
    al, be, _, kd = O.lanczos(P, 0.0, v, 12)
    assert kd == 5
    assert O.ga_quad(al, be, 30.0) == pytest.approx(O.gauss_quad(al, be, 30.0), abs=1e-9)
    al1, be1, _, _ = O.lanczos(P, 0.0, v, 1)
    assert O.ga_quad(al1, be1, 30.0) == O.gauss_quad(al1, be1, 30.0)


# ------------------------------------------ T^{-1}-inner-product Lanczos

def test_tinv_lanczos_equals_algorithm1_dense():
    # Eq. lanT1 with y_1 = M q_1 (Sec. 4) reproduces Algorithm 1's tridiagonal
    # for C = M (A - tau I) M, and so its Gauss quadrature
    from oracle.lanczos_tinv import lanczos_tinv
    n, tau, k = 60, 0.3, 14
    A = I.random_symmetric_dense(n, seed=21)
    rng = np.random.default_rng(22)
    Qm, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = (Qm * rng.uniform(0.5, 2.0, n)) @ Qm.T
    M = 0.5 * (M + M.T)
    T = M @ M
    P = O.Problem.dense_matrix(A, O.PREC_DENSE, denseM=M)
    v = O.probe_vector(0, 5, n)
    al, be, _, kd = O.lanczos(P, tau, v, k)
    q1 = v / np.linalg.norm(v)
    a2, b2, k2 = lanczos_tinv(lambda x: A @ x - tau * x, lambda x: T @ x, M @ q1,
                              np.linalg.solve(M, q1), k)
    assert k2 == kd == k
    np.testing.assert_allclose(a2, al, rtol=1e-9, atol=1e-11)
    np.testing.assert_allclose(b2, be, rtol=1e-9, atol=1e-11)
    assert O.gauss_quad(a2, b2, n) == pytest.approx(O.gauss_quad(al, be, n), abs=1e-9)
    # a planted mistake -- z_1 = M q_1 instead of T^{-1} y_1 = M^{-1} q_1 --
    # leaves alpha_1 = y_1^T (A - tau I) y_1 alone but breaks beta_2 and alpha_2
    a3, b3, _ = lanczos_tinv(lambda x: A @ x - tau * x, lambda x: T @ x, M @ q1, M @ q1, 3)
    assert abs(a3[0] - al[0]) < 1e-10
    assert abs(b3[1] - be[1]) > 1e-3 * abs(be[1]) or abs(a3[1] - al[1]) > 1e-3


def test_tinv_lanczos_equals_algorithm1_chebyshev_stencil():
    # the kinetic Chebyshev preconditioner of the stencil oracle, T = p_8(K)^2
    from oracle.lanczos_tinv import lanczos_tinv
    N, h, tau, k = 4, 0.3, -1.0, 10
    V = I.gaussian_wells(N, h, nwells=3, seed=1)
    P = O.Problem.stencil(N, h, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    n = N ** 3
    Mdense = np.stack([O.apply_M(P, tau, e) for e in np.eye(n)], axis=1)
    v = O.probe_vector(1, 3, n)
    al, be, _, kd = O.lanczos(P, tau, v, k)
    q1 = v / np.linalg.norm(v)
    a2, b2, k2 = lanczos_tinv(lambda x: O.apply_A(P, x) - tau * x,
                              lambda x: O.apply_M(P, tau, O.apply_M(P, tau, x)),
                              O.apply_M(P, tau, q1), np.linalg.solve(Mdense, q1), k)
    assert k2 == kd
    np.testing.assert_allclose(a2, al, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(b2, be, rtol=1e-8, atol=1e-9)


def test_tinv_lanczos_equals_algorithm1_jacobi_csr():
    # the diagonal case: Jacobi T = M^2 = diag(1/(|a_rr - tau| + eps)) on a
    # sparse indefinite matrix, z_1 = M^{-1} q_1 by division, T^{-1} never
    # formed; Algorithm 1 runs on the CSR oracle with its own Jacobi M
    from oracle.lanczos_tinv import lanczos_tinv
    n, tau, k, eps = 80, 0.4, 16, 1e-3
    A = I.random_symmetric_dense(n, seed=31)
    A[np.abs(A) < 1.0] = 0.0
    A = 0.5 * (A + A.T) + np.diag(np.linspace(-2, 2, n))
    csr = I.dense_to_csr(A)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI, jac_eps=eps)
    mdiag = O.apply_M(P, tau, np.ones(n))
    # the oracle's M is the Jacobi scaling itself
    np.testing.assert_allclose(mdiag, 1.0 / np.sqrt(np.abs(np.diag(A) - tau) + eps), rtol=1e-14)
    v = O.probe_vector(3, 2, n)
    al, be, _, kd = O.lanczos(P, tau, v, k)
    q1 = v / np.linalg.norm(v)
    a2, b2, k2 = lanczos_tinv(lambda x: A @ x - tau * x, lambda x: mdiag ** 2 * x, mdiag * q1,
                              q1 / mdiag, k)
    assert k2 == kd == k
    np.testing.assert_allclose(a2, al, rtol=1e-9, atol=1e-10)
    np.testing.assert_allclose(b2, be, rtol=1e-9, atol=1e-10)
    assert O.gauss_quad(a2, b2, n) == pytest.approx(O.gauss_quad(al, be, n), abs=1e-9)
