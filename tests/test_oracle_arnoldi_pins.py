"""Pins of the Arnoldi-type oracle (Sec. 4) to facts outside itself.

* T = I and symmetric A: the Arnoldi process is the Lanczos process, so the
  Arnoldi quadrature equals the Gauss quadrature of the (independent, C)
  Lanczos oracle and H_k is tridiagonal.
* k = n: the quadrature is v^T h(T(A - tau I)) v, computed here from a dense
  eigen-decomposition of the n x n non-symmetric matrix; over the full
  Sylvester-Hadamard probe set (H H^T = n I) the mean is trace h(T(A - tau I)),
  the negative inertia of A - tau I (T(A - tau I) is similar to M(A - tau I)M).
  A non-scalar T makes H_k non-symmetric, so a row of Z^{-1} used in place of
  its first column fails these.
* p distinct eigenvalues of T(A - tau I): the process stops at k = p and the
  quadrature is exact (the Arnoldi analogue of Proposition 1).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import arnoldi as AR
from oracle import oracle as O
from paper_1602_02306_gb300 import inputs as I


def _dense_op(P, tau):
    n = P.n
    return np.column_stack([AR.apply_TA(P, tau, e) for e in np.eye(n)])


def _h_dense(Cm, v):
    w, Z = np.linalg.eig(Cm)
    hw = (w.real < 0).astype(float)
    return float(np.real(v @ (Z @ np.diag(hw) @ np.linalg.inv(Z)) @ v))


def test_identity_T_reduces_to_lanczos():
    A = I.random_symmetric_dense(40, seed=11)
    P = O.Problem.dense_matrix(A)
    for tau, k in ((0.3, 8), (-0.6, 14)):
        v = O.probe_vector(5, 2, 40)
        H, kd = AR.arnoldi(P, tau, v, k)
        assert kd == k
        Hk = H[:k, :k]
        assert np.max(np.abs(np.triu(Hk, 2))) < 1e-10
        al, be, _, kl = O.lanczos(P, tau, v, k)
        np.testing.assert_allclose(np.diag(Hk), al, rtol=0, atol=1e-10)
        np.testing.assert_allclose(np.diag(H, -1)[:k], be[1:k + 1], rtol=0, atol=1e-10)
        assert AR.arnoldi_quad(Hk, v @ v) == pytest.approx(O.gauss_quad(al, be, v @ v), abs=1e-9)


@pytest.mark.parametrize("prec", [O.PREC_JACOBI, O.PREC_NONE])
def test_full_krylov_space_quadrature_is_the_quadratic_form(prec):
    A = I.random_symmetric_dense(16, seed=21) + np.diag(np.linspace(-2, 3, 16))
    A = 0.5 * (A + A.T)
    P = O.Problem.dense_matrix(A, prec)
    tau = 0.35
    Cm = _dense_op(P, tau)
    v = O.probe_vector(1, 4, 16)
    H, kd = AR.arnoldi(P, tau, v, 16)
    assert AR.arnoldi_quad(H[:kd, :kd], v @ v) == pytest.approx(_h_dense(Cm, v), abs=1e-8)


@pytest.mark.parametrize("prec", [O.PREC_JACOBI, O.PREC_NONE])
def test_exhaustive_hadamard_equals_inertia(prec):
    A = I.random_symmetric_dense(16, seed=23) + np.diag(np.linspace(-3, 2, 16))
    A = 0.5 * (A + A.T)
    lam = np.linalg.eigvalsh(A)
    P = O.Problem.dense_matrix(A, prec)
    Hm = sla.hadamard(16).astype(np.float64)
    for tau in (-0.7, 0.9):
        tot = 0.0
        for v in Hm:
            H, kd = AR.arnoldi(P, tau, v, 16)
            tot += AR.arnoldi_quad(H[:kd, :kd], v @ v)
        assert tot / 16 == pytest.approx(float((lam < tau).sum()), abs=1e-7)


def test_exhaustive_stencil_chebyshev_T():
    # 4^3 periodic Hamiltonian with T = p_8(K)^2
    N, h = 4, 0.3
    V = I.gaussian_wells(N, h, nwells=2, seed=1)
    P = O.Problem.stencil(N, h, 2, V, O.PREC_CHEB, cheb_degree=8, cheb_c=1.0)
    Hd = np.column_stack([O.apply_A(P, e) for e in np.eye(64)])
    lam = np.linalg.eigvalsh(0.5 * (Hd + Hd.T))
    tau = float(0.5 * (lam[20] + lam[21]))
    Hm = sla.hadamard(64).astype(np.float64)
    tot = 0.0
    for v in Hm:
        H, kd = AR.arnoldi(P, tau, v, 64)
        tot += AR.arnoldi_quad(H[:kd, :kd], v @ v)
    assert tot / 64 == pytest.approx(21.0, abs=1e-6)


def test_exact_at_p_distinct_eigenvalues():
    distinct = [-2.0, -0.5, 0.7, 1.5, 3.0]
    A = I.random_symmetric_dense(30, seed=4, distinct=distinct)
    P = O.Problem.dense_matrix(A)
    v = O.probe_vector(9, 1, 30)
    w, U = np.linalg.eigh(A)
    exact = float(np.sum((U[:, w < 0].T @ v) ** 2))
    H, kd = AR.arnoldi(P, 0.0, v, 12)
    assert kd == len(distinct)
    assert AR.arnoldi_quad(H[:kd, :kd], v @ v) == pytest.approx(exact, abs=1e-9)
    H3, _ = AR.arnoldi(P, 0.0, v, 3)
    assert abs(AR.arnoldi_quad(H3[:3, :3], v @ v) - exact) > 1e-6


def test_count_means_and_stop_rule():
    csr = I.laplace2d_dirichlet(8)
    P = O.Problem.csr_matrix(csr, O.PREC_JACOBI)
    shifts = [1.0, 2.3]
    quad, steps, L = AR.count(P, shifts, 5, 16, tol=0.3, seed=4)
    np.testing.assert_allclose(L, quad.mean(axis=1), rtol=1e-15)
    for s, tau in enumerate(shifts):
        assert 3 <= steps[s] <= 16
        q1, _, _ = AR.count(P, [tau], 5, int(steps[s]), seed=4)
        np.testing.assert_allclose(q1[0], quad[s], rtol=0, atol=1e-12)
