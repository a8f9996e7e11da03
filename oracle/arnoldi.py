"""FP64 oracle of the preconditioned Arnoldi-type estimator (Sec. 4).

TEST INFRASTRUCTURE ONLY, like the rest of this package.  Plain numpy, the
paper's steps in the paper's order:

* Algorithm 3 (the Arnoldi procedure for T(A - tau I)): q_1 = v/||v||; for
  j = 1..k, w = T (A - tau I) q_j, modified Gram-Schmidt against q_1..q_j
  (h_ij = q_i^T w, w -= h_ij q_i), h_{j+1,j} = ||w||, q_{j+1} = w / h_{j+1,j}.
  T is applied unfactored as T = M M, where M is the factor the Lanczos
  oracle uses (Jacobi: T = diag(1/(|a_ii - tau| + eps)); Chebyshev: T = p_d(K)^2).
* The Arnoldi quadrature (Eq. arnoldi_quad): eigen-decomposition H_k = Z Theta Z^{-1};
  ||v||^2 Re( sum over eigenvalues with negative real part of z_i(1) s_i ),
  s = the first column of S = Z^{-1} (the paper's text says the first column;
  its algorithm listing writes S(1,:) -- the product e_1^T Z h(Theta) Z^{-1} e_1
  needs the column).
* The estimator A_tau(k, m) (Eq. rand_prec_quad_arn): the mean over m probes,
  with the same counter-hashed Rademacher probes and the same stop rule as the
  Lanczos oracle.

Parity unpinned parts: none -- the pins are in tests/test_oracle_arnoldi_pins.py
(Arnoldi = Lanczos for T = I and symmetric A; exact count from exhaustive
Sylvester-Hadamard probes at k = n; exactness at p distinct eigenvalues).
"""
from __future__ import annotations

import numpy as np

from . import oracle as O


def apply_T(P: O.Problem, tau, x):
    """T x with T = M M (Sec. 4: T used without its factorisation)."""
    return O.apply_M(P, tau, O.apply_M(P, tau, x))


def apply_TA(P: O.Problem, tau, x):
    """T (A - tau I) x."""
    return apply_T(P, tau, O.apply_A(P, x) - tau * x)


def arnoldi(P: O.Problem, tau, v, k, breakdown_rel=O.BREAKDOWN_REL):
    """Algorithm 3.  Returns (H[k_done+1, k_done], k_done): the extended upper
    Hessenberg matrix.  A breakdown h_{j+1,j} <= breakdown_rel * max|H| stops
    the process at k_done = j (the Krylov space is invariant)."""
    n = v.size
    Q = np.zeros((k + 1, n))
    H = np.zeros((k + 1, k))
    Q[0] = v / np.linalg.norm(v)
    scale = 0.0
    for j in range(k):
        w = apply_TA(P, tau, Q[j])
        for i in range(j + 1):
            H[i, j] = Q[i] @ w
            w = w - H[i, j] * Q[i]
        H[j + 1, j] = np.linalg.norm(w)
        scale = max(scale, float(np.max(np.abs(H[: j + 1, j]))))
        if H[j + 1, j] <= breakdown_rel * max(scale, H[j + 1, j]) or j + 1 == n:
            return H[: j + 2, : j + 1], j + 1
        Q[j + 1] = w / H[j + 1, j]
    return H, k


def arnoldi_quad(Hk, vnorm2):
    """Eq. arnoldi_quad: ||v||^2 Re(e_1^T Z h(Theta) Z^{-1} e_1), h = 1 on the
    open left half-plane."""
    theta, Z = np.linalg.eig(Hk)
    S = np.linalg.inv(Z)
    neg = theta.real < 0
    return float(vnorm2 * np.real(np.sum(Z[0, neg] * S[neg, 0])))


def count(P: O.Problem, shifts, m, kmax, tol=0.0, seed=0, probe_ids=None,
          breakdown_rel=O.BREAKDOWN_REL, min_steps=3):
    """The Arnoldi-type estimator for every shift: (quad[S, m], steps[S], L[S]).

    Stop rule as in the Lanczos oracle: with tol > 0, a shift stops at the
    first step i >= max(3, min_steps) where L changed by at most tol over each
    of the last two steps; after a breakdown H stays H_{k_done}."""
    shifts = np.asarray(shifts, dtype=np.float64)
    S = shifts.size
    kmax = min(kmax, P.n)
    hist = np.zeros((S, m, kmax))
    for s in range(S):
        for j in range(m):
            pid = int(probe_ids[j]) if probe_ids is not None else j
            v = O.probe_vector(seed, pid, P.n)
            vn2 = float(v @ v)
            H, kd = arnoldi(P, shifts[s], v, kmax, breakdown_rel)
            for i in range(1, kmax + 1):
                if tol <= 0.0 and i < kmax:
                    continue
                ki = min(i, kd)
                hist[s, j, i - 1] = arnoldi_quad(H[:ki, :ki], vn2)
    quad = np.zeros((S, m))
    steps = np.zeros(S, dtype=np.int32)
    L = np.zeros(S)
    for s in range(S):
        ks = kmax
        if tol > 0.0:
            prev = prev2 = 0.0
            for i in range(1, kmax + 1):
                Li = float(np.mean(hist[s, :, i - 1]))
                if i >= 3 and i >= min_steps and abs(Li - prev) <= tol and abs(prev - prev2) <= tol:
                    ks = i
                    break
                prev2, prev = prev, Li
        quad[s] = hist[s, :, ks - 1]
        steps[s] = ks
        L[s] = float(np.mean(quad[s]))
    return quad, steps, L
