"""FP64 oracle of the T^{-1}-inner-product Lanczos process (Sec. 4, Eq. lanT1).

TEST INFRASTRUCTURE ONLY, like the rest of this package.  Plain numpy.

The process works with the unfactored preconditioned operator T (A - tau I)
and is orthogonal in the inner product <x, y> = x^T T^{-1} y:

    T (A - tau I) Y_k = Y_{k+1} J_{k+1,k},   Y_{k+1}^T T^{-1} Y_{k+1} = I,

started from y_1 = M q_1 (T = M M with M symmetric, q_1 = v/||v||), so that
Y_k = M Q_k and J is the tridiagonal of Algorithm 1 on C = M (A - tau I) M.
The T^{-1} inner products need T^{-1} Y, which the process carries along as
Z = T^{-1} Y without ever applying T^{-1}: with u = (A - tau I) y_i,

    w = T u - beta_i y_{i-1},           T^{-1} w = u - beta_i z_{i-1},
    alpha_i = y_i^T (T^{-1} w),
    w -= alpha_i y_i, T^{-1} w -= alpha_i z_i  (the same coefficients),
    one classical Gram-Schmidt pass in the T^{-1} inner product against
    y_1..y_i: c = Z_i^T w, w -= Y_i c, T^{-1} w -= Z_i c,
    beta_{i+1} = sqrt(w^T T^{-1} w),  y_{i+1} = w/beta_{i+1},
    z_{i+1} = T^{-1} w / beta_{i+1}.

Only the start needs the factor: y_1 = M q_1 and z_1 = T^{-1} y_1 = M^{-1} q_1.
The quadrature is Eq. gauss_quad of the resulting J_k.

Pins: tests/test_oracle_pins.py (the tridiagonal equals Algorithm 1's for
the same T; the Gauss quadrature then equals the oracle's per-probe value).
"""
from __future__ import annotations

import numpy as np


def lanczos_tinv(apply_shifted_A, apply_T, y1, z1, k, breakdown_rel=1e-12):
    """Eq. lanT1: returns (alpha[k_done], beta[k_done + 1], k_done).

    apply_shifted_A(x) = (A - tau I) x, apply_T(x) = T x; y1 = M q_1 and
    z1 = T^{-1} y1 = M^{-1} q_1 for a unit q_1.  A breakdown beta_{i+1} <=
    breakdown_rel * max(|alpha|, beta) stops the process at k_done = i."""
    n = y1.size
    Y = np.zeros((k + 1, n))
    Z = np.zeros((k + 1, n))
    Y[0], Z[0] = y1, z1
    alpha = np.zeros(k)
    beta = np.zeros(k + 1)
    scale = 0.0
    for i in range(k):
        u = apply_shifted_A(Y[i])
        w = apply_T(u)
        t = u.copy()                                   # T^{-1} w
        if i > 0:
            w -= beta[i] * Y[i - 1]
            t -= beta[i] * Z[i - 1]
        alpha[i] = Y[i] @ t
        w -= alpha[i] * Y[i]
        t -= alpha[i] * Z[i]
        c = Z[: i + 1] @ w                             # <y_j, w> in the T^{-1} product
        w -= c @ Y[: i + 1]
        t -= c @ Z[: i + 1]
        b = float(np.sqrt(max(w @ t, 0.0)))
        beta[i + 1] = b
        scale = max(scale, abs(alpha[i]), beta[i])
        if b <= breakdown_rel * max(scale, b) or i + 1 == n:
            return alpha[: i + 1], beta[: i + 2], i + 1
        Y[i + 1] = w / b
        Z[i + 1] = t / b
    return alpha, beta, k
