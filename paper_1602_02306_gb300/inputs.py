"""Seeded synthetic problem generators (host, numpy).

This module builds the *inputs* of an eigenvalue-count problem and nothing
else: sparse matrices in CSR form and the local potential of a finite-
difference Hamiltonian. It holds none of the estimator's arithmetic (no
operator application, no preconditioner, no Lanczos, no quadrature), so both
the CUDA path and the FP64 oracle can consume what it returns.

Workload families (the paper's own matrices are not available, these stand in
for them):

* ``laplace2d_dirichlet`` -- the 5-point Dirichlet Laplacian on an N x N
  interior grid, the paper's "Laplace" test problem (Sec. 7, Table 1) when
  scaled by 1/h^2, and the small plain-FP64 case (diag 4, off-diagonal -1).
* ``gaussian_wells`` -- the potential V of a real-space DFT-like Hamiltonian
  H = -1/2 Lap_h + V on a periodic N^3 grid: a sum of Gaussian wells with
  seeded depths and centres. It stands in for the paper's PARSEC / KSSOLV
  Hamiltonians (Sec. 7, Table 1 "Benzene", "H2").
* ``powerlaw_symmetric`` -- a generic sparse symmetric indefinite matrix with
  power-law row lengths, values N(0,1), diagonal U(-5,5).
* ``random_symmetric_dense`` -- tiny dense symmetric matrices for pins.

Grid points of an N^3 stencil problem are numbered p = x + N*(y + N*z).
"""
from __future__ import annotations

import numpy as np


def laplace2d_dirichlet(N: int, scale: float = 1.0):
    """5-point Dirichlet Laplacian on the N x N interior grid, CSR.

    Diagonal 4*scale, nearest-neighbour off-diagonals -scale. Row r = x + N*y.
    Returns (row_ptr int64[n+1], col int32[nnz], val float64[nnz]) with the
    columns of each row sorted.
    """
    n = N * N
    rows, cols, vals = [], [], []
    idx = np.arange(n, dtype=np.int64)
    x = idx % N
    y = idx // N
    entries = [(0, 0, 4.0), (-1, 0, -1.0), (1, 0, -1.0), (0, -1, -1.0), (0, 1, -1.0)]
    for dx, dy, v in entries:
        xx, yy = x + dx, y + dy
        ok = (xx >= 0) & (xx < N) & (yy >= 0) & (yy < N)
        rows.append(idx[ok])
        cols.append((xx + N * yy)[ok])
        vals.append(np.full(int(ok.sum()), v * scale))
    return coo_to_csr(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def coo_to_csr(n: int, r, c, v, sum_duplicates: bool = True):
    """Sort COO triplets by (row, col), optionally summing duplicates, into CSR."""
    r = np.asarray(r, dtype=np.int64)
    c = np.asarray(c, dtype=np.int64)
    v = np.asarray(v, dtype=np.float64)
    key = r * np.int64(n) + c
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    if sum_duplicates and key.size:
        uniq, start = np.unique(key, return_index=True)
        v = np.add.reduceat(v, start)
        key = uniq
    r = key // n
    c = key % n
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(r, minlength=n), out=row_ptr[1:])
    return row_ptr, c.astype(np.int32), v


def gaussian_wells(N: int, h: float, nwells: int = 32, depth=(2.0, 6.0),
                   width: float = 1.0, seed: int = 1) -> np.ndarray:
    """Local potential V of an N^3 periodic grid with spacing h, float64[N^3].

    V(r) = -sum_w d_w exp(-|r - c_w|^2 / (2 width^2)), with the minimum-image
    distance in the periodic box [0, N h)^3, depths d_w ~ U(depth) and centres
    uniform in the box, all drawn from numpy's PCG64 stream seeded by `seed`.
    """
    rng = np.random.default_rng(seed)
    L = N * h
    d = rng.uniform(depth[0], depth[1], size=nwells)
    cen = rng.uniform(0.0, L, size=(nwells, 3))
    g = np.arange(N, dtype=np.float64) * h
    V = np.zeros((N, N, N), dtype=np.float64)   # indexed [z, y, x]
    for w in range(nwells):
        def mi(axis_c):
            t = g - axis_c
            t -= L * np.round(t / L)
            return t * t
        dx2, dy2, dz2 = mi(cen[w, 0]), mi(cen[w, 1]), mi(cen[w, 2])
        r2 = dz2[:, None, None] + dy2[None, :, None] + dx2[None, None, :]
        V -= d[w] * np.exp(-r2 / (2.0 * width * width))
    return V.reshape(-1)


def powerlaw_symmetric(n: int, mean_row: float = 30.0, cap: int = 1000,
                       diag_range=(-5.0, 5.0), seed: int = 2, alpha: float = 2.2):
    """Sparse symmetric indefinite A = B + B^T with power-law row lengths, CSR.

    Out-degrees of B follow a discrete Pareto law with exponent `alpha`, capped
    at `cap`, rescaled so that the mean stored row length of A is about
    `mean_row`; columns are uniform, values N(0,1), duplicates are summed and
    the diagonal is replaced by U(diag_range).
    """
    rng = np.random.default_rng(seed)
    raw = (rng.pareto(alpha - 1.0, size=n) + 1.0)
    raw = np.minimum(raw, cap)
    # Each off-diagonal entry of B appears twice in A (b_ij and b_ji).
    target = max(mean_row - 1.0, 0.0) / 2.0
    deg = np.minimum(np.maximum(np.round(raw * (target / raw.mean())), 0), cap).astype(np.int64)
    nnz_b = int(deg.sum())
    r = np.repeat(np.arange(n, dtype=np.int64), deg)
    c = rng.integers(0, n, size=nnz_b, dtype=np.int64)
    v = rng.standard_normal(nnz_b)
    keep = r != c
    r, c, v = r[keep], c[keep], v[keep]
    d = rng.uniform(diag_range[0], diag_range[1], size=n)
    rr = np.concatenate([r, c, np.arange(n, dtype=np.int64)])
    cc = np.concatenate([c, r, np.arange(n, dtype=np.int64)])
    vv = np.concatenate([v, v, d])
    return coo_to_csr(n, rr, cc, vv)


def random_symmetric_dense(n: int, seed: int, distinct=None) -> np.ndarray:
    """Tiny dense symmetric matrix, float64[n, n].

    With `distinct` (a sequence of eigenvalues), the matrix is Q diag(lam) Q^T
    with Q a seeded random orthogonal matrix and lam cycling through
    `distinct`, so it has exactly len(distinct) distinct eigenvalues.
    """
    rng = np.random.default_rng(seed)
    if distinct is None:
        G = rng.standard_normal((n, n))
        return 0.5 * (G + G.T)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.array([distinct[i % len(distinct)] for i in range(n)], dtype=np.float64)
    A = (Q * lam) @ Q.T
    return 0.5 * (A + A.T)


def dense_to_csr(A: np.ndarray):
    """Dense float64 matrix to CSR (explicit zeros dropped)."""
    n = A.shape[0]
    r, c = np.nonzero(A)
    return coo_to_csr(n, r, c, A[r, c])
