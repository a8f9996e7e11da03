"""The seeded input generators both sides use (no GPU): each against a
brute-force restatement of the recipe it documents."""
import numpy as np
import pytest

from paper_1602_02306_gb300 import inputs as I


def test_gaussian_wells_brute_force_minimum_image():
    N, h, nw, width = 5, 0.7, 3, 1.0
    V = I.gaussian_wells(N, h, nwells=nw, seed=4, width=width)
    rng = np.random.default_rng(4)                       # the documented draw order
    d = rng.uniform(2.0, 6.0, size=nw)
    cen = rng.uniform(0.0, N * h, size=(nw, 3))
    L = N * h
    for z in range(N):
        for y in range(N):
            for x in range(N):
                p = np.array([x, y, z]) * h
                v = 0.0
                for w in range(nw):
                    r2 = 0.0
                    for a in range(3):
                        t = p[a] - cen[w, a]
                        t = min((t - k * L for k in (-1, 0, 1)), key=abs)   # nearest image
                        r2 += t * t
                    v -= d[w] * np.exp(-r2 / (2 * width * width))
                assert V[(z * N + y) * N + x] == pytest.approx(v, abs=1e-13)
    assert np.all(V < 0) and V.min() >= -d.sum()


def test_gaussian_wells_seeded():
    a = I.gaussian_wells(8, 0.3, nwells=4, seed=1)
    b = I.gaussian_wells(8, 0.3, nwells=4, seed=1)
    c = I.gaussian_wells(8, 0.3, nwells=4, seed=2)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_powerlaw_symmetric_structure():
    n = 20000
    rp, col, val = I.powerlaw_symmetric(n, cap=300, seed=2)
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 1)
    rows = np.repeat(np.arange(n), np.diff(rp))
    # sorted, unique columns per row (duplicates summed)
    key = rows * n + col
    assert np.all(np.diff(key) > 0)
    # symmetric in pattern and value
    A = {(int(r), int(c)): v for r, c, v in zip(rows, col, val)}
    for (r, c), v in list(A.items())[:: max(1, len(A) // 20000)]:
        assert A[(c, r)] == v
    diag = np.array([A[(i, i)] for i in range(n)])
    assert diag.min() >= -5.0 and diag.max() <= 5.0
    lens = np.diff(rp)
    assert abs(lens.mean() - 30.0) < 3.0            # the documented mean row length
    assert lens.max() <= 2 * 300 + 1                 # cap per half, plus the diagonal
    assert lens.max() > 5 * lens.mean()              # heavy tail


def test_coo_to_csr_sums_duplicates():
    rp, col, val = I.coo_to_csr(3, np.array([2, 0, 2, 0, 1]), np.array([1, 2, 1, 0, 1]),
                                np.array([1.0, 2.0, 3.0, 4.0, 5.0]))
    assert list(rp) == [0, 2, 3, 4]
    assert list(col) == [0, 2, 1, 1] and list(val) == [4.0, 2.0, 5.0, 4.0]


def test_random_symmetric_dense_has_exactly_the_distinct_eigenvalues():
    distinct = [-2.0, 0.5, 3.0]
    A = I.random_symmetric_dense(12, seed=5, distinct=distinct)
    w = np.linalg.eigvalsh(A)
    for lam in distinct:
        assert np.sum(np.abs(w - lam) < 1e-10) == 4
    assert np.allclose(A, A.T)


def test_laplace_family_exact_counts():
    # the closed-form count against a dense eigendecomposition of the assembled
    # matrix on the small meshes, and against Table 1's printed 226 at h = 2^-7
    import json
    import os
    from paper_1602_02306_gb300 import workloads as W
    for e in (3, 4, 5):
        h = 2.0 ** -e
        rp, col, val = I.laplace2d_dirichlet(2 ** e - 1, scale=1.0 / h ** 2)
        n = len(rp) - 1
        A = np.zeros((n, n))
        for r in range(n):
            A[r, col[rp[r]:rp[r + 1]]] = val[rp[r]:rp[r + 1]]
        lam = np.linalg.eigvalsh(A)
        for tau in (100.0, 0.37 * lam.max(), 3000.0):
            assert W.laplace_exact_below(e, tau) == int((lam < tau).sum())
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_table1_laplace.json")))
    assert W.laplace_exact_below(7, g["tau"]) == g["exact_negative_inertia"]
    assert [W.laplace_exact_below(e) for e in range(6, 11)] == [230, 226, 222, 220, 220]
