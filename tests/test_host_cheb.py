"""Host side of the kinetic Chebyshev preconditioner M = p_d(K) (no GPU).

evc_cheb_kinetic returns what evc_set_precond builds: the interval [a, b],
the coefficients of p_d (the interpolant of x^(-1/2) at Chebyshev points of
the first kind), the minimum of p_d over the spectrum of K on an N^3 grid, and
the factored form the stencil passes apply.  They are checked against the
oracle's own construction, against numpy's Chebyshev-series roots and
evaluation, and against the spectrum of K computed from dense circulant
matrices (not from the stencil symbol the library uses)."""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npc

from oracle import oracle as O
from paper_1602_02306_gb300 import evc

DEGREES = [1, 2, 3, 5, 8, 12, 16]


@pytest.fixture(scope="module")
def lib():
    from paper_1602_02306_gb300 import build
    build.build()
    return evc.load()


def _product(r, x):
    p = np.full_like(x, r["sign"])
    g = r["g"]
    for re, im, pair in r["factors"]:
        p = p * (g * g * ((x - re) ** 2 + im * im) if pair else g * (x - re))
    return p


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("degree", DEGREES)
def test_interval_and_coefficients_match_the_oracle(lib, order, degree):
    h, c = 0.3, 1.0
    r = evc.evc_cheb_kinetic(order, h, degree, c)
    P = O.Problem.stencil(4, h, order, np.zeros(64), O.PREC_CHEB, cheb_degree=degree, cheb_c=c)
    a, b = O.kinetic_interval(P)
    assert r["a"] == pytest.approx(a, rel=1e-15) and r["b"] == pytest.approx(b, rel=1e-15)
    ref = O.cheb_coeffs(degree, a, b)
    np.testing.assert_allclose(r["coef"], ref, rtol=0, atol=1e-13 * np.max(np.abs(ref)))


@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("degree", DEGREES)
def test_factored_form_reproduces_the_series(lib, order, degree):
    r = evc.evc_cheb_kinetic(order, 0.3, degree, 1.0)
    a, b = r["a"], r["b"]
    assert r["factors"], "the factorisation is expected to pass its check here"
    pairs = [f for f in r["factors"] if f[2]]
    reals = [f for f in r["factors"] if not f[2]]
    assert 2 * len(pairs) + len(reals) == degree
    assert r["factors"] == pairs + reals                        # pairs first
    assert [f[0] for f in pairs] == sorted(f[0] for f in pairs)
    assert [f[0] for f in reals] == sorted(f[0] for f in reals)
    assert all(f[1] > 0 for f in pairs) and all(f[1] == 0 for f in reals)
    x = np.linspace(a, b, 2001)
    ref = npc.chebval((2 * x - a - b) / (b - a), r["coef"])
    assert np.max(np.abs(_product(r, x) - ref) / np.abs(ref)) < 1e-9
    # the roots themselves, against numpy's (companion-matrix) roots of the series
    t = npc.chebroots(r["coef"])
    want = np.sort_complex(0.5 * (b - a) * t + 0.5 * (a + b))
    ours = [complex(re, s * im) for re, im, pair in pairs for s in (1, -1)] + \
           [complex(re, 0.0) for re, _, _ in reals]
    got = np.sort_complex(np.array(ours))
    np.testing.assert_allclose(got, want, rtol=1e-7, atol=1e-7 * (b - a))


def _circulant_spectrum(N, h, order):
    """Eigenvalues of -1/2 d^2/dx^2 on a periodic line of N points (dense)."""
    w = {2: [(0, -2.0), (1, 1.0)], 4: [(0, -2.5), (1, 4.0 / 3.0), (2, -1.0 / 12.0)]}[order]
    D = np.zeros((N, N))
    for i in range(N):
        for off, val in w:
            D[i, (i + off) % N] += val
            if off:
                D[i, (i - off) % N] += val
    return np.linalg.eigvalsh(-0.5 * D / (h * h))


@pytest.mark.parametrize("order,N,degree", [(2, 8, 8), (4, 10, 8), (2, 12, 3), (4, 6, 12)])
def test_positivity_on_the_exact_spectrum(lib, order, N, degree):
    h, c = 0.3, 1.0
    r = evc.evc_cheb_kinetic(order, h, degree, c, N=N)
    lam = _circulant_spectrum(N, h, order)
    spec = c + lam[:, None, None] + lam[None, :, None] + lam[None, None, :]
    assert spec.min() >= r["a"] - 1e-9 and spec.max() <= r["b"] + 1e-9   # [a, b] bounds spec(K)
    a, b = r["a"], r["b"]
    pmin = np.min(npc.chebval((2 * spec - a - b) / (b - a), r["coef"]))
    assert r["pmin"] == pytest.approx(pmin, rel=1e-10)
    assert r["pmin"] > 0
    assert evc.evc_cheb_kinetic(order, h, degree, c)["pmin"] == 0.0    # N = 0: not evaluated


@pytest.mark.parametrize("args", [(3, 0.3, 8, 1.0), (2, 0.0, 8, 1.0), (2, 0.3, 0, 1.0),
                                  (2, 0.3, 33, 1.0), (4, 0.3, 8, 0.0), (2, -1.0, 8, 1.0)])
def test_invalid_arguments(lib, args):
    with pytest.raises(evc.EvcError):
        evc.evc_cheb_kinetic(*args)
    with pytest.raises(evc.EvcError):
        evc.evc_cheb_kinetic(2, 0.3, 8, 1.0, N=-1)
