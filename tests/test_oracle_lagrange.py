"""Pins of the oracle's centered Lagrange fractional-delay read (Sec. "Implementation").

Independent of the oracle's product formula: exact rational moment equations, scipy's
barycentric interpolator, polynomial reproduction, the delta property at integer shifts.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy.interpolate import BarycentricInterpolator

import oracle

ORDERS = [1, 3, 5, 7, 11, 25, 41]


def exact_weights(p: int, eps: Fraction):
    """Weights w_j solving the moment equations sum_j w_j j^k = eps^k (k = 0..p) exactly,
    i.e. the unique rule that reproduces every polynomial of degree <= p."""
    h = (p - 1) // 2
    nodes = [Fraction(j - h) for j in range(p + 1)]
    n = p + 1
    A = [[nodes[j] ** k for j in range(n)] + [eps ** k] for k in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if A[r][c] != 0)
        A[c], A[piv] = A[piv], A[c]
        for r in range(n):
            if r != c and A[r][c] != 0:
                f = A[r][c] / A[c][c]
                A[r] = [a - f * b for a, b in zip(A[r], A[c])]
    return [A[j][n] / A[j][j] for j in range(n)]


@pytest.mark.parametrize("p", [1, 3, 5, 25])
@pytest.mark.parametrize("eps", [Fraction(1, 3), Fraction(2, 7), Fraction(999, 1000)])
def test_weights_match_exact_rational(p, eps):
    w = oracle.lagrange_weights(p, float(eps))
    ex = np.array([float(x) for x in exact_weights(p, eps)])
    assert np.max(np.abs(w - ex)) <= 1e-14 * max(1.0, np.max(np.abs(ex)))


@pytest.mark.parametrize("p", ORDERS)
def test_integer_shift_is_exact_delta(p):
    w = oracle.lagrange_weights(p, 0.0)
    h = (p - 1) // 2
    expect = np.zeros(p + 1)
    expect[h] = 1.0
    assert np.array_equal(w, expect)
    s = np.random.default_rng(1).normal(size=200)
    for base in [50, 51, 120]:
        assert oracle.lagrange_read(s, base, 0.0, p) == s[base]
        assert oracle.lagrange_read(s, base, 3.0, p) == s[base + 3]
        assert oracle.lagrange_read(s, base, -7.0, p) == s[base - 7]


@pytest.mark.parametrize("p", ORDERS)
def test_partition_of_unity(p):
    for eps in np.random.default_rng(p).uniform(0, 1, 20):
        assert abs(oracle.lagrange_weights(p, eps).sum() - 1.0) < 1e-13


@pytest.mark.parametrize("p", [1, 3, 5, 11, 25])
def test_reproduces_polynomials_up_to_degree_p(p):
    rng = np.random.default_rng(100 + p)
    coef = rng.normal(size=p + 1)
    centre, scale = 100.0, 20.0
    poly = lambda x: np.polyval(coef, (x - centre) / scale)
    s = poly(np.arange(200.0))
    for u in rng.uniform(-5, 5, 30):
        got = oracle.lagrange_read(s, 100, u, p)
        assert abs(got - poly(100 + u)) <= 1e-11 * (1 + abs(poly(100 + u)))
    # one degree more is NOT reproduced (for p < 25 the error is visible)
    if p <= 11:
        c2 = np.concatenate([[1.0], np.zeros(p + 1)])
        q = lambda x: np.polyval(c2, (x - centre) / 2.0)
        sq = q(np.arange(200.0))
        assert abs(oracle.lagrange_read(sq, 100, 0.5, p) - q(100.5)) > 1e-6


@pytest.mark.parametrize("p", [3, 7, 25])
def test_matches_scipy_barycentric(p):
    rng = np.random.default_rng(7 + p)
    s = rng.normal(size=300)
    h = (p - 1) // 2
    for u in rng.uniform(-3, 3, 15):
        m = 150 + int(np.floor(u))
        nodes = np.arange(m - h, m + h + 2, dtype=float)
        ref = BarycentricInterpolator(nodes, s[m - h:m + h + 2])(150 + u)
        assert abs(oracle.lagrange_read(s, 150, u, p) - ref) < 1e-11 * np.abs(s).max()


def test_zero_extension_outside_series():
    s = np.ones(10)
    # the stencil of p = 3 around x = 0.5 touches index -1, which is treated as 0
    w = oracle.lagrange_weights(3, 0.5)
    assert abs(oracle.lagrange_read(s, 0, 0.5, 3) - w[1:].sum()) < 1e-15
    assert oracle.lagrange_read(s, 100, 0.25, 3) == 0.0


def test_convergence_to_sinusoid_with_order():
    omega = 0.6
    j = np.arange(400.0)
    s = np.cos(omega * j)
    errs = []
    for p in [1, 3, 5, 7, 9, 11]:
        e = max(abs(oracle.lagrange_read(s, 200, u, p) - np.cos(omega * (200 + u))) for u in [0.1, 0.37, 0.5, 0.81])
        errs.append(e)
    assert all(b < a for a, b in zip(errs, errs[1:]))
    assert errs[-1] < 1e-6


@pytest.mark.parametrize("p", [1, 3, 11, 25])
def test_derivative_weights_reproduce_polynomial_derivatives(p):
    rng = np.random.default_rng(300 + p)
    for eps in rng.uniform(0, 1, 5):
        dw = oracle.lagrange_dweights(p, eps)
        h = (p - 1) // 2
        j = np.arange(p + 1) - h
        for k in range(min(p, 6) + 1):
            expect = 0.0 if k == 0 else k * eps ** (k - 1)
            assert abs(np.sum(dw * j.astype(float) ** k) - expect) < 1e-9 * (1 + abs(expect)) * (h + 1) ** k
        # central difference of the weights
        d = 1e-6
        fd = (oracle.lagrange_weights(p, eps + d) - oracle.lagrange_weights(p, eps - d)) / (2 * d)
        assert np.max(np.abs(fd - dw)) < 1e-6 * max(1, np.abs(dw).max())
