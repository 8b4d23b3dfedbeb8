"""Pins of the oracle's quadrature rules (Section II.A: m-point rule on each
triangle; n-point rule on each source edge) against closed-form moments."""
import math

import numpy as np
import pytest

import oracle as O

DEGREE = {1: 1, 3: 2, 4: 3, 6: 4, 7: 5}


def exact_monomial(i, j):
    # mean of x^i y^j over the triangle (0,0),(1,0),(0,1): 2 i! j! / (i+j+2)!
    return 2.0 * math.factorial(i) * math.factorial(j) / math.factorial(i + j + 2)


@pytest.mark.parametrize("npts", sorted(DEGREE))
def test_rule_exact_to_its_degree(npts):
    b, w = O.rule(npts)
    assert b.shape == (npts, 3)
    np.testing.assert_allclose(b.sum(axis=1), 1.0, atol=1e-15)
    assert (b > 0).all()
    x, y = b[:, 1], b[:, 2]
    deg = DEGREE[npts]
    for i in range(deg + 1):
        for j in range(deg + 1 - i):
            got = float(np.sum(w * x**i * y**j))
            assert abs(got - exact_monomial(i, j)) < 1e-14, (npts, i, j)
    # and not exact one degree higher (the rule has the degree it claims)
    errs = [abs(float(np.sum(w * x**i * y**(deg + 1 - i))) - exact_monomial(i, deg + 1 - i))
            for i in range(deg + 2)]
    assert max(errs) > 1e-6


def test_six_point_rule_matches_published_decimals():
    # Dunavant's degree-4 6-point rule as published (16-digit decimals); the
    # oracle derives it from the moment equations instead.
    b, w = O.rule(6)
    a = sorted(set(np.round(np.median(b, axis=1), 12)))  # the repeated coordinate
    assert abs(a[0] - 0.091576213509771) < 1e-12
    assert abs(a[1] - 0.445948490915965) < 1e-12
    ws = sorted(set(np.round(w, 12)))
    assert abs(ws[0] - 0.109951743655322) < 1e-12
    assert abs(ws[1] - 0.223381589678011) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3, 8, 16, 32])
def test_gauss_legendre_exact(n):
    x, w = O.gauss_legendre(n)
    for p in range(2 * n):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.sum(w * x**p) - exact) < 1e-13
