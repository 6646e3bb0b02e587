"""Pins of the oracle's quadrature rules: exactness on polynomials (Sec. 2.2/2.3 Gauss points)."""
from math import factorial

import numpy as np
import pytest

from oracle.quadrature import DEGREE, gauss_legendre, triangle_rule


def _exact_monomial(a, b):
    # mean of x^a y^b over the reference triangle (0,0),(1,0),(0,1)
    return 2.0 * factorial(a) * factorial(b) / factorial(a + b + 2)


@pytest.mark.parametrize("K", [1, 3, 7, 19])
def test_triangle_rule_exact_to_degree(K):
    lam, w = triangle_rule(K)
    assert lam.shape == (K, 3)
    assert abs(w.sum() - 1.0) < 1e-14
    assert np.allclose(lam.sum(1), 1.0, atol=1e-15)
    x, y = lam[:, 1], lam[:, 2]
    deg = DEGREE[K]
    for a in range(deg + 1):
        for b in range(deg + 1 - a):
            ex = _exact_monomial(a, b)
            assert abs((w * x ** a * y ** b).sum() - ex) <= 2e-14 * max(1.0, ex), (K, a, b)
    # and not exact one degree higher (the stated degree is sharp)
    errs = [abs((w * x ** a * y ** (deg + 1 - a)).sum() - _exact_monomial(a, deg + 1 - a))
            for a in range(deg + 2)]
    assert max(errs) > 1e-10


def test_triangle_rule_symmetric():
    for K in (3, 7, 19):
        lam, w = triangle_rule(K)
        for perm in ([1, 2, 0], [0, 2, 1]):
            p = lam[:, perm]
            for row, wt in zip(p, w):
                d = np.abs(lam - row).sum(1)
                j = np.argmin(d)
                assert d[j] < 1e-14 and abs(w[j] - wt) < 1e-15


@pytest.mark.parametrize("n", [1, 3, 5, 8])
def test_gauss_legendre_exact(n):
    x, w = gauss_legendre(n)
    for d in range(2 * n):
        ex = 0.0 if d % 2 else 2.0 / (d + 1)
        assert abs((w * x ** d).sum() - ex) < 1e-14
