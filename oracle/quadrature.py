"""Quadrature rules on triangles and on intervals (Sec. 2.2, 2.3 "Treecode-accelerated BEM").

The paper integrates every panel with Gauss points: K points per panel in the
regular case (K = 1 in Table 1, K = 3 in Table 3) and K_fine points in the
near-singular region (K_fine = 19 in Tables 4 and 6).  The semi-analytical
singular rule uses N_k Gauss points along each triangle side (N_k = 5).

Rules are stored as barycentric coordinates (l0, l1, l2) with weights summing
to 1, so that the integral over a panel of area A is A * sum_k w_k f(y_k) with
y_k = l0 v0 + l1 v1 + l2 v2.

Pins (tests/test_oracle_quadrature.py): polynomial exactness of each rule on
all monomials up to its stated degree.
"""
from __future__ import annotations

import itertools

import numpy as np


def _orbit(bary):
    return sorted(set(itertools.permutations(bary)))


# Published symmetric rules (D. A. Dunavant, "High degree efficient symmetrical
# Gaussian quadrature rules for the triangle", 1985): (weight, orbit generator).
_DUNAVANT = {
    1: [(1.0, (1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0))],
    3: [(1.0 / 3.0, (2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0))],
    7: [(0.225, (1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)),
        (0.132394152788506, (0.059715871789770, 0.470142064105115, 0.470142064105115)),
        (0.125939180544827, (0.797426985353087, 0.101286507323456, 0.101286507323456))],
    19: [(0.097135796282799, (1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)),
         (0.031334700227139, (0.020634961602525, 0.489682519198738, 0.489682519198738)),
         (0.077827541004774, (0.125820817014127, 0.437089591492937, 0.437089591492937)),
         (0.079647738927210, (0.623592928761935, 0.188203535619033, 0.188203535619033)),
         (0.025577675658698, (0.910540973211095, 0.044729513394453, 0.044729513394453)),
         (0.043283539377289, (0.036838412054736, 0.221962989160766, 0.741198598784498))],
}
DEGREE = {1: 1, 3: 2, 7: 5, 19: 9}


def triangle_rule(K: int):
    """Barycentric nodes [K,3] and weights [K] (sum 1) of the K-point rule."""
    if K not in _DUNAVANT:
        raise ValueError(f"no {K}-point triangle rule")
    nodes, weights = [], []
    for w, gen in _DUNAVANT[K]:
        # K = 3 keeps the node order (2/3,1/6,1/6), (1/6,2/3,1/6), (1/6,1/6,2/3)
        orb = _orbit(gen) if K != 3 else [gen, gen[1:2] + gen[0:1] + gen[2:], gen[1:] + gen[:1]]
        for b in orb:
            nodes.append(b)
            weights.append(w)
    nodes = np.array(nodes, dtype=np.float64)
    weights = np.array(weights, dtype=np.float64)
    assert nodes.shape[0] == K
    return nodes, weights


def gauss_legendre(n: int):
    """n-point Gauss-Legendre nodes and weights on [-1, 1]."""
    return np.polynomial.legendre.leggauss(n)
