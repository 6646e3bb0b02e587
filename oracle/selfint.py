"""Semi-analytical singular (self-panel) integrals (Sec. 2.3, "Treecode-accelerated BEM").

The paper integrates the singular self-panel terms with the semi-analytical
technique of Zhu, Huang, Song & White (2001), using N_k Gauss points per side
of the triangle (N_k = 5 in Tables 4 and 6).  Reading used here: the panel is
split into three sub-triangles with apex at the collocation point c (the
centroid).  In polar coordinates about c the radial integral is done in closed
form,

    int_0^rho G_L(r) r dr = rho / (4 pi)
    int_0^rho G_Y(r) r dr = (1 - exp(-kappa rho)) / (4 pi kappa),

and the remaining integral over the polar angle is taken edge by edge.  For an
edge at in-plane distance h from c, with u the arclength along the edge from
the foot of the perpendicular dropped from c, d(angle) = h du / (h^2 + u^2)
and the edge lies at rho = sqrt(h^2 + u^2).  Substituting u = h sinh(s)
(rho = h cosh s, d(angle) = ds / cosh s) gives

    I_edge = int_{s1}^{s2} F(h cosh s) / cosh s ds,   s_{1,2} = asinh(u_{1,2} / h),
    F(rho) = rho  or  (1 - exp(-kappa rho)) / kappa,

integrated with N_k-point Gauss-Legendre in s.  The Laplace integrand is the
constant h, so the rule reproduces the closed form h (s2 - s1) exactly; the
Yukawa integrand is smooth and bounded for every triangle shape.  (Gauss
points in u, or in the polar angle itself, lose 10-30% on thin panels.)  The
double-layer self term is zero for a flat panel collocated in its own plane.

Pins (tests/test_oracle_selfint.py): the Laplace edge integral has the closed
form h [asinh(u2/h) - asinh(u1/h)]; both kernels are compared with an
independent Duffy-transformed adaptive 2-D quadrature; the Yukawa value tends
to the Laplace value as kappa -> 0.
"""
from __future__ import annotations

import numpy as np

from .quadrature import gauss_legendre

FOUR_PI = 4.0 * np.pi


def _edges(verts, tris):
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    v0, v1, v2 = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    c = ((v0 + v1) + v2) / 3.0
    return c, [(v0, v1), (v1, v2), (v2, v0)]


def _edge_params(c, va, vb):
    e = vb - va
    ln = np.sqrt((e * e).sum(1))
    eh = e / ln[:, None]
    s0 = ((c - va) * eh).sum(1)
    foot = va + s0[:, None] * eh
    h = np.sqrt(((c - foot) ** 2).sum(1))
    return h, -s0, ln - s0


def self_single_layer(verts, tris, kappa: float, Nk: int = 5):
    """V_ii = int_{panel i} G(c_i, y) dA_y for every panel, by the semi-analytical rule."""
    c, edges = _edges(verts, tris)
    xi, wi = gauss_legendre(Nk)
    total = np.zeros(c.shape[0])
    for va, vb in edges:
        h, u1, u2 = _edge_params(c, va, vb)
        s1 = np.arcsinh(u1 / h)
        s2 = np.arcsinh(u2 / h)
        half = 0.5 * (s2 - s1)
        mid = 0.5 * (s2 + s1)
        for x, w in zip(xi, wi):
            ch = np.cosh(mid + half * x)
            rho = h * ch
            if kappa == 0.0:
                F = rho
            else:
                F = -np.expm1(-kappa * rho) / kappa
            total += w * half * F / ch
    return total / FOUR_PI


def self_single_layer_laplace_exact(verts, tris):
    """Closed form of the same Laplace self integral: sum_edges h [asinh(u2/h) - asinh(u1/h)] / 4pi."""
    c, edges = _edges(verts, tris)
    total = np.zeros(c.shape[0])
    for va, vb in edges:
        h, u1, u2 = _edge_params(c, va, vb)
        total += h * (np.arcsinh(u2 / h) - np.arcsinh(u1 / h))
    return total / FOUR_PI


def _dF_dkappa(rho, kappa):
    """d/dkappa of the Yukawa radial integral (1 - exp(-kappa rho)) / kappa.

    Closed form (kappa rho exp(-kappa rho) + expm1(-kappa rho)) / kappa^2; for
    kappa rho < 0.1 its power series rho^2 sum_{n>=2} (-1)^(n-1) (n-1)/n! (kappa rho)^(n-2),
    which avoids the cancellation; at kappa = 0 it is -rho^2 / 2.
    """
    x = kappa * rho
    series = np.zeros_like(rho)
    fact = 1.0
    for n in range(2, 16):
        fact *= n
        series += (-1.0) ** (n - 1) * (n - 1) / fact * x ** (n - 2)
    series *= rho * rho
    if kappa == 0.0:
        return series
    closed = (x * np.exp(-x) + np.expm1(-x)) / (kappa * kappa)
    return np.where(x < 0.1, series, closed)


def self_single_layer_dkappa(verts, tris, kappa: float, Nk: int = 5):
    """d V_ii / d kappa of the Yukawa self integral by the same semi-analytical rule.

    The radial integral of dG_Y/dkappa = -exp(-kappa r) / (4 pi) is the kappa
    derivative of (1 - exp(-kappa rho)) / kappa; the angular integral uses the
    same N_k-point rule in s = asinh(u / h) as self_single_layer.
    """
    c, edges = _edges(verts, tris)
    xi, wi = gauss_legendre(Nk)
    total = np.zeros(c.shape[0])
    for va, vb in edges:
        h, u1, u2 = _edge_params(c, va, vb)
        s1 = np.arcsinh(u1 / h)
        s2 = np.arcsinh(u2 / h)
        half = 0.5 * (s2 - s1)
        mid = 0.5 * (s2 + s1)
        for x, w in zip(xi, wi):
            ch = np.cosh(mid + half * x)
            total += w * half * _dF_dkappa(h * ch, kappa) / ch
    return total / FOUR_PI
