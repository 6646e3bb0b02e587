"""Pins of the semi-analytical self integrals (Sec. 2.3, Zhu et al. technique, N_k = 5)."""
import numpy as np
import pytest
from scipy import integrate

from oracle.selfint import self_single_layer, self_single_layer_laplace_exact
from synth.molecule import gaussian_surface, synthetic_atoms


def _tri_set():
    rng = np.random.default_rng(7)
    tris = [np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float),
            np.array([[0, 0, 0], [3, 0, 0], [0.2, 0.15, 0]], float),   # sliver
            np.array([[1, 2, 3], [1.5, 2.1, 2.7], [0.8, 2.6, 3.3]], float)]
    for _ in range(3):
        tris.append(rng.normal(size=(3, 3)))
    return tris


def _duffy(tri, kappa):
    """Adaptive 2-D integral of G over the triangle with the singular point at the centroid.

    Each sub-triangle (c, a, b) is mapped by y = c + s((a - c) + t(b - a)),
    whose Jacobian s |(a - c) x (b - a)| cancels the 1/r singularity.
    """
    c = tri.mean(0)
    tot = 0.0
    for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
        J = np.linalg.norm(np.cross(a - c, b - a))

        def f(s, t):
            w = (a - c) + t * (b - a)
            r = s * np.linalg.norm(w)
            return np.exp(-kappa * r) * J / (4 * np.pi * np.linalg.norm(w))

        val, _ = integrate.dblquad(f, 0.0, 1.0, 0.0, 1.0, epsabs=1e-14, epsrel=1e-13)
        tot += val
    return tot


@pytest.mark.parametrize("kappa", [0.0, 0.125, 2.0])
def test_self_integral_vs_duffy(kappa):
    for tri in _tri_set():
        v = tri
        t = np.array([[0, 1, 2]])
        exact = _duffy(tri, kappa)
        approx = self_single_layer(v, t, kappa, Nk=5)[0]
        fine = self_single_layer(v, t, kappa, Nk=40)[0]
        assert abs(fine - exact) < 1e-10 * abs(exact)
        # N_k = 5 (Tables 4 and 6): Laplace is exact; the Yukawa error grows with
        # kappa * panel size (worst case here: the 3 A sliver)
        tol = {0.0: 1e-13, 0.125: 5e-6, 2.0: 1e-3}[kappa]
        assert abs(approx - exact) < tol * abs(exact)


def test_laplace_closed_form():
    for tri in _tri_set():
        t = np.array([[0, 1, 2]])
        ex = self_single_layer_laplace_exact(tri, t)[0]
        assert abs(ex - _duffy(tri, 0.0)) < 1e-11 * abs(ex)
        for Nk in (1, 2, 5):
            assert abs(self_single_layer(tri, t, 0.0, Nk)[0] - ex) < 1e-14 * abs(ex)


def test_yukawa_tends_to_laplace():
    tri = _tri_set()[2]
    t = np.array([[0, 1, 2]])
    lap = self_single_layer(tri, t, 0.0, 5)[0]
    for k in (1e-3, 1e-6):
        assert abs(self_single_layer(tri, t, k, 5)[0] - lap) < 2 * k * abs(lap)


def test_equilateral_closed_form_value():
    # equilateral triangle side s: V = (3 / (4 pi)) h asinh(sqrt(3)) * 2 with h = s / (2 sqrt 3)
    s = 1.3
    tri = np.array([[0, 0, 0], [s, 0, 0], [s / 2, s * np.sqrt(3) / 2, 0]])
    h = s / (2 * np.sqrt(3))
    val = 3 * h * 2 * np.arcsinh(np.sqrt(3)) / (4 * np.pi)
    assert abs(self_single_layer_laplace_exact(tri, np.array([[0, 1, 2]]))[0] - val) < 1e-15 * 10
