"""Pins of the adjoint gradient oracle (oracle/gradient.py).

The gradient is checked against central finite differences of the energy
(dense LU solves), against the exact identities q . dE/dq = 2E and
sum_R eps_R dE/deps_R = -E, and against derivatives of the Kirkwood closed
form; the self-integral kappa derivative against adaptive quadrature of its
defining integral.
"""
import copy

import numpy as np
import pytest
from scipy import integrate

from oracle.closed_forms import kirkwood_energy
from oracle.gradient import energy_only, solvation_gradient
from oracle.selfint import self_single_layer, self_single_layer_dkappa
from synth.configs import cavity_sphere_problem, layered_sphere_problem, sphere_problem

P = dict(K=3, K_fine=19, N_k=5, thres=2.0)


def _problems():
    sph = sphere_problem(level=2, charges="both")
    sph["charges"]["q"] = np.array([0.7, -0.4])
    lay = layered_sphere_problem(level=2)
    lay["charges"]["q"] = np.array([1.0, 0.5])
    cav = cavity_sphere_problem(level=2)
    return {"sphere": sph, "layered": lay, "cavity": cav}


PROBLEMS = _problems()


def _fd(problem, mutate, h):
    a = copy.deepcopy(problem)
    b = copy.deepcopy(problem)
    mutate(a, h)
    mutate(b, -h)
    return (energy_only(a, P) - energy_only(b, P)) / (2 * h)


@pytest.fixture(scope="module")
def grads():
    return {k: solvation_gradient(v, P) for k, v in PROBLEMS.items()}


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_identities(name, grads):
    g = grads[name]
    pr = PROBLEMS[name]
    q = np.asarray(pr["charges"]["q"])
    assert abs(q @ g["dq"] - 2 * g["E"]) < 1e-11 * abs(g["E"])
    eps = np.array([r["eps"] for r in pr["regions"]])
    assert abs(eps @ g["deps"] + g["E"]) < 1e-10 * abs(g["E"])
    assert abs(g["E"] - energy_only(pr, P)) < 1e-12 * abs(g["E"])


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_charge_gradients_vs_fd(name, grads):
    g = grads[name]
    pr = PROBLEMS[name]
    nc = len(pr["charges"]["q"])
    for k in range(nc):
        def mq(p, h, k=k):
            p["charges"]["q"] = np.array(p["charges"]["q"], dtype=float)
            p["charges"]["q"][k] += h
        fd = _fd(pr, mq, 1e-3)
        assert abs(fd - g["dq"][k]) < 1e-9 * max(1.0, abs(fd)), (k, fd, g["dq"][k])
        for d in range(3):
            def mr(p, h, k=k, d=d):
                p["charges"]["xyz"] = np.array(p["charges"]["xyz"], dtype=float)
                p["charges"]["xyz"][k, d] += h
            fd = _fd(pr, mr, 1e-5)
            scale = np.abs(g["dxyz"]).max()
            assert abs(fd - g["dxyz"][k, d]) < 1e-6 * scale, (k, d, fd, g["dxyz"][k, d])


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_region_gradients_vs_fd(name, grads):
    g = grads[name]
    pr = PROBLEMS[name]
    for r in range(len(pr["regions"])):
        def me(p, h, r=r):
            p["regions"][r]["eps"] += h * p["regions"][r]["eps"]
        fd = _fd(pr, me, 1e-5) / pr["regions"][r]["eps"]
        assert abs(fd - g["deps"][r]) < 1e-6 * max(abs(g["E"]) / pr["regions"][r]["eps"], abs(fd)), (r, fd, g["deps"][r])

        def mk(p, h, r=r):
            p["regions"][r]["kappa"] += h
        fd = _fd(pr, mk, 1e-5)
        assert abs(fd - g["dkappa"][r]) < 1e-6 * max(1.0, abs(fd)), (r, fd, g["dkappa"][r])


def test_adjoint_solves_transposed_system(grads):
    g = grads["layered"]
    A, Rm = g["A"], g["Rm"]
    q = np.asarray(PROBLEMS["layered"]["charges"]["q"])
    C0 = 0.5 * 1389.3545764 * 4 * np.pi
    assert np.linalg.norm(A.T @ g["lam"] - C0 * Rm.T @ q) < 1e-12 * np.linalg.norm(C0 * Rm.T @ q)
    # E = lambda . b
    assert abs(g["lam"] @ (g["B"] @ q) - g["E"]) < 1e-11 * abs(g["E"])


def test_kirkwood_derivatives():
    """BEM gradient at 2,048 panels against derivatives of the Kirkwood series (discretisation error)."""
    pr = sphere_problem(level=4, charges="off")
    g = solvation_gradient(pr, P)
    a, e1, e2, k = 4.0, 4.0, 80.0, 0.125
    xyz = np.array([[2.0, 0.0, 0.0]])
    q = np.ones(1)
    E0 = kirkwood_energy(a, e1, e2, k, xyz, q)
    h = 1e-5
    dk = (kirkwood_energy(a, e1, e2, k + h, xyz, q) - kirkwood_energy(a, e1, e2, k - h, xyz, q)) / (2 * h)
    dx = (kirkwood_energy(a, e1, e2, k, xyz + [[h, 0, 0]], q)
          - kirkwood_energy(a, e1, e2, k, xyz - [[h, 0, 0]], q)) / (2 * h)
    de1 = (kirkwood_energy(a, e1 + h, e2, k, xyz, q) - kirkwood_energy(a, e1 - h, e2, k, xyz, q)) / (2 * h)
    de2 = (kirkwood_energy(a, e1, e2 + h, k, xyz, q) - kirkwood_energy(a, e1, e2 - h, k, xyz, q)) / (2 * h)
    assert abs(g["E"] - E0) < 5e-3 * abs(E0)
    assert abs(g["dkappa"][1] - dk) < 2e-2 * abs(dk)
    assert abs(g["dxyz"][0, 0] - dx) < 2e-2 * abs(dx)
    assert abs(g["dxyz"][0, 1]) < 1e-3 * abs(dx) and abs(g["dxyz"][0, 2]) < 1e-3 * abs(dx)
    assert abs(g["deps"][0] - de1) < 1e-2 * abs(de1)
    assert abs(g["deps"][1] - de2) < 2e-2 * abs(de2)
    assert abs(g["dq"][0] - 2 * E0) < 5e-3 * abs(2 * E0)


def _duffy_dkappa(tri, kappa):
    """Adaptive integral of dG_Y/dkappa = -exp(-kappa r)/(4 pi) over the triangle (Duffy map at the centroid)."""
    c = tri.mean(0)
    tot = 0.0
    for a, b in ((tri[0], tri[1]), (tri[1], tri[2]), (tri[2], tri[0])):
        J = np.linalg.norm(np.cross(a - c, b - a))

        def f(s, t):
            w = (a - c) + t * (b - a)
            return -np.exp(-kappa * s * np.linalg.norm(w)) * s * J / (4 * np.pi)

        val, _ = integrate.dblquad(f, 0.0, 1.0, 0.0, 1.0, epsabs=1e-15, epsrel=1e-13)
        tot += val
    return tot


@pytest.mark.parametrize("kappa", [0.0, 1e-3, 0.125, 2.0])
def test_self_integral_dkappa(kappa):
    rng = np.random.default_rng(11)
    tris = [np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], float),
            np.array([[0, 0, 0], [3, 0, 0], [0.2, 0.15, 0]], float),
            rng.normal(size=(3, 3))]
    t = np.array([[0, 1, 2]])
    for tri in tris:
        exact = _duffy_dkappa(tri, kappa)
        fine = self_single_layer_dkappa(tri, t, kappa, Nk=40)[0]
        assert abs(fine - exact) < 1e-10 * abs(exact)
        # N_k = 5 (the paper's rule) on the 3 A sliver is the worst case
        tol = 5e-3 if kappa == 2.0 else 1e-3
        assert abs(self_single_layer_dkappa(tri, t, kappa, Nk=5)[0] - exact) < tol * abs(exact)
        if kappa >= 1e-3:
            # the derivative of the N_k = 5 rule itself (what the discrete operator uses)
            h = 1e-6
            fd = (self_single_layer(tri, t, kappa + h, 5)[0] - self_single_layer(tri, t, kappa - h, 5)[0]) / (2 * h)
            assert abs(fd - self_single_layer_dkappa(tri, t, kappa, 5)[0]) < 1e-7 * abs(fd)
