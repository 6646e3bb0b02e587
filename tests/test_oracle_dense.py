"""Pins of the dense FP64 oracle (Sec. 2.2 Eqs. nBEM_disc, matrix, matel, reac_integral, solv).

Nothing here compares the oracle with itself: entries are checked against
adaptive 2-D quadrature of the defining integrals, the operator against
Gauss's law, energies against the Kirkwood and layered-sphere closed forms
and their invariances.
"""
import numpy as np
import pytest
from scipy import integrate

from oracle import formulation as F
from oracle.cdense import DenseOperator
from oracle.cdense import solve as cdense_solve
from oracle.closed_forms import kirkwood_energy, layered_sphere_energy
from oracle.dense import (KJ_PER_MOL, SurfaceData, coulomb_energy, kernel_matrices,
                          operator_matrix, rhs, solve_dense)
from oracle.gmres import gmres
from synth.configs import cavity_sphere_problem, layered_sphere_problem, sphere_problem
from synth.meshes import octasphere


def _panel_integral(x, v, nrm, kappa, double):
    e1, e2 = v[1] - v[0], v[2] - v[0]
    J = np.linalg.norm(np.cross(e1, e2))

    def f(t, s):
        y = v[0] + s * e1 + t * e2
        r = x - y
        rho = np.linalg.norm(r)
        g = np.exp(-kappa * rho) / (4 * np.pi * rho)
        if not double:
            return g * J
        return np.dot(r, nrm) * (1 + kappa * rho) * g / rho ** 2 * J

    val, _ = integrate.dblquad(f, 0.0, 1.0, 0.0, lambda s: 1.0 - s, epsabs=1e-15, epsrel=1e-12)
    return val


@pytest.mark.parametrize("kappa", [0.0, 0.125])
def test_entries_vs_adaptive_quadrature(kappa):
    v, t = octasphere(2, 4.0)
    sd = SurfaceData(v, t, 19, 19)
    V, K = kernel_matrices(sd.cen, sd, kappa, dict(thres=0.0))
    rng = np.random.default_rng(0)
    done = 0
    while done < 12:
        i, j = rng.choice(t.shape[0], 2, replace=False)
        if np.linalg.norm(sd.cen[i] - sd.cen[j]) < 3.0 * sd.L[j]:
            continue            # the 19-point rule is accurate away from the panel
        done += 1
        tri = v[t[j]]
        ev = _panel_integral(sd.cen[i], tri, sd.normal[j], kappa, False)
        ek = _panel_integral(sd.cen[i], tri, sd.normal[j], kappa, True)
        assert abs(V[i, j] - ev) < 2e-5 * abs(ev)
        assert abs(K[i, j] - ek) < 2e-5 * abs(ek) + 1e-12


def test_normals_point_outward():
    v, t = octasphere(2, 4.0)
    sd = SurfaceData(v, t, 3, 19)
    assert np.all((sd.normal * sd.cen).sum(1) > 0)
    assert abs(sd.area.sum() - 4 * np.pi * 16) < 0.1 * 4 * np.pi * 16


@pytest.mark.parametrize("level", [2, 3])
def test_gauss_law(level):
    # (1/2 I + K_L) 1 = 0 on a closed surface: the double-layer potential of unit
    # density is -1/2 on the surface (solid angle), up to quadrature error
    v, t = octasphere(level, 4.0)
    sd = SurfaceData(v, t, 3, 19)
    _, K = kernel_matrices(sd.cen, sd, 0.0, {}, self_rows=np.arange(sd.n))
    resid = 0.5 + K.sum(1)
    assert np.abs(resid).max() < 2e-2 / 4 ** (level - 2)
    # and -1 at an interior point, 0 outside (no singular panel involved)
    _, Ki = kernel_matrices(np.array([[0.5, -0.3, 0.2]]), sd, 0.0, {})
    _, Ko = kernel_matrices(np.array([[9.0, 1.0, -2.0]]), sd, 0.0, {})
    assert abs(Ki.sum() + 1.0) < 1e-3
    assert abs(Ko.sum()) < 1e-3


def test_kirkwood_convergence_and_richardson():
    # BEM error is first order in the panel area (observed order 1.013, Sec. 3.1)
    for charges in ("centre", "both"):
        f = []
        for level in (2, 3, 4):
            pr = sphere_problem(level=level, charges=charges)
            f.append(solve_dense(pr)["dG"])
        ex = kirkwood_energy(4.0, 4.0, 80.0, 0.125, pr["charges"]["xyz"], pr["charges"]["q"])
        p = np.log((f[0] - f[1]) / (f[1] - f[2])) / np.log(4.0)    # Eq. observed_order
        assert 0.9 < p < 1.1
        rich = f[2] + (f[2] - f[1]) / (4.0 ** p - 1.0)              # Eq. rich_extr
        assert abs(rich - ex) < 1e-4 * abs(ex)
        assert abs(f[2] - ex) < 5e-3 * abs(ex)


def test_kirkwood_kappa0_paper_value():
    # the paper's analytic value for the centred charge, kappa = 0 (Sec. 3.1)
    assert abs(kirkwood_energy(4.0, 4.0, 80.0, 0.0, [[0, 0, 0]], [1.0]) - (-41.2465)) < 5e-5


def test_energy_scalings():
    pr = sphere_problem(level=2, charges="both")
    base = solve_dense(pr)["dG"]
    pr2 = sphere_problem(level=2, charges="both")
    pr2["charges"]["q"] = 3.0 * pr2["charges"]["q"]
    assert abs(solve_dense(pr2)["dG"] - 9.0 * base) < 1e-12 * abs(base)
    pr3 = sphere_problem(level=2, charges="both", eps_in=8.0, eps_out=160.0)
    assert solve_dense(pr3)["dG"] == base / 2.0          # power-of-two scaling is exact


def test_superposition():
    pa = sphere_problem(level=2, charges="centre")
    pb = sphere_problem(level=2, charges="off")
    pab = sphere_problem(level=2, charges="both")
    ra, rb, rab = solve_dense(pa), solve_dense(pb), solve_dense(pab)
    assert np.allclose(ra["x"] + rb["x"], rab["x"], rtol=0, atol=1e-13 * np.abs(rab["x"]).max())


def _refinement_study(make, levels=(2, 3, 4)):
    """Energies on three meshes (panel area / 4 per level), the observed order
    (Eq. observed_order) and the Richardson value (Eq. rich_extr)."""
    f = [cdense_solve(make(lv), tol=1e-10)["dG"] for lv in levels]
    p = np.log((f[0] - f[1]) / (f[1] - f[2])) / np.log(4.0)
    return f, p, f[2] + (f[2] - f[1]) / (4.0 ** p - 1.0)


XY2 = [[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]]
# (Stern eps, Stern kappa, solvent kappa): the configuration's Stern layer
# (eps_solvent, kappa 0, Sec. 2.2 "Multi-surface problems"), a high-contrast one
# (eps 20) and a screened one (Yukawa kernels on both sides of the Stern surface)
STERN_CASES = [(80.0, 0.0, 0.125), (20.0, 0.0, 0.125), (80.0, 0.05, 0.25)]
STERN_TOL = 2e-4


@pytest.mark.parametrize("eps_s,kap_s,kap_o", STERN_CASES)
def test_stern_layer_richardson_vs_layered_closed_form(eps_s, kap_s, kap_o):
    # the extrapolated energy must land on the layered-sphere series well inside
    # the gap to what a wrong kernel choice for the Stern blocks would give
    eps, kap = (4.0, eps_s, 80.0), (0.0, kap_s, kap_o)
    ex = layered_sphere_energy([4.0, 6.0], eps, kap, 0, XY2, [1.0, 1.0])
    wrong = [layered_sphere_energy([4.0, 6.0], eps, (0.0, kap_o, kap_o), 0, XY2, [1.0, 1.0]),
             layered_sphere_energy([4.0, 6.0], (4.0, 80.0, 80.0), kap, 0, XY2, [1.0, 1.0]),
             kirkwood_energy(4.0, 4.0, 80.0, kap_o, XY2, [1.0, 1.0])]
    gaps = [abs(w - ex) / abs(ex) for w in wrong if w != ex]
    assert min(gaps) > 5 * STERN_TOL
    f, p, rich = _refinement_study(lambda lv: layered_sphere_problem(level=lv, eps=eps, kappa=kap, charges="both"))
    assert 0.9 < p < 1.1
    assert abs(rich - ex) < STERN_TOL * abs(ex)


def _planted(monkeypatch, kappa_from=None, eps_from=None):
    """Plant a mistake in the oracle's multi-surface rule: the Stern region (1)
    takes the solvent's (2) kappa in its kernels, or its eps in the c factors."""
    if kappa_from is not None:
        orig_blocks = F.blocks

        def blocks(problem):
            return [F.Block(b.s, kappa_from if b.R == 1 else b.R, b.row_side, b.t, b.sigma, b.c)
                    for b in orig_blocks(problem)]
        monkeypatch.setattr(F, "blocks", blocks)
    if eps_from is not None:
        orig_sc = F.sigma_c

        def sigma_c(problem, R, t):
            sg, c = orig_sc(problem, R, t)
            if R == 1 and sg < 0:
                eps = [r["eps"] for r in problem["regions"]]
                c = eps[problem["surfaces"][t]["inner"]] / eps[eps_from]
            return sg, c
        monkeypatch.setattr(F, "sigma_c", sigma_c)


@pytest.mark.parametrize("mistake", ["stern_kappa", "stern_eps"])
def test_stern_pin_catches_a_planted_mistake(monkeypatch, mistake):
    # the same study with the Stern blocks given the solvent's kappa (configuration
    # case) or eps (high-contrast case) misses the closed form by far more than the bound
    eps_s = 80.0 if mistake == "stern_kappa" else 20.0
    eps, kap = (4.0, eps_s, 80.0), (0.0, 0.0, 0.125)
    ex = layered_sphere_energy([4.0, 6.0], eps, kap, 0, XY2, [1.0, 1.0])
    _planted(monkeypatch, kappa_from=2 if mistake == "stern_kappa" else None,
             eps_from=2 if mistake == "stern_eps" else None)
    f, p, rich = _refinement_study(lambda lv: layered_sphere_problem(level=lv, eps=eps, kappa=kap, charges="both"))
    assert abs(rich - ex) > 5 * STERN_TOL * abs(ex)


def test_layered_closed_form_centred_charge():
    # a centred charge sees only the n = 0 term: phi_reac(0) = sum over interfaces
    # of (1/eps_outer - 1/eps_inner)/a, with 1/(eps (1 + kappa a)) for a screened outer region
    for eps_s in (80.0, 20.0):
        ex = layered_sphere_energy([4.0, 6.0], [4.0, eps_s, 80.0], [0.0, 0.0, 0.125], 0, [[0, 0, 0]], [1.0])
        phi = (1 / eps_s - 1 / 4.0) / 4.0 + (1 / (80.0 * (1 + 0.125 * 6.0)) - 1 / eps_s) / 6.0
        assert abs(ex - 0.5 * KJ_PER_MOL * phi) < 1e-12 * abs(ex)
    # a Stern layer with the solvent's eps and kappa reduces to Kirkwood exactly
    for x in ([[0, 0, 0]], XY2):
        q = np.ones(len(x))
        a = layered_sphere_energy([4.0, 6.0], [4, 80, 80], [0, 0.125, 0.125], 0, x, q)
        assert abs(a - kirkwood_energy(4, 4, 80, 0.125, x, q)) < 1e-11 * abs(a)


def test_cavity_richardson_vs_layered_closed_form():
    # cavity r < 1.5 (eps 80) inside the protein shell, Stern layer to 6 A; the
    # charge sits 1 A from the cavity, so three levels reach order ~1.1 and the
    # extrapolation ~2e-4; an absent cavity (eps_cav = eps_protein) is 18% away
    ex = layered_sphere_energy([1.5, 4.0, 6.0], [80, 4, 80, 80], [0, 0, 0, 0.125], 1, [[2.5, 0, 0]], [1.0])
    f, p, rich = _refinement_study(lambda lv: cavity_sphere_problem(level=lv, cavity_coarsening=0))
    assert 0.9 < p < 1.2
    assert abs(rich - ex) < 5e-4 * abs(ex)


def test_invisible_interfaces():
    # a Stern layer with the solvent's eps and kappa, or a cavity with the
    # protein's eps, changes nothing but the discretisation
    pr = layered_sphere_problem(level=3, eps=(4, 80, 80), kappa=(0, 0.125, 0.125), charges="both")
    ex = kirkwood_energy(4, 4, 80, 0.125, pr["charges"]["xyz"], pr["charges"]["q"])
    assert abs(solve_dense(pr)["dG"] - ex) < 2e-2 * abs(ex)
    pc = cavity_sphere_problem(level=3, eps_cav=4.0)
    exc = layered_sphere_energy([4.0, 6.0], [4, 80, 80], [0, 0, 0.125], 0, [[2.5, 0, 0]], [1.0])
    assert abs(solve_dense(pc)["dG"] - exc) < 3e-2 * abs(exc)


def test_single_surface_block_structure():
    # the multi-surface rule reproduces Eq. matrix on one surface
    pr = sphere_problem(level=1)
    A = operator_matrix(pr)
    sd = SurfaceData(pr["surfaces"][0]["verts"], pr["surfaces"][0]["tris"], 3, 19)
    n = sd.n
    VL, KL = kernel_matrices(sd.cen, sd, 0.0, {}, self_rows=np.arange(n))
    VY, KY = kernel_matrices(sd.cen, sd, 0.125, {}, self_rows=np.arange(n))
    I = np.eye(n)
    ref = np.block([[0.5 * I + KL, -VL], [0.5 * I - KY, (4.0 / 80.0) * VY]])
    assert np.array_equal(A, ref)
    b = rhs(pr)
    assert np.all(b[n:] == 0.0)


def test_coulomb_two_charges():
    xyz = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0]])
    assert abs(coulomb_energy(xyz, [1.0, -2.0], 4.0) - KJ_PER_MOL * (-2.0) / (4.0 * 5.0)) < 1e-12


def test_c_oracle_equals_numpy_oracle():
    pr = layered_sphere_problem(level=2, charges="both")
    A = operator_matrix(pr)
    op = DenseOperator(pr)
    x = np.random.default_rng(3).normal(size=A.shape[0])
    assert np.linalg.norm(op(x) - A @ x) < 1e-14 * np.linalg.norm(A @ x)


def test_gmres_matches_lu():
    pr = sphere_problem(level=3, charges="both")
    A = operator_matrix(pr)
    b = rhs(pr)
    x, it, res, _ = gmres(lambda v: A @ v, b, tol=1e-10, restart=20)
    assert res < 1e-10
    xs = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xs) < 1e-8 * np.linalg.norm(xs)


def test_block_jacobi_preconditioned_gmres_same_solution():
    # right preconditioning changes the iteration count, not the solution
    from oracle.formulation import block_jacobi
    from oracle.dense import surfaces_data
    pr = layered_sphere_problem(level=2, charges="both")
    sd = surfaces_data(pr)
    A = operator_matrix(pr, sdata=sd)
    b = rhs(pr, sdata=sd)
    M = block_jacobi(pr, lambda s, k: sd[s].self_V(k, 5))
    x, it, res, _ = gmres(lambda v: A @ v, b, tol=1e-11, restart=30, M_inv=M)
    xs = np.linalg.solve(A, b)
    assert res < 1e-11 and np.linalg.norm(x - xs) < 1e-9 * np.linalg.norm(xs)
    # applying M to the block-diagonal part of A gives the identity on each 2x2 block
    D = np.zeros_like(A)
    for s in range(2):
        for side in (0, 1):
            rs = F.row_slice(pr, s, side)
            for c in F.unknown_slices(pr)[s]:
                D[rs, c] = np.diag(np.diag(A[rs, c]))
    cols = np.random.default_rng(0).choice(A.shape[0], 5, replace=False)
    for j in cols:
        e = np.zeros(A.shape[0]); e[j] = 1.0
        assert np.allclose(M(D @ e), e, atol=1e-12)
