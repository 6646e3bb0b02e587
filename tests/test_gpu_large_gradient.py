"""Adjoint gradients against central finite differences of the GPU energy.

Small case (FP64 direct summation, 512-panel sphere, h = 1e-4, GMRES tol
1e-12): the adjoint gradient and the finite differences agree to 1e-5
relative (direct summation has no acceptance test a step could flip).

Large case: a 30,000-atom globule meshed on the device (~480k panels),
FP32-mixed treecode, GMRES tol 1e-7; 16 charges, 16 position coordinates,
eps_in, eps_out and kappa.  The mixed operator's energy carries noise of
about tol |E| (4.6e-3 kJ/mol here), so a central difference with step h is
good to about tol |E| / h: h = 0.05 keeps that floor near 0.1 kJ/mol per e
(per A) while the truncation error of the step stays below 1e-3 relative.
Bound: |FD - adjoint| <= 2e-2 |adjoint| + 2 tol |E| / h (the mixed
adjoint is itself good to about 1e-3).
"""
import numpy as np
import pytest

from gpu_util import ctx
from synth.configs import large_protein_problem, sphere_problem

pytestmark = pytest.mark.gpu


def test_small_fp64_gradient_matches_finite_differences():
    from paper_1309_4018_b300 import pbbem
    d = sphere_problem(level=3, charges="both")
    d["charges"]["q"] = np.array([0.7, -0.4])
    P = dict(precision="fp64", theta=-1.0, ncrit=64, gmres_tol=1e-12)
    pb = pbbem.Problem.from_dict(ctx(), d)
    pb.setup(**P)
    pb.solve()
    g = pb.gradient()
    xyz, q = d["charges"]["xyz"].copy(), d["charges"]["q"].copy()
    h = 1e-4

    def energy(xx, qq):
        pb.set_charges(xx, qq, 0)
        pb.setup(**P)
        return pb.solve().dG_solv

    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd = (energy(xyz, q + e) - energy(xyz, q - e)) / (2 * h)
        assert abs(fd - g["dq"][k]) <= 1e-5 * abs(g["dq"][k])
        for a in range(3):
            xp, xm = xyz.copy(), xyz.copy()
            xp[k, a] += h
            xm[k, a] -= h
            fd = (energy(xp, q) - energy(xm, q)) / (2 * h)
            assert abs(fd - g["dxyz"][k, a]) <= 1e-5 * np.abs(g["dxyz"]).max()
    pb.close()


def test_large_mixed_gradient_matches_finite_differences():
    from paper_1309_4018_b300 import pbbem
    tol, h = 1e-7, 0.05
    P = dict(precision="mixed", theta=0.5, P=6, ncrit=300, gmres_tol=tol)
    d = large_protein_problem()
    pb = pbbem.Problem.from_dict(ctx(), d)
    assert pb.surface_info(0)["nt"] > 400_000
    pb.setup(**P)
    r = pb.solve()
    x0 = pb.solution()
    g = pb.gradient()
    E0 = r.dG_solv
    floor = 2 * tol * abs(E0) / h
    xyz, q = d["charges"]["xyz"].copy(), d["charges"]["q"].copy()

    def energy(xx, qq):
        pb.set_charges(xx, qq, 0)
        pb.setup(**P)
        return pb.solve(x0).dG_solv

    rng = np.random.default_rng(0)
    for k in rng.choice(q.size, 16, replace=False):
        qp, qm = q.copy(), q.copy()
        qp[k] += h
        qm[k] -= h
        fd = (energy(xyz, qp) - energy(xyz, qm)) / (2 * h)
        assert abs(fd - g["dq"][k]) <= 2e-2 * abs(g["dq"][k]) + floor, (k, fd, g["dq"][k])
    for _ in range(16):
        k, a = int(rng.integers(q.size)), int(rng.integers(3))
        xp, xm = xyz.copy(), xyz.copy()
        xp[k, a] += h
        xm[k, a] -= h
        fd = (energy(xp, q) - energy(xm, q)) / (2 * h)
        assert abs(fd - g["dxyz"][k, a]) <= 2e-2 * abs(g["dxyz"][k, a]) + floor, (k, a, fd, g["dxyz"][k, a])
    pb.close()
    # region parameters: eps_in, eps_out, kappa (the device mesh is rebuilt identically each time)
    for reg, key, grad in ((0, "eps", g["deps"][0]), (1, "eps", g["deps"][1]), (1, "kappa", g["dkappa"][1])):
        e = []
        for s in (1, -1):
            dd = dict(d, regions=[dict(x) for x in d["regions"]])
            dd["regions"][reg][key] += s * h * (0.1 if key == "kappa" else 1.0)
            p = pbbem.Problem.from_dict(ctx(), dd)
            p.setup(**P)
            e.append(p.solve(x0).dG_solv)
            p.close()
        step = h * (0.1 if key == "kappa" else 1.0)
        fd = (e[0] - e[1]) / (2 * step)
        assert abs(fd - grad) <= 2e-2 * abs(grad) + 2 * tol * abs(E0) / step, (reg, key, fd, grad)
