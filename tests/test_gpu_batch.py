"""Batched solves (lock-step GMRES on pool streams) and the binding energy (Eq. bind_energy).

A batched problem runs exactly the kernels of a single solve on another
stream, and every reduction has a fixed order, so its energy equals the
single solve's bit for bit.  The binding energy of a small synthetic complex
is checked against the dense oracle (LU) and the Coulomb energies.
"""
import numpy as np
import pytest

from gpu_util import ctx, problem
from oracle import dense as OD
from synth.configs import binding_triplet, layered_sphere_problem, ligand_fleet, sphere_problem

pytestmark = pytest.mark.gpu

DIRECT = dict(theta=-1.0, precision="fp64", ncrit=64, gmres_tol=1e-10)
MIXED = dict(precision="mixed", gmres_tol=1e-5)


def _batch(dicts, params):
    from paper_1309_4018_b300 import pbbem
    single = []
    for d in dicts:
        single.append(problem(d, **params).solve())
    probs = [problem(d, **params) for d in dicts]
    return single, pbbem.solve_batch(ctx(), probs)


def test_batch_equals_single_direct():
    dicts = [sphere_problem(level=3, charges="both"), sphere_problem(level=4, charges="off"),
             layered_sphere_problem(level=2)]
    single, batch = _batch(dicts, DIRECT)
    for a, b in zip(single, batch):
        assert b.converged and a.iterations == b.iterations
        assert a.dG_solv == b.dG_solv


def test_batch_equals_single_treecode_fleet():
    dicts = ligand_fleet(count=6, n_min=150, n_max=600, spacing=1.4)
    single, batch = _batch(dicts, MIXED)
    for a, b in zip(single, batch):
        assert b.converged and a.iterations == b.iterations
        assert a.dG_solv == b.dG_solv


def test_binding_energy_vs_oracle():
    from paper_1309_4018_b300 import pbbem
    cx, rec, lig = binding_triplet(n_rec=80, n_lig=30, spacing=2.0)
    probs = [problem(d, **DIRECT) for d in (cx, rec, lig)]
    ddG = pbbem.binding_energy(ctx(), *probs)
    E = []
    for d in (cx, rec, lig):
        ref = OD.solve_dense(d)
        E.append(ref["dG"] + OD.coulomb_energy(d["charges"]["xyz"], d["charges"]["q"], d["regions"][0]["eps"]))
    ref_ddG = E[0] - E[1] - E[2]
    assert abs(ddG - ref_ddG) <= 1e-8 * max(abs(e) for e in E)
    # the batch solved every member: each problem's own energy is available and matches
    assert abs(probs[1].solve().dG_solv - (E[1] - OD.coulomb_energy(rec["charges"]["xyz"], rec["charges"]["q"], 4.0))) \
        <= 1e-8 * abs(E[1])


def test_batch_rejects_foreign_and_repeated_problems():
    from paper_1309_4018_b300 import pbbem
    d = sphere_problem(level=2)
    p = problem(d, **DIRECT)
    with pytest.raises(pbbem.PBError):
        pbbem.solve_batch(ctx(), [p, p])
    other = pbbem.Context(0)
    q = pbbem.Problem.from_dict(other, d)
    q.setup(**DIRECT)
    with pytest.raises(pbbem.PBError):
        pbbem.solve_batch(ctx(), [p, q])
