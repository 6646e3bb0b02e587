"""Batched solves and the binding energy (Eq. bind_energy).

A batch of single-surface FP32-mixed molecules runs its operator
applications as one persistent launch per GMRES step over a queue of
(problem, phase, tile) entries; other batches run every problem's GMRES
cycle as a device-driven graph on a pool stream.  Both compute exactly the
arithmetic of a single solve, and every reduction has a fixed order, so the
energies equal the single solves' bit for bit.  The binding energy of a small
synthetic complex is checked against the dense oracle (LU) and the Coulomb
energies.  The persistent launch's bounded wait is made to run out (a count
that nothing reaches, PB_FAULT=wait, in a child process): the batch returns
PB_ETIMEOUT and the context stays usable.
"""
import contextlib
import json
import os
import subprocess
import sys

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


@contextlib.contextmanager
def persistent(on):
    from paper_1309_4018_b300 import pbbem
    ctx().set_option(pbbem.PB_OPT_BATCH_PERSISTENT, on)
    try:
        yield
    finally:
        ctx().set_option(pbbem.PB_OPT_BATCH_PERSISTENT, 0)


@pytest.mark.parametrize("on", [1, 0])
def test_batch_equals_single_treecode_fleet(on):
    with persistent(on):
        dicts = ligand_fleet(count=6, n_min=150, n_max=600, spacing=1.4)
        single, batch = _batch(dicts, MIXED)
    for a, b in zip(single, batch):
        assert b.converged and a.iterations == b.iterations
        assert a.dG_solv == b.dG_solv


def test_batch_persistent_mixed_triplet_and_theta_variants():
    # the binding triplet's three molecules, FP32-mixed, at two treecode settings;
    # equal to single solves whether or not a member reaches the tolerance
    from paper_1309_4018_b300 import pbbem
    cx, rec, lig = binding_triplet(n_rec=400, n_lig=120, spacing=1.4)
    for kw in (dict(theta=0.5, P=6, ncrit=100), dict(theta=0.6, P=4, ncrit=60)):
        params = dict(precision="mixed", gmres_tol=1e-4, max_iter=200, **kw)
        single = [problem(d, **params).solve(check=False) for d in (cx, rec, lig)]
        with persistent(1):
            batch = pbbem.solve_batch(ctx(), [problem(d, **params) for d in (cx, rec, lig)], check=False)
        for a, b in zip(single, batch):
            assert a.converged == b.converged and a.iterations == b.iterations and a.dG_solv == b.dG_solv
        assert all(np.isfinite(b.dG_solv) and b.dG_solv < 0 for b in batch)


def test_batch_option_rejects_bad_values():
    from paper_1309_4018_b300 import pbbem
    with pytest.raises(pbbem.PBError):
        ctx().set_option(pbbem.PB_OPT_BATCH_PERSISTENT, 2)
    with pytest.raises(pbbem.PBError):
        ctx().set_option(99, 1)


_TIMEOUT = r"""
import json, sys
sys.path.insert(0, {root!r})
from paper_1309_4018_b300 import pbbem
from synth.configs import ligand_fleet
ctx = pbbem.Context(0)
ctx.set_option(pbbem.PB_OPT_BATCH_PERSISTENT, 1)
dicts = ligand_fleet(count=3, n_min=150, n_max=400, spacing=1.6)
def probs():
    out = []
    for d in dicts:
        p = pbbem.Problem.from_dict(ctx, d)
        p.setup(precision="mixed", gmres_tol=1e-5)
        out.append(p)
    return out
out = {{}}
try:
    pbbem.solve_batch(ctx, probs())
    out["batch"] = "ok"
except pbbem.PBError as e:
    out["batch"] = [e.code, str(e)]
# the context is still usable: single solves and the per-problem batch path
ps = probs()
out["single"] = [p.solve().dG_solv for p in ps]
ctx.set_option(pbbem.PB_OPT_BATCH_PERSISTENT, 0)
out["graphs"] = [r.dG_solv for r in pbbem.solve_batch(ctx, probs())]
print(json.dumps(out))
"""


def test_persistent_batch_bounded_wait_times_out():
    from paper_1309_4018_b300 import pbbem
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PB_FAULT="wait")
    p = subprocess.run([sys.executable, "-c", _TIMEOUT.format(root=root)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    out = json.loads(p.stdout.strip().splitlines()[-1])
    assert out["batch"][0] == pbbem.PB_ETIMEOUT and "bounded wait" in out["batch"][1]
    assert out["graphs"] == out["single"]


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
