"""Malformed inputs and failure paths of the C-ABI: every one returns a status
code with a message, and the context stays usable afterwards.

Faults are made on the host only: malformed meshes and charges, an iteration
cap that GMRES cannot meet, and an allocation request that the library's
PB_FAULT hook turns into PB_ENOMEM.  Nothing here faults the GPU.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from gpu_util import ctx, problem
from synth.configs import cavity_sphere_problem, sphere_problem

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _pbbem():
    from paper_1309_4018_b300 import pbbem
    return pbbem


def _expect_einval(d, words, params=None):
    pbbem = _pbbem()
    with pytest.raises(pbbem.PBError) as ei:
        pb = pbbem.Problem.from_dict(ctx(), d)
        pb.setup(**(params or dict(theta=-1.0, precision="fp64", ncrit=64)))
    assert ei.value.code == pbbem.PB_EINVAL
    assert all(w in str(ei.value) for w in words), str(ei.value)


def _sphere(**kw):
    d = sphere_problem(level=2, charges="both")
    s = dict(d["surfaces"][0], **kw)
    return dict(d, surfaces=[s])


def test_open_mesh_rejected():
    t = sphere_problem(level=2)["surfaces"][0]["tris"]
    _expect_einval(_sphere(tris=t[1:]), ["closed 2-manifold", "1 triangle"])


def test_flipped_triangle_rejected():
    t = sphere_problem(level=2)["surfaces"][0]["tris"].copy()
    t[7] = t[7][[0, 2, 1]]
    _expect_einval(_sphere(tris=t), ["consistently oriented"])


def test_repeated_vertex_rejected():
    t = sphere_problem(level=2)["surfaces"][0]["tris"].copy()
    t[3, 1] = t[3, 0]
    _expect_einval(_sphere(tris=t), ["repeats a vertex"])


def test_inverted_winding_rejected():
    # a reversed mesh would put the solvent inside: the signed volume is negative
    t = sphere_problem(level=2)["surfaces"][0]["tris"][:, ::-1].copy()
    _expect_einval(_sphere(tris=t), ["signed volume", "counter-clockwise"])


def test_charge_outside_its_region_rejected():
    d = sphere_problem(level=3, charges="both")
    d["charges"] = dict(d["charges"], xyz=np.array([[0.0, 0.0, 0.0], [4.5, 0.3, -0.2]]))
    _expect_einval(d, ["1 charge(s) lie outside their region", "charge 1"])
    # the same with the treecode's settings
    _expect_einval(d, ["outside their region"], dict(theta=0.5, P=6, ncrit=40, precision="mixed"))


def test_charge_inside_a_cavity_rejected():
    d = cavity_sphere_problem(level=2)
    # region 1 is the shell 1.5 < r < 4: a charge at the centre sits in the cavity
    d["charges"] = dict(d["charges"], xyz=np.array([[0.2, 0.1, 0.0]]))
    _expect_einval(d, ["outside their region"])


def test_valid_problems_still_accepted_after_errors():
    d = sphere_problem(level=3, charges="both")
    r = problem(d, theta=-1.0, precision="fp64", ncrit=64, gmres_tol=1e-8).solve()
    assert r.converged and r.dG_solv < 0.0


def test_enoconv_writes_the_partial_result():
    pbbem = _pbbem()
    d = sphere_problem(level=3, charges="both")
    pb = problem(d, theta=0.5, P=6, ncrit=40, precision="mixed", gmres_tol=1e-10, max_iter=1)
    with pytest.raises(pbbem.PBError) as ei:
        pb.solve()
    assert ei.value.code == pbbem.PB_ENOCONV and "max_iter" in str(ei.value)
    r = pb.solve(check=False)
    assert not r.converged and r.iterations == 1
    assert np.isfinite(r.dG_solv) and r.dG_solv < 0.0 and r.residual > 1e-10
    assert np.all(np.isfinite(pb.solution()))


_INJECT = r"""
import json, sys
sys.path.insert(0, {root!r})
from paper_1309_4018_b300 import pbbem
from synth.configs import sphere_problem
ctx = pbbem.Context(0)
d = sphere_problem(level=3, charges="both")
out = {{}}
for attempt in (0, 1):
    try:
        pb = pbbem.Problem.from_dict(ctx, d)
        pb.setup(theta=0.5, P=6, ncrit=40, precision="mixed", gmres_tol=1e-6)
        out[attempt] = dict(ok=True, dG=pb.solve().dG_solv)
        pb.close()
    except pbbem.PBError as e:
        out[attempt] = dict(ok=False, code=e.code, msg=str(e))
print(json.dumps(out))
"""


@pytest.mark.parametrize("nth", [1, 4, 25])
def test_injected_allocation_failure_gives_enomem(nth):
    env = dict(os.environ, PB_FAULT=f"alloc:{nth}")
    p = subprocess.run([sys.executable, "-c", _INJECT.format(root=ROOT)], env=env, capture_output=True,
                       text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    out = json.loads(p.stdout.strip().splitlines()[-1])
    first, second = out["0"], out["1"]
    from paper_1309_4018_b300 import pbbem
    assert not first["ok"] and first["code"] == pbbem.PB_ENOMEM and "injected" in first["msg"]
    # the fault fires once: the same work then succeeds in the same context
    assert second["ok"] and second["dG"] < 0.0
