"""pbbem.Energy, the torch.autograd.Function over (q, xyz, eps, kappa): its
value is the solvation energy of Eq. solv and its gradient, taken by
torch.autograd.grad through the library's adjoint solve, equals the dense
oracle's adjoint gradient (oracle/gradient.py, LU solves)."""
import numpy as np
import pytest

from gpu_util import ctx
from oracle.gradient import solvation_gradient
from synth.configs import layered_sphere_problem, sphere_problem

pytestmark = pytest.mark.gpu

DIRECT = dict(theta=-1.0, precision="fp64", ncrit=64, gmres_tol=1e-12)


def _inputs(d, torch):
    ch = d["charges"]
    q = torch.tensor(np.asarray(ch["q"], dtype=np.float64), requires_grad=True)
    xyz = torch.tensor(np.asarray(ch["xyz"], dtype=np.float64), requires_grad=True)
    eps = torch.tensor([r["eps"] for r in d["regions"]], dtype=torch.float64, requires_grad=True)
    kap = torch.tensor([r["kappa"] for r in d["regions"]], dtype=torch.float64, requires_grad=True)
    return q, xyz, eps, kap


@pytest.mark.parametrize("case", ["sphere", "layered"])
def test_energy_autograd_matches_oracle_adjoint(case):
    import torch
    from paper_1309_4018_b300 import pbbem
    d = sphere_problem(level=3, charges="both") if case == "sphere" else layered_sphere_problem(level=2)
    d["charges"] = dict(d["charges"], q=np.array([0.7, -0.4]))
    ref = solvation_gradient(d)
    q, xyz, eps, kap = _inputs(d, torch)
    E = pbbem.Energy.apply(d, q, xyz, eps, kap, ctx(), DIRECT)
    assert abs(E.item() - ref["E"]) <= 1e-9 * abs(ref["E"])
    gq, gx, ge, gk = torch.autograd.grad(2.0 * E, [q, xyz, eps, kap])
    scale = max(np.abs(ref[k]).max() for k in ("dq", "dxyz", "deps", "dkappa"))
    for got, key in ((gq, "dq"), (gx, "dxyz"), (ge, "deps"), (gk, "dkappa")):
        assert np.abs(got.numpy() - 2.0 * ref[key]).max() <= 2e-9 * scale, key


def test_energy_without_backward_and_without_grad():
    import torch
    from paper_1309_4018_b300 import pbbem
    d = sphere_problem(level=3, charges="both")
    q, xyz, eps, kap = _inputs(d, torch)
    with torch.no_grad():
        E0 = pbbem.Energy.apply(d, q, xyz, eps, kap, ctx(), DIRECT)
    E1 = pbbem.Energy.apply(d, q.detach(), xyz.detach(), eps.detach(), kap.detach(), ctx(), DIRECT)
    assert not E1.requires_grad
    assert E0.item() == E1.item()
