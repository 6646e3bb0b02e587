"""GPU parity of the transposed treecode and the adjoint energy gradient.

Direct summation (theta < 0, FP64) must reproduce the dense oracle's A^T and
its LU-based adjoint gradient to rounding; the treecode paths agree within
their truncation (FP64) and FP32 (mixed) error.  At the 40k-panel protein
the oracle cannot run, so the exact identities q . dE/dq = 2E and
sum_R eps_R dE/deps_R = -E hold to the solver tolerance.
"""
import numpy as np
import pytest

from gpu_util import problem, rel_l2
from oracle import dense as OD
from oracle.gradient import solvation_gradient
from synth.configs import cavity_sphere_problem, layered_sphere_problem, protein_problem, sphere_problem

pytestmark = pytest.mark.gpu

DIRECT = dict(theta=-1.0, precision="fp64", ncrit=64)
TREE64 = dict(theta=0.5, P=6, ncrit=60, precision="fp64")
TREE32 = dict(theta=0.5, P=6, ncrit=60, precision="mixed")


def _cases():
    sph = sphere_problem(level=3, charges="both")
    sph["charges"]["q"] = np.array([0.7, -0.4])
    lay = layered_sphere_problem(level=2)
    lay["charges"]["q"] = np.array([1.0, 0.5])
    return {"sphere": sph, "layered": lay, "cavity": cavity_sphere_problem(level=2)}


CASES = _cases()


@pytest.fixture(scope="module")
def oracle_grads():
    return {k: solvation_gradient(v) for k, v in CASES.items()}


@pytest.mark.parametrize("name", list(CASES))
def test_transpose_direct_matches_dense(name):
    d = CASES[name]
    pb = problem(d, **DIRECT)
    A = OD.operator_matrix(d)
    rng = np.random.default_rng(3)
    for _ in range(2):
        y = rng.normal(size=A.shape[0])
        assert rel_l2(pb.apply_transpose(y), A.T @ y) <= 1e-12


@pytest.mark.parametrize("params,P,tol", [(TREE64, 6, 1e-4), (TREE64, 10, 3e-6), (TREE32, 6, 1e-4)])
def test_transpose_treecode(params, P, tol):
    d = sphere_problem(level=4, charges="both")
    pb = problem(d, **dict(params, P=P))
    A = OD.operator_matrix(d)
    y = np.random.default_rng(5).normal(size=A.shape[0])
    et = rel_l2(pb.apply_transpose(y), A.T @ y)
    ef = rel_l2(pb.apply(y), A @ y)
    # truncation of the same order as the forward treecode's, falling with P
    assert et <= tol and et <= 5 * ef + 1e-9, (et, ef)
    # the adjoint identity (A x) . y = x . (A^T y) up to the same truncation
    x = np.random.default_rng(6).normal(size=A.shape[0])
    lhs, rhs = pb.apply(x) @ y, x @ pb.apply_transpose(y)
    assert abs(lhs - rhs) <= 5 * tol * np.linalg.norm(A @ x) * np.linalg.norm(y)


def _compare(g, ref, tol):
    for k in ("dq", "dxyz", "deps", "dkappa"):
        a, b = np.asarray(g[k]).ravel(), np.asarray(ref[k]).ravel()
        scale = max(np.abs(b).max(), abs(ref["E"]) * 1e-3)
        assert np.abs(a - b).max() <= tol * scale, (k, a, b)


@pytest.mark.parametrize("name", list(CASES))
def test_gradient_direct_matches_oracle(name, oracle_grads):
    d = CASES[name]
    pb = problem(d, gmres_tol=1e-13, max_iter=400, **DIRECT)
    r = pb.solve()
    g = pb.gradient()
    ref = oracle_grads[name]
    assert abs(r.dG_solv - ref["E"]) <= 1e-10 * abs(ref["E"])
    assert g["residual"] < 1e-13
    _compare(g, ref, 1e-9)


@pytest.mark.parametrize("name", ["sphere", "layered"])
@pytest.mark.parametrize("params,tol", [(TREE64, 1e-4), (TREE32, 1e-3)])
def test_gradient_treecode(name, params, tol, oracle_grads):
    d = CASES[name]
    pb = problem(d, gmres_tol=1e-10 if params["precision"] == "fp64" else 1e-6, max_iter=400, **params)
    pb.solve()
    _compare(pb.gradient(), oracle_grads[name], tol)


def test_gradient_identities_protein():
    d = protein_problem()
    pb = problem(d, precision="mixed", gmres_tol=1e-6)
    r = pb.solve()
    g = pb.gradient()
    q = d["charges"]["q"]
    eps = np.array([reg["eps"] for reg in d["regions"]])
    assert abs(q @ g["dq"] - 2 * r.dG_solv) <= 1e-4 * abs(r.dG_solv)
    assert abs(eps @ g["deps"] + r.dG_solv) <= 1e-4 * abs(r.dG_solv)
    assert np.all(np.isfinite(g["dxyz"])) and np.all(np.isfinite(g["dkappa"]))


@pytest.mark.parametrize("P", [2, 6, 8])
def test_mixed_transpose_matches_fp64_transpose(P):
    # same trees and lists in both precisions: the FP32 transposed operator
    # (radial-form M2P of the Laplace + Yukawa pairs) differs from the FP64 one
    # by rounding only; bound 2e-6 as for the forward operator
    d = layered_sphere_problem(level=3, charges="both")
    kw = dict(theta=0.5, P=P, ncrit=40)
    x = np.random.default_rng(P).normal(size=2 * sum(s["tris"].shape[0] for s in d["surfaces"]))
    y64 = problem(d, precision="fp64", **kw).apply_transpose(x)
    y32 = problem(d, precision="mixed", **kw).apply_transpose(x)
    assert rel_l2(y32, y64) <= 2e-6
