"""GPU treecode (P2P + P2M/M2M + M2P + near field) against the oracle treecode and dense operator."""
import numpy as np
import pytest

from gpu_util import problem, rel_l2
from oracle import dense as OD
from oracle import formulation as F
from oracle.treecode import TreecodeOracle
from synth.configs import layered_sphere_problem, sphere_problem

pytestmark = pytest.mark.gpu


def _rows_rel(out, y, d, rows):
    num = den = 0.0
    for (s, side), ref in out.items():
        got = y[F.row_slice(d, s, side)][rows[s]]
        num += ((got - ref) ** 2).sum()
        den += (ref ** 2).sum()
    return np.sqrt(num / den)


@pytest.mark.parametrize("P", [2, 6, 10])
def test_fp64_treecode_matches_oracle_treecode(P):
    d = sphere_problem(level=4, charges="both")
    prm = dict(theta=0.5, P=P, ncrit=40)
    pb = problem(d, precision="fp64", **prm)
    x = np.random.default_rng(P).normal(size=2 * 2048)
    y = pb.apply(x)
    tc = TreecodeOracle(d, prm)
    rows = {0: np.arange(0, 2048, 61 if P < 10 else 257)}
    assert _rows_rel(tc.matvec(x, rows), y, d, rows) <= 1e-12


def test_fp64_treecode_multisurface():
    d = layered_sphere_problem(level=3, charges="both")
    prm = dict(theta=0.5, P=4, ncrit=25)
    pb = problem(d, precision="fp64", **prm)
    x = np.random.default_rng(3).normal(size=4 * 512)
    y = pb.apply(x)
    tc = TreecodeOracle(d, prm)
    rows = {0: np.arange(0, 512, 23), 1: np.arange(5, 512, 29)}
    assert _rows_rel(tc.matvec(x, rows), y, d, rows) <= 1e-12


def test_mixed_matvec_close_to_dense():
    d = sphere_problem(level=4, charges="both")
    A = OD.operator_matrix(d)
    x = np.random.default_rng(5).normal(size=A.shape[0])
    yd = A @ x
    pb = problem(d, precision="mixed", theta=-1.0, ncrit=64)
    assert rel_l2(pb.apply(x), yd) <= 2e-6
    pb2 = problem(d, precision="mixed", theta=0.5, P=6, ncrit=40)
    assert rel_l2(pb2.apply(x), yd) <= 1e-4


def test_mixed_energy_within_1e4_of_fp64():
    d = sphere_problem(level=4, charges="both")
    e64 = problem(d, precision="fp64", theta=-1.0, gmres_tol=1e-10).solve().dG_solv
    em = problem(d, precision="mixed", theta=0.5, P=6, ncrit=40, gmres_tol=1e-6).solve().dG_solv
    assert abs(em - e64) <= 1e-4 * abs(e64)


def test_mixed_rhs_close_to_oracle():
    from synth.configs import protein_problem
    d = protein_problem()
    pb = problem(d, precision="mixed", theta=0.5, P=6, ncrit=300)
    b = pb.rhs()
    n = d["surfaces"][0]["tris"].shape[0]
    rows = np.arange(0, n, 97)
    sd = OD.surfaces_data(d)
    ref = OD._green(sd[0].cen[rows], np.asarray(d["charges"]["xyz"]), 0.0) @ d["charges"]["q"] / 4.0
    assert rel_l2(b[rows], ref) <= 1e-5
    assert np.all(b[n:] == 0.0)


@pytest.mark.parametrize("P", [1, 3, 6, 8, 9])
def test_mixed_treecode_matches_fp64_treecode(P):
    # same tree, same lists, same truncation: the FP32 path (radial-form M2P for
    # P <= 8, recurrences above) differs from the FP64 treecode only by FP32
    # rounding (measured 2.3e-7 .. 2.7e-7; FP32 unit roundoff 6e-8 times a few
    # for the sums' cancellation); bound 2e-6.
    d = layered_sphere_problem(level=3, charges="both")
    kw = dict(theta=0.5, P=P, ncrit=40)
    x = np.random.default_rng(P).normal(size=2 * sum(s["tris"].shape[0] for s in d["surfaces"]))
    y64 = problem(d, precision="fp64", **kw).apply(x)
    y32 = problem(d, precision="mixed", **kw).apply(x)
    assert rel_l2(y32, y64) <= 2e-6


def test_mixed_protein_operator_matches_fp64_treecode():
    # the 40k-panel protein of the benchmark, its default settings: measured
    # 2.9e-6 (coordinates relative to the root centre reach 30 A, panels 0.6 A:
    # the FP32 differences of the near terms lose more); bound 2e-5
    from synth.configs import protein_problem
    d = protein_problem()
    kw = dict(theta=0.5, P=6, ncrit=300)
    x = np.random.default_rng(0).normal(size=2 * d["surfaces"][0]["tris"].shape[0])
    y64 = problem(d, precision="fp64", **kw).apply(x)
    y32 = problem(d, precision="mixed", **kw).apply(x)
    assert rel_l2(y32, y64) <= 2e-5


def test_m2p_tensor_pipe_variant():
    # the radial contraction on the tensor pipe (split TF32 operands, FP32
    # accumulation) against the FP32-pipe path and the FP64 treecode on the
    # 40k-panel protein: rounding differences only
    from synth.configs import protein_problem
    d = protein_problem()
    kw = dict(theta=0.5, P=6, ncrit=300)
    x = np.random.default_rng(0).normal(size=2 * d["surfaces"][0]["tris"].shape[0])
    y64 = problem(d, precision="fp64", **kw).apply(x)
    y32 = problem(d, precision="mixed", **kw).apply(x)
    ytc = problem(d, precision="mixed", m2p_variant=1, **kw).apply(x)
    assert rel_l2(ytc, y64) <= 2e-5
    assert rel_l2(ytc, y32) <= 1e-5
    e0 = problem(d, precision="mixed", gmres_tol=1e-6, **kw).solve().dG_solv
    e1 = problem(d, precision="mixed", gmres_tol=1e-6, m2p_variant=1, **kw).solve().dG_solv
    assert abs(e1 - e0) <= 1e-6 * abs(e0)


@pytest.mark.parametrize("n_atoms", [101, 103])
def test_mixed_gather_partial_lane_groups(n_atoms):
    # the FP32 gather takes four targets per warp: with 101 or 103 charges the
    # reaction potential's last warp holds one or three targets (the other
    # lane groups only join the shuffles).  Same tree, lists and truncation as
    # the FP64 treecode: the operator within the FP32 bound of the benchmark
    # protein's (2e-5), the energy within 1e-5 (FP64 solved to 1e-8, the
    # FP32 operator to 1e-6, near its rounding floor).
    from synth.configs import protein_problem
    d = protein_problem(n_atoms=n_atoms, seed=5 if n_atoms == 101 else 6)
    assert d["charges"]["q"].size % 4 != 0
    kw = dict(theta=0.5, P=6, ncrit=300)
    x = np.random.default_rng(n_atoms).normal(size=2 * d["surfaces"][0]["tris"].shape[0])
    y64 = problem(d, precision="fp64", **kw).apply(x)
    y32 = problem(d, precision="mixed", **kw).apply(x)
    assert rel_l2(y32, y64) <= 2e-5
    e64 = problem(d, precision="fp64", gmres_tol=1e-8, **kw).solve().dG_solv
    e32 = problem(d, precision="mixed", gmres_tol=1e-6, **kw).solve().dG_solv
    assert abs(e32 - e64) <= 1e-5 * abs(e64)
