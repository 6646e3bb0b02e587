"""Full-size parity against the oracle's stored values.

tests/golden/*.json were written by tests/golden/make_golden.py, which calls
only the oracle and the seeded input generators.  Each file fingerprints the
meshes it was made on (panel counts, a hash of the triangles, vertex sums),
and the tests first check that the regenerated inputs match.

protein40k (the benchmark workload, 40,144 panels): the FP64 direct operator
equals the dense oracle on 200 sampled rows (<= 1e-12); the FP64 treecode
equals the oracle's treecode there (<= 1e-12: same lists, moments by M2M
instead of directly, coefficients by recurrence instead of jets); the mixed
treecode stays within FP32 rounding of it; the energies of Eq. solv are within
1e-6 (FP64 direct) and 1e-4 (FP32-mixed treecode at the benchmark's settings)
of the oracle's GMRES solve at tol 1e-8.

multisurface400 (four surfaces, Sec. 2.2 "Multi-surface problems"): the FP64
direct operator of the full model on sampled rows of every surface, and the
energy of each of the four model variants, FP64 direct and mixed.
"""
import json
import hashlib
import os

import numpy as np
import pytest

from gpu_util import ctx, problem
from oracle import formulation as F
from synth import configs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(GOLDEN, name + ".json")) as f:
        return json.load(f)


def _check_mesh(d, fps):
    for s, fp in zip(d["surfaces"], fps):
        v = np.asarray(s["verts"], dtype=np.float64)
        t = np.ascontiguousarray(np.asarray(s["tris"], dtype=np.int32))
        assert t.shape[0] == fp["n_panels"] and v.shape[0] == fp["n_verts"]
        assert hashlib.sha256(t.tobytes()).hexdigest() == fp["tris_sha256"]
        assert abs(v.sum() - fp["verts_sum"]) <= 1e-12 * np.abs(v).sum()
        assert abs((v * v).sum() - fp["verts_sumsq"]) <= 1e-12 * fp["verts_sumsq"]


def _x(d, seed):
    return np.random.default_rng(seed).normal(size=2 * configs.panel_count(d))


def _rows_rel(y, d, ref):
    num = den = 0.0
    for s, r in enumerate(ref):
        rows = np.asarray(r["rows"])
        for side, key in ((0, "inner"), (1, "outer")):
            got = y[F.row_slice(d, s, side)][rows]
            want = np.asarray(r[key])
            num += ((got - want) ** 2).sum()
            den += (want ** 2).sum()
    return float(np.sqrt(num / den))


def _ref_rel(a, b):
    num = den = 0.0
    for ra, rb in zip(a, b):
        for key in ("inner", "outer"):
            num += ((np.asarray(ra[key]) - np.asarray(rb[key])) ** 2).sum()
            den += (np.asarray(rb[key]) ** 2).sum()
    return float(np.sqrt(num / den))


@pytest.fixture(scope="module")
def protein():
    g = _load("protein40k")
    d = configs.protein_problem()
    _check_mesh(d, g["mesh"])
    return d, g


def test_protein_direct_operator_rows(protein):
    d, g = protein
    y = problem(d, precision="fp64", theta=-1.0, ncrit=300).apply(_x(d, g["x_seed"]))
    assert _rows_rel(y, d, g["dense_rows"]) <= 1e-12


def test_protein_treecode_rows(protein):
    d, g = protein
    tc = g["treecode"]
    kw = dict(theta=tc["theta"], P=tc["P"], ncrit=tc["ncrit"])
    x = _x(d, g["x_seed"])
    assert _rows_rel(problem(d, precision="fp64", **kw).apply(x), d, tc["rows"]) <= 1e-12
    # FP32 rounding of the mixed path at this size: 2.9e-6 against the FP64 treecode
    ym = problem(d, precision="mixed", **kw).apply(x)
    assert _rows_rel(ym, d, tc["rows"]) <= 2e-5
    # and against the exact operator within the treecode's own truncation error plus that
    trunc = _ref_rel(tc["rows"], g["dense_rows"])
    assert _rows_rel(ym, d, g["dense_rows"]) <= trunc + 2e-5


def test_protein_energy_fp64_direct(protein):
    d, g = protein
    r = problem(d, precision="fp64", theta=-1.0, ncrit=300, gmres_tol=1e-8).solve()
    assert r.converged
    assert abs(r.dG_solv - g["dG"]) <= 1e-6 * abs(g["dG"])


def test_protein_energy_mixed_benchmark_settings(protein):
    # the benchmark's step: theta 0.5, P 6, ncrit 300, GMRES tol 1e-4, FP32-mixed
    d, g = protein
    r = problem(d, precision="mixed", theta=0.5, P=6, ncrit=300, gmres_tol=1e-4).solve()
    assert r.converged
    assert abs(r.dG_solv - g["dG"]) <= 1e-4 * abs(g["dG"])


@pytest.fixture(scope="module")
def multisurface():
    g = _load("multisurface400")
    v = configs.reduced_model_variants()
    for name, d in v.items():
        _check_mesh(d, g["variants"][name]["mesh"])
    return v, g


def test_multisurface_direct_operator_rows(multisurface):
    v, g = multisurface
    d = v["full"]
    y = problem(d, precision="fp64", theta=-1.0, ncrit=300).apply(_x(d, g["x_seed"]))
    assert _rows_rel(y, d, g["full_dense_rows"]) <= 1e-12


def test_multisurface_model_variants_energy(multisurface):
    from paper_1309_4018_b300 import pbbem
    v, g = multisurface
    names = list(v)
    probs = [problem(v[k], precision="mixed", theta=0.5, P=6, ncrit=300, gmres_tol=1e-6) for k in names]
    mixed = dict(zip(names, pbbem.solve_batch(ctx(), probs)))
    for k in names:
        ref = g["variants"][k]["dG"]
        assert mixed[k].converged
        assert abs(mixed[k].dG_solv - ref) <= 1e-4 * abs(ref), k
        e64 = problem(v[k], precision="fp64", theta=-1.0, ncrit=300, gmres_tol=1e-8).solve().dG_solv
        assert abs(e64 - ref) <= 1e-6 * abs(ref), k
