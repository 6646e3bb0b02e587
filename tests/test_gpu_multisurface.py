"""The multi-surface molecule at full size (~103k panels: molecular surface,
Stern layer, two solvent-filled cavities) and its four solvent models
(Sec. 2.2 "Multi-surface problems"; the Single / Cavity / Stern / Full
comparison of Sec. 3).

Parity at this size: the FP32-mixed energy of every model is within 1e-4 of
the FP64 treecode's; a cavity whose permittivity equals the protein's is
invisible (its energy equals the single-surface model's to discretisation
error); the octrees and interaction lists of cross-surface pairs equal the
oracle's bit for bit on sampled targets.
"""
import copy

import numpy as np
import pytest

from gpu_util import ctx, problem
from test_gpu_tree import _check_lists, _check_tree
from synth.configs import EPS_IN, model_variants

pytestmark = pytest.mark.gpu

MIXED = dict(precision="mixed", gmres_tol=1e-6)
FP64 = dict(precision="fp64", gmres_tol=1e-8)


@pytest.fixture(scope="module")
def variants():
    return model_variants()


def test_model_variants_mixed_vs_fp64(variants):
    from paper_1309_4018_b300 import pbbem
    names = list(variants)
    probs = [problem(variants[k], **MIXED) for k in names]
    res = dict(zip(names, pbbem.solve_batch(ctx(), probs)))
    for k in names:
        assert res[k].converged and res[k].dG_solv < 0.0
    e64 = problem(variants["full"], **FP64).solve().dG_solv
    assert abs(res["full"].dG_solv - e64) <= 1e-4 * abs(e64)
    single = res["single"].dG_solv
    for k in ("cavity", "stern", "full"):
        assert abs(res[k].dG_solv - single) < 0.1 * abs(single)
    # the Stern layer removes salt from the first 2 A: the reaction field weakens
    assert res["stern"].dG_solv > single


def test_invisible_cavity(variants):
    d = copy.deepcopy(variants["cavity"])
    d["regions"][0]["eps"] = EPS_IN
    d["regions"][1]["eps"] = EPS_IN
    e_cav = problem(d, **MIXED).solve().dG_solv
    e_single = problem(variants["single"], **MIXED).solve().dG_solv
    assert abs(e_cav - e_single) < 1e-3 * abs(e_single)


def test_full_size_cross_surface_lists(variants):
    d = variants["full"]
    pb = problem(d, ncrit=300, theta=0.5, P=6, precision="mixed")
    rng = np.random.default_rng(5)
    _check_tree(pb, d, 3, 3, 300)
    for tgt, src in ((3, 2), (2, 3), (2, 0), (0, 2)):
        n = d["surfaces"][tgt]["tris"].shape[0]
        sample = np.sort(rng.choice(n, min(n, 200), replace=False))
        _check_lists(pb, d, tgt, src, 3, 300, 0.5, 2.0, sample=sample)
