"""Bit-exact parity of the integer work (Morton keys, octree, interaction lists) with the oracle (Sec. 2.3)."""
import numpy as np
import pytest

from gpu_util import problem
from oracle.dense import SurfaceData
from oracle.tree import Octree, interaction_lists, near_lists
from synth.configs import layered_sphere_problem, protein_problem, sphere_problem

pytestmark = pytest.mark.gpu


def _check_tree(pb, d, surface, K, ncrit):
    s = d["surfaces"][surface]
    sd = SurfaceData(s["verts"], s["tris"], K, 19)
    ref = Octree(sd.y.reshape(-1, 3), ncrit)
    got = pb.tree(surface)
    assert np.array_equal(got["corner"], ref.corner) and got["side"] == ref.side
    assert np.array_equal(got["keys"], ref.keys)
    assert np.array_equal(got["perm"], ref.perm)
    assert np.array_equal(got["level"], ref.level)
    assert np.array_equal(got["start"], ref.start)
    assert np.array_equal(got["count"], ref.count)
    assert np.array_equal(got["nchild"], ref.nchild)
    assert np.array_equal(got["first_child"], np.where(ref.nchild > 0, ref.first_child, -1))


def _check_lists(pb, d, tgt, src, K, ncrit, theta, thres, sample=None):
    sd_t = SurfaceData(d["surfaces"][src]["verts"], d["surfaces"][src]["tris"], K, 19)
    tree = Octree(sd_t.y.reshape(-1, 3), ncrit)
    if tgt >= 0:
        sd_s = SurfaceData(d["surfaces"][tgt]["verts"], d["surfaces"][tgt]["tris"], K, 19)
        x = sd_s.cen
    else:
        x = np.asarray(d["charges"]["xyz"], dtype=np.float64)
    mp, mb, pp, pb_ = interaction_lists(tree, x, theta)
    got = pb.lists(tgt, src)
    assert np.array_equal(got["m2p_ptr"], mp) and np.array_equal(got["m2p"], mb)
    assert np.array_equal(got["p2p_ptr"], pp) and np.array_equal(got["p2p"], pb_)
    rows = np.arange(x.shape[0]) if sample is None else sample
    selfp = rows if tgt == src else -np.ones(rows.size, np.int64)
    sub_ptr = np.concatenate([[0], np.cumsum(pp[rows + 1] - pp[rows])])
    sub = np.concatenate([pb_[pp[i]:pp[i + 1]] for i in rows])
    nptr, npan, excl, sexcl = near_lists(tree, K, x[rows], selfp, sd_t.cen, sd_t.L, thres, sub_ptr, sub)
    for r, i in enumerate(rows):
        assert np.array_equal(got["near"][got["near_ptr"][i]:got["near_ptr"][i + 1]], npan[nptr[r]:nptr[r + 1]])
    if sample is None:
        assert got["n_near_excluded"] == excl and got["n_self_excluded"] == sexcl


@pytest.mark.parametrize("ncrit,theta", [(20, 0.5), (64, 0.7), (300, 0.5)])
def test_sphere_tree_and_lists_bit_exact(ncrit, theta):
    d = sphere_problem(level=4, charges="both")
    pb = problem(d, ncrit=ncrit, theta=theta, precision="fp64")
    _check_tree(pb, d, 0, 3, ncrit)
    _check_lists(pb, d, 0, 0, 3, ncrit, theta, 2.0)
    _check_lists(pb, d, -1, 0, 3, ncrit, theta, 2.0)


def test_multisurface_lists_bit_exact():
    d = layered_sphere_problem(level=3, charges="both")
    pb = problem(d, ncrit=30, theta=0.5, precision="fp64")
    for s in (0, 1):
        _check_tree(pb, d, s, 3, 30)
    for t, s in ((0, 0), (0, 1), (1, 0), (1, 1)):
        _check_lists(pb, d, t, s, 3, 30, 0.5, 2.0)


def test_protein_tree_and_lists_bit_exact():
    # the ~40k-panel synthetic protein at the production parameters
    d = protein_problem()
    pb = problem(d, ncrit=300, theta=0.5, P=6, precision="mixed")
    _check_tree(pb, d, 0, 3, 300)
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(d["surfaces"][0]["tris"].shape[0], 300, replace=False))
    _check_lists(pb, d, 0, 0, 3, 300, 0.5, 2.0, sample=sample)
    _check_lists(pb, d, -1, 0, 3, 300, 0.5, 2.0, sample=np.arange(0, 2000, 7))
