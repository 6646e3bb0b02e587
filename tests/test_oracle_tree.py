"""Pins of the oracle's octree, Morton keys and interaction lists (Sec. 2.3, Eq. MAC).

The lists are checked against their definitions: the accepted boxes and the
direct-sum leaves of every target partition the sources exactly once, every
accepted box satisfies the MAC, every opened box fails it, and the
near-singular lists equal a brute-force scan.
"""
import numpy as np
import pytest

from oracle.dense import SurfaceData
from oracle.tree import Octree, interaction_lists, morton_keys, near_lists, root_cube
from synth.configs import protein_problem, sphere_problem


def _sphere_points(level=4, K=3):
    pr = sphere_problem(level=level)
    s = pr["surfaces"][0]
    return SurfaceData(s["verts"], s["tris"], K, 19)


def _decode(key):
    q = np.zeros((key.size, 3), dtype=np.int64)
    k = key.astype(np.uint64)
    for b in range(21):
        for a, sh in ((0, 2), (1, 1), (2, 0)):
            q[:, a] |= (((k >> np.uint64(3 * b + sh)) & np.uint64(1)).astype(np.int64) << b)
    return q


def test_morton_keys_roundtrip():
    rng = np.random.default_rng(1)
    p = rng.uniform(-3, 5, size=(500, 3))
    corner, side = root_cube(p)
    assert np.all(corner <= p.min(0)) and np.all(corner + side >= p.max(0))
    key = morton_keys(p, corner, side)
    q = _decode(key)
    cell = side / 2 ** 21
    lo = corner + q * cell
    assert np.all(p >= lo - 1e-12) and np.all(p <= lo + cell + 1e-12)
    # x-major interleave: the top bit of x is bit 62
    assert np.all(((key >> np.uint64(62)) & np.uint64(1)).astype(int) == (q[:, 0] >> 20))


@pytest.mark.parametrize("ncrit", [20, 60, 300])
def test_octree_invariants(ncrit):
    sd = _sphere_points()
    pts = sd.y.reshape(-1, 3)
    tr = Octree(pts, ncrit)
    # permutation sorts keys stably
    k = morton_keys(pts, tr.corner, tr.side)
    assert np.all(np.diff(tr.keys.astype(np.float64)) >= 0)
    assert np.array_equal(np.sort(tr.perm), np.arange(pts.shape[0]))
    eq = tr.keys[1:] == tr.keys[:-1]
    assert np.all(tr.perm[1:][eq] > tr.perm[:-1][eq])
    assert np.array_equal(k[tr.perm], tr.keys)
    for b in range(tr.n_nodes):
        s, c = tr.start[b], tr.count[b]
        sp = pts[tr.perm[s:s + c]]
        half = tr.side_l[b] / 2
        assert np.all(np.abs(sp - tr.centre[b]) <= half * (1 + 1e-12))
        if tr.is_leaf[b]:
            assert c < ncrit or tr.level[b] == 21
        else:
            fc, nc = tr.first_child[b], tr.nchild[b]
            assert tr.start[fc] == s
            assert tr.count[fc:fc + nc].sum() == c
            assert np.all(tr.parent[fc:fc + nc] == b)
            assert np.all(tr.level[fc:fc + nc] == tr.level[b] + 1)
    # leaves partition the points
    assert tr.count[tr.is_leaf].sum() == pts.shape[0]


@pytest.mark.parametrize("theta", [0.0, 0.5, 0.7])
def test_lists_partition_sources_and_respect_mac(theta):
    sd = _sphere_points()
    pts = sd.y.reshape(-1, 3)
    tr = Octree(pts, 40)
    mp, mb, pp, pb = interaction_lists(tr, sd.cen, theta)
    th2 = theta * theta
    for i in range(0, sd.n, 37):
        x = sd.cen[i]
        covered = np.zeros(pts.shape[0], int)
        for b in mb[mp[i]:mp[i + 1]]:
            d = x - tr.centre[b]
            assert tr.rb2[b] < th2 * ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
            covered[tr.start[b]:tr.start[b] + tr.count[b]] += 1
            # the parent was opened, so it failed the MAC
            par = tr.parent[b]
            if par >= 0:
                dp = x - tr.centre[par]
                assert not tr.rb2[par] < th2 * ((dp[0] * dp[0] + dp[1] * dp[1]) + dp[2] * dp[2])
        for b in pb[pp[i]:pp[i + 1]]:
            assert tr.is_leaf[b]
            d = x - tr.centre[b]
            assert not tr.rb2[b] < th2 * ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2])
            covered[tr.start[b]:tr.start[b] + tr.count[b]] += 1
        assert np.all(covered == 1)
        # depth-first pre-order within each list
        assert np.all(np.diff(tr.preorder[mb[mp[i]:mp[i + 1]]]) > 0)
        assert np.all(np.diff(tr.preorder[pb[pp[i]:pp[i + 1]]]) > 0)
    if theta == 0.0:
        assert mp[-1] == 0


def test_near_lists_brute_force():
    sd = _sphere_points(level=4)
    tr = Octree(sd.y.reshape(-1, 3), 40)
    mp, mb, pp, pb = interaction_lists(tr, sd.cen, 0.5)
    thres = 2.0
    ptr, pan, excl, self_excl = near_lists(tr, 3, sd.cen, np.arange(sd.n), sd.cen, sd.L, thres, pp, pb)
    assert self_excl == 0
    n_near = 0
    for i in range(0, sd.n, 11):
        d = np.sqrt(((sd.cen - sd.cen[i]) ** 2).sum(1))
        brute = set(np.nonzero(d < thres * sd.L)[0].tolist()) - {i}
        got = set(pan[ptr[i]:ptr[i + 1]].tolist())
        assert got <= brute
        n_near += len(brute)
        assert np.all(np.diff(pan[ptr[i]:ptr[i + 1]]) > 0)
    assert n_near > 0
    assert ptr[-1] + excl == sum(
        len(set(np.nonzero(np.sqrt(((sd.cen - sd.cen[i]) ** 2).sum(1)) < thres * sd.L)[0].tolist()) - {i})
        for i in range(sd.n))


def test_direct_list_is_all_leaves():
    sd = _sphere_points(level=3)
    tr = Octree(sd.y.reshape(-1, 3), 30)
    mp, mb, pp, pb = interaction_lists(tr, sd.cen, 0.0)
    leaves = np.nonzero(tr.is_leaf)[0]
    order = leaves[np.argsort(tr.preorder[leaves])]
    for i in range(sd.n):
        assert np.array_equal(pb[pp[i]:pp[i + 1]], order)
