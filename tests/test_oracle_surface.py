"""Pins of the oracle's Gaussian-density surface (marching tetrahedra, outer
component, smoothing) against closed forms, invariants and an independent mesher."""
import itertools

import numpy as np
import pytest

from oracle import surface as OS


def _mesh_stats(v, t):
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    directed = set(map(tuple, e))
    und = {tuple(sorted(x)) for x in directed}
    vol = np.einsum("ij,ij->i", v[t[:, 0]], np.cross(v[t[:, 1]], v[t[:, 2]])).sum() / 6.0
    return directed, und, vol


def _freudenthal(fc, u):
    """Piecewise-linear interpolant of corner values fc[8] at local coords u (Freudenthal's formula)."""
    order = np.argsort(-u, kind="stable")
    val, corner = fc[0], 0
    for a in order:
        nxt = corner | (1 << a)
        val += u[a] * (fc[nxt] - fc[corner])
        corner = nxt
    return val


def test_tets_positive_and_cover_the_cube():
    vol = 0.0
    for tet in OS.TETS:
        w = OS.CORNER[list(tet)].astype(float)
        d = np.linalg.det(np.stack([w[1] - w[0], w[2] - w[0], w[3] - w[0]]))
        assert d > 0
        vol += d / 6.0
    assert abs(vol - 1.0) < 1e-15


@pytest.mark.parametrize("seed", range(20))
def test_random_cube_triangles_lie_on_the_linear_level_set(seed):
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.0, 2.0, size=(2, 2, 2))
    fc = np.array([rho[c[0], c[1], c[2]] for c in OS.CORNER])
    h, lo = 0.7, np.array([1.0, -2.0, 0.5])
    v, t, _ = OS.marching_tetrahedra(rho, lo, h, 1.0, 0.0)
    if fc.min() >= 1.0 or fc.max() < 1.0:
        assert t.shape[0] == 0
        return
    assert t.shape[0] > 0
    for tri in t:
        P = v[tri]
        for _ in range(4):
            b = rng.dirichlet(np.ones(3))
            u = ((b @ P) - lo) / h
            assert abs(_freudenthal(fc, u) - 1.0) < 1e-12
        # the normal points down the interpolant: gradient from finite differences at the centroid
        c = (P.mean(0) - lo) / h
        n = np.cross(P[1] - P[0], P[2] - P[0])
        area = 0.5 * np.linalg.norm(n)
        if area < 1e-10:
            continue
        g = np.array([_freudenthal(fc, c + 1e-7 * np.eye(3)[k]) - _freudenthal(fc, c - 1e-7 * np.eye(3)[k])
                      for k in range(3)])
        assert n @ g < 0


def test_corner_cut_gives_three_squares():
    rho = np.zeros((2, 2, 2))
    rho[0, 0, 0] = 2.0
    h = 0.8
    v, t, _ = OS.marching_tetrahedra(rho, np.zeros(3), h, 1.0, 0.0)
    assert v.shape[0] == 7 and t.shape[0] == 6
    n = np.cross(v[t[:, 1]] - v[t[:, 0]], v[t[:, 2]] - v[t[:, 0]])
    assert abs(0.5 * np.linalg.norm(n, axis=1).sum() - 3 * (h / 2) ** 2) < 1e-14
    # every piece lies in a plane x, y or z = h/2 and faces away from the inside corner
    for tri, nn in zip(t, n):
        a = int(np.argmax(np.abs(nn)))
        assert np.allclose(v[tri][:, a], h / 2, atol=1e-15) and nn[a] > 0
        assert np.allclose(np.delete(nn, a), 0.0, atol=1e-15)


def _sphere(h, **kw):
    return OS.gaussian_surface(np.zeros((1, 3)), np.array([2.0]), h, **kw)


def test_single_atom_is_a_closed_sphere_converging_as_h_squared():
    errs = []
    for h in (0.4, 0.2):
        s = _sphere(h, smooth_iters=-1, tclamp=0.0)
        v, t = s["verts"], s["tris"]
        directed, und, vol = _mesh_stats(v, t)
        assert len(directed) == 3 * t.shape[0]                     # no directed edge twice
        assert all((b, a) in directed for a, b in directed)        # closed, consistently oriented
        assert v.shape[0] - len(und) + t.shape[0] == 2             # genus 0
        assert s["components"] == 1
        assert vol > 0
        r = np.linalg.norm(v, axis=1)
        errs.append(np.abs(r - 2.0).max())
        assert abs(vol - 4.0 / 3.0 * np.pi * 8.0) < 0.05 * 4.0 / 3.0 * np.pi * 8.0
    assert 3.0 < errs[0] / errs[1] < 5.0, errs


def test_smoothed_single_atom_lies_on_the_sphere():
    s = _sphere(0.4)
    assert s["rounds"] == 5
    r = np.linalg.norm(s["verts"], axis=1)
    assert np.abs(r - 2.0).max() < 1e-9
    assert OS.folded(s["verts"], s["tris"], np.zeros((1, 3)), np.array([2.0]), OS.DEFAULTS) == 0
    assert OS.folded(s["verts"], s["tris"][:, [0, 2, 1]], np.zeros((1, 3)), np.array([2.0]),
                     OS.DEFAULTS) == s["tris"].shape[0]


def test_laplacian_round_keeps_a_regular_planar_grid_interior():
    n = 6
    P = np.array([[i + 0.5 * j, j * np.sqrt(3) / 2, 0.0] for j in range(n) for i in range(n)])
    tris = []
    for j, i in itertools.product(range(n - 1), range(n - 1)):
        a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i, (j + 1) * n + i + 1
        tris += [(a, b, c), (b, d, c)]
    tris = np.array(tris)
    p = dict(OS.DEFAULTS, newton_steps=0, relax=1.0)
    e = OS.neighbours(P.shape[0], tris)
    v = OS.smooth_round(P, e, np.zeros((1, 3)), np.array([1.0]), p)
    interior = [j * n + i for j in range(1, n - 1) for i in range(1, n - 1)]
    assert np.abs(v[interior] - P[interior]).max() < 1e-14
    assert np.abs(v - P).max() > 0.1


def test_laplacian_shrinks_a_convex_surface():
    s = _sphere(0.4, smooth_iters=-1)
    e = OS.neighbours(s["verts"].shape[0], s["tris"])
    v = OS.smooth_round(s["verts"], e, np.zeros((1, 3)), np.array([2.0]), dict(OS.DEFAULTS, newton_steps=0))
    # the umbrella step pulls a round surface inwards: smaller mean radius and volume
    assert np.linalg.norm(v, axis=1).mean() < np.linalg.norm(s["verts"], axis=1).mean() - 1e-4
    assert _mesh_stats(v, s["tris"])[2] < _mesh_stats(s["verts"], s["tris"])[2]


def test_hollow_shell_keeps_the_outer_surface():
    k = np.arange(500) + 0.5
    phi, th = np.arccos(1 - 2 * k / 500), np.pi * (1 + 5 ** 0.5) * k
    xyz = 8.0 * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    s = OS.gaussian_surface(xyz, np.full(500, 1.5), 0.6, smooth_iters=-1)
    assert s["components"] == 2
    raw_r = np.linalg.norm(s["raw_verts"], axis=1)
    assert raw_r.min() < 8.0 < raw_r.max()
    assert np.linalg.norm(s["verts"], axis=1).min() > 8.0
    _, _, vol = _mesh_stats(s["verts"], s["tris"])
    assert vol > 4.0 / 3.0 * np.pi * 8.0 ** 3


def test_vertex_set_matches_the_independent_mesher():
    from synth.molecule import marching_tetrahedra, outer_component, synthetic_atoms
    at = synthetic_atoms(200, 9.0, seed=11)
    s = OS.gaussian_surface(at["xyz"], at["radius"], 1.0, smooth_iters=-1)
    assert np.abs(s["rho"] - 1.0).min() > 1e-10
    v2, t2 = marching_tetrahedra(s["rho"].copy(), s["lo"], 1.0, level=1.0, tclamp=0.02)
    assert np.array_equal(v2, s["raw_verts"])
    assert t2.shape[0] == s["raw_tris"].shape[0]
    v3, t3 = outer_component(v2, t2)
    assert np.array_equal(v3, s["verts"]) and t3.shape[0] == s["tris"].shape[0]
    # same closed surface: same enclosed volume up to the quadrilateral diagonals
    _, _, vol = _mesh_stats(s["verts"], s["tris"])
    _, _, vol3 = _mesh_stats(v3, t3)
    assert abs(vol - vol3) < 1e-3 * vol


def test_separate_blobs_keep_the_one_of_largest_x():
    xyz = np.array([[-6.0, 0.0, 0.0], [6.0, 0.5, 0.0]])
    s = OS.gaussian_surface(xyz, np.array([2.0, 1.5]), 0.5, smooth_iters=-1)
    assert s["components"] == 2
    d = np.linalg.norm(s["verts"] - xyz[1], axis=1)
    assert np.abs(d - 1.5).max() < 0.1        # the other blob is 12 A away
