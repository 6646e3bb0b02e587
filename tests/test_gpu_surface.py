"""GPU parity of the device surface generator against the oracle (oracle/surface.py).

Integer results (triangles, vertex numbering, component count, grid, rounds)
must be identical; vertex coordinates agree to rounding of the density sums
(FP64 on both sides, summed in a different order).  Each case first checks
that no grid node's density is within 1e-10 of the level, so the inside test
is decided the same way by both sides.
"""
import numpy as np
import pytest

from gpu_util import ctx
from oracle import surface as OS
from synth.configs import protein_atoms, sphere_problem
from synth.molecule import synthetic_atoms

pytestmark = pytest.mark.gpu


def _gpu_surface(xyz, radius, **params):
    from paper_1309_4018_b300 import pbbem
    pb = pbbem.Problem(ctx())
    pb.add_region(4.0, 0.0)
    pb.add_region(80.0, 0.125)
    sid = pb.add_gaussian_surface(xyz, radius, 0, 1, **params)
    v, t = pb.surface_mesh(sid)
    info = pb.surface_info(sid)
    pb.close()
    return v, t, info


def _shell(n=500, r=8.0):
    k = np.arange(n) + 0.5
    phi, th = np.arccos(1 - 2 * k / n), np.pi * (1 + 5 ** 0.5) * k
    return r * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)


CASES = {
    "molecule200": (lambda: synthetic_atoms(200, 9.0, seed=11), dict(spacing=1.0)),
    "molecule200_fine_stern": (lambda: synthetic_atoms(200, 9.0, seed=12), dict(spacing=0.7, radius_offset=2.0)),
    "shell": (lambda: {"xyz": _shell(), "radius": np.full(500, 1.5)}, dict(spacing=0.8)),
    # the grid moves with the atoms: a margin off the lattice keeps every node off rho = 1 exactly
    "two_blobs": (lambda: {"xyz": np.array([[-6.0, 0.0, 0.0], [6.0, 0.5, 0.0]]), "radius": np.array([2.0, 1.5])},
                  dict(spacing=0.5, margin=4.0123)),
    "atom": (lambda: {"xyz": np.zeros((1, 3)), "radius": np.array([2.0])}, dict(spacing=0.4, beta=0.8, margin=4.0123)),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_unsmoothed_mesh_matches_oracle(name):
    make, params = CASES[name]
    at = make()
    ref = OS.gaussian_surface(at["xyz"], at["radius"], smooth_iters=-1, **params)
    assert np.abs(ref["rho"] - 1.0).min() > 1e-10
    v, t, info = _gpu_surface(at["xyz"], at["radius"], smooth_iters=-1, **params)
    assert info["generated"] and info["rounds"] == 0
    assert info["grid"] == tuple(ref["shape"])
    assert info["raw_nv"] == ref["raw_verts"].shape[0] and info["raw_nt"] == ref["raw_tris"].shape[0]
    assert info["components"] == ref["components"]
    assert np.array_equal(t, ref["tris"])
    assert np.abs(v - ref["verts"]).max() <= 1e-9


@pytest.mark.parametrize("name", ["molecule200", "molecule200_fine_stern", "atom"])
def test_smoothed_mesh_matches_oracle(name):
    make, params = CASES[name]
    at = make()
    ref = OS.gaussian_surface(at["xyz"], at["radius"], **params)
    v, t, info = _gpu_surface(at["xyz"], at["radius"], **params)
    assert info["rounds"] == ref["rounds"]
    assert np.array_equal(t, ref["tris"])
    assert np.abs(v - ref["verts"]).max() <= 1e-8


def test_fold_fallback_uses_fewer_rounds():
    # a sharper density, full umbrella steps and tiny projections: the fifth round
    # folds more triangles than the unsmoothed mesh, so both sides keep four rounds
    at = synthetic_atoms(200, 9.0, seed=11)
    params = dict(spacing=1.6, beta=1.2, relax=1.0, newton_steps=1, max_step=0.02)
    ref = OS.gaussian_surface(at["xyz"], at["radius"], **params)
    assert ref["rounds"] == 4
    v, t, info = _gpu_surface(at["xyz"], at["radius"], **params)
    assert info["rounds"] == 4
    assert np.array_equal(t, ref["tris"]) and np.abs(v - ref["verts"]).max() <= 1e-8


def test_smoothing_kept_when_the_unsmoothed_mesh_already_folds():
    # ligand 60 of the 64-ligand fleet: marching tetrahedra folds 3 triangles, every
    # smoothing round leaves 1, so all five rounds are kept
    from synth.configs import PROTEIN_SPACING, fleet_atoms, fleet_sizes
    at = fleet_atoms(60, fleet_sizes(64)[60])
    ref = OS.gaussian_surface(at["xyz"], at["radius"], PROTEIN_SPACING)
    assert ref["rounds"] == 5
    v, t, info = _gpu_surface(at["xyz"], at["radius"], spacing=PROTEIN_SPACING)
    assert info["rounds"] == 5
    assert np.array_equal(t, ref["tris"]) and np.abs(v - ref["verts"]).max() <= 1e-8


def _ring(nbrs, c, depth):
    seen, front = {c}, [c]
    for _ in range(depth):
        front = [w for u in front for w in nbrs[u] if w not in seen]
        seen.update(front)
    return np.array(sorted(seen))


def test_full_size_protein_surface():
    # the 2,000-atom synthetic protein at 1.17 A: topology identical to the oracle's
    # unsmoothed mesh; smoothed vertices sampled against the oracle's smoothing of
    # their 5-ring neighbourhood (after r rounds only vertices r rings inside a
    # patch depend on nothing outside it); closed, no folds
    at = protein_atoms(2000, 2)
    ref = OS.gaussian_surface(at["xyz"], at["radius"], 1.17, smooth_iters=-1)
    assert np.abs(ref["rho"] - 1.0).min() > 1e-10
    v0, t, info = _gpu_surface(at["xyz"], at["radius"], spacing=1.17, smooth_iters=-1)
    assert np.array_equal(t, ref["tris"]) and np.abs(v0 - ref["verts"]).max() <= 1e-9
    v, t2, info = _gpu_surface(at["xyz"], at["radius"], spacing=1.17)
    assert np.array_equal(t2, t) and info["rounds"] == 5
    e = OS.neighbours(v.shape[0], ref["tris"])
    nbrs = np.split(e[:, 1], np.cumsum(np.bincount(e[:, 0], minlength=v.shape[0]))[:-1])
    p = dict(OS.DEFAULTS)
    for c in np.random.default_rng(0).choice(v.shape[0], 24, replace=False):
        ids = _ring(nbrs, c, 5)
        local = -np.ones(v.shape[0], dtype=np.int64)
        local[ids] = np.arange(ids.size)
        tr = ref["tris"][(local[ref["tris"]] >= 0).all(1)]
        sub_t = local[tr]
        sub_e = OS.neighbours(ids.size, sub_t)
        x = ref["verts"][ids]
        for _ in range(5):
            x = OS.smooth_round(x, sub_e, at["xyz"], at["radius"], p)
        assert np.abs(x[local[c]] - v[c]).max() <= 1e-8
    rho = OS.density(v[np.random.default_rng(1).choice(v.shape[0], 2000, replace=False)], at["xyz"], at["radius"],
                     0.5, 2.7)
    assert np.median(np.abs(rho - 1.0)) < 1e-12          # most vertices reach the level set exactly
    assert OS.folded(v, t, at["xyz"], at["radius"], OS.DEFAULTS) == 0
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    directed = set(map(tuple, e))
    assert len(directed) == e.shape[0] and all((b, a) in directed for a, b in directed)


def test_generated_surface_solves_like_the_uploaded_mesh():
    from paper_1309_4018_b300 import pbbem
    at = synthetic_atoms(200, 9.0, seed=11)
    ref = OS.gaussian_surface(at["xyz"], at["radius"], 1.0)
    regions = [{"eps": 4.0, "kappa": 0.0}, {"eps": 80.0, "kappa": 0.125}]
    charges = {"xyz": at["xyz"], "q": at["q"], "region": 0}
    up = {"regions": regions, "surfaces": [{"verts": ref["verts"], "tris": ref["tris"], "inner": 0, "outer": 1}],
          "charges": charges}
    gen = {"regions": regions, "charges": charges,
           "surfaces": [{"atoms": {"xyz": at["xyz"], "radius": at["radius"]}, "surf_params": {"spacing": 1.0},
                         "inner": 0, "outer": 1}]}
    e = []
    for d in (up, gen):
        pb = pbbem.Problem.from_dict(ctx(), d)
        pb.setup(precision="fp64", theta=0.5, P=6, ncrit=100, gmres_tol=1e-10)
        e.append(pb.solve().dG_solv)
        pb.close()
    assert abs(e[0] - e[1]) <= 1e-9 * abs(e[0])


def test_bad_inputs_are_clean_errors():
    from paper_1309_4018_b300 import pbbem
    at = synthetic_atoms(20, 4.0, seed=1)
    for kw, radius in ((dict(spacing=0.0), at["radius"]), (dict(spacing=1.0), -at["radius"]),
                       (dict(spacing=1.0, level=1e6), at["radius"]), (dict(spacing=1e-3), at["radius"]),
                       (dict(spacing=1.0, tclamp=0.6), at["radius"])):
        with pytest.raises(pbbem.PBError) as ei:
            _gpu_surface(at["xyz"], radius, **kw)
        assert ei.value.code == pbbem.PB_EINVAL
    # the context is still usable
    v, t, info = _gpu_surface(at["xyz"], at["radius"], spacing=1.0)
    assert t.shape[0] > 0


def test_sphere_problem_from_device_surface_matches_kirkwood():
    # a single 4 A atom at the origin: its smoothed surface is the r = 4 sphere
    from oracle.closed_forms import kirkwood_energy
    from paper_1309_4018_b300 import pbbem
    ch = sphere_problem(level=2, charges="both")["charges"]
    d = {"regions": [{"eps": 4.0, "kappa": 0.0}, {"eps": 80.0, "kappa": 0.125}], "charges": ch,
         "surfaces": [{"atoms": {"xyz": np.zeros((1, 3)), "radius": np.array([4.0])},
                       "surf_params": {"spacing": 0.35}, "inner": 0, "outer": 1}]}
    pb = pbbem.Problem.from_dict(ctx(), d)
    pb.setup(precision="fp64", theta=0.5, P=8, ncrit=100, gmres_tol=1e-8)
    r = pb.solve()
    ex = kirkwood_energy(4.0, 4.0, 80.0, 0.125, ch["xyz"], ch["q"])
    assert abs(r.dG_solv - ex) < 1e-2 * abs(ex)
    pb.close()


def test_mesh_tool_writes_the_device_mesh(tmp_path, capsys):
    from paper_1309_4018_b300 import mesh as M
    at = synthetic_atoms(60, 6.0, seed=5)
    p = tmp_path / "a.xyzr"
    np.savetxt(p, np.hstack([at["xyz"], at["radius"][:, None]]))
    M.main([str(p), "--spacing", "1.0", "--out", str(tmp_path / "m.npz")])
    z = np.load(tmp_path / "m.npz")
    ref = OS.gaussian_surface(*M.read_xyzr(str(p)), 1.0)
    assert np.array_equal(z["tris"], ref["tris"]) and np.abs(z["verts"] - ref["verts"]).max() <= 1e-8
    assert '"generated": true' in capsys.readouterr().out
