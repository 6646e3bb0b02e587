"""Problem descriptions for the synthetic workloads.

A problem is a plain dict of input data:

    {"regions":  [{"eps": float, "kappa": float}, ...],
     "surfaces": [{"verts": f64[nv,3], "tris": i32[nt,3], "inner": int, "outer": int}, ...],
     "charges":  {"xyz": f64[nc,3], "q": f64[nc], "region": int}}

Triangles are wound counter-clockwise seen from the surface's outer region.
Nothing here evaluates the method; the oracle and the CUDA library both read
these dicts.
"""
from __future__ import annotations

import functools

import numpy as np

from .meshes import icosphere, octasphere
from .molecule import gaussian_surface, synthetic_atoms

EPS_IN, EPS_OUT, KAPPA = 4.0, 80.0, 0.125


def sphere_problem(level=4, radius=4.0, charges="both", eps_in=EPS_IN, eps_out=EPS_OUT,
                   kappa=KAPPA, mesh="octa"):
    """Kirkwood sphere: one surface, charges at the centre and/or 2 A off-centre.

    level 4 octasphere = 2,048 panels (level 3: 512, level 5: 8,192).
    """
    v, t = (octasphere if mesh == "octa" else icosphere)(level, radius)
    xyz = {"centre": [[0.0, 0.0, 0.0]], "off": [[2.0, 0.0, 0.0]],
           "both": [[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]]}[charges]
    xyz = np.array(xyz, dtype=np.float64)
    return {
        "regions": [{"eps": eps_in, "kappa": 0.0}, {"eps": eps_out, "kappa": kappa}],
        "surfaces": [{"verts": v, "tris": t, "inner": 0, "outer": 1}],
        "charges": {"xyz": xyz, "q": np.ones(xyz.shape[0]), "region": 0},
    }


def layered_sphere_problem(level=3, a=4.0, b=6.0, stern_level=None, eps=(4.0, 80.0, 80.0),
                           kappa=(0.0, 0.0, 0.125), charges="both"):
    """Sphere with a concentric Stern layer: protein | Stern (r<b) | solvent."""
    v1, t1 = octasphere(level, a)
    v2, t2 = octasphere(stern_level if stern_level is not None else level, b)
    xyz = {"centre": [[0.0, 0.0, 0.0]], "off": [[2.0, 0.0, 0.0]],
           "both": [[0.0, 0.0, 0.0], [2.0, 0.0, 0.0]]}[charges]
    xyz = np.array(xyz, dtype=np.float64)
    return {
        "regions": [{"eps": eps[i], "kappa": kappa[i]} for i in range(3)],
        "surfaces": [{"verts": v1, "tris": t1, "inner": 0, "outer": 1},
                     {"verts": v2, "tris": t2, "inner": 1, "outer": 2}],
        "charges": {"xyz": xyz, "q": np.ones(xyz.shape[0]), "region": 0},
    }


def cavity_sphere_problem(level=3, eps_cav=80.0, cavity_coarsening=1):
    """Cavity r < 1.5 | protein shell to 4 | Stern to 6 | solvent, charge at 2.5 A.

    The cavity sphere is meshed `cavity_coarsening` octasphere levels below the
    two outer spheres (0: the same level, as a refinement study needs)."""
    vc, tc = octasphere(max(level - cavity_coarsening, 1), 1.5)
    v1, t1 = octasphere(level, 4.0)
    v2, t2 = octasphere(level, 6.0)
    return {
        "regions": [{"eps": eps_cav, "kappa": 0.0}, {"eps": 4.0, "kappa": 0.0},
                    {"eps": 80.0, "kappa": 0.0}, {"eps": 80.0, "kappa": 0.125}],
        "surfaces": [{"verts": vc, "tris": tc, "inner": 0, "outer": 1},
                     {"verts": v1, "tris": t1, "inner": 1, "outer": 2},
                     {"verts": v2, "tris": t2, "inner": 2, "outer": 3}],
        "charges": {"xyz": np.array([[2.5, 0.0, 0.0]]), "q": np.ones(1), "region": 1},
    }


# Grid spacings (A) of the marching-tetrahedra mesher that give the stated
# panel counts for the seeded molecules below.
PROTEIN_SPACING = 1.17      # ~40k panels for the 2,000-atom seed-2 molecule
STERN_SPACING = 1.16        # ~60k panels for the +2 A Stern surface of the seed-3 molecule


@functools.lru_cache(maxsize=8)
def protein_atoms(n_atoms=2000, seed=2, cavities=False, cavity_x=7.0, cavity_r=3.0):
    """Atoms of a synthetic protein; with `cavities`, atom centres keep
    cavity_r + 2.0 + 1.4 A away from (+-cavity_x, 0, 0) to leave room for two
    solvent-filled cavities of radius cavity_r."""
    radius = 20.0 * (n_atoms / 2000.0) ** (1.0 / 3.0)
    exclude = ()
    if cavities:
        gap = cavity_r + 2.0 + 1.4
        exclude = (((cavity_x, 0.0, 0.0), gap), ((-cavity_x, 0.0, 0.0), gap))
    return synthetic_atoms(n_atoms, radius, seed, exclude=exclude)


def protein_problem(n_atoms=2000, seed=2, spacing=PROTEIN_SPACING):
    """Synthetic globular protein, single dielectric interface (~40k panels)."""
    at = protein_atoms(n_atoms, seed)
    v, t = gaussian_surface(at["xyz"], at["radius"], spacing)
    return {
        "regions": [{"eps": EPS_IN, "kappa": 0.0}, {"eps": EPS_OUT, "kappa": KAPPA}],
        "surfaces": [{"verts": v, "tris": t, "inner": 0, "outer": 1}],
        "charges": {"xyz": at["xyz"].copy(), "q": at["q"].copy(), "region": 0},
    }


def multisurface_problem(n_atoms=2000, seed=3, spacing=PROTEIN_SPACING,
                         stern_spacing=STERN_SPACING, cavity_level=3, cavity_x=7.0, cavity_r=3.0):
    """Protein SES + Stern surface (+2 A) + two solvent-filled cavities of
    radius cavity_r at (+-cavity_x, 0, 0) (3 A at +-7 A for the 2,000-atom molecule).

    Regions: 0 cav1, 1 cav2, 2 protein (charged), 3 Stern (eps_out, kappa 0),
    4 solvent (eps_out, kappa).  Surfaces: C1, C2, SES, Stern.
    """
    at = protein_atoms(n_atoms, seed, cavities=True, cavity_x=cavity_x, cavity_r=cavity_r)
    vs, ts = gaussian_surface(at["xyz"], at["radius"], spacing)
    vt, tt = gaussian_surface(at["xyz"], at["radius"], stern_spacing, radius_offset=2.0)
    c1v, c1t = icosphere(cavity_level, cavity_r, (cavity_x, 0.0, 0.0))
    c2v, c2t = icosphere(cavity_level, cavity_r, (-cavity_x, 0.0, 0.0))
    return {
        "regions": [{"eps": EPS_OUT, "kappa": 0.0}, {"eps": EPS_OUT, "kappa": 0.0},
                    {"eps": EPS_IN, "kappa": 0.0}, {"eps": EPS_OUT, "kappa": 0.0},
                    {"eps": EPS_OUT, "kappa": KAPPA}],
        "surfaces": [{"verts": c1v, "tris": c1t, "inner": 0, "outer": 2},
                     {"verts": c2v, "tris": c2t, "inner": 1, "outer": 2},
                     {"verts": vs, "tris": ts, "inner": 2, "outer": 3},
                     {"verts": vt, "tris": tt, "inner": 3, "outer": 4}],
        "charges": {"xyz": at["xyz"].copy(), "q": at["q"].copy(), "region": 2},
    }


def panel_count(problem):
    return sum(int(np.asarray(s["tris"]).shape[0]) for s in problem["surfaces"])


def _ball_radius(n_atoms):
    return 20.0 * (n_atoms / 2000.0) ** (1.0 / 3.0)


def place_ligand(rec_xyz, lig_xyz, gap=3.0, direction=(1.0, 0.0, 0.0)):
    """Translate the ligand along `direction` until its closest atom centre is `gap` A from the receptor's."""
    from scipy.spatial import cKDTree
    tree = cKDTree(rec_xyz)
    u = np.asarray(direction, dtype=np.float64)
    u = u / np.linalg.norm(u)
    lo, hi = 0.0, float(np.ptp(rec_xyz, axis=0).max() + np.ptp(lig_xyz, axis=0).max() + 2 * gap)

    def dmin(t):
        return float(tree.query(lig_xyz + t * u)[0].min())

    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if dmin(mid) < gap:
            lo = mid
        else:
            hi = mid
    return lig_xyz + hi * u


def _molecule_problem(xyz, radius, q, spacing):
    v, t = gaussian_surface(xyz, radius, spacing)
    return {
        "regions": [{"eps": EPS_IN, "kappa": 0.0}, {"eps": EPS_OUT, "kappa": KAPPA}],
        "surfaces": [{"verts": v, "tris": t, "inner": 0, "outer": 1}],
        "charges": {"xyz": np.array(xyz, dtype=np.float64), "q": np.array(q, dtype=np.float64), "region": 0},
    }


def binding_triplet(n_rec=8000, n_lig=1500, seed=4, spacing=PROTEIN_SPACING, gap=3.0):
    """Receptor, ligand and complex of a synthetic binding pair (Eq. bind_energy).

    Receptor and ligand atoms are drawn like protein_atoms (ball radius
    20 (N/2000)^(1/3) A, seeds `seed` and `seed` + 1); the ligand is moved
    along +x until its closest atom centre is `gap` A from the receptor's.
    The complex is the union of both atom sets (its own Gaussian surface).
    Returns (complex, receptor, ligand) problem dicts.
    """
    rec = synthetic_atoms(n_rec, _ball_radius(n_rec), seed)
    lig = synthetic_atoms(n_lig, _ball_radius(n_lig), seed + 1)
    lxyz = place_ligand(rec["xyz"], lig["xyz"], gap)
    cx_xyz = np.vstack([rec["xyz"], lxyz])
    cx_r = np.concatenate([rec["radius"], lig["radius"]])
    cx_q = np.concatenate([rec["q"], lig["q"]])
    return (_molecule_problem(cx_xyz, cx_r, cx_q, spacing),
            _molecule_problem(rec["xyz"], rec["radius"], rec["q"], spacing),
            _molecule_problem(lxyz, lig["radius"], lig["q"], spacing))


def fleet_sizes(count=64, n_min=300, n_max=3000, seed=4):
    """Atom counts of a ligand fleet: log-uniform in [n_min, n_max]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return [int(n) for n in np.exp(rng.uniform(np.log(n_min), np.log(n_max), size=count)).astype(int)]


def fleet_atoms(i, n_atoms, seed=4):
    """Atoms of ligand i of a fleet: n_atoms atoms drawn with seed + 1 + i."""
    return synthetic_atoms(int(n_atoms), _ball_radius(int(n_atoms)), seed + 1 + i)


def molecule_problem(xyz, radius, q, spacing=PROTEIN_SPACING):
    """One molecule (charges in eps 4, solvent eps 80 / kappa 0.125) meshed on the CPU."""
    return _molecule_problem(xyz, radius, q, spacing)


def fleet_ligand(i, n_atoms, seed=4, spacing=PROTEIN_SPACING):
    """Ligand i of a fleet: n_atoms atoms drawn with seed + 1 + i."""
    at = fleet_atoms(i, n_atoms, seed)
    return _molecule_problem(at["xyz"], at["radius"], at["q"], spacing)


def ligand_fleet(count=64, n_min=300, n_max=3000, seed=4, spacing=PROTEIN_SPACING):
    """`count` synthetic ligands with atom counts log-uniform in [n_min, n_max] (seed + 1 + i each)."""
    return [fleet_ligand(i, n, seed, spacing) for i, n in enumerate(fleet_sizes(count, n_min, n_max, seed))]


def protein_refinements(levels=2, spacing=2.0 * PROTEIN_SPACING, n_atoms=2000, seed=2):
    """The synthetic protein on nested meshes: its surface at `spacing`, then
    `levels` refinements that split every panel into four on the same level set
    (panel area / 4 per level).  Returns problem dicts, coarsest first."""
    from .molecule import refine_on_level_set
    at = protein_atoms(n_atoms, seed)
    base = protein_problem(n_atoms, seed, spacing)
    s = base["surfaces"][0]
    out = [base]
    for v, t in refine_on_level_set(s["verts"], s["tris"], at["xyz"], at["radius"], levels):
        d = dict(base)
        d["surfaces"] = [dict(s, verts=v, tris=t)]
        out.append(d)
    return out


def model_variants(n_atoms=2000, seed=3, spacing=PROTEIN_SPACING, stern_spacing=STERN_SPACING, cavity_level=3,
                   cavity_x=7.0, cavity_r=3.0):
    """The four solvent models of the multi-surface molecule (the paper's Single /
    Cavity / Stern / Full comparison) on the same atoms and meshes:
    single: molecular surface only; cavity: + the two solvent-filled cavities;
    stern: + the Stern layer; full: all four surfaces (= multisurface_problem)."""
    full = multisurface_problem(n_atoms, seed, spacing, stern_spacing, cavity_level, cavity_x, cavity_r)
    c1, c2, ses, stern = full["surfaces"]
    ch = full["charges"]
    ew, eo, kap = EPS_OUT, EPS_IN, KAPPA

    def mk(regions, surfaces, creg):
        return {"regions": regions, "surfaces": surfaces, "charges": dict(ch, region=creg)}

    single = mk([{"eps": eo, "kappa": 0.0}, {"eps": ew, "kappa": kap}],
                [dict(ses, inner=0, outer=1)], 0)
    cavity = mk([{"eps": ew, "kappa": 0.0}, {"eps": ew, "kappa": 0.0}, {"eps": eo, "kappa": 0.0},
                 {"eps": ew, "kappa": kap}],
                [dict(c1, inner=0, outer=2), dict(c2, inner=1, outer=2), dict(ses, inner=2, outer=3)], 2)
    stern_m = mk([{"eps": eo, "kappa": 0.0}, {"eps": ew, "kappa": 0.0}, {"eps": ew, "kappa": kap}],
                 [dict(ses, inner=0, outer=1), dict(stern, inner=1, outer=2)], 0)
    return {"single": single, "cavity": cavity, "stern": stern_m, "full": full}



# Reduced multi-surface molecule, small enough for the dense oracle to solve
# its four model variants on host cores in minutes: 400 atoms (ball radius
# 11.7 A), two 2 A cavities at (+-4.5, 0, 0) meshed as 320-panel icospheres,
# SES and Stern surface on a 1.4 A grid (10,324 + 19,568 + 2 x 320 panels).
REDUCED_MULTISURFACE = dict(n_atoms=400, seed=3, spacing=1.4, stern_spacing=1.4, cavity_level=2,
                            cavity_x=4.5, cavity_r=2.0)


def reduced_model_variants():
    return model_variants(**REDUCED_MULTISURFACE)


def large_protein_problem(n_atoms=30000, seed=2, spacing=0.8):
    """A 30,000-atom seeded globule (drawn like protein_atoms: ball radius
    20 (N/2000)^(1/3) = 49 A) whose surface the device mesher builds from the
    atoms (~480k panels at 0.8 A)."""
    at = protein_atoms(n_atoms, seed)
    return {
        "regions": [{"eps": EPS_IN, "kappa": 0.0}, {"eps": EPS_OUT, "kappa": KAPPA}],
        "surfaces": [{"atoms": {"xyz": at["xyz"], "radius": at["radius"]}, "surf_params": {"spacing": spacing},
                      "inner": 0, "outer": 1}],
        "charges": {"xyz": at["xyz"].copy(), "q": at["q"].copy(), "region": 0},
    }
