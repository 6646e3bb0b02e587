"""Mesh a molecule on the device: atoms -> Gaussian-density surface.

    python -m paper_1309_4018_b300.mesh atoms.xyzr --spacing 1.17 --out mesh.npz
    python -m paper_1309_4018_b300.mesh --synthetic 2000 --repeat 3

Input: an .xyzr file (one atom per line: x y z radius, Angstrom; the format
MSMS reads) or a seeded synthetic protein of N atoms.  The surface is built
by pb_add_gaussian_surface (every step on the GPU); the mesh is written as
.npz (verts float64 [nv, 3], tris int32 [nt, 3]) or .off, and the device
time of each generation is printed.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import pbbem


def read_xyzr(path):
    a = np.loadtxt(path, dtype=np.float64, ndmin=2)
    if a.shape[1] < 4:
        raise ValueError(f"{path}: expected x y z radius per line")
    return a[:, :3].copy(), a[:, 3].copy()


def write_mesh(path, verts, tris):
    if path.endswith(".off"):
        with open(path, "w") as f:
            f.write(f"OFF\n{verts.shape[0]} {tris.shape[0]} 0\n")
            np.savetxt(f, verts, fmt="%.17g")
            np.savetxt(f, np.hstack([np.full((tris.shape[0], 1), 3), tris]), fmt="%d")
    else:
        np.savez(path, verts=verts, tris=tris)


def mesh(ctx, xyz, radius, **params):
    """(verts, tris, info) of the device surface of the atoms (params: pb_surf_params fields)."""
    pb = pbbem.Problem(ctx)
    try:
        pb.add_region(1.0, 0.0)
        pb.add_region(1.0, 0.0)
        sid = pb.add_gaussian_surface(xyz, radius, 0, 1, **params)
        v, t = pb.surface_mesh(sid)
        return v, t, pb.surface_info(sid)
    finally:
        pb.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("xyzr", nargs="?", help="atoms file (x y z radius per line)")
    ap.add_argument("--synthetic", type=int, default=0, help="mesh the seeded synthetic protein of N atoms")
    ap.add_argument("--spacing", type=float, default=1.17)
    ap.add_argument("--radius-offset", type=float, default=0.0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--out", default="")
    a = ap.parse_args(argv)
    if a.synthetic:
        from synth.configs import protein_atoms
        at = protein_atoms(a.synthetic, 2)
        xyz, radius = at["xyz"], at["radius"]
    elif a.xyzr:
        xyz, radius = read_xyzr(a.xyzr)
    else:
        ap.error("give an .xyzr file or --synthetic N")
    ctx = pbbem.Context(a.device)
    for _ in range(max(1, a.repeat)):
        v, t, info = mesh(ctx, xyz, radius, spacing=a.spacing, radius_offset=a.radius_offset)
        print(json.dumps(info))
    if a.out:
        write_mesh(a.out, v, t)
    ctx.close()


if __name__ == "__main__":
    main()
