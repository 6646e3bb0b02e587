"""Seeded synthetic molecules and their Gaussian-density surfaces.

A synthetic "protein" is a set of atoms placed uniformly in a ball with a
minimum pair distance, with radii and partial charges drawn from a seeded
generator.  Its molecular surface is the level set rho(x) = 1 of the Gaussian
density rho(x) = sum_a exp(-beta (|x - x_a|^2 / R_a^2 - 1)), triangulated by
marching tetrahedra on a uniform grid (a Kuhn split of every grid cube into six
tetrahedra, which has no ambiguous cases and gives a closed, consistently
oriented surface).  Only the outer connected component is kept.  A few rounds
of Laplacian vertex smoothing, each followed by a Newton projection back onto
the level set, even out the thin triangles marching tetrahedra leaves.

beta = 0.5 gives a smooth, solvent-excluded-like envelope (the probe-rolled
surface of a protein has no atom-scale crevices); sharper densities
(beta ~ 2.3) give folded van der Waals-like surfaces whose panels nearly touch,
where the K-point integration of the boundary operator breaks down.

This module produces inputs only; it holds none of the boundary-element
arithmetic, and both the oracle and the CUDA path read its output.
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

BETA = 0.5
CUTOFF = 2.7        # an atom contributes to rho within CUTOFF * R_a


def synthetic_atoms(n_atoms: int, ball_radius: float, seed: int,
                    min_dist: float = 1.0, exclude=()):
    """Atoms uniform in a ball, pair distance >= min_dist, by rejection.

    exclude: iterable of (center(3), radius) balls that atom centres avoid.
    Returns dict(xyz [n,3] f64, radius [n] f64, q [n] f64) with net charge 0.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = np.empty((0, 3))
    exclude = [(np.asarray(c, dtype=np.float64), float(r)) for c, r in exclude]
    while pts.shape[0] < n_atoms:
        cand = rng.uniform(-ball_radius, ball_radius, size=(4 * n_atoms, 3))
        cand = cand[(cand * cand).sum(1) <= ball_radius * ball_radius]
        for c, r in exclude:
            cand = cand[((cand - c) ** 2).sum(1) > r * r]
        for p in cand:
            if pts.shape[0] >= n_atoms:
                break
            if pts.shape[0]:
                d2 = ((pts - p) ** 2).sum(1)
                if d2.min() < min_dist * min_dist:
                    continue
            pts = np.vstack([pts, p[None]])
    radius = rng.uniform(1.2, 2.0, size=n_atoms)
    q = rng.normal(0.0, 0.4, size=n_atoms)
    q = q - q.mean()
    return {"xyz": pts, "radius": radius, "q": q}


def _density_grid(xyz, radius, lo, h, shape, beta=BETA, cutoff=CUTOFF):
    """rho on grid nodes lo + h*(i,j,k); each atom contributes within cutoff*R."""
    rho = np.zeros(shape, dtype=np.float64)
    axes = [lo[d] + h * np.arange(shape[d]) for d in range(3)]
    for p, r in zip(xyz, radius):
        rc = cutoff * r
        i0 = [max(0, int(np.floor((p[d] - rc - lo[d]) / h))) for d in range(3)]
        i1 = [min(shape[d], int(np.ceil((p[d] + rc - lo[d]) / h)) + 1) for d in range(3)]
        gx = axes[0][i0[0]:i1[0]] - p[0]
        gy = axes[1][i0[1]:i1[1]] - p[1]
        gz = axes[2][i0[2]:i1[2]] - p[2]
        d2 = gx[:, None, None] ** 2 + gy[None, :, None] ** 2 + gz[None, None, :] ** 2
        contrib = np.exp(-beta * (d2 / (r * r) - 1.0))
        contrib[d2 > rc * rc] = 0.0
        rho[i0[0]:i1[0], i0[1]:i1[1], i0[2]:i1[2]] += contrib
    return rho


# Kuhn split of the unit cube into 6 tetrahedra along the (0,0,0)-(1,1,1) diagonal.
_CUBE_CORNERS = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0],
                          [0, 0, 1], [1, 0, 1], [0, 1, 1], [1, 1, 1]])
_KUHN = np.array([[0, 1, 3, 7], [0, 3, 2, 7], [0, 2, 6, 7],
                  [0, 6, 4, 7], [0, 4, 5, 7], [0, 5, 1, 7]])


def marching_tetrahedra(field: np.ndarray, lo, h, level: float = 1.0,
                        tclamp: float = 0.02):
    """Triangulate {field > level} boundary; normals point to field < level."""
    nx, ny, nz = field.shape
    f = field - level
    f[f == 0.0] = 1e-12
    ci, cj, ck = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1),
                             indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    # keep only cubes whose corners straddle the level
    corner_ids = []
    for c in _CUBE_CORNERS:
        corner_ids.append(((ci + c[0]) * ny + (cj + c[1])) * nz + (ck + c[2]))
    corner_ids = np.stack(corner_ids, axis=1)            # [ncube, 8]
    fv = f.ravel()[corner_ids]
    inside = fv > 0
    mixed = inside.any(1) & ~inside.all(1)
    corner_ids, fv, inside = corner_ids[mixed], fv[mixed], inside[mixed]

    tet_ids = corner_ids[:, _KUHN].reshape(-1, 4)        # [ntet, 4] node ids
    tet_f = fv[:, _KUHN].reshape(-1, 4)
    tet_in = inside[:, _KUHN].reshape(-1, 4)
    nin = tet_in.sum(1)
    keep = (nin > 0) & (nin < 4)
    tet_ids, tet_f, tet_in, nin = tet_ids[keep], tet_f[keep], tet_in[keep], nin[keep]

    node_xyz = lambda ids: np.stack(np.unravel_index(ids, (nx, ny, nz)), axis=1) * h + lo

    # every triangle vertex is a grid edge (inside node, outside node); vertices
    # shared by neighbouring tetrahedra are merged by their edge key
    tri_a, tri_b = [], []
    order = np.argsort(~tet_in, axis=1, kind="stable")   # inside nodes first
    ids_s = np.take_along_axis(tet_ids, order, 1)
    for nI in (1, 2, 3):
        ids = ids_s[nin == nI]
        if ids.shape[0] == 0:
            continue
        ins, outs = ids[:, :nI], ids[:, nI:]
        if nI == 1:
            tri_a.append(np.stack([ins[:, 0]] * 3, 1)); tri_b.append(outs[:, :3])
        elif nI == 3:
            tri_a.append(ins[:, :3]); tri_b.append(np.stack([outs[:, 0]] * 3, 1))
        else:
            p = (ins[:, 0], outs[:, 0]); q = (ins[:, 0], outs[:, 1])
            r = (ins[:, 1], outs[:, 1]); s = (ins[:, 1], outs[:, 0])
            tri_a.append(np.stack([p[0], q[0], r[0]], 1)); tri_b.append(np.stack([p[1], q[1], r[1]], 1))
            tri_a.append(np.stack([p[0], r[0], s[0]], 1)); tri_b.append(np.stack([p[1], r[1], s[1]], 1))
    tri_a = np.concatenate(tri_a); tri_b = np.concatenate(tri_b)
    nn = nx * ny * nz
    keys = np.minimum(tri_a, tri_b) * nn + np.maximum(tri_a, tri_b)
    ukeys, inv = np.unique(keys.ravel(), return_inverse=True)
    tris = inv.reshape(-1, 3)
    ek = np.stack([ukeys // nn, ukeys % nn], 1)
    fa, fb = f.ravel()[ek[:, 0]], f.ravel()[ek[:, 1]]
    t = np.clip(fa / (fa - fb), tclamp, 1.0 - tclamp)
    pa, pb = node_xyz(ek[:, 0]), node_xyz(ek[:, 1])
    verts = pa + t[:, None] * (pb - pa)

    # orient: normal must point from the inside node of an edge to its outside node
    v0, v1, v2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    e0 = ek[tris[:, 0]]
    ins_node = np.where(fa[tris[:, 0]] > 0, e0[:, 0], e0[:, 1])
    out_node = np.where(fa[tris[:, 0]] > 0, e0[:, 1], e0[:, 0])
    direc = node_xyz(out_node) - node_xyz(ins_node)
    flip = np.einsum("ij,ij->i", nrm, direc) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts, tris


def outer_component(verts, tris):
    """Keep the connected component holding the vertex of largest x."""
    nv = verts.shape[0]
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]]])
    g = coo_matrix((np.ones(e.shape[0]), (e[:, 0], e[:, 1])), shape=(nv, nv))
    _, lab = connected_components(g, directed=False)
    used = np.zeros(nv, bool)
    used[tris.ravel()] = True
    cand = np.where(used)[0]
    top = cand[np.argmax(verts[cand, 0])]
    keep_t = lab[tris[:, 0]] == lab[top]
    tris = tris[keep_t]
    used = np.zeros(nv, bool)
    used[tris.ravel()] = True
    remap = -np.ones(nv, dtype=np.int64)
    remap[used] = np.arange(used.sum())
    return verts[used], remap[tris]


def density_and_gradient(p, xyz, radius, beta=BETA, cutoff=CUTOFF, tree=None):
    """rho and grad rho at points p [m,3] (same truncation as the grid)."""
    p = np.asarray(p, dtype=np.float64)
    tree = tree if tree is not None else cKDTree(xyz)
    lists = tree.query_ball_point(p, cutoff * float(np.max(radius)))
    cnt = np.array([len(l) for l in lists])
    vi = np.repeat(np.arange(p.shape[0]), cnt)
    ai = np.concatenate([np.asarray(l, dtype=np.int64) for l in lists]) if cnt.sum() else np.zeros(0, np.int64)
    d = p[vi] - xyz[ai]
    d2 = (d * d).sum(1)
    R2 = radius[ai] ** 2
    e = np.exp(-beta * (d2 / R2 - 1.0))
    e[d2 > (cutoff * cutoff) * R2] = 0.0
    rho = np.bincount(vi, weights=e, minlength=p.shape[0])
    g = np.stack([np.bincount(vi, weights=e * (-2.0 * beta) * d[:, k] / R2, minlength=p.shape[0])
                  for k in range(3)], 1)
    return rho, g


def smooth_on_level_set(verts, tris, xyz, radius, beta=BETA, iters=5, relax=0.5, level=1.0):
    """Laplacian smoothing of the vertices, each round projected back onto rho = level."""
    v = np.array(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    nv = v.shape[0]
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    e = np.concatenate([e, e[:, ::-1]])
    e = np.unique(e, axis=0)
    deg = np.bincount(e[:, 0], minlength=nv).astype(np.float64)
    tree = cKDTree(xyz)
    for _ in range(iters):
        avg = np.stack([np.bincount(e[:, 0], weights=v[e[:, 1], k], minlength=nv) for k in range(3)], 1)
        v = v + relax * (avg / deg[:, None] - v)
        for _ in range(3):
            f, g = density_and_gradient(v, xyz, radius, beta, tree=tree)
            g2 = (g * g).sum(1)
            step = np.where(g2 > 1e-12, (f - level) / np.maximum(g2, 1e-12), 0.0)
            dv = step[:, None] * g
            n = np.sqrt((dv * dv).sum(1))
            dv *= np.minimum(1.0, 0.3 / np.maximum(n, 1e-30))[:, None]
            v = v - dv
    return v


def gaussian_surface(xyz, radius, spacing: float, radius_offset: float = 0.0,
                     beta: float = BETA, margin: float = 4.0, smooth_iters: int = 5):
    """Closed outward-oriented triangulation of the level set rho = 1.

    radius_offset enlarges every atomic radius (a Stern surface uses +2 A).
    Returns (verts f64 [nv,3], tris int32 [nt,3]).
    """
    r = np.asarray(radius, dtype=np.float64) + radius_offset
    lo = xyz.min(0) - r.max() - margin
    hi = xyz.max(0) + r.max() + margin
    shape = tuple(int(np.ceil((hi[d] - lo[d]) / spacing)) + 1 for d in range(3))
    rho = _density_grid(xyz, r, lo, spacing, shape, beta=beta)
    v, t = marching_tetrahedra(rho, lo, spacing)
    v, t = outer_component(v, t)
    # smoothing must not fold a triangle over (outward normals still point down
    # the density); where it would, fewer rounds are used, down to none
    for it in range(smooth_iters, 0, -1):
        vs = smooth_on_level_set(v, t, xyz, r, beta=beta, iters=it)
        a, b, c = vs[t[:, 0]], vs[t[:, 1]], vs[t[:, 2]]
        nrm = np.cross(b - a, c - a)
        _, g = density_and_gradient((a + b + c) / 3.0, xyz, r, beta)
        if not np.any(np.einsum("ij,ij->i", nrm, g) >= 0.0):
            return vs, t.astype(np.int32)
    return v, t.astype(np.int32)


def _split4(verts, tris):
    """Split every triangle into four at its edge midpoints (shared midpoints, winding kept)."""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    key = np.minimum(e[:, 0], e[:, 1]) * v.shape[0] + np.maximum(e[:, 0], e[:, 1])
    uk, inv = np.unique(key, return_inverse=True)
    a, b = uk // v.shape[0], uk % v.shape[0]
    mid = 0.5 * (v[a] + v[b])
    m = v.shape[0] + inv.reshape(3, -1).T          # midpoint index of edges (01, 12, 20) per triangle
    nv = np.vstack([v, mid])
    t0, t1, t2 = t[:, 0], t[:, 1], t[:, 2]
    m01, m12, m20 = m[:, 0], m[:, 1], m[:, 2]
    nt = np.concatenate([np.stack([t0, m01, m20], 1), np.stack([t1, m12, m01], 1),
                         np.stack([t2, m20, m12], 1), np.stack([m01, m12, m20], 1)])
    return nv, nt


def refine_on_level_set(verts, tris, xyz, radius, levels=1, radius_offset=0.0, beta=BETA, level=1.0):
    """Nested refinements of a level-set mesh: each level splits every triangle
    into four and moves the new vertices onto rho = level (Newton steps along
    grad rho), so the panel area shrinks by 4 per level on the same surface.
    Returns [(verts, tris int32)] for levels 1..levels.
    """
    r = np.asarray(radius, dtype=np.float64) + radius_offset
    tree = cKDTree(xyz)
    out = []
    v, t = np.asarray(verts, dtype=np.float64), np.asarray(tris, dtype=np.int64)
    for _ in range(levels):
        n_old = v.shape[0]
        v, t = _split4(v, t)
        p = v[n_old:]
        for _ in range(6):
            f, g = density_and_gradient(p, xyz, r, beta, tree=tree)
            g2 = (g * g).sum(1)
            step = np.where(g2 > 1e-12, (f - level) / np.maximum(g2, 1e-12), 0.0)
            dv = step[:, None] * g
            n = np.sqrt((dv * dv).sum(1))
            dv *= np.minimum(1.0, 0.3 / np.maximum(n, 1e-30))[:, None]
            p = p - dv
        v = np.vstack([v[:n_old], p])
        out.append((v.copy(), t.astype(np.int32)))
    return out
