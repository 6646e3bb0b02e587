"""Gaussian-density molecular surface (oracle of the device surface generator).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper meshes the solvent-excluded surface with MSMS (Sec. 2.2, Sec. 3);
this library builds instead the level set rho(x) = level of a Gaussian
density of the atoms,

    rho(x) = sum_a [ |x - x_a| <= cutoff R_a ]  exp(-beta (|x - x_a|^2 / R_a^2 - 1)),

with R_a the atomic radius plus an optional offset (a Stern layer takes +2 A).
The steps, written here in their plainest form:

1. Grid.  lo = min_a x_a - max_a R_a - margin (per axis), hi likewise with max
   and +; n_d = ceil((hi_d - lo_d) / h) + 1 nodes per axis, node (i, j, k) at
   lo + h (i, j, k), linear id (i n_y + j) n_z + k.  rho is summed at every node.
2. Inside test.  A node is inside when rho >= level.
3. Marching tetrahedra.  Every grid cube is split into six tetrahedra along
   its (0,0,0)-(1,1,1) diagonal (Kuhn / Freudenthal split: one tetrahedron per
   monotone corner path).  Every tetrahedron edge joins two nodes of which one
   is reached from the other by a positive step in a subset of the axes, so an
   edge is (lower node p, upper node q > p).  A surface vertex sits on every
   edge whose two nodes differ in the inside test, at
       t = f_p / (f_p - f_q),  f = rho - level,  t clamped to [tclamp, 1 - tclamp],
       v = x_p + t (x_q - x_p);
   vertices are numbered by ascending (p, q), so the vertex of an edge shared
   by several tetrahedra is one vertex.  A tetrahedron with one node on one side
   gives one triangle, with two on each side a quadrilateral cut into two
   triangles.  Without the clamp the triangles are exactly the level set of the
   piecewise-linear interpolant of rho on the tetrahedra.
4. Orientation, by integer logic alone.  The six tetrahedra are listed with a
   positive orientation (det[w1-w0, w2-w0, w3-w0] > 0).  For an even
   permutation (a, b, c, d) of a positively oriented tetrahedron, the triangle
   through the edges ab, ac, ad has its normal pointing away from a; so with
   a the lone inside node the triangle is (ab, ac, ad), with a the lone
   outside node it is (ab, ad, ac); with a, b inside and c, d outside the
   quadrilateral is (ac, ad, bd) + (ac, bd, bc).  Every normal then points from
   the inside (rho >= level) to the outside, i.e. into the outer region.
   Triangles are listed by cube (ascending lower-corner node id), then
   tetrahedron, then the order above.
5. Outer component.  Triangles sharing a vertex are connected; the component
   holding the vertex of largest (p, q), i.e. the last vertex, is kept: its
   lower node has the largest x index of any crossing, and every node beyond
   that x index is outside, so that vertex borders the exterior.  Kept
   vertices are renumbered in ascending order.
6. Smoothing (rounds r = 1 .. R).  Each round moves every vertex a fraction
   relax towards the mean of its edge neighbours, then takes newton_steps
   projections onto rho = level along grad rho (step (rho - level) / |grad|^2,
   zero where |grad|^2 <= 1e-12, capped at max_step in length).  A triangle is
   folded when its normal has a non-negative dot product with grad rho at its
   centroid; a round count is acceptable when it leaves no more folded
   triangles than the unsmoothed mesh has (marching tetrahedra itself can fold
   a few where a quadrilateral is cut along the diagonal the grid fixes).  The
   largest acceptable count <= R is used, none when no count is.

Parity status: pinned (tests/test_oracle_surface.py): the triangles of a random
cube lie on the piecewise-linear level set computed by Freudenthal's formula,
the corner-cut cube gives three exact squares, a single atom gives a closed
genus-0 sphere of radius R (h^2 convergence unsmoothed, on the sphere to 1e-9
smoothed), the outer surface of a hollow shell of atoms is kept and its cavity
dropped, of two separate blobs the one of larger x is kept, and the vertex set equals that of the independent mesher the
synthetic inputs use.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

DEFAULTS = dict(beta=0.5, cutoff=2.7, radius_offset=0.0, margin=4.0, level=1.0, tclamp=0.02,
                relax=0.5, max_step=0.3, smooth_iters=5, newton_steps=3)

# Cube corners: bit 0 = +x, bit 1 = +y, bit 2 = +z.
CORNER = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)])
# The six Kuhn tetrahedra (monotone corner paths 0 -> e_a -> e_a + e_b -> 7),
# each listed with a positive orientation: paths of even axis permutations as
# they are, odd ones with their last two corners exchanged.
TETS = [(0, 1, 3, 7), (0, 1, 7, 5), (0, 2, 7, 3), (0, 2, 6, 7), (0, 4, 5, 7), (0, 4, 7, 6)]
# even permutation of (0,1,2,3) that starts with a given vertex
EVEN_FROM = {0: (0, 1, 2, 3), 1: (1, 0, 3, 2), 2: (2, 3, 0, 1), 3: (3, 2, 1, 0)}


def _even_pair_split(ins):
    """(a, b, c, d) even permutation with {a, b} = ins (a < b) and c, d the others."""
    a, b = sorted(ins)
    c, d = sorted(set(range(4)) - {a, b})
    perm = (a, b, c, d)
    inv = sum(1 for i in range(4) for j in range(i + 1, 4) if perm[i] > perm[j])
    return perm if inv % 2 == 0 else (a, b, d, c)


def tet_triangles(inside):
    """Triangles of one positively oriented tetrahedron (step 4).

    inside: 4 booleans.  Returns a list of triangles, each a tuple of three
    tetrahedron edges (u, w) as pairs of local vertex numbers.
    """
    ins = [i for i in range(4) if inside[i]]
    if len(ins) in (0, 4):
        return []
    if len(ins) == 1:
        a, b, c, d = EVEN_FROM[ins[0]]
        return [((a, b), (a, c), (a, d))]
    if len(ins) == 3:
        a, b, c, d = EVEN_FROM[next(i for i in range(4) if not inside[i])]
        return [((a, b), (a, d), (a, c))]
    a, b, c, d = _even_pair_split(ins)
    return [((a, c), (a, d), (b, d)), ((a, c), (b, d), (b, c))]


def grid_spec(xyz, r_eff, spacing, margin):
    """Step 1: lower corner and node counts of the grid."""
    xyz = np.asarray(xyz, dtype=np.float64)
    rmax = float(np.max(r_eff))
    lo = xyz.min(0) - rmax - margin
    hi = xyz.max(0) + rmax + margin
    shape = tuple(int(math.ceil((hi[d] - lo[d]) / spacing)) + 1 for d in range(3))
    return lo, shape


def node_coords(lo, h, shape):
    """Coordinates of every node, [n_x, n_y, n_z, 3]: lo + h * index per axis."""
    ax = [lo[d] + h * np.arange(shape[d], dtype=np.float64) for d in range(3)]
    X, Y, Z = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
    return np.stack([X, Y, Z], -1)


def _chunk(na):
    return max(16, 2_000_000 // max(int(na), 1))


def density(points, xyz, r_eff, beta, cutoff):
    """rho at `points` [m, 3] by its definition (sum over every atom)."""
    points = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    xyz = np.asarray(xyz, dtype=np.float64)
    chunk = _chunk(xyz.shape[0])
    R = np.asarray(r_eff, dtype=np.float64)
    out = np.zeros(points.shape[0])
    for s in range(0, points.shape[0], chunk):
        p = points[s:s + chunk]
        g = p[:, None, :] - xyz[None, :, :]
        d2 = g[..., 0] ** 2 + g[..., 1] ** 2 + g[..., 2] ** 2
        e = np.exp(-beta * (d2 / (R * R) - 1.0))
        rc = cutoff * R
        e[d2 > rc * rc] = 0.0
        out[s:s + chunk] = e.sum(1)
    return out


def density_gradient(points, xyz, r_eff, beta, cutoff):
    """rho and grad rho at `points` [m, 3]: d/dx of every term is -2 beta (x - x_a) / R_a^2 times it."""
    points = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    xyz = np.asarray(xyz, dtype=np.float64)
    chunk = _chunk(xyz.shape[0])
    R = np.asarray(r_eff, dtype=np.float64)
    rho = np.zeros(points.shape[0])
    grad = np.zeros((points.shape[0], 3))
    for s in range(0, points.shape[0], chunk):
        g = points[s:s + chunk, None, :] - xyz[None, :, :]
        d2 = g[..., 0] ** 2 + g[..., 1] ** 2 + g[..., 2] ** 2
        e = np.exp(-beta * (d2 / (R * R) - 1.0))
        rc = cutoff * R
        e[d2 > rc * rc] = 0.0
        rho[s:s + chunk] = e.sum(1)
        for k in range(3):
            grad[s:s + chunk, k] = (e * (-2.0 * beta) * g[..., k] / (R * R)).sum(1)
    return rho, grad


def marching_tetrahedra(rho, lo, h, level, tclamp):
    """Steps 2-4 on a node array rho [n_x, n_y, n_z].  Returns (verts, tris, edges [nv, 2])."""
    nx, ny, nz = rho.shape
    f = rho.ravel() - level
    inside = f >= 0.0
    X = node_coords(lo, h, rho.shape).reshape(-1, 3)
    # cubes by lower corner, ascending node id
    ci, cj, ck = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), np.arange(nz - 1), indexing="ij")
    cube0 = ((ci * ny + cj) * nz + ck).ravel()
    corner_id = np.stack([cube0 + (c[0] * ny + c[1]) * nz + c[2] for c in CORNER], 1)   # [ncube, 8]
    cin = inside[corner_id]
    mixed = cin.any(1) & ~cin.all(1)
    tri_edges = []                       # per triangle: three (p, q) node pairs
    for cube in np.nonzero(mixed)[0]:
        ids, ins = corner_id[cube], cin[cube]
        for tet in TETS:
            w = [ids[c] for c in tet]
            for tri in tet_triangles([ins[c] for c in tet]):
                tri_edges.append([(min(w[u], w[v]), max(w[u], w[v])) for u, v in tri])
    if not tri_edges:
        return np.zeros((0, 3)), np.zeros((0, 3), np.int64), np.zeros((0, 2), np.int64)
    te = np.asarray(tri_edges, dtype=np.int64)              # [nt, 3, 2]
    nn = nx * ny * nz
    keys = te[..., 0] * nn + te[..., 1]
    ukeys, inv = np.unique(keys.ravel(), return_inverse=True)
    tris = inv.reshape(-1, 3)
    edges = np.stack([ukeys // nn, ukeys % nn], 1)
    fp, fq = f[edges[:, 0]], f[edges[:, 1]]
    t = np.clip(fp / (fp - fq), tclamp, 1.0 - tclamp)
    xp, xq = X[edges[:, 0]], X[edges[:, 1]]
    verts = xp + t[:, None] * (xq - xp)
    return verts, tris, edges


def components(nv, tris):
    """Connected-component label of every vertex (triangles sharing a vertex are connected)."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]]])
    g = coo_matrix((np.ones(e.shape[0]), (e[:, 0], e[:, 1])), shape=(nv, nv))
    return connected_components(g, directed=False)


def outer_component(verts, tris):
    """Step 5: the component of the last vertex; vertices renumbered in ascending order."""
    nv = verts.shape[0]
    ncomp, lab = components(nv, tris)
    keep_t = lab[tris[:, 0]] == lab[nv - 1]
    keep_v = lab == lab[nv - 1]
    new = -np.ones(nv, dtype=np.int64)
    new[keep_v] = np.arange(int(keep_v.sum()))
    return verts[keep_v], new[tris[keep_t]], ncomp


def neighbours(nv, tris):
    """Sorted unique undirected edges, both directions: rows (a, b) ascending."""
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    e = np.concatenate([e, e[:, ::-1]])
    return np.unique(e, axis=0)


def smooth_round(v, edges, xyz, r_eff, p):
    """One round of step 6: Laplacian move, then the level-set projections."""
    nv = v.shape[0]
    deg = np.bincount(edges[:, 0], minlength=nv).astype(np.float64)
    avg = np.stack([np.bincount(edges[:, 0], weights=v[edges[:, 1], k], minlength=nv) for k in range(3)], 1)
    v = v + p["relax"] * (avg / deg[:, None] - v)
    for _ in range(p["newton_steps"]):
        rho, g = density_gradient(v, xyz, r_eff, p["beta"], p["cutoff"])
        g2 = g[:, 0] * g[:, 0] + g[:, 1] * g[:, 1] + g[:, 2] * g[:, 2]
        ok = g2 > 1e-12
        step = np.where(ok, (rho - p["level"]) / np.where(ok, g2, 1.0), 0.0)
        dv = step[:, None] * g
        n = np.sqrt(dv[:, 0] * dv[:, 0] + dv[:, 1] * dv[:, 1] + dv[:, 2] * dv[:, 2])
        dv = dv * np.minimum(1.0, p["max_step"] / np.maximum(n, 1e-30))[:, None]
        v = v - dv
    return v


def folded(v, tris, xyz, r_eff, p):
    """Number of triangles whose normal does not point down the density."""
    a, b, c = v[tris[:, 0]], v[tris[:, 1]], v[tris[:, 2]]
    n = np.cross(b - a, c - a)
    _, g = density_gradient((a + b + c) / 3.0, xyz, r_eff, p["beta"], p["cutoff"])
    return int(np.count_nonzero((n * g).sum(1) >= 0.0))


def gaussian_surface(xyz, radius, spacing, **params):
    """Steps 1-6.  Returns dict(verts, tris, shape, lo, rounds, components, raw_verts, raw_tris, rho)."""
    p = dict(DEFAULTS)
    p.update(params)
    xyz = np.asarray(xyz, dtype=np.float64)
    r_eff = np.asarray(radius, dtype=np.float64) + p["radius_offset"]
    lo, shape = grid_spec(xyz, r_eff, spacing, p["margin"])
    rho = density(node_coords(lo, spacing, shape).reshape(-1, 3), xyz, r_eff, p["beta"], p["cutoff"]).reshape(shape)
    raw_v, raw_t, _ = marching_tetrahedra(rho, lo, spacing, p["level"], p["tclamp"])
    v, t, ncomp = outer_component(raw_v, raw_t)
    snaps = [v]
    if p["smooth_iters"] > 0:
        e = neighbours(v.shape[0], t)
        for _ in range(p["smooth_iters"]):
            snaps.append(smooth_round(snaps[-1], e, xyz, r_eff, p))
    rounds = 0
    if len(snaps) > 1:
        f0 = folded(snaps[0], t, xyz, r_eff, p)
        for r in range(len(snaps) - 1, 0, -1):
            if folded(snaps[r], t, xyz, r_eff, p) <= f0:
                rounds = r
                break
    return {"verts": snaps[rounds], "tris": t, "shape": shape, "lo": lo, "rounds": rounds,
            "components": ncomp, "raw_verts": raw_v, "raw_tris": raw_t, "rho": rho}
