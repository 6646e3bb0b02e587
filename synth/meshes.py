"""Seeded/deterministic sphere meshes used as synthetic inputs.

These generators only produce geometry (vertex coordinates and triangle
connectivity).  They contain none of the boundary-element arithmetic and are
shared by the oracle-side tests and the CUDA-side tests and benchmark.

Triangles are oriented counter-clockwise when seen from outside, so that the
right-hand normal (v1 - v0) x (v2 - v0) points out of the enclosed region.
"""
from __future__ import annotations

import numpy as np

_OCTA_VERTS = np.array(
    [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]],
    dtype=np.float64,
)
_OCTA_TRIS = np.array(
    [[0, 2, 4], [2, 1, 4], [1, 3, 4], [3, 0, 4],
     [2, 0, 5], [1, 2, 5], [3, 1, 5], [0, 3, 5]],
    dtype=np.int64,
)

_PHI = (1.0 + 5.0 ** 0.5) / 2.0
_ICO_VERTS = np.array(
    [[-1, _PHI, 0], [1, _PHI, 0], [-1, -_PHI, 0], [1, -_PHI, 0],
     [0, -1, _PHI], [0, 1, _PHI], [0, -1, -_PHI], [0, 1, -_PHI],
     [_PHI, 0, -1], [_PHI, 0, 1], [-_PHI, 0, -1], [-_PHI, 0, 1]],
    dtype=np.float64,
)
_ICO_TRIS = np.array(
    [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
     [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
     [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
     [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]],
    dtype=np.int64,
)


def _subdivide(verts: np.ndarray, tris: np.ndarray, levels: int):
    """Split every triangle into four, ``levels`` times, sharing edge midpoints."""
    verts = [tuple(v) for v in verts]
    for _ in range(levels):
        mid = {}
        new_tris = []

        def midpoint(a, b):
            key = (a, b) if a < b else (b, a)
            if key not in mid:
                va, vb = verts[a], verts[b]
                verts.append(((va[0] + vb[0]) * 0.5, (va[1] + vb[1]) * 0.5,
                              (va[2] + vb[2]) * 0.5))
                mid[key] = len(verts) - 1
            return mid[key]

        for a, b, c in tris:
            ab, bc, ca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
            new_tris += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = np.array(new_tris, dtype=np.int64)
    return np.array(verts, dtype=np.float64), np.asarray(tris, dtype=np.int64)


def _project(verts: np.ndarray, radius: float, center) -> np.ndarray:
    nrm = np.sqrt((verts * verts).sum(axis=1))[:, None]
    return verts / nrm * radius + np.asarray(center, dtype=np.float64)[None, :]


def octasphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Octahedron subdivided ``level`` times, vertices projected to the sphere.

    Face count is 8 * 4**level (level 3: 512, level 4: 2048, level 5: 8192).
    Returns (verts float64 [nv,3], tris int32 [nt,3]).
    """
    v, t = _subdivide(_OCTA_VERTS, _OCTA_TRIS, level)
    return _project(v, radius, center), t.astype(np.int32)


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Icosahedron subdivided ``level`` times (20 * 4**level faces)."""
    v, t = _subdivide(_ICO_VERTS, _ICO_TRIS, level)
    return _project(v, radius, center), t.astype(np.int32)


def flip_orientation(tris: np.ndarray) -> np.ndarray:
    """Reverse triangle winding (normals then point into the enclosed region)."""
    t = np.array(tris, copy=True)
    t[:, [1, 2]] = t[:, [2, 1]]
    return t


def closed_and_oriented(tris: np.ndarray) -> bool:
    """True when every directed edge appears once and its reverse once."""
    t = np.asarray(tris, dtype=np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    nv = int(t.max()) + 1
    fwd = e[:, 0] * nv + e[:, 1]
    rev = e[:, 1] * nv + e[:, 0]
    if np.unique(fwd).size != fwd.size:
        return False
    return bool(np.all(np.isin(rev, fwd)))


def signed_volume(verts: np.ndarray, tris: np.ndarray) -> float:
    """Enclosed volume by the divergence theorem (positive for outward winding)."""
    v0, v1, v2 = (verts[tris[:, k]] for k in range(3))
    return float(np.einsum("ij,ij->i", v0, np.cross(v1, v2)).sum() / 6.0)
