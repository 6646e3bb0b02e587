"""Flat-triangle panel geometry and Gauss points (Sec. 2.2, Eq. nBEM_disc).

Panels are flat triangles with constant phi and dphi/dn; the collocation point
of panel i is its centroid r_i (Eq. nBEM_disc).  The unit normal is
(v1 - v0) x (v2 - v0) normalised: with counter-clockwise winding seen from the
outer region it points from the inner region to the outer one.  The
characteristic length of a panel, used by the near-singular test of the
treecode-accelerated BEM (Table 4), is read as L = sqrt(2 A).

All arithmetic is FP64 and written out operation by operation (numpy never
fuses a multiply and an add), so that the Morton keys and the near-singular
decisions that depend on these values are reproducible bit for bit.
"""
from __future__ import annotations

import numpy as np

from .quadrature import triangle_rule


def panel_geometry(verts: np.ndarray, tris: np.ndarray):
    """Centroid [N,3], unit normal [N,3], area [N], characteristic length [N]."""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    v0, v1, v2 = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    cen = ((v0 + v1) + v2) / 3.0
    a = v1 - v0
    b = v2 - v0
    cx = a[:, 1] * b[:, 2] - a[:, 2] * b[:, 1]
    cy = a[:, 2] * b[:, 0] - a[:, 0] * b[:, 2]
    cz = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
    nrm2 = (cx * cx + cy * cy) + cz * cz
    nlen = np.sqrt(nrm2)
    normal = np.stack([cx / nlen, cy / nlen, cz / nlen], axis=1)
    area = 0.5 * nlen
    L = np.sqrt(2.0 * area)
    return cen, normal, area, L


def gauss_points(verts: np.ndarray, tris: np.ndarray, K: int):
    """Quadrature points of every panel (Sec. 2.3: they are the treecode sources).

    Returns y [N*K,3] (point k of panel j at row j*K+k), weight*area [N*K],
    owning panel id [N*K].
    """
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    lam, w = triangle_rule(K)
    v0, v1, v2 = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    _, _, area, _ = panel_geometry(verts, tris)
    n = t.shape[0]
    y = np.empty((n, K, 3))
    wa = np.empty((n, K))
    for k in range(K):
        y[:, k, :] = (lam[k, 0] * v0 + lam[k, 1] * v1) + lam[k, 2] * v2
        wa[:, k] = w[k] * area
    pid = np.repeat(np.arange(n), K)
    return y.reshape(n * K, 3), wa.reshape(n * K), pid
