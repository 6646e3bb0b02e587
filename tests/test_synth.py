"""The synthetic inputs: closed, consistently oriented meshes of the stated sizes."""
import numpy as np

from synth.configs import panel_count, protein_problem, sphere_problem
from synth.meshes import closed_and_oriented, icosphere, octasphere, signed_volume


def test_sphere_meshes():
    for level, n in ((3, 512), (4, 2048), (5, 8192)):
        v, t = octasphere(level, 4.0)
        assert t.shape[0] == n and closed_and_oriented(t) and signed_volume(v, t) > 0
    v, t = icosphere(3, 3.0, (7, 0, 0))
    assert t.shape[0] == 1280 and closed_and_oriented(t) and signed_volume(v, t) > 0
    assert panel_count(sphere_problem(level=4)) == 2048


def test_protein_surface():
    pr = protein_problem()
    n = panel_count(pr)
    assert 38000 <= n <= 42000
    s = pr["surfaces"][0]
    assert closed_and_oriented(s["tris"]) and signed_volume(s["verts"], s["tris"]) > 0
    q = pr["charges"]["q"]
    assert q.size == 2000 and abs(q.sum()) < 1e-10
    # every charge is inside: winding number of the closed surface is 1
    v, t = s["verts"], s["tris"].astype(np.int64)
    for p in pr["charges"]["xyz"][::97]:
        a, b, c = v[t[:, 0]] - p, v[t[:, 1]] - p, v[t[:, 2]] - p
        la, lb, lc = (np.linalg.norm(z, axis=1) for z in (a, b, c))
        num = np.einsum("ij,ij->i", a, np.cross(b, c))
        den = la * lb * lc + np.einsum("ij,ij->i", a, b) * lc + np.einsum("ij,ij->i", b, c) * la \
            + np.einsum("ij,ij->i", c, a) * lb
        w = 2 * np.arctan2(num, den).sum() / (4 * np.pi)
        assert abs(w - 1.0) < 1e-6


def test_binding_triplet_geometry():
    from scipy.spatial import cKDTree
    from synth.configs import binding_triplet
    cx, rec, lig = binding_triplet(n_rec=80, n_lig=30, spacing=2.0)
    for d in (cx, rec, lig):
        t = d["surfaces"][0]["tris"]
        assert closed_and_oriented(t)
        assert signed_volume(d["surfaces"][0]["verts"], t) > 0
    dmin = cKDTree(rec["charges"]["xyz"]).query(lig["charges"]["xyz"])[0].min()
    assert abs(dmin - 3.0) < 1e-6
    assert cx["charges"]["q"].size == rec["charges"]["q"].size + lig["charges"]["q"].size
