"""Host-side file handling of the device mesher's command line tool (no GPU)."""
import numpy as np

from paper_1309_4018_b300 import mesh as M


def test_xyzr_round_trip(tmp_path):
    a = np.array([[0.5, -1.25, 3.0, 1.6], [2.0, 0.0, -0.5, 1.2]])
    p = tmp_path / "m.xyzr"
    np.savetxt(p, a)
    xyz, r = M.read_xyzr(str(p))
    assert np.array_equal(xyz, a[:, :3]) and np.array_equal(r, a[:, 3])


def test_mesh_writers(tmp_path):
    v = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0 / 3.0]])
    t = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]], dtype=np.int32)
    M.write_mesh(str(tmp_path / "m.npz"), v, t)
    z = np.load(tmp_path / "m.npz")
    assert np.array_equal(z["verts"], v) and np.array_equal(z["tris"], t)
    M.write_mesh(str(tmp_path / "m.off"), v, t)
    lines = (tmp_path / "m.off").read_text().split("\n")
    assert lines[0] == "OFF" and lines[1] == "4 4 0"
    vv = np.array([[float(x) for x in l.split()] for l in lines[2:6]])
    tt = np.array([[int(x) for x in l.split()] for l in lines[6:10]])
    assert np.array_equal(vv, v) and np.array_equal(tt[:, 1:], t) and np.all(tt[:, 0] == 3)
