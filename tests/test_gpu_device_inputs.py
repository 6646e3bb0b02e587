"""Inputs handed over by device pointer (pb_add_surface_dev, pb_set_charges_dev),
the pointer checks of the device-pointer calls, and the one-call pbbem.solve.

A problem built from CUDA tensors must solve to the same bits as the same
problem built from host arrays (same device copies, same kernels); malformed
device inputs are refused with PB_EINVAL by device-side checks, and a pointer
that is not device memory is refused on the host before any kernel runs.
"""
import ctypes

import numpy as np
import pytest

from gpu_util import ctx
from synth.configs import layered_sphere_problem, sphere_problem

pytestmark = pytest.mark.gpu

FP64 = dict(theta=-1.0, precision="fp64", ncrit=64, gmres_tol=1e-8)
MIXED = dict(theta=0.5, P=6, ncrit=40, precision="mixed", gmres_tol=1e-6)


def _pbbem():
    from paper_1309_4018_b300 import pbbem
    return pbbem


def _from_tensors(d):
    import torch
    pbbem = _pbbem()
    pb = pbbem.Problem(ctx())
    for r in d["regions"]:
        pb.add_region(r["eps"], r["kappa"])
    for s in d["surfaces"]:
        pb.add_surface(torch.as_tensor(s["verts"], dtype=torch.float64, device="cuda"),
                       torch.as_tensor(s["tris"], dtype=torch.int32, device="cuda"), s["inner"], s["outer"])
    ch = d["charges"]
    pb.set_charges(torch.as_tensor(ch["xyz"], dtype=torch.float64, device="cuda"),
                   torch.as_tensor(ch["q"], dtype=torch.float64, device="cuda"), ch["region"])
    return pb


@pytest.mark.parametrize("params", [FP64, MIXED], ids=["fp64", "mixed"])
def test_device_inputs_solve_like_host_inputs(params):
    pbbem = _pbbem()
    d = layered_sphere_problem(level=3, stern_level=3)
    host = pbbem.Problem.from_dict(ctx(), d)
    host.setup(**params)
    r_host = host.solve()
    dev = _from_tensors(d)
    dev.setup(**params)
    r_dev = dev.solve()
    assert r_dev.dG_solv == r_host.dG_solv
    assert r_dev.iterations == r_host.iterations
    np.testing.assert_array_equal(dev.solution(), host.solution())
    v, t = dev.surface_mesh(1)
    np.testing.assert_array_equal(v, d["surfaces"][1]["verts"])
    np.testing.assert_array_equal(t, d["surfaces"][1]["tris"])


def test_device_mesh_checks():
    import torch
    pbbem = _pbbem()
    d = sphere_problem(level=2)
    v = torch.as_tensor(d["surfaces"][0]["verts"], dtype=torch.float64, device="cuda")
    t = torch.as_tensor(d["surfaces"][0]["tris"], dtype=torch.int32, device="cuda")
    cases = []
    vb = v.clone()
    vb[5, 1] = float("nan")
    cases.append((vb, t, ["non-finite vertex coordinate", "element 16"]))
    tb = t.clone()
    tb[4, 2] = v.shape[0]
    cases.append((v, tb, ["triangle vertex index out of range", "element 14"]))
    cases.append((v, t[1:].contiguous(), ["closed 2-manifold"]))
    cases.append((v, t.flip(1).contiguous(), ["signed volume"]))
    for vv, tt, words in cases:
        pb = pbbem.Problem(ctx())
        pb.add_region(1.0, 0.0)
        pb.add_region(80.0, 0.125)
        with pytest.raises(pbbem.PBError) as ei:
            pb.add_surface(vv, tt, 0, 1)
        assert ei.value.code == pbbem.PB_EINVAL
        assert all(w in str(ei.value) for w in words), str(ei.value)
    # the context stays usable
    pb = pbbem.Problem(ctx())
    pb.add_region(1.0, 0.0)
    pb.add_region(80.0, 0.125)
    assert pb.add_surface(v, t, 0, 1) == 0


def test_device_charge_checks():
    import torch
    pbbem = _pbbem()
    d = sphere_problem(level=3)
    pb = pbbem.Problem.from_dict(ctx(), d)
    xyz = torch.zeros((2, 3), dtype=torch.float64, device="cuda")
    xyz[1, 2] = float("inf")
    q = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(pbbem.PBError) as ei:
        pb.set_charges(xyz, q, 0)
    assert ei.value.code == pbbem.PB_EINVAL and "non-finite charge position" in str(ei.value)
    with pytest.raises(TypeError):
        pb.set_charges(xyz.float(), q, 0)
    # a failed device call leaves no charges: setting valid ones makes the problem whole again
    pb.set_charges(torch.as_tensor(d["charges"]["xyz"], device="cuda"), torch.as_tensor(d["charges"]["q"],
                                                                                         device="cuda"), 0)
    pb.setup(**FP64)
    r = pb.solve()
    ref = pbbem.Problem.from_dict(ctx(), d)
    ref.setup(**FP64)
    assert r.dG_solv == ref.solve().dG_solv


def test_host_pointers_refused_where_device_pointers_are_required():
    import torch
    pbbem = _pbbem()
    lib = pbbem._lib
    d = sphere_problem(level=3)
    v = np.ascontiguousarray(d["surfaces"][0]["verts"])
    t = np.ascontiguousarray(d["surfaces"][0]["tris"], dtype=np.int32)
    pb = pbbem.Problem(ctx())
    pb.add_region(1.0, 0.0)
    pb.add_region(80.0, 0.125)
    sid = ctypes.c_int()
    rc = lib.pb_add_surface_dev(pb._h, ctypes.c_void_p(v.ctypes.data), v.shape[0], ctypes.c_void_p(t.ctypes.data),
                                t.shape[0], 0, 1, ctypes.byref(sid))
    assert rc == pbbem.PB_EINVAL and b"not device memory" in lib.pb_last_error(ctx().handle)
    pinned = torch.zeros(12, dtype=torch.float64).pin_memory()
    rc = lib.pb_set_charges_dev(pb._h, ctypes.c_void_p(pinned.data_ptr()), ctypes.c_void_p(pinned.data_ptr()), 4, 0)
    assert rc == pbbem.PB_EINVAL and b"not device memory" in lib.pb_last_error(ctx().handle)
    # the device-pointer operator calls check their pointers too
    full = pbbem.Problem.from_dict(ctx(), d)
    full.setup(**FP64)
    x = np.ones(full.n_unknowns)
    y = np.empty_like(x)
    for fn in (lib.pb_apply_operator, lib.pb_apply_transpose):
        rc = fn(full._h, ctypes.c_void_p(x.ctypes.data), ctypes.c_void_p(y.ctypes.data), 1)
        assert rc == pbbem.PB_EINVAL and b"not device memory" in lib.pb_last_error(ctx().handle)
    xd = torch.ones(full.n_unknowns, dtype=torch.float64, device="cuda")
    np.testing.assert_array_equal(full.apply(xd).cpu().numpy(), full.apply(x))


def test_one_call_solve():
    pbbem = _pbbem()
    d = sphere_problem(level=3)
    pb = pbbem.Problem.from_dict(ctx(), d)
    pb.setup(**MIXED)
    ref = pb.solve()
    r = pbbem.solve(d, context=ctx(), **MIXED)
    assert r.dG_solv == ref.dG_solv and r.iterations == ref.iterations
    r2, x = pbbem.solve(d, return_solution=True, **MIXED)   # its own context
    assert r2.dG_solv == ref.dG_solv
    np.testing.assert_array_equal(x, pb.solution())
