"""Thin ctypes binding of the pbbem C-ABI (include/pbbem.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Importing this module loads ``libpbbem.so`` (built in-tree by
``paper_1309_4018_b300/build.py``); if it is missing the import fails loudly —
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import functools
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpbbem.so")

PB_OK, PB_EINVAL, PB_ENOMEM, PB_ECUDA, PB_ENOCONV, PB_ETIMEOUT, PB_ENOTSETUP = range(7)
PB_FP64, PB_MIXED = 0, 1
PB_OPT_BATCH_PERSISTENT = 1
_ERRNAMES = {1: "PB_EINVAL", 2: "PB_ENOMEM", 3: "PB_ECUDA", 4: "PB_ENOCONV", 5: "PB_ETIMEOUT",
             6: "PB_ENOTSETUP"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"pbbem CUDA library not built: {LIB_PATH} is missing "
                      "(run paper_1309_4018_b300/build.py)")
_lib = ctypes.CDLL(LIB_PATH)


class pb_params(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("K_fine", ctypes.c_int), ("N_k", ctypes.c_int),
                ("thres", ctypes.c_double), ("P", ctypes.c_int), ("theta", ctypes.c_double),
                ("ncrit", ctypes.c_int), ("gmres_tol", ctypes.c_double), ("restart", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("precision", ctypes.c_int), ("no_precond", ctypes.c_int),
                ("ncrit_adjoint", ctypes.c_int), ("p2p_tile", ctypes.c_int), ("m2p_variant", ctypes.c_int),
                ("precond_block", ctypes.c_int)]


class pb_result(ctypes.Structure):
    _fields_ = [("dG_solv", ctypes.c_double), ("residual", ctypes.c_double),
                ("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("pad_", ctypes.c_int), ("setup_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("p2p_pairs", ctypes.c_int64), ("m2p_pairs", ctypes.c_int64),
                ("near_pairs", ctypes.c_int64), ("near_excluded", ctypes.c_int64)]


class pb_grad(ctypes.Structure):
    _fields_ = [("dq", ctypes.c_void_p), ("dxyz", ctypes.c_void_p), ("deps", ctypes.c_void_p),
                ("dkappa", ctypes.c_void_p), ("energy", ctypes.c_double), ("residual", ctypes.c_double),
                ("iterations", ctypes.c_int), ("matvecs", ctypes.c_int), ("grad_ms", ctypes.c_double)]


class pb_surf_params(ctypes.Structure):
    _fields_ = [("spacing", ctypes.c_double), ("beta", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("radius_offset", ctypes.c_double), ("margin", ctypes.c_double), ("level", ctypes.c_double),
                ("tclamp", ctypes.c_double), ("relax", ctypes.c_double), ("max_step", ctypes.c_double),
                ("smooth_iters", ctypes.c_int), ("newton_steps", ctypes.c_int)]


class pb_surface_info(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("nt", ctypes.c_int64), ("generated", ctypes.c_int),
                ("grid", ctypes.c_int * 3), ("rounds", ctypes.c_int), ("pad_", ctypes.c_int),
                ("components", ctypes.c_int64), ("raw_nv", ctypes.c_int64), ("raw_nt", ctypes.c_int64),
                ("gen_ms", ctypes.c_double)]


class pb_tree_info(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_nodes", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("corner", ctypes.c_double * 3), ("side", ctypes.c_double)]


_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double
_SIGS = {
    "pb_ctx_create": ([_int, ctypes.POINTER(_vp)], _int),
    "pb_ctx_destroy": ([_vp], None),
    "pb_last_error": ([_vp], ctypes.c_char_p),
    "pb_ctx_stream": ([_vp], _vp),
    "pb_ctx_set_option": ([_vp, _int, ctypes.c_longlong], _int),
    "pb_problem_create": ([_vp, ctypes.POINTER(_vp)], _int),
    "pb_problem_destroy": ([_vp], None),
    "pb_add_region": ([_vp, _dbl, _dbl, ctypes.POINTER(_int)], _int),
    "pb_add_surface": ([_vp, _vp, _i64, _vp, _i64, _int, _int, ctypes.POINTER(_int)], _int),
    "pb_set_charges": ([_vp, _vp, _vp, _i64, _int], _int),
    "pb_add_surface_dev": ([_vp, _vp, _i64, _vp, _i64, _int, _int, ctypes.POINTER(_int)], _int),
    "pb_set_charges_dev": ([_vp, _vp, _vp, _i64, _int], _int),
    "pb_add_gaussian_surface": ([_vp, _vp, _vp, _i64, ctypes.POINTER(pb_surf_params), _int, _int,
                                 ctypes.POINTER(_int)], _int),
    "pb_surface_info_get": ([_vp, _int, ctypes.POINTER(pb_surface_info)], _int),
    "pb_surface_export": ([_vp, _int, _vp, _vp], _int),
    "pb_setup": ([_vp, ctypes.POINTER(pb_params)], _int),
    "pb_num_unknowns": ([_vp], _i64),
    "pb_apply_operator": ([_vp, _vp, _vp, _int], _int),
    "pb_rhs": ([_vp, _vp], _int),
    "pb_solve": ([_vp, _vp, ctypes.POINTER(pb_result)], _int),
    "pb_get_solution": ([_vp, _vp], _int),
    "pb_gradient": ([_vp, ctypes.POINTER(pb_grad)], _int),
    "pb_solve_batch": ([_vp, _vp, _int, _vp], _int),
    "pb_binding_energy": ([_vp, _vp, _vp, _vp, ctypes.POINTER(_dbl)], _int),
    "pb_apply_transpose": ([_vp, _vp, _vp, _int], _int),
    "pb_reaction_potential": ([_vp, _vp, _vp], _int),
    "pb_coulomb_energy": ([_vp, ctypes.POINTER(_dbl)], _int),
    "pb_profile_operator": ([_vp, _vp, _int, _vp], _int),
    "pb_launch_count": ([], ctypes.c_longlong),
    "pb_coulomb_energy_noalloc": ([_int, _vp, _vp, _i64, _dbl, _vp, _vp, ctypes.POINTER(ctypes.c_char_p)], _int),
    "pb_tree_info_get": ([_vp, _int, ctypes.POINTER(pb_tree_info)], _int),
    "pb_tree_export": ([_vp, _int, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _int),
    "pb_lists_export": ([_vp, _int, _int, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _int),
}
for _name, (_args, _ret) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = _ret

EXPORTED = tuple(_SIGS)


def launch_count() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(_lib.pb_launch_count())


def coulomb_energy_noalloc(device: int, xyz_ptr: int, q_ptr: int, nc: int, eps: float, out_ptr: int,
                           stream: int = 0):
    """Coulomb energy into *out_ptr from device arrays, with no device allocation.

    Returns (status code, message).  The work is queued on `stream`.
    """
    msg = ctypes.c_char_p()
    rc = _lib.pb_coulomb_energy_noalloc(int(device), _vp(xyz_ptr), _vp(q_ptr), int(nc), float(eps), _vp(out_ptr),
                                        _vp(stream), ctypes.byref(msg))
    return rc, (msg.value or b"").decode()


class PBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_ERRNAMES.get(code, code)}: {msg}")
        self.code = code


def _ptr(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _is_cuda_tensor(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _cuda_arg(a, dtype: str, cols):
    """A CUDA torch tensor of the given dtype, contiguous, with `cols` columns
    (or flat); the current torch stream is synchronised so the library's
    stream sees its contents."""
    import torch
    if not _is_cuda_tensor(a):
        raise TypeError("device arguments must all be CUDA tensors")
    want = getattr(torch, dtype)
    if a.dtype != want:
        raise TypeError(f"expected a {dtype} tensor, got {a.dtype}")
    a = a.contiguous()
    a = a.reshape(-1, cols) if cols else a.reshape(-1)
    torch.cuda.current_stream(a.device).synchronize()
    return a


class Context:
    """One CUDA device and stream (pb_ctx)."""

    def __init__(self, device: int = 0):
        h = _vp()
        rc = _lib.pb_ctx_create(device, ctypes.byref(h))
        if rc != PB_OK:
            raise PBError(rc, "pb_ctx_create failed")
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def stream(self) -> int:
        return _lib.pb_ctx_stream(self._h) or 0

    def set_option(self, option: int, value: int):
        """pb_ctx_set_option (PB_OPT_BATCH_PERSISTENT: 1 or 0)."""
        self.check(_lib.pb_ctx_set_option(self._h, int(option), int(value)))

    def check(self, rc):
        if rc != PB_OK:
            raise PBError(rc, _lib.pb_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _lib.pb_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


@dataclass
class Result:
    dG_solv: float
    residual: float
    iterations: int
    converged: bool
    matvecs: int
    setup_ms: float
    solve_ms: float
    p2p_pairs: int
    m2p_pairs: int
    near_pairs: int
    near_excluded: int


def make_params(**kw) -> pb_params:
    p = pb_params()
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = {"fp64": PB_FP64, "mixed": PB_MIXED}[v]
        setattr(p, k, v)
    return p


def _result(r) -> "Result":
    return Result(r.dG_solv, r.residual, r.iterations, bool(r.converged), r.matvecs, r.setup_ms,
                  r.solve_ms, r.p2p_pairs, r.m2p_pairs, r.near_pairs, r.near_excluded)


def solve_batch(ctx: "Context", problems, check=True):
    """Solve set-up problems of one context together (pb_solve_batch); one Result each."""
    n = len(problems)
    handles = (ctypes.c_void_p * max(1, n))(*[p._h for p in problems])
    res = (pb_result * max(1, n))()
    rc = _lib.pb_solve_batch(ctx.handle, handles, n, res)
    if check or rc not in (PB_OK, PB_ENOCONV):
        ctx.check(rc)
    return [_result(res[i]) for i in range(n)]


def solve(problem: dict, context: "Context | None" = None, return_solution: bool = False, check: bool = True,
          **params):
    """One problem in one call: build it from its description (Problem.from_dict),
    set it up with the pb_params fields given as keywords, solve it, free it.

    Returns the Result, or (Result, x) with the solution x (2 N host doubles)
    when return_solution is set.  A context made here is closed again.
    """
    ctx = context if context is not None else Context(0)
    try:
        pb = Problem.from_dict(ctx, problem)
        try:
            pb.setup(**params)
            r = pb.solve(check=check)
            return (r, pb.solution()) if return_solution else r
        finally:
            pb.close()
    finally:
        if context is None:
            ctx.close()


def binding_energy(ctx: "Context", cx, rec, lig) -> float:
    """ddG = E_complex - E_receptor - E_ligand (solvation + Coulomb), kJ/mol (pb_binding_energy)."""
    out = _dbl()
    ctx.check(_lib.pb_binding_energy(ctx.handle, cx._h, rec._h, lig._h, ctypes.byref(out)))
    return out.value


class Problem:
    """A molecule: regions, surfaces and charges (pb_problem)."""

    def __init__(self, ctx: Context):
        self.ctx = ctx
        h = _vp()
        ctx.check(_lib.pb_problem_create(ctx.handle, ctypes.byref(h)))
        self._h = h
        self.n_charges = 0
        self.n_regions = 0

    @classmethod
    def from_dict(cls, ctx: Context, d: dict) -> "Problem":
        """Build from the plain input description used by the synthetic workloads."""
        pb = cls(ctx)
        for r in d["regions"]:
            pb.add_region(r["eps"], r["kappa"])
        for s in d["surfaces"]:
            if "atoms" in s:      # generated on the device: {"xyz", "radius"} plus pb_surf_params fields
                pb.add_gaussian_surface(s["atoms"]["xyz"], s["atoms"]["radius"], s["inner"], s["outer"],
                                        **s.get("surf_params", {}))
            else:
                pb.add_surface(s["verts"], s["tris"], s["inner"], s["outer"])
        ch = d.get("charges")
        if ch is not None:
            pb.set_charges(ch["xyz"], ch["q"], ch["region"])
        return pb

    def add_region(self, eps, kappa) -> int:
        rid = _int()
        self.ctx.check(_lib.pb_add_region(self._h, float(eps), float(kappa), ctypes.byref(rid)))
        self.n_regions = rid.value + 1
        return rid.value

    def add_surface(self, verts, tris, inner, outer) -> int:
        """verts [nv, 3], tris [nt, 3]: numpy arrays (host), or CUDA torch tensors
        (float64, int32) handed over by device pointer (pb_add_surface_dev)."""
        if _is_cuda_tensor(verts) or _is_cuda_tensor(tris):
            v, t = _cuda_arg(verts, "float64", 3), _cuda_arg(tris, "int32", 3)
            sid = _int()
            self.ctx.check(_lib.pb_add_surface_dev(self._h, _vp(v.data_ptr()), v.shape[0], _vp(t.data_ptr()),
                                                   t.shape[0], int(inner), int(outer), ctypes.byref(sid)))
            return sid.value
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tris, dtype=np.int32)
        sid = _int()
        self.ctx.check(_lib.pb_add_surface(self._h, _ptr(v), v.shape[0], _ptr(t), t.shape[0], int(inner),
                                           int(outer), ctypes.byref(sid)))
        return sid.value

    def add_gaussian_surface(self, xyz, radius, inner, outer, **params) -> int:
        """Surface generated on the device from atoms (pb_add_gaussian_surface); params are
        pb_surf_params fields (spacing required)."""
        x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        r = np.ascontiguousarray(radius, dtype=np.float64).ravel()
        sp = pb_surf_params()
        for k, v in params.items():
            if not hasattr(sp, k):
                raise TypeError(f"unknown surface parameter {k}")
            setattr(sp, k, v)
        sid = _int()
        self.ctx.check(_lib.pb_add_gaussian_surface(self._h, _ptr(x), _ptr(r), r.size, ctypes.byref(sp), int(inner),
                                                    int(outer), ctypes.byref(sid)))
        return sid.value

    def surface_info(self, surface: int) -> dict:
        inf = pb_surface_info()
        self.ctx.check(_lib.pb_surface_info_get(self._h, int(surface), ctypes.byref(inf)))
        return dict(nv=inf.nv, nt=inf.nt, generated=bool(inf.generated), grid=tuple(inf.grid), rounds=inf.rounds,
                    components=inf.components, raw_nv=inf.raw_nv, raw_nt=inf.raw_nt, gen_ms=inf.gen_ms)

    def surface_mesh(self, surface: int):
        """(verts [nv, 3] float64, tris [nt, 3] int32) of a surface, copied from the device."""
        inf = self.surface_info(surface)
        v = np.empty((inf["nv"], 3))
        t = np.empty((inf["nt"], 3), dtype=np.int32)
        self.ctx.check(_lib.pb_surface_export(self._h, int(surface), _ptr(v), _ptr(t)))
        return v, t

    def set_charges(self, xyz, q, region):
        """xyz [nc, 3], q [nc]: numpy arrays (host), or CUDA torch float64 tensors
        handed over by device pointer (pb_set_charges_dev)."""
        if _is_cuda_tensor(xyz) or _is_cuda_tensor(q):
            x, qq = _cuda_arg(xyz, "float64", 3), _cuda_arg(q, "float64", None)
            if x.shape[0] != qq.numel():
                raise ValueError("xyz and q hold different numbers of charges")
            self.ctx.check(_lib.pb_set_charges_dev(self._h, _vp(x.data_ptr()), _vp(qq.data_ptr()), qq.numel(),
                                                   int(region)))
            self.n_charges = qq.numel()
            return
        x = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
        qq = np.ascontiguousarray(q, dtype=np.float64).ravel()
        self.ctx.check(_lib.pb_set_charges(self._h, _ptr(x), _ptr(qq), qq.size, int(region)))
        self.n_charges = qq.size

    def setup(self, **params):
        p = make_params(**params)
        self.ctx.check(_lib.pb_setup(self._h, ctypes.byref(p)))

    @property
    def n_unknowns(self) -> int:
        return int(_lib.pb_num_unknowns(self._h))

    def apply(self, x):
        """y = A x.  x: numpy array (host) or a CUDA torch tensor (device pointers)."""
        if hasattr(x, "data_ptr"):
            import torch
            y = torch.empty_like(x)
            self.ctx.check(_lib.pb_apply_operator(self._h, _vp(x.data_ptr()), _vp(y.data_ptr()), 1))
            return y
        xx = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(xx)
        self.ctx.check(_lib.pb_apply_operator(self._h, _ptr(xx), _ptr(y), 0))
        return y

    def apply_transpose(self, x):
        """y = A^T x by the transposed treecode.  x: numpy array (host) or a CUDA torch tensor."""
        if hasattr(x, "data_ptr"):
            import torch
            y = torch.empty_like(x)
            self.ctx.check(_lib.pb_apply_transpose(self._h, _vp(x.data_ptr()), _vp(y.data_ptr()), 1))
            return y
        xx = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(xx)
        self.ctx.check(_lib.pb_apply_transpose(self._h, _ptr(xx), _ptr(y), 0))
        return y

    def gradient(self, check=True) -> dict:
        """Adjoint gradient of the last solve's energy: dq, dxyz, deps, dkappa (per region) and stats."""
        g = pb_grad()
        out = dict(dq=np.empty(self.n_charges), dxyz=np.empty((self.n_charges, 3)),
                   deps=np.empty(self.n_regions), dkappa=np.empty(self.n_regions))
        g.dq, g.dxyz = out["dq"].ctypes.data, out["dxyz"].ctypes.data
        g.deps, g.dkappa = out["deps"].ctypes.data, out["dkappa"].ctypes.data
        rc = _lib.pb_gradient(self._h, ctypes.byref(g))
        if check or rc not in (PB_OK, PB_ENOCONV):
            self.ctx.check(rc)
        out.update(energy=g.energy, residual=g.residual, iterations=g.iterations, matvecs=g.matvecs,
                   grad_ms=g.grad_ms)
        return out

    def apply_device(self, x_ptr: int, y_ptr: int):
        """y = A x on raw device pointers (2 N doubles each)."""
        self.ctx.check(_lib.pb_apply_operator(self._h, _vp(x_ptr), _vp(y_ptr), 1))

    def rhs(self):
        b = np.empty(self.n_unknowns)
        self.ctx.check(_lib.pb_rhs(self._h, _ptr(b)))
        return b

    def solve(self, x0=None, check=True) -> Result:
        r = pb_result()
        xx = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        rc = _lib.pb_solve(self._h, _ptr(xx), ctypes.byref(r))
        if check or rc not in (PB_OK, PB_ENOCONV):
            self.ctx.check(rc)
        return _result(r)

    def solution(self):
        x = np.empty(self.n_unknowns)
        self.ctx.check(_lib.pb_get_solution(self._h, _ptr(x)))
        return x

    def reaction_potential(self, x):
        xx = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty(self.n_charges)
        self.ctx.check(_lib.pb_reaction_potential(self._h, _ptr(xx), _ptr(out)))
        return out

    def coulomb_energy(self) -> float:
        e = _dbl()
        self.ctx.check(_lib.pb_coulomb_energy(self._h, ctypes.byref(e)))
        return e.value

    def profile(self, x, reps: int = 10) -> dict:
        """Average device ms per phase of one operator application."""
        xx = np.ascontiguousarray(x, dtype=np.float64)
        out = np.zeros(6)
        self.ctx.check(_lib.pb_profile_operator(self._h, _ptr(xx), int(reps), _ptr(out)))
        return dict(zip(("upward", "p2p", "m2p", "gather_near", "combine", "total"), out.tolist()))

    def tree(self, surface: int) -> dict:
        info = pb_tree_info()
        self.ctx.check(_lib.pb_tree_info_get(self._h, surface, ctypes.byref(info)))
        n, m = info.n_points, info.n_nodes
        out = dict(keys=np.empty(n, np.uint64), perm=np.empty(n, np.int32), level=np.empty(m, np.int32),
                   start=np.empty(m, np.int64), count=np.empty(m, np.int64),
                   first_child=np.empty(m, np.int32), nchild=np.empty(m, np.int32))
        self.ctx.check(_lib.pb_tree_export(self._h, surface, *[_ptr(out[k]) for k in
                                                               ("keys", "perm", "level", "start", "count",
                                                                "first_child", "nchild")]))
        out.update(corner=np.array(info.corner[:]), side=info.side, n_leaves=info.n_leaves)
        return out

    def lists(self, target_surface: int, source_surface: int) -> dict:
        counts = np.zeros(6, np.int64)
        self.ctx.check(_lib.pb_lists_export(self._h, target_surface, source_surface, _ptr(counts),
                                            None, None, None, None, None, None))
        m = int(counts[5])
        out = dict(m2p_ptr=np.empty(m + 1, np.int64), m2p=np.empty(max(1, counts[0]), np.int32),
                   p2p_ptr=np.empty(m + 1, np.int64), p2p=np.empty(max(1, counts[1]), np.int32),
                   near_ptr=np.empty(m + 1, np.int64), near=np.empty(max(1, counts[2]), np.int32))
        self.ctx.check(_lib.pb_lists_export(self._h, target_surface, source_surface, _ptr(counts),
                                            *[_ptr(out[k]) for k in ("m2p_ptr", "m2p", "p2p_ptr", "p2p",
                                                                     "near_ptr", "near")]))
        out["m2p"] = out["m2p"][:counts[0]]
        out["p2p"] = out["p2p"][:counts[1]]
        out["near"] = out["near"][:counts[2]]
        out.update(n_near_excluded=int(counts[3]), n_self_excluded=int(counts[4]))
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.pb_problem_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


@functools.lru_cache(maxsize=1)
def _energy_autograd():
    import torch

    class Energy(torch.autograd.Function):
        """Solvation energy (kJ/mol) as a differentiable function of (q, xyz, eps, kappa).

        forward(problem_dict, q [nc], xyz [nc,3], eps [n_regions], kappa [n_regions], context=None, params=None)
        builds the problem with these values, sets it up and solves it (Eq. solv).
        When an input needs a gradient the set-up problem is kept, and backward
        runs the adjoint solve (pb_gradient) once, on its first call; a forward
        that no backward follows costs one solve.  The mesh is held fixed.
        """

        @staticmethod
        def forward(fctx, problem, q, xyz, eps, kappa, context=None, params=None):
            d = dict(problem)
            d["regions"] = [{"eps": float(e), "kappa": float(k)}
                            for e, k in zip(eps.detach().cpu().tolist(), kappa.detach().cpu().tolist())]
            d["charges"] = dict(problem["charges"], q=q.detach().cpu().double().numpy(),
                                xyz=xyz.detach().cpu().double().numpy())
            c = context or Context(0)
            pb = Problem.from_dict(c, d)
            pb.setup(**(params or {}))
            r = pb.solve()
            if any(fctx.needs_input_grad[1:5]):
                fctx.pb = pb
            else:
                pb.close()
            fctx.like = (q.dtype, q.device)
            return torch.as_tensor(r.dG_solv, dtype=q.dtype, device=q.device)

        @staticmethod
        def backward(fctx, gout):
            g = fctx.pb.gradient()
            fctx.pb.close()
            fctx.pb = None
            dt, dev = fctx.like
            out = [gout * torch.as_tensor(g[k], dtype=dt, device=dev) for k in ("dq", "dxyz", "deps", "dkappa")]
            return (None, *out, None, None)

    return Energy


def __getattr__(name):
    if name == "Energy":
        return _energy_autograd()
    raise AttributeError(name)
