"""ctypes front end of the C/OpenMP matrix-free dense oracle (oracle/csrc/bem_dense.c).

Same discrete operator as oracle.dense (Sec. 2.2), evaluated row by row
without storing the matrix, so that ~10^5-panel problems can be checked and
timed on the host.  Test infrastructure only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from . import formulation as F
from .dense import full_params, surfaces_data, rhs, KJ_PER_MOL, FOUR_PI
from .gmres import gmres

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "csrc", "bem_dense.c")
_LIB = os.path.join(_HERE, "csrc", "libbemdense.so")


def build():
    """Compile the C oracle (gcc, OpenMP, no FMA contraction)."""
    if (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               _SRC, "-o", _LIB, "-lm"])
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.POINTER(ctypes.c_int64)
        _lib.bem_dense_block_sums.argtypes = [ctypes.c_int64, d, i64, ctypes.c_int64, d, d, d,
                                              ctypes.c_int, d, d, ctypes.c_int, d, d, d,
                                              ctypes.c_double, ctypes.c_double, d, d, d, d]
        _lib.bem_dense_block_sums.restype = None
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def block_sums(x, src, kappa, params, phi, dphi, self_idx=None):
    """(V_i, K_i) of targets x [m,3] against the panels of SurfaceData ``src``."""
    lib = _load()
    p = full_params(params)
    x = np.ascontiguousarray(x, dtype=np.float64)
    m = x.shape[0]
    V = np.zeros(m)
    K = np.zeros(m)
    selfV = np.ascontiguousarray(src.self_V(kappa, p["N_k"]))
    si = None
    if self_idx is not None:
        si = np.ascontiguousarray(self_idx, dtype=np.int64)
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in
            (src.cen, src.normal, src.L, src.y, src.wa, src.yf, src.waf, phi, dphi)]
    lib.bem_dense_block_sums(m, _p(x), si.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)) if si is not None else None,
                             src.n, _p(arrs[0]), _p(arrs[1]), _p(arrs[2]),
                             src.y.shape[1], _p(arrs[3]), _p(arrs[4]),
                             src.yf.shape[1], _p(arrs[5]), _p(arrs[6]), _p(selfV),
                             float(p["thres"]), float(kappa), _p(arrs[7]), _p(arrs[8]), _p(V), _p(K))
    return V, K


class DenseOperator:
    """y = A x for the full (multi-surface) system, optionally on sampled rows."""

    def __init__(self, problem, params=None):
        self.problem = problem
        self.p = full_params(params)
        self.sd = surfaces_data(problem, self.p)
        self.n = 2 * sum(F.n_panels(problem))

    def apply(self, x, rows_per_surface=None):
        pr = self.problem
        us = F.unknown_slices(pr)
        kap = [r["kappa"] for r in pr["regions"]]
        out = {}
        cache = {}
        for s in range(len(pr["surfaces"])):
            rows = np.arange(self.sd[s].n) if rows_per_surface is None else np.asarray(rows_per_surface[s])
            for side in (0, 1):
                out[(s, side)] = 0.5 * x[us[s][0]][rows]
        for blk in F.blocks(pr):
            s, t = blk.s, blk.t
            rows = np.arange(self.sd[s].n) if rows_per_surface is None else np.asarray(rows_per_surface[s])
            key = (s, t, kap[blk.R])
            if key not in cache:
                cache[key] = block_sums(self.sd[s].cen[rows], self.sd[t], kap[blk.R], self.p,
                                        x[us[t][0]], x[us[t][1]], rows if s == t else None)
            V, K = cache[key]
            out[(s, blk.row_side)] = out[(s, blk.row_side)] + blk.sigma * K - blk.sigma * blk.c * V
        return out

    def __call__(self, x):
        out = self.apply(x)
        y = np.empty(self.n)
        for (s, side), v in out.items():
            y[F.row_slice(self.problem, s, side)] = v
        return y

    def phi_reac(self, x):
        pr = self.problem
        ch = pr["charges"]
        Rc = ch["region"]
        kap = pr["regions"][Rc]["kappa"]
        us = F.unknown_slices(pr)
        out = np.zeros(len(ch["q"]))
        for t in F.region_surfaces(pr, Rc):
            sg, c = F.sigma_c(pr, Rc, t)
            V, K = block_sums(np.asarray(ch["xyz"]), self.sd[t], kap, self.p, x[us[t][0]], x[us[t][1]])
            out += sg * c * V - sg * K
        return out


def solve(problem, params=None, tol=None, precond=False, log=None):
    """GMRES solve with the dense matrix-free operator; returns dict(x, dG, iters, resid).

    precond: right block-Jacobi preconditioner from the panels' 2x2 self blocks
    (oracle.formulation.block_jacobi); it changes the iteration count, not the
    solution, and keeps the stopping test on the true residual.
    log: optional callable(str) told of every operator application."""
    op = DenseOperator(problem, params)
    b = rhs(problem, op.p, op.sd)
    M = F.block_jacobi(problem, lambda s, k: op.sd[s].self_V(k, op.p["N_k"])) if precond else None
    count = [0]

    def apply(v):
        count[0] += 1
        if log is not None:
            log(f"operator application {count[0]}")
        return op(v)
    x, it, res, _ = gmres(apply, b, tol=tol if tol is not None else op.p["gmres_tol"],
                          restart=op.p["restart"], max_iter=op.p["max_iter"], M_inv=M)
    phr = op.phi_reac(x)
    dG = 0.5 * KJ_PER_MOL * float(np.dot(problem["charges"]["q"], FOUR_PI * phr))
    return dict(x=x, dG=dG, iters=it, resid=res, phi_reac=phr)
