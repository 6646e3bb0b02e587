"""Mesh-refinement convergence study (Sec. 3, "Richardson extrapolation").

Solves one molecule on a sequence of meshes whose panel size shrinks by a
constant ratio r (r = h_coarse / h_fine, with h the panel area or spacing)
and reports, from the three finest results f1 (finest), f2, f3 (coarsest):

  * the observed order of convergence (Eq. observed_order)
        p = log((f3 - f2) / (f2 - f1)) / log(r),
  * the extrapolated value (Eq. rich_extr)
        f_exact ~ f1 + (f1 - f2) / (r**p - 1).

A result is in the asymptotic range when p matches the method's expected
order (one, in the panel area, for flat panels with centroid collocation).
Every solve runs through the CUDA library; this module only sequences them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import pbbem


def observed_order(f1: float, f2: float, f3: float, r: float) -> float:
    """Eq. observed_order: order from three results refined by a constant ratio r (f1 finest).

    NaN when the two differences have opposite signs (or one is zero): the
    results are not converging monotonically, i.e. not in the asymptotic range.
    """
    q = (f3 - f2) / (f2 - f1) if f2 != f1 else float("nan")
    return math.log(q) / math.log(r) if q > 0 else float("nan")


def extrapolate(f1: float, f2: float, r: float, p: float) -> float:
    """Eq. rich_extr: estimate of the exact value from the two finest results."""
    return f1 + (f1 - f2) / (r ** p - 1.0)


@dataclass
class Study:
    panels: list = field(default_factory=list)
    energies: list = field(default_factory=list)
    solve_s: list = field(default_factory=list)
    iterations: list = field(default_factory=list)
    ratio: float = 0.0
    order: float = float("nan")
    extrapolated: float = float("nan")


def study(problems, ratio: float, ctx: pbbem.Context | None = None, **params) -> Study:
    """Solve `problems` (problem dicts, coarsest first, refined by `ratio`) and extrapolate.

    params are pb_params fields (precision, theta, P, gmres_tol, ...).
    """
    ctx = ctx or pbbem.Context(0)
    out = Study(ratio=float(ratio))
    for d in problems:
        pb = pbbem.Problem.from_dict(ctx, d)
        pb.setup(**params)
        r = pb.solve()
        out.panels.append(int(sum(int(s["tris"].shape[0]) for s in d["surfaces"])))
        out.energies.append(r.dG_solv)
        out.solve_s.append((r.setup_ms + r.solve_ms) / 1e3)
        out.iterations.append(r.iterations)
        pb.close()
    if len(out.energies) >= 3:
        f3, f2, f1 = out.energies[-3:]
        out.order = observed_order(f1, f2, f3, ratio)
        if out.order == out.order:
            out.extrapolated = extrapolate(f1, f2, ratio, out.order)
    return out
