"""Accuracy-versus-time sweeps (Sec. 3: time to solution against the error of
the solvation energy, for mesh refinement and the treecode/solver settings).

`sweep` solves each (problem, parameters) case through the library and
records the device time of setup + solve and the relative error of the energy
against a reference value; `pareto_front` keeps the cases no other case beats
in both time and error.  Every solve runs in the CUDA library; this module
only sequences them.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import pbbem


@dataclass
class Case:
    label: str
    params: dict
    panels: int
    time_s: float
    energy: float
    rel_error: float
    iterations: int


def sweep(cases, reference: float, ctx: pbbem.Context | None = None):
    """cases: iterable of (label, problem dict, pb_params dict).  Returns [Case]."""
    ctx = ctx or pbbem.Context(0)
    out = []
    for label, d, params in cases:
        pb = pbbem.Problem.from_dict(ctx, d)
        pb.setup(**params)
        r = pb.solve()
        pb.close()
        out.append(Case(label, dict(params), int(sum(int(s["tris"].shape[0]) for s in d["surfaces"])),
                        (r.setup_ms + r.solve_ms) / 1e3, r.dG_solv, abs(r.dG_solv - reference) / abs(reference),
                        r.iterations))
    return out


def pareto_front(cases):
    """The cases not dominated in (time, error), fastest first."""
    front, best = [], float("inf")
    for c in sorted(cases, key=lambda c: (c.time_s, c.rel_error)):
        if c.rel_error < best:
            front.append(c)
            best = c.rel_error
    return front
