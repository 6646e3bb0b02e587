"""Autotuner of the treecode settings (theta, P, ncrit) and the P2P tile for batched solves.

The treecode's cost splits between the direct sums (P2P, whose source tile is
a leaf of fewer than ncrit points, swept by a warp for up to p2p_tile
targets at a time) and the expansions (M2P, whose work grows with P and the
number of accepted boxes, i.e. falls as theta grows).  Which setting is
fastest at a given energy accuracy depends on the molecule's size and shape,
so the tuner measures it:

* `tune` solves one problem with every candidate setting, times setup +
  solve on the device (the library's CUDA events, best of `repeats`),
  measures the energy's error against an accurate reference (theta = 0.3,
  P = 10, tight GMRES tolerance), and keeps the fastest candidate whose
  error is at most `target` / `safety`; then it times that setting with
  every P2P tile (targets per work item: the energy does not depend on it)
  and keeps the fastest.
* `Schedule` bins problems by panel count (factor-of-two classes), tunes one
  representative per class (the median problem) and hands every problem the
  setting of its class.

Every solve runs in the CUDA library; this module only sequences them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

from . import pbbem

# (theta, P) pairs of roughly balanced accuracy, times leaf sizes
THETA_P = ((0.7, 3), (0.6, 4), (0.5, 5), (0.5, 6), (0.4, 7), (0.4, 8))
NCRIT = (100, 200, 300, 500)
P2P_TILES = (64, 32, 16, 8)
REFERENCE = dict(theta=0.3, P=10, gmres_tol=1e-7)


@dataclass
class Choice:
    theta: float
    P: int
    ncrit: int
    time_s: float
    rel_error: float
    p2p_tile: int = 64

    def params(self) -> dict:
        return dict(theta=self.theta, P=self.P, ncrit=self.ncrit, p2p_tile=self.p2p_tile)


def candidates(theta_p=THETA_P, ncrit=NCRIT):
    return [dict(theta=t, P=p, ncrit=n) for t, p in theta_p for n in ncrit]


def _energy_and_time(ctx, d, params, repeats):
    pb = pbbem.Problem.from_dict(ctx, d)
    try:
        best, e = math.inf, None
        for _ in range(max(1, repeats)):
            pb.setup(**params)
            r = pb.solve()
            best = min(best, (r.setup_ms + r.solve_ms) / 1e3)
            e = r.dG_solv
        return e, best
    finally:
        pb.close()


def pick(measured, target, safety=2.0):
    """Fastest (params, time, error) within target / safety; the most accurate one if none is."""
    ok = [m for m in measured if m[2] <= target / safety]
    if ok:
        return min(ok, key=lambda m: m[1])
    return min(measured, key=lambda m: m[2])


def tune(ctx, d, target=1e-4, base=None, cands=None, repeats=2, safety=2.0, reference=None,
         tiles=P2P_TILES) -> Choice:
    """Fastest candidate setting for problem dict `d` within `target` relative energy error.

    base: other pb_params fields (precision, gmres_tol, K, ...), mixed precision by default.
    reference: the accurate energy if already known.
    """
    base = dict(dict(precision="mixed", gmres_tol=1e-4), **(base or {}))
    if reference is None:
        reference, _ = _energy_and_time(ctx, d, dict(base, **REFERENCE), 1)
    measured = []
    for c in cands or candidates():
        e, t = _energy_and_time(ctx, d, dict(base, **c), repeats)
        measured.append((c, t, abs(e - reference) / abs(reference)))
    c, t, err = pick(measured, target, safety)
    tile = c.get("p2p_tile", 64)
    for tl in tiles:
        if tl == tile:
            continue
        _, tt = _energy_and_time(ctx, d, dict(base, **dict(c, p2p_tile=tl)), repeats)
        if tt < t:
            tile, t = tl, tt
    return Choice(c["theta"], c["P"], c["ncrit"], t, err, tile)


def panel_count(d) -> int:
    n = 0
    for s in d["surfaces"]:
        if "tris" in s:
            n += int(len(s["tris"]))
        else:
            raise ValueError("panel_count needs meshes; generate device surfaces first")
    return n


def size_class(panels: int) -> int:
    """Factor-of-two bin of a panel count."""
    return int(math.floor(math.log2(max(1, panels))))


@dataclass
class Schedule:
    choices: dict = field(default_factory=dict)     # size class -> Choice

    @classmethod
    def build(cls, ctx, problems, target=1e-4, base=None, cands=None, repeats=2, safety=2.0):
        """Tune the median problem of every size class present in `problems` (problem dicts)."""
        by = {}
        for d in problems:
            by.setdefault(size_class(panel_count(d)), []).append(d)
        out = cls()
        for k, ds in sorted(by.items()):
            ds = sorted(ds, key=panel_count)
            out.choices[k] = tune(ctx, ds[len(ds) // 2], target, base, cands, repeats, safety)
        return out

    def params_for(self, d) -> dict:
        """Setting of the problem's size class (the nearest tuned class if its own was not tuned)."""
        k = size_class(panel_count(d))
        if k not in self.choices:
            k = min(self.choices, key=lambda c: abs(c - k))
        return self.choices[k].params()
