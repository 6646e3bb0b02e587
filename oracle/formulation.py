"""Block structure of the single- and multi-surface boundary-integral system.

Single surface (Sec. 2.2, Eqs. nBEM, nBEM_disc, matrix, matel): for the
protein region Omega_1 (Poisson, eps_1, charges) inside Gamma and the solvent
Omega_2 (linearised PB, eps_2, kappa) outside, the unknowns are phi_1 and
dphi_1/dn at the panel centroids and the 2N x 2N system is

    [ 1/2 I + K_L      -V_L          ] [ phi   ]   [ Q ]
    [ 1/2 I - K_Y   (eps1/eps2) V_Y  ] [ dphi  ] = [ 0 ].

Readings where the paper is garbled or silent (Sec. 2.1 Eqs. nBEM, reac_integral; Sec. 2.2 Eqs. nBEM_disc, matrix, matel):
  * The ratio on V_Y is eps1/eps2 (Eqs. nBEM_disc and matrix); the eps2/eps1
    printed in Eq. nBEM contradicts flux continuity and is read as a typo.
  * Every kernel, Q and phi_reac keep the 1/(4 pi) of Eqs. nBEM/nBEM_disc
    (Eq. matel drops it, which is inconsistent with the 1/2 jump term).
  * Charge sums run over k = 1..N_c.
  * Multi-surface problems (Sec. 2.2 "Multi-surface problems" defers to
    Altman et al. 2009): every surface t carries phi_t and dphi_t/dn taken on
    its inner side.  For every region R and every surface s on its boundary
    there is one equation collocated on s,

        1/2 phi_s - sum_{t in dR} sigma_{R,t} [c_{R,t} V_R(s,t) dphi_t - K_R(s,t) phi_t]
            = [R charged] sum_k q_k G_R(x, r_k) / eps_R,

    with sigma = +1 when R is t's inner region and -1 when it is t's outer
    region, c = 1 when R is t's inner region and eps_inner(t)/eps_R otherwise,
    and G_R the Laplace kernel if kappa_R = 0, else the Yukawa kernel.  With
    one surface this is exactly Eq. matrix.  Unknown and row order: surface by
    surface, [phi_1, dphi_1, phi_2, dphi_2, ...]; the two row blocks of
    surface s are its inner-region equation, then its outer-region equation.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class Block:
    s: int          # collocation (target) surface
    R: int          # region whose Green's function is used
    row_side: int   # 0: s's inner-region equation, 1: outer-region equation
    t: int          # source surface
    sigma: float
    c: float


def n_panels(problem):
    return [int(np.asarray(s["tris"]).shape[0]) for s in problem["surfaces"]]


def offsets(problem):
    """Start of each surface's panel range in the concatenated panel list."""
    n = n_panels(problem)
    return np.concatenate([[0], np.cumsum(n)]).astype(np.int64)


def region_surfaces(problem, R):
    return [t for t, s in enumerate(problem["surfaces"]) if s["inner"] == R or s["outer"] == R]


def sigma_c(problem, R, t):
    surf = problem["surfaces"][t]
    eps = [r["eps"] for r in problem["regions"]]
    if surf["inner"] == R:
        return 1.0, 1.0
    if surf["outer"] == R:
        return -1.0, eps[surf["inner"]] / eps[R]
    raise ValueError("surface does not bound region")


def blocks(problem):
    out = []
    for s, surf in enumerate(problem["surfaces"]):
        for side, R in enumerate((surf["inner"], surf["outer"])):
            for t in region_surfaces(problem, R):
                sg, c = sigma_c(problem, R, t)
                out.append(Block(s, R, side, t, sg, c))
    return out


def unknown_slices(problem):
    """(phi slice, dphi slice) of every surface in the 2N unknown vector."""
    off = offsets(problem)
    n = n_panels(problem)
    return [(slice(2 * off[t], 2 * off[t] + n[t]), slice(2 * off[t] + n[t], 2 * off[t] + 2 * n[t]))
            for t in range(len(n))]


def row_slice(problem, s, side):
    off = offsets(problem)
    n = n_panels(problem)
    return slice(2 * off[s] + side * n[s], 2 * off[s] + (side + 1) * n[s])


def block_jacobi(problem, self_V):
    """Right preconditioner from the 2x2 self blocks of every panel.

    The paper names no preconditioner; this optional variant inverts, panel by
    panel, the diagonal entries of the four (s, s) blocks: [1/2, cV_in V_in,ii;
    1/2, cV_out V_out,ii], with K_ii = 0 and cV = -sigma c of the row's region.
    self_V(s, kappa) -> semi-analytical V_ii of the panels of surface s.
    Returns z -> M^-1 z on the 2N unknown vector.
    """
    eps = [r["eps"] for r in problem["regions"]]
    kap = [r["kappa"] for r in problem["regions"]]
    blocks_ = []
    for s, surf in enumerate(problem["surfaces"]):
        coef = []
        for R in (surf["inner"], surf["outer"]):
            sg, c = sigma_c(problem, R, s)
            coef.append(-sg * c * self_V(s, kap[R]))
        a11 = 0.5
        a12 = coef[0]
        a21 = 0.5
        a22 = coef[1]
        det = a11 * a22 - a12 * a21
        blocks_.append((a22 / det, -a12 / det, -a21 / det, a11 / det))
    us = unknown_slices(problem)

    def apply(z):
        out = np.empty_like(z)
        for s, (m11, m12, m21, m22) in enumerate(blocks_):
            ps, ds = us[s]
            u1 = z[row_slice(problem, s, 0)]
            u2 = z[row_slice(problem, s, 1)]
            out[ps] = m11 * u1 + m12 * u2
            out[ds] = m21 * u1 + m22 * u2
        return out

    return apply
