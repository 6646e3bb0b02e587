"""Dense FP64 collocation BEM: operator, right-hand side, reaction potential, energy.

This is the exact discrete problem that the treecode approximates (Sec. 2.2
and 2.3, "Treecode-accelerated BEM"), written out entry by entry:

  * V_R,ij = sum_k w_k A_j G_R(x_i, y_jk) and
    K_R,ij = sum_k w_k A_j n_j . grad_y G_R(x_i, y_jk)           (Eq. matel, with 1/4pi)
    with the K-point rule in the regular case;
  * the K_fine-point rule when |x_i - c_j| < thres * L_j (near-singular region);
  * the semi-analytical self integral for V and K_ii = 0 when i = j on the
    same surface (singular panel).

G_L = 1 / (4 pi r),  G_Y = exp(-kappa r) / (4 pi r)   (Eq. nBEM),
grad_y G = (x - y) (1 + kappa r) exp(-kappa r) / (4 pi r^3).

The reaction potential at the charges follows Eq. reac_integral and the
solvation energy Eq. solv, converted to kJ/mol with
C = e^2 N_A / (4 pi eps_0 * 1 Angstrom) / 1000 = 1389.3545764 kJ A mol^-1 e^-2
(CODATA 2018; the paper states no constants).  With the 1/(4 pi) kernels the
energy is dG = 1/2 * C * sum_k q_k * 4 pi phi_reac(r_k).
"""
from __future__ import annotations

import numpy as np

from . import formulation as F
from .geometry import gauss_points, panel_geometry
from .selfint import self_single_layer

FOUR_PI = 4.0 * np.pi
KJ_PER_MOL = 1389.3545764  # e^2 N_A / (4 pi eps0 * 1 A) / 1000, CODATA 2018

DEFAULT_PARAMS = dict(K=3, K_fine=19, N_k=5, thres=2.0, P=6, theta=0.5, ncrit=300,
                      gmres_tol=1e-4, restart=50, max_iter=1000)


def full_params(params=None):
    p = dict(DEFAULT_PARAMS)
    if params:
        p.update(params)
    return p


class SurfaceData:
    """Geometry and quadrature of one surface."""

    def __init__(self, verts, tris, K, K_fine):
        self.verts = np.asarray(verts, dtype=np.float64)
        self.tris = np.asarray(tris, dtype=np.int64)
        self.cen, self.normal, self.area, self.L = panel_geometry(self.verts, self.tris)
        self.n = self.tris.shape[0]
        y, wa, _ = gauss_points(self.verts, self.tris, K)
        self.y = y.reshape(self.n, K, 3)
        self.wa = wa.reshape(self.n, K)
        yf, waf, _ = gauss_points(self.verts, self.tris, K_fine)
        self.yf = yf.reshape(self.n, K_fine, 3)
        self.waf = waf.reshape(self.n, K_fine)
        self._sa = {}

    def self_V(self, kappa, Nk):
        key = (float(kappa), int(Nk))
        if key not in self._sa:
            self._sa[key] = self_single_layer(self.verts, self.tris, kappa, Nk)
        return self._sa[key]


def _kernel_sums(x, y, wa, normal, kappa):
    """sum_k wa_k G(x, y_k) and sum_k wa_k n . grad_y G(x, y_k) for pairs.

    x [..., 3], y [..., Kq, 3], wa [..., Kq], normal [..., 3] broadcastable.
    """
    r = x[..., None, :] - y
    rho2 = (r * r).sum(-1)
    rho = np.sqrt(rho2)
    rn = (r * normal[..., None, :]).sum(-1)
    if kappa == 0.0:
        g = 1.0 / rho
        dg = rn / (rho2 * rho)
    else:
        e = np.exp(-kappa * rho)
        g = e / rho
        dg = rn * (1.0 + kappa * rho) * e / (rho2 * rho)
    V = (wa * g).sum(-1) / FOUR_PI
    K = (wa * dg).sum(-1) / FOUR_PI
    return V, K


def kernel_matrices(x, src: SurfaceData, kappa, params, self_rows=None, chunk=None):
    """V [m,n] and K [m,n] of targets x [m,3] against the panels of ``src``.

    self_rows: None, or an int array [m] giving for each target the panel of
    ``src`` it is collocated on (-1 for none); that entry uses the
    semi-analytical rule (V) and K = 0.
    """
    p = full_params(params)
    x = np.asarray(x, dtype=np.float64)
    m, n = x.shape[0], src.n
    V = np.empty((m, n))
    K = np.empty((m, n))
    tl = p["thres"] * src.L
    tl2 = tl * tl
    if chunk is None:
        chunk = max(1, int(2_000_000 // max(1, n * src.y.shape[1])))
    with np.errstate(divide="ignore", invalid="ignore"):
        for a in range(0, m, chunk):
            b = min(m, a + chunk)
            xa = x[a:b]
            Vc, Kc = _kernel_sums(xa[:, None, :], src.y[None], src.wa[None], src.normal[None], kappa)
            d = xa[:, None, :] - src.cen[None]
            d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
            near = d2 < tl2[None, :]
            if self_rows is not None:
                sr = np.asarray(self_rows[a:b])
                has = sr >= 0
                near[np.where(has)[0], sr[has]] = False
            ii, jj = np.nonzero(near)
            if ii.size:
                Vf, Kf = _kernel_sums(xa[ii], src.yf[jj], src.waf[jj], src.normal[jj], kappa)
                Vc[ii, jj] = Vf
                Kc[ii, jj] = Kf
            if self_rows is not None:
                sr = np.asarray(self_rows[a:b])
                has = np.where(sr >= 0)[0]
                if has.size:
                    sa = src.self_V(kappa, p["N_k"])
                    Vc[has, sr[has]] = sa[sr[has]]
                    Kc[has, sr[has]] = 0.0
            V[a:b] = Vc
            K[a:b] = Kc
    return V, K


def surfaces_data(problem, params=None):
    p = full_params(params)
    return [SurfaceData(s["verts"], s["tris"], p["K"], p["K_fine"]) for s in problem["surfaces"]]


def operator_matrix(problem, params=None, sdata=None):
    """The 2N x 2N collocation matrix of the (multi-surface) system."""
    p = full_params(params)
    sd = sdata or surfaces_data(problem, p)
    n_tot = 2 * sum(F.n_panels(problem))
    A = np.zeros((n_tot, n_tot))
    us = F.unknown_slices(problem)
    kap = [r["kappa"] for r in problem["regions"]]
    cache = {}
    for blk in F.blocks(problem):
        rows = F.row_slice(problem, blk.s, blk.row_side)
        key = (blk.s, blk.t, kap[blk.R])
        if key not in cache:
            selfr = np.arange(sd[blk.s].n) if blk.s == blk.t else None
            cache[key] = kernel_matrices(sd[blk.s].cen, sd[blk.t], kap[blk.R], p, self_rows=selfr)
        V, K = cache[key]
        phi_t, dphi_t = us[blk.t]
        A[rows, phi_t] += blk.sigma * K
        A[rows, dphi_t] += -blk.sigma * blk.c * V
    for s in range(len(problem["surfaces"])):
        phi_s, _ = us[s]
        for side in (0, 1):
            rows = F.row_slice(problem, s, side)
            idx = np.arange(rows.start, rows.stop)
            A[idx, np.arange(phi_s.start, phi_s.stop)] += 0.5
    return A


def _green(x, y, kappa):
    d = x[:, None, :] - y[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    if kappa == 0.0:
        return 1.0 / (FOUR_PI * r)
    return np.exp(-kappa * r) / (FOUR_PI * r)


def rhs(problem, params=None, sdata=None):
    """b: sum_k q_k G_R(x_i, r_k) / eps_R on the rows of the charged region (Eq. matel Q)."""
    p = full_params(params)
    sd = sdata or surfaces_data(problem, p)
    n_tot = 2 * sum(F.n_panels(problem))
    b = np.zeros(n_tot)
    ch = problem.get("charges")
    if ch is None or len(ch["q"]) == 0:
        return b
    Rc = ch["region"]
    reg = problem["regions"][Rc]
    xyz = np.asarray(ch["xyz"], dtype=np.float64)
    q = np.asarray(ch["q"], dtype=np.float64)
    for s, surf in enumerate(problem["surfaces"]):
        for side, R in enumerate((surf["inner"], surf["outer"])):
            if R != Rc:
                continue
            rows = F.row_slice(problem, s, side)
            b[rows] += _green(sd[s].cen, xyz, reg["kappa"]) @ q / reg["eps"]
    return b


def reaction_matrix(problem, params=None, sdata=None):
    """Rm [N_c, 2N] with phi_reac(r_k) = (Rm x)_k (Eq. reac_integral, multi-surface form)."""
    p = full_params(params)
    sd = sdata or surfaces_data(problem, p)
    ch = problem["charges"]
    Rc = ch["region"]
    kap = problem["regions"][Rc]["kappa"]
    xyz = np.asarray(ch["xyz"], dtype=np.float64)
    n_tot = 2 * sum(F.n_panels(problem))
    Rm = np.zeros((xyz.shape[0], n_tot))
    us = F.unknown_slices(problem)
    for t in F.region_surfaces(problem, Rc):
        sg, c = F.sigma_c(problem, Rc, t)
        V, K = kernel_matrices(xyz, sd[t], kap, p)
        phi_t, dphi_t = us[t]
        Rm[:, dphi_t] += sg * c * V
        Rm[:, phi_t] += -sg * K
    return Rm


def solvation_energy_from_phi_reac(q, phi_reac):
    """Eq. solv in kJ/mol: 1/2 C sum_k q_k 4 pi phi_reac(r_k)."""
    return 0.5 * KJ_PER_MOL * float(np.dot(q, FOUR_PI * phi_reac))


def coulomb_energy(xyz, q, eps):
    """Coulomb energy of the point charges in a uniform dielectric eps, kJ/mol.

    The paper names this term (Eq. total_energy) without a formula; reading:
    E_C = 1/2 C sum_{i != j} q_i q_j / (eps r_ij).
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    d = xyz[:, None, :] - xyz[None, :, :]
    r = np.sqrt((d * d).sum(-1))
    np.fill_diagonal(r, np.inf)
    return 0.5 * KJ_PER_MOL * float((q[:, None] * q[None, :] / r).sum()) / eps


def solve_dense(problem, params=None):
    """LU solve of the dense system; returns dict(x, A, b, Rm, phi_reac, dG)."""
    p = full_params(params)
    sd = surfaces_data(problem, p)
    A = operator_matrix(problem, p, sd)
    b = rhs(problem, p, sd)
    x = np.linalg.solve(A, b)
    Rm = reaction_matrix(problem, p, sd)
    phi_reac = Rm @ x
    dG = solvation_energy_from_phi_reac(problem["charges"]["q"], phi_reac)
    return dict(x=x, A=A, b=b, Rm=Rm, phi_reac=phi_reac, dG=dG)
