"""Exact gradient of the discrete solvation energy by the adjoint method (dense FP64).

TEST INFRASTRUCTURE ONLY (see the package header).

The solvation energy of Eq. solv is, with the discrete operator A (Eq. matrix
and its multi-surface form), the right-hand side b = B q (Eq. matel, Q) and
the reaction-potential map phi_reac = Rm x (Eq. reac_integral),

    E(q, r, eps, kappa) = c0 q^T Rm x,   A x = B q,   c0 = 1/2 C 4 pi.

With the adjoint lambda of A^T lambda = c0 Rm^T q (so that E = lambda^T b):

    dE/dq   = c0 Rm x + B^T lambda
    dE/dr_k = c0 q_k grad_r (Rm x)_k + q_k sum_i lambda_i grad_r B_ik
    dE/dp   = c0 q^T (dRm/dp) x + lambda^T (dB/dp) q - lambda^T (dA/dp) x

for p = eps_R or kappa_R of any region R.  Every derivative matrix is the
derivative of the entries exactly as the dense oracle defines them: K-point
rule far, K_fine rule for near-singular pairs, the semi-analytical rule on the
panel itself (its kappa derivative by the same rule), so the result is the
derivative of the discrete energy.  The rule choice (near or far) is held
fixed, as a derivative must.

Kernel derivatives (r = x - y, rho = |r|, e = exp(-kappa rho), all / 4 pi):
    dG/dkappa                   = -e
    d(n . grad_y G)/dkappa      = -kappa (r . n) e / rho
    grad_x G_L                  = -r / rho^3
    grad_x (n . grad_y G_L)     = n / rho^3 - 3 (r . n) r / rho^5
    grad_r G_L(x_i, r)          = (x_i - r) / rho^3
Charges sit in a kappa = 0 region (Laplace kernel), as in the paper's
molecules; the position gradient is written for that kernel only.

Pins (tests/test_oracle_gradient.py): central finite differences of the
energy in every q_k, every coordinate of r_k, every eps_R and kappa_R;
q . dE/dq = 2E (E is quadratic in q); sum_R eps_R dE/deps_R = -E (E scales
as 1/alpha when every eps is multiplied by alpha); the kappa and charge-
position derivatives of the Kirkwood closed form.
"""
from __future__ import annotations

import numpy as np

from . import formulation as F
from .dense import (FOUR_PI, KJ_PER_MOL, full_params, operator_matrix, reaction_matrix, rhs,
                    surfaces_data, kernel_matrices)
from .selfint import self_single_layer_dkappa

C0 = 0.5 * KJ_PER_MOL * FOUR_PI


def _near_mask(x, src, thres, self_rows):
    """The dense oracle's rule choice: K_fine where |x_i - c_j| < thres L_j, not on the own panel."""
    tl = thres * src.L
    d = x[:, None, :] - src.cen[None]
    d2 = (d[..., 0] * d[..., 0] + d[..., 1] * d[..., 1]) + d[..., 2] * d[..., 2]
    near = d2 < (tl * tl)[None, :]
    if self_rows is not None:
        sr = np.asarray(self_rows)
        has = np.where(sr >= 0)[0]
        near[has, sr[has]] = False
    return near


def _dkappa_sums(x, y, wa, normal, kappa):
    r = x[..., None, :] - y
    rho = np.sqrt((r * r).sum(-1))
    rn = (r * normal[..., None, :]).sum(-1)
    e = np.exp(-kappa * rho)
    dV = (wa * -e).sum(-1) / FOUR_PI
    dK = (wa * (-kappa * rn * e / rho)).sum(-1) / FOUR_PI
    return dV, dK


def kernel_matrices_dkappa(x, src, kappa, params, self_rows=None):
    """dV/dkappa [m,n] and dK/dkappa [m,n] of targets x against the panels of src."""
    p = full_params(params)
    x = np.asarray(x, dtype=np.float64)
    dV, dK = _dkappa_sums(x[:, None, :], src.y[None], src.wa[None], src.normal[None], kappa)
    near = _near_mask(x, src, p["thres"], self_rows)
    ii, jj = np.nonzero(near)
    if ii.size:
        fV, fK = _dkappa_sums(x[ii], src.yf[jj], src.waf[jj], src.normal[jj], kappa)
        dV[ii, jj] = fV
        dK[ii, jj] = fK
    if self_rows is not None:
        sr = np.asarray(self_rows)
        has = np.where(sr >= 0)[0]
        if has.size:
            sd = self_single_layer_dkappa(src.verts, src.tris, kappa, p["N_k"])
            dV[has, sr[has]] = sd[sr[has]]
            dK[has, sr[has]] = 0.0
    return dV, dK


def _grad_sums(x, y, wa, normal):
    r = x[..., None, :] - y
    rho2 = (r * r).sum(-1)
    rho = np.sqrt(rho2)
    rn = (r * normal[..., None, :]).sum(-1)
    i3 = 1.0 / (rho2 * rho)
    gV = (wa[..., None] * (-r * i3[..., None])).sum(-2) / FOUR_PI
    gK = (wa[..., None] * (normal[..., None, :] * i3[..., None]
                           - 3.0 * (rn * i3 / rho2)[..., None] * r)).sum(-2) / FOUR_PI
    return gV, gK


def kernel_matrices_grad(x, src, params):
    """grad_x V_L [m,n,3] and grad_x K_L [m,n,3] (targets off the surface, Laplace kernel)."""
    p = full_params(params)
    x = np.asarray(x, dtype=np.float64)
    gV, gK = _grad_sums(x[:, None, :], src.y[None], src.wa[None], src.normal[None])
    near = _near_mask(x, src, p["thres"], None)
    ii, jj = np.nonzero(near)
    if ii.size:
        fV, fK = _grad_sums(x[ii], src.yf[jj], src.waf[jj], src.normal[jj])
        gV[ii, jj] = fV
        gK[ii, jj] = fK
    return gV, gK


def charge_matrix(problem, sdata):
    """B [2N, N_c] with b = B q: G_Rc(c_i, r_k) / eps_Rc on the rows of the charged region."""
    ch = problem["charges"]
    Rc = ch["region"]
    reg = problem["regions"][Rc]
    xyz = np.asarray(ch["xyz"], dtype=np.float64)
    n_tot = 2 * sum(F.n_panels(problem))
    B = np.zeros((n_tot, xyz.shape[0]))
    dBk = np.zeros_like(B)           # d/dkappa_Rc
    gB = np.zeros((n_tot, xyz.shape[0], 3))   # d/dr_k (Laplace)
    for s, surf in enumerate(problem["surfaces"]):
        for side, R in enumerate((surf["inner"], surf["outer"])):
            if R != Rc:
                continue
            rows = F.row_slice(problem, s, side)
            d = sdata[s].cen[:, None, :] - xyz[None, :, :]
            r = np.sqrt((d * d).sum(-1))
            e = np.exp(-reg["kappa"] * r)
            B[rows] = e / (FOUR_PI * r) / reg["eps"]
            dBk[rows] = -e / FOUR_PI / reg["eps"]
            gB[rows] = d / (r ** 3)[..., None] / FOUR_PI / reg["eps"]
    return B, dBk, gB


def _dc(problem, R, t, p):
    """d c_{R,t} / d eps_p, with c = 1 (R inner of t) or eps_inner(t) / eps_R (R outer of t)."""
    surf = problem["surfaces"][t]
    if surf["inner"] == R:
        return 0.0
    eps = [r["eps"] for r in problem["regions"]]
    i = surf["inner"]
    out = 0.0
    if p == i:
        out += 1.0 / eps[R]
    if p == R:
        out -= eps[i] / eps[R] ** 2
    return out


def operator_derivatives(problem, params, sd):
    """dA/deps_p and dA/dkappa_p for every region p (lists of 2N x 2N matrices)."""
    nreg = len(problem["regions"])
    n_tot = 2 * sum(F.n_panels(problem))
    us = F.unknown_slices(problem)
    kap = [r["kappa"] for r in problem["regions"]]
    dAe = [np.zeros((n_tot, n_tot)) for _ in range(nreg)]
    dAk = [np.zeros((n_tot, n_tot)) for _ in range(nreg)]
    Vc, Dc = {}, {}
    for blk in F.blocks(problem):
        rows = F.row_slice(problem, blk.s, blk.row_side)
        phi_t, dphi_t = us[blk.t]
        key = (blk.s, blk.t, kap[blk.R])
        selfr = np.arange(sd[blk.s].n) if blk.s == blk.t else None
        if key not in Vc:
            Vc[key] = kernel_matrices(sd[blk.s].cen, sd[blk.t], kap[blk.R], params, self_rows=selfr)[0]
            Dc[key] = kernel_matrices_dkappa(sd[blk.s].cen, sd[blk.t], kap[blk.R], params, self_rows=selfr)
        for p in range(nreg):
            dc = _dc(problem, blk.R, blk.t, p)
            if dc:
                dAe[p][rows, dphi_t] += -blk.sigma * dc * Vc[key]
        dV, dK = Dc[key]
        dAk[blk.R][rows, phi_t] += blk.sigma * dK
        dAk[blk.R][rows, dphi_t] += -blk.sigma * blk.c * dV
    return dAe, dAk


def reaction_derivatives(problem, params, sd):
    """dRm/deps_p, dRm/dkappa_Rc and grad_r Rm (row k's gradient in r_k) [N_c, 2N, 3]."""
    ch = problem["charges"]
    Rc = ch["region"]
    kap = problem["regions"][Rc]["kappa"]
    if kap != 0.0:
        raise ValueError("charges must sit in a kappa = 0 region")
    xyz = np.asarray(ch["xyz"], dtype=np.float64)
    nreg = len(problem["regions"])
    n_tot = 2 * sum(F.n_panels(problem))
    us = F.unknown_slices(problem)
    dRe = [np.zeros((xyz.shape[0], n_tot)) for _ in range(nreg)]
    dRk = np.zeros((xyz.shape[0], n_tot))
    gR = np.zeros((xyz.shape[0], n_tot, 3))
    for t in F.region_surfaces(problem, Rc):
        sg, c = F.sigma_c(problem, Rc, t)
        phi_t, dphi_t = us[t]
        V, _ = kernel_matrices(xyz, sd[t], kap, params)
        for p in range(nreg):
            dc = _dc(problem, Rc, t, p)
            if dc:
                dRe[p][:, dphi_t] += sg * dc * V
        dV, dK = kernel_matrices_dkappa(xyz, sd[t], kap, params)
        dRk[:, dphi_t] += sg * c * dV
        dRk[:, phi_t] += -sg * dK
        gV, gK = kernel_matrices_grad(xyz, sd[t], params)
        gR[:, dphi_t, :] += sg * c * gV
        gR[:, phi_t, :] += -sg * gK
    return dRe, dRk, gR


def solvation_gradient(problem, params=None):
    """Energy, solution, adjoint and gradient of the discrete solvation energy (LU solves).

    Returns dict(E, x, lam, dq [N_c], dxyz [N_c,3], deps [n_regions], dkappa [n_regions]).
    """
    p = full_params(params)
    sd = surfaces_data(problem, p)
    ch = problem["charges"]
    q = np.asarray(ch["q"], dtype=np.float64)
    Rc = ch["region"]
    A = operator_matrix(problem, p, sd)
    B, dBk, gB = charge_matrix(problem, sd)
    b = B @ q
    x = np.linalg.solve(A, b)
    Rm = reaction_matrix(problem, p, sd)
    E = C0 * float(q @ (Rm @ x))
    lam = np.linalg.solve(A.T, C0 * (Rm.T @ q))
    dq = C0 * (Rm @ x) + B.T @ lam
    dRe, dRk, gR = reaction_derivatives(problem, p, sd)
    dxyz = C0 * q[:, None] * np.einsum("kjd,j->kd", gR, x) + q[:, None] * np.einsum("ikd,i->kd", gB, lam)
    dAe, dAk = operator_derivatives(problem, p, sd)
    nreg = len(problem["regions"])
    eps_rc = problem["regions"][Rc]["eps"]
    deps = np.zeros(nreg)
    dkap = np.zeros(nreg)
    for r in range(nreg):
        dB_e = -B / eps_rc if r == Rc else None
        deps[r] = C0 * float(q @ (dRe[r] @ x)) - float(lam @ (dAe[r] @ x))
        if dB_e is not None:
            deps[r] += float(lam @ (dB_e @ q))
        dkap[r] = -float(lam @ (dAk[r] @ x))
        if r == Rc:
            dkap[r] += C0 * float(q @ (dRk @ x)) + float(lam @ (dBk @ q))
    return dict(E=E, x=x, lam=lam, dq=dq, dxyz=dxyz, deps=deps, dkappa=dkap, A=A, Rm=Rm, B=B)


def energy_only(problem, params=None):
    """Discrete solvation energy by LU (for finite differences)."""
    p = full_params(params)
    sd = surfaces_data(problem, p)
    A = operator_matrix(problem, p, sd)
    b = rhs(problem, p, sd)
    x = np.linalg.solve(A, b)
    Rm = reaction_matrix(problem, p, sd)
    return C0 * float(np.asarray(problem["charges"]["q"]) @ (Rm @ x))
