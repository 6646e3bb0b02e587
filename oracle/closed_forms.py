"""Closed-form solvation energies of spherical molecules (test pins for the BEM).

Kirkwood (1934) sphere: a ball of radius a, permittivity eps1, holding point
charges, in a solvent eps2 with inverse Debye length kappa.  Expanding the
potential in Legendre polynomials about the centre and imposing continuity of
phi and eps dphi/dr at r = a (Eq. pde) gives the reaction potential

  phi_reac(r_j) = sum_i q_i sum_n f_n (r_i r_j)^n / a^(2n+1) P_n(cos g_ij),
  f_n = [(n+1) + (eps2/eps1) g_n] / (eps1 n - eps2 g_n),
  g_n = x k_n'(x) / k_n(x),  x = kappa a   (g_n = -(n+1) when kappa = 0),

with k_n the modified spherical Bessel function of the second kind, and
dG = 1/2 C sum_j q_j phi_reac(r_j) (Eq. solv).  The paper quotes the centred
kappa = 0 case as -41.2465 kJ/mol (Sec. 3.1).

Layered spheres: concentric interfaces a_1 < ... < a_L, region m between
a_m and a_{m+1} with (eps_m, kappa_m); per Legendre order n the general
solution in region m is A r^n + B r^-(n+1) (kappa = 0) or A i_n(kappa r) +
B k_n(kappa r), plus the free-space potential of the charges in their region.
Continuity of phi and eps dphi/dr at each interface gives a 2L x 2L system per n.
This is the multi-surface (Stern layer, cavity) pin.
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_legendre, spherical_in, spherical_kn

KJ_PER_MOL = 1389.3545764


def _cosg(ri, rj):
    ni, nj = np.linalg.norm(ri), np.linalg.norm(rj)
    if ni == 0.0 or nj == 0.0:
        return 1.0
    return float(np.clip(np.dot(ri, rj) / (ni * nj), -1.0, 1.0))


def kirkwood_energy(a, eps1, eps2, kappa, xyz, q, nmax=80):
    """Solvation energy (kJ/mol) of charges inside a sphere centred at the origin."""
    a, eps1, eps2, kappa = float(a), float(eps1), float(eps2), float(kappa)
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).ravel()
    n = np.arange(nmax + 1, dtype=np.float64)
    if kappa == 0.0:
        g = -(n + 1.0)
    else:
        x = kappa * a
        ni = np.arange(nmax + 1)
        g = x * spherical_kn(ni, x, derivative=True) / spherical_kn(ni, x)
    f = ((n + 1.0) + (eps2 / eps1) * g) / (eps1 * n - eps2 * g)
    E = 0.0
    for i in range(len(q)):
        for j in range(len(q)):
            ri, rj = np.linalg.norm(xyz[i]), np.linalg.norm(xyz[j])
            c = _cosg(xyz[i], xyz[j])
            terms = f * (ri * rj / (a * a)) ** n / a * eval_legendre(n.astype(int), c)
            E += q[i] * q[j] * terms.sum()
    return 0.5 * KJ_PER_MOL * E


def _radial(n, kappa, r, which):
    """Regular (0) / decaying (1) radial solution and its r-derivative."""
    if kappa == 0.0:
        if which == 0:
            return r ** n, n * r ** (n - 1) if n > 0 else 0.0
        return r ** (-(n + 1.0)), -(n + 1.0) * r ** (-(n + 2.0))
    x = kappa * r
    if which == 0:
        return spherical_in(n, x), kappa * spherical_in(n, x, derivative=True)
    return spherical_kn(n, x), kappa * spherical_kn(n, x, derivative=True)


def layered_sphere_energy(radii, eps, kappa, charge_region, xyz, q, nmax=60):
    """Solvation energy of charges in concentric layers (kJ/mol).

    radii: interface radii a_1 < ... < a_L; eps, kappa: L+1 region values from
    the innermost ball outwards; charge_region: index of the region holding all
    charges.  The reference state is the charges' own region filling space.
    """
    radii = np.asarray(radii, dtype=np.float64)
    eps = [float(e) for e in eps]
    kappa = [float(k) for k in kappa]
    L = radii.size
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64).ravel()
    epsc = eps[charge_region]
    E = 0.0
    for i in range(len(q)):
        b = np.linalg.norm(xyz[i])
        # reaction coefficients for the source charge i, order by order
        for n in range(nmax + 1):
            # unknowns: region m has (A_m, B_m); region 0 only A, region L only B
            # the homogeneous solution in the charged region is the reaction field
            idx = {}
            k = 0
            for m in range(L + 1):
                if m < L:
                    idx[(m, 0)] = k; k += 1
                if m > 0:
                    idx[(m, 1)] = k; k += 1
            M = np.zeros((k, k))
            rhs = np.zeros(k)
            for j in range(L):
                a = radii[j]
                inner, outer = j, j + 1
                # free-space term of the charge (q/eps_c) b^n/r^(n+1) (r > b) or r^n/b^(n+1)
                def free(r):
                    if r > b:
                        return b ** n / r ** (n + 1.0), -(n + 1.0) * b ** n / r ** (n + 2.0)
                    return r ** n / b ** (n + 1.0), (n * r ** (n - 1) if n > 0 else 0.0) / b ** (n + 1.0)
                for m, sgn in ((inner, 1.0), (outer, -1.0)):
                    for which in (0, 1):
                        if (m, which) not in idx:
                            continue
                        f0, f1 = _radial(n, kappa[m], a, which)
                        M[2 * j, idx[(m, which)]] += sgn * f0
                        M[2 * j + 1, idx[(m, which)]] += sgn * eps[m] * f1
                    if m == charge_region:
                        g0, g1 = free(a)
                        rhs[2 * j] -= sgn * g0 / epsc
                        rhs[2 * j + 1] -= sgn * eps[m] * g1 / epsc
            coef = np.linalg.solve(M, rhs)
            m = charge_region
            for j2 in range(len(q)):
                rj = np.linalg.norm(xyz[j2])
                c = _cosg(xyz[i], xyz[j2])
                val = 0.0
                for which in (0, 1):
                    if (m, which) in idx:
                        val += coef[idx[(m, which)]] * _radial(n, kappa[m], rj, which)[0]
                E += q[i] * q[j2] * val * eval_legendre(n, c)
    return 0.5 * KJ_PER_MOL * E
