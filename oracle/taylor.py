"""Taylor coefficients and multipole moments of the treecode (Sec. 2.3, Eqs. taylor, multexp).

The far field of a box with centre y_c is

    V(x) ~ sum_{|k| <= P} a^k(x, y_c) m_c^k,   a^k = (1/k!) D_y^k psi(x, y_c),
                                              m_c^k = sum_j q_j (y_j - y_c)^k.

The paper computes a^k with the recurrences of Duan & Krasny (Laplace) and
Li, Johnston & Krasny (Yukawa).  The oracle deliberately does NOT use any
recurrence: it obtains a^k as the coefficients of the truncated multivariate
power series (a "jet") of psi(x, y_c + h) in h, built from the series of
rho^2 = sum_a (u_a + h_a)^2 (u = y_c - x) by the univariate expansions of
sqrt, 1/x and exp.  Any error in a recurrence then shows up as a mismatch.

Double-layer terms use the moments of the dipole sources d_j:
n_j . grad_y psi(x, y_j) ~ sum_k a^k D^k with
D^k = sum_j sum_l d_{j,l} k_l (y_j - y_c)^(k - e_l).

Pins (tests/test_oracle_taylor.py): axis-aligned coefficients equal the 1-D
derivatives of 1/r and exp(-kappa r)/r written in closed form; the jets
satisfy the screened-Laplace equation term by term; the truncated series
reproduces psi(x, y) with an error O(|h|^(P+1)).
"""
from __future__ import annotations

import functools
from math import comb

import numpy as np

FOUR_PI = 4.0 * np.pi


@functools.lru_cache(maxsize=None)
def multi_indices(P: int):
    """All k = (k1, k2, k3) with |k| <= P, graded by |k| then lexicographic."""
    out = []
    for n in range(P + 1):
        for k1 in range(n, -1, -1):
            for k2 in range(n - k1, -1, -1):
                out.append((k1, k2, n - k1 - k2))
    return tuple(out)


@functools.lru_cache(maxsize=None)
def _index_map(P):
    return {k: i for i, k in enumerate(multi_indices(P))}


@functools.lru_cache(maxsize=None)
def _product_table(P):
    ks = multi_indices(P)
    idx = _index_map(P)
    a, b, c = [], [], []
    for i, ki in enumerate(ks):
        for j, kj in enumerate(ks):
            s = (ki[0] + kj[0], ki[1] + kj[1], ki[2] + kj[2])
            if sum(s) <= P:
                a.append(i); b.append(j); c.append(idx[s])
    return np.array(a), np.array(b), np.array(c)


def jet_mul(A, B, P):
    """Truncated product of two jets [..., nterms]."""
    ia, ib, ic = _product_table(P)
    out = np.zeros(np.broadcast_shapes(A.shape, B.shape))
    prod = A[..., ia] * B[..., ib]
    for t in range(out.shape[-1]):
        sel = ic == t
        out[..., t] = prod[..., sel].sum(-1)
    return out


def _compose(c0, H, coeffs, P):
    """sum_m coeffs[m] H^m with H a jet of zero constant term."""
    out = np.zeros(H.shape)
    out[..., 0] = coeffs[0]
    Hm = None
    for m in range(1, P + 1):
        Hm = H.copy() if Hm is None else jet_mul(Hm, H, P)
        out += coeffs[m][..., None] * Hm
    return out


def green_jets(u, kappa, P):
    """a^k (including 1/4pi) of G(x, y_c + h) for u = y_c - x [..., 3]."""
    u = np.asarray(u, dtype=np.float64)
    ks = multi_indices(P)
    idx = _index_map(P)
    nt = len(ks)
    r2 = np.zeros(u.shape[:-1] + (nt,))
    r2[..., 0] = (u * u).sum(-1)
    for a in range(3):
        e = [0, 0, 0]; e[a] = 1
        r2[..., idx[tuple(e)]] += 2.0 * u[..., a]
        if P >= 2:
            e[a] = 2
            r2[..., idx[tuple(e)]] += 1.0
    c0 = r2[..., 0]
    H = r2.copy(); H[..., 0] = 0.0
    # rho^-1 = (c0 + H)^(-1/2) = c0^(-1/2) sum_m binom(-1/2, m) (H/c0)^m
    binm = [1.0]
    for m in range(1, P + 1):
        binm.append(binm[-1] * (-0.5 - (m - 1)) / m)
    inv_r = _compose(c0, H, [binm[m] * c0 ** (-0.5 - m) for m in range(P + 1)], P)
    if kappa == 0.0:
        return inv_r / FOUR_PI
    # rho = (c0 + H)^(1/2)
    binh = [1.0]
    for m in range(1, P + 1):
        binh.append(binh[-1] * (0.5 - (m - 1)) / m)
    rho = _compose(c0, H, [binh[m] * c0 ** (0.5 - m) for m in range(P + 1)], P)
    r0 = rho[..., 0]
    Hr = rho.copy(); Hr[..., 0] = 0.0
    # exp(-kappa rho) = exp(-kappa r0) sum_m (-kappa)^m Hr^m / m!
    fact = [1.0]
    for m in range(1, P + 1):
        fact.append(fact[-1] * m)
    ex = _compose(r0, Hr, [np.exp(-kappa * r0) * (-kappa) ** m / fact[m] for m in range(P + 1)], P)
    return jet_mul(ex, inv_r, P) / FOUR_PI


def monomials(h, P):
    """h^k for every multi-index, h [..., 3] -> [..., nterms]."""
    ks = multi_indices(P)
    h = np.asarray(h, dtype=np.float64)
    out = np.empty(h.shape[:-1] + (len(ks),))
    for i, k in enumerate(ks):
        out[..., i] = h[..., 0] ** k[0] * h[..., 1] ** k[1] * h[..., 2] ** k[2]
    return out


def monopole_moments(y, s, yc, P):
    """M^k = sum_j s_j (y_j - y_c)^k."""
    return (s[:, None] * monomials(y - yc[None, :], P)).sum(0)


def dipole_moments(y, d, yc, P):
    """D^k = sum_j sum_l d_{j,l} k_l (y_j - y_c)^(k - e_l)."""
    ks = multi_indices(P)
    h = y - yc[None, :]
    out = np.zeros(len(ks))
    for i, k in enumerate(ks):
        tot = np.zeros(h.shape[0])
        for l in range(3):
            if k[l] == 0:
                continue
            km = list(k); km[l] -= 1
            tot += d[:, l] * k[l] * h[:, 0] ** km[0] * h[:, 1] ** km[1] * h[:, 2] ** km[2]
        out[i] = tot.sum()
    return out


def n_terms(P):
    return comb(P + 3, 3)
