"""Pins of the oracle's Taylor coefficients and moments (Sec. 2.3, Eqs. taylor, multexp).

The jet coefficients a^k = (1/k!) D_y^k G are checked against closed-form
one-dimensional derivatives on the axes, against the screened Laplace
equation (Delta - kappa^2) G = 0 written for the coefficients, and against
the exact kernel through the O(|h|^(P+1)) remainder.  The far-field sums are
checked against direct sums.
"""
from math import comb, factorial

import numpy as np
import pytest

from oracle.taylor import (dipole_moments, green_jets, monomials, monopole_moments,
                           multi_indices, n_terms)


def test_multi_index_count():
    for P in (0, 2, 6, 12):
        assert len(multi_indices(P)) == n_terms(P) == (P + 1) * (P + 2) * (P + 3) // 6


@pytest.mark.parametrize("kappa", [0.0, 0.125, 0.9])
def test_axis_coefficients_closed_form(kappa):
    P = 8
    z0 = 2.3
    ks = multi_indices(P)
    for axis in range(3):
        u = np.zeros(3); u[axis] = z0
        a = green_jets(u, kappa, P)
        for n in range(P + 1):
            k = [0, 0, 0]; k[axis] = n
            # (1/n!) d^n/dz^n [exp(-kappa z) / z] at z0 (Leibniz rule)
            ex = sum(comb(n, m) * (-kappa) ** m * np.exp(-kappa * z0)
                     * (-1) ** (n - m) * factorial(n - m) / z0 ** (n - m + 1)
                     for m in range(n + 1)) / factorial(n) / (4 * np.pi)
            assert abs(a[ks.index(tuple(k))] - ex) <= 1e-14 * abs(ex) + 1e-18


@pytest.mark.parametrize("kappa", [0.0, 0.125, 0.9])
def test_coefficients_satisfy_screened_laplace(kappa):
    # sum_l (k_l+2)(k_l+1) a_{k+2e_l} = kappa^2 a_k for |k| <= P-2
    P = 8
    ks = multi_indices(P)
    idx = {k: i for i, k in enumerate(ks)}
    a = green_jets(np.array([0.7, -1.9, 1.3]), kappa, P)
    for k in ks:
        if sum(k) > P - 2:
            continue
        lap = 0.0
        for l in range(3):
            kk = list(k); kk[l] += 2
            lap += (k[l] + 2) * (k[l] + 1) * a[idx[tuple(kk)]]
        assert abs(lap - kappa ** 2 * a[idx[k]]) < 1e-12 * np.abs(a).max()


@pytest.mark.parametrize("kappa", [0.0, 0.125])
def test_taylor_remainder_order(kappa):
    P = 6
    u = np.array([1.1, -0.4, 2.0])
    a = green_jets(u, kappa, P)
    errs = []
    for s in (0.08, 0.04):
        h = s * np.array([0.3, 0.8, -0.5])
        r = np.linalg.norm(u + h)
        ex = np.exp(-kappa * r) / (4 * np.pi * r)
        errs.append(abs((a * monomials(h, P)).sum() - ex))
    assert 2 ** (P + 1) / 1.5 < errs[0] / errs[1] < 2 ** (P + 1) * 1.5


def test_far_field_sums_converge_to_direct():
    rng = np.random.default_rng(5)
    yc = np.array([0.2, 0.1, -0.3])
    y = yc + rng.uniform(-0.5, 0.5, size=(40, 3))
    s = rng.normal(size=40)
    d = rng.normal(size=(40, 3))
    x = np.array([3.0, 2.0, -1.5])
    kappa = 0.125
    r = x - y
    rho = np.linalg.norm(r, axis=1)
    e = np.exp(-kappa * rho)
    Vd = (s * e / rho).sum() / (4 * np.pi)
    Kd = ((r * d).sum(1) * (1 + kappa * rho) * e / rho ** 3).sum() / (4 * np.pi)
    prev = None
    for P in (2, 4, 6, 8):
        a = green_jets(yc - x, kappa, P)
        err = (abs((a * monopole_moments(y, s, yc, P)).sum() - Vd) / abs(Vd),
               abs((a * dipole_moments(y, d, yc, P)).sum() - Kd) / abs(Kd))
        if prev is not None:
            assert err[0] < prev[0] and err[1] < prev[1]
        prev = err
    assert prev[0] < 1e-6 and prev[1] < 1e-5
