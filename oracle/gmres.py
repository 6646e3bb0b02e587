"""Restarted GMRES(m) with modified Gram-Schmidt and Givens rotations.

The paper solves the BEM system with a Krylov method that needs one treecode
evaluation per iteration (Sec. 2.3, last paragraph) and stops at a relative
residual gmres_tol (Tables 1 and 3).  It names no variant; this is textbook
restarted GMRES (Saad & Schultz 1986): x0 = 0, Arnoldi by modified
Gram-Schmidt, the Hessenberg least-squares problem reduced by Givens
rotations, stop when |g_{j+1}| / ||b|| < tol, restart after m steps, and on
reaching the estimate check the true residual ||b - A x|| / ||b|| and restart
if it is still above tol.

Optional right preconditioning (solve A M^-1 u = b, x = M^-1 u) keeps the
stopping test on the true residual of A x = b.
"""
from __future__ import annotations

import numpy as np


def gmres(apply_A, b, tol=1e-4, restart=50, max_iter=1000, x0=None, M_inv=None):
    """Returns (x, iterations, relative true residual, history of estimates).

    M_inv: optional right preconditioner z -> M^-1 z.
    """
    prec = M_inv if M_inv is not None else (lambda z: z)
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, 0, 0.0, []
    hist = []
    it = 0
    while True:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta / bnorm < tol or it >= max_iter:
            return x, it, beta / bnorm, hist
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            w = apply_A(prec(V[j]))
            for i in range(j + 1):
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm < tol or it >= max_iter:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + prec(V[:j_done].T @ y)
