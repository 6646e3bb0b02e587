"""Plain FP64 treecode matrix-vector product (Sec. 2.3, Eqs. nbody, taylor, multexp, MAC).

For every block (target surface s, source surface t, region kernel G_R) the
treecode-accelerated BEM (Sec. 2.3 "Treecode-accelerated BEM") evaluates, at
each collocation point x_i of s,

  V_i = sum_j V_ij dphi_j  and  K_i = sum_j K_ij phi_j

as an N-body sum whose sources are the K Gauss points of the panels of t,
with strengths s_p = w_p A_j dphi_j (single layer) and dipoles
d_p = w_p A_j phi_j n_j (double layer):

  * direct sum over the points of the leaves that fail the MAC (Eq. MAC),
    skipping the target's own panel;
  * Taylor far field sum_k a^k M^k and sum_k a^k D^k over the accepted boxes
    (Eq. multexp), with moments taken directly from each box's points
    (no M2M shifting, so that the CUDA library's upward pass is checked
    against the definition) and coefficients from jets (oracle.taylor);
  * the near-singular correction (K_fine rule minus the K-point value the
    direct sum used) for the panels of the near list, and the semi-analytical
    self integral for the target's own panel.

The oracle evaluates any subset of rows, so that large problems can be
checked on sampled outputs.
"""
from __future__ import annotations

import numpy as np

from . import formulation as F
from .dense import FOUR_PI, _kernel_sums, full_params, surfaces_data
from .taylor import dipole_moments, green_jets, monopole_moments
from .tree import Octree, interaction_lists, near_lists


class TreecodeOracle:
    def __init__(self, problem, params=None, sdata=None):
        self.problem = problem
        self.p = full_params(params)
        self.sd = sdata or surfaces_data(problem, self.p)
        K = self.p["K"]
        self.trees = [Octree(s.y.reshape(-1, 3), self.p["ncrit"]) for s in self.sd]
        self.pairs = sorted({(b.s, b.t) for b in F.blocks(problem)})
        self.lists = {}
        for s, t in self.pairs:
            self.lists[(s, t)] = interaction_lists(self.trees[t], self.sd[s].cen, self.p["theta"])

    def near(self, s, t, rows):
        K = self.p["K"]
        mp, mb, pp, pb = self.lists[(s, t)]
        rows = np.asarray(rows)
        sub_ptr = np.concatenate([[0], np.cumsum(pp[rows + 1] - pp[rows])])
        sub_nodes = np.concatenate([pb[pp[i]:pp[i + 1]] for i in rows]) if rows.size else np.zeros(0, np.int64)
        selfp = rows if s == t else -np.ones(rows.size, dtype=np.int64)
        st = self.sd[t]
        return near_lists(self.trees[t], K, self.sd[s].cen[rows], selfp, st.cen, st.L,
                          self.p["thres"], sub_ptr, sub_nodes)

    def block_sums(self, s, t, kappa, phi_t, dphi_t, rows):
        """(V_i, K_i) for the targets ``rows`` of surface s against surface t."""
        p = self.p
        P, K = p["P"], p["K"]
        st, tree = self.sd[t], self.trees[t]
        mp, mb, pp, pb = self.lists[(s, t)]
        y = st.y.reshape(-1, 3)
        wa = st.wa.reshape(-1)
        pid = np.repeat(np.arange(st.n), K)
        sp = wa * dphi_t[pid]
        dp = (wa * phi_t[pid])[:, None] * st.normal[pid]
        x = self.sd[s].cen
        rows = np.asarray(rows)
        V = np.zeros(rows.size)
        Kd = np.zeros(rows.size)
        mom_cache = {}
        nptr, npan, _, _ = self.near(s, t, rows)
        for r, i in enumerate(rows):
            xi = x[i]
            # direct part
            leaves = pb[pp[i]:pp[i + 1]]
            if leaves.size:
                idx = np.concatenate([tree.perm[tree.start[b]:tree.start[b] + tree.count[b]] for b in leaves])
                if s == t:
                    idx = idx[pid[idx] != i]
                rr = xi[None, :] - y[idx]
                rho2 = (rr * rr).sum(1)
                rho = np.sqrt(rho2)
                e = np.exp(-kappa * rho) if kappa != 0.0 else np.ones_like(rho)
                V[r] += (sp[idx] * e / rho).sum() / FOUR_PI
                Kd[r] += ((rr * dp[idx]).sum(1) * (1.0 + kappa * rho) * e / (rho2 * rho)).sum() / FOUR_PI
            # far part
            boxes = mb[mp[i]:mp[i + 1]]
            if boxes.size:
                for b in boxes:
                    if b not in mom_cache:
                        ids = tree.perm[tree.start[b]:tree.start[b] + tree.count[b]]
                        mom_cache[b] = (monopole_moments(y[ids], sp[ids], tree.centre[b], P),
                                        dipole_moments(y[ids], dp[ids], tree.centre[b], P))
                a = green_jets(tree.centre[boxes] - xi[None, :], kappa, P)
                M = np.stack([mom_cache[b][0] for b in boxes])
                D = np.stack([mom_cache[b][1] for b in boxes])
                V[r] += (a * M).sum()
                Kd[r] += (a * D).sum()
            # near-singular corrections and the self panel
            nj = npan[nptr[r]:nptr[r + 1]]
            if nj.size:
                Vf, Kf = _kernel_sums(np.repeat(xi[None], nj.size, 0), st.yf[nj], st.waf[nj], st.normal[nj], kappa)
                Vk, Kk = _kernel_sums(np.repeat(xi[None], nj.size, 0), st.y[nj], st.wa[nj], st.normal[nj], kappa)
                V[r] += ((Vf - Vk) * dphi_t[nj]).sum()
                Kd[r] += ((Kf - Kk) * phi_t[nj]).sum()
            if s == t:
                V[r] += st.self_V(kappa, p["N_k"])[i] * dphi_t[i]
        return V, Kd

    def matvec(self, x, rows_per_surface=None):
        """y = A x on the requested rows: dict s -> target indices (default all).

        Returns dict (s, side) -> values on those targets.
        """
        pr = self.problem
        us = F.unknown_slices(pr)
        kap = [r["kappa"] for r in pr["regions"]]
        out = {}
        cache = {}
        for s in range(len(pr["surfaces"])):
            rows = np.arange(self.sd[s].n) if rows_per_surface is None else np.asarray(rows_per_surface[s])
            for side in (0, 1):
                out[(s, side)] = 0.5 * x[us[s][0]][rows]
        for blk in F.blocks(pr):
            s, t = blk.s, blk.t
            rows = np.arange(self.sd[s].n) if rows_per_surface is None else np.asarray(rows_per_surface[s])
            key = (s, t, kap[blk.R])
            if key not in cache:
                cache[key] = self.block_sums(s, t, kap[blk.R], x[us[t][0]], x[us[t][1]], rows)
            V, Kd = cache[key]
            out[(s, blk.row_side)] = out[(s, blk.row_side)] + blk.sigma * Kd - blk.sigma * blk.c * V
        return out
