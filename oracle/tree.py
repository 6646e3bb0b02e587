"""Octree, Morton keys and per-target interaction lists (Sec. 2.3, Eq. MAC).

The treecode clusters the sources (the Gauss points of the panels, Sec. 2.3
"Treecode-accelerated BEM") in an octree whose leaves hold fewer than ncrit
sources, and traverses it for every target from the root, using the Taylor
expansion of a box when theta > r_b / r_tb (Eq. MAC), opening it otherwise,
and summing directly at the leaves.

The paper fixes none of the integer details; the readings used here (and in
the CUDA library, which must reproduce these results bit for bit) are:

  * Root cube: centre = midpoint of the FP64 bounding box of the sources,
    side = largest extent * (1 + 2^-20); lower corner = centre - side / 2.
  * Morton key: q_a = min(2^21 - 1, floor((p_a - corner_a) * (2^21 / side)))
    per axis, bits interleaved with x the most significant of each triple;
    sources are sorted by key, ties kept in input order (stable).
  * A box with count >= ncrit below level 21 splits into its non-empty
    octants (children in octant order); nodes are numbered breadth first.
  * Box centre corner_a + (i_a + 0.5) * side_l, side_l = side / 2^l;
    r_b = half diagonal, r_b^2 = (side_l * side_l) * 0.75; r_tb = distance
    from the target to the box centre.  Accept when
    r_b^2 < theta^2 * ((dx*dx + dy*dy) + dz*dz), all in FP64 without fused
    multiply-add; theta <= 0 never accepts (direct summation).
  * Lists are ordered by the boxes' depth-first pre-order rank (the order a
    recursive traversal visits them).
  * Near-singular list of target i: panels j (j != i on the target's own
    surface) with |x_i - c_j|^2 < (thres * L_j)^2 whose quadrature points all
    lie in i's direct-sum leaves, in ascending j.  Near panels with some point
    in an accepted box are left uncorrected and counted (the paper states the
    near region always falls in the direct part, Sec. 2.3).
"""
from __future__ import annotations

import numpy as np

MAXLEVEL = 21
NBITS = 2097152.0  # 2^21


def root_cube(points):
    p = np.asarray(points, dtype=np.float64)
    lo = p.min(0)
    hi = p.max(0)
    centre = (lo + hi) * 0.5
    ext = hi - lo
    side = max(ext[0], ext[1], ext[2]) * (1.0 + 2.0 ** -20)
    if side == 0.0:
        side = 1.0
    corner = centre - side * 0.5
    return corner, side


def morton_keys(points, corner, side):
    p = np.asarray(points, dtype=np.float64)
    scale = NBITS / side
    q = np.floor((p - corner[None, :]) * scale)
    q = np.clip(q, 0, 2 ** 21 - 1).astype(np.uint64)
    key = np.zeros(p.shape[0], dtype=np.uint64)
    for b in range(MAXLEVEL):
        for a, sh in ((0, 2), (1, 1), (2, 0)):
            bit = (q[:, a] >> np.uint64(b)) & np.uint64(1)
            key |= bit << np.uint64(3 * b + sh)
    return key


class Octree:
    """Octree over one set of source points (one surface)."""

    def __init__(self, points, ncrit):
        self.points = np.asarray(points, dtype=np.float64)
        self.corner, self.side = root_cube(self.points)
        keys = morton_keys(self.points, self.corner, self.side)
        self.perm = np.argsort(keys, kind="stable")
        self.keys = keys[self.perm]
        n = self.points.shape[0]
        level, start, count, ijk, first_child, nchild, parent = [], [], [], [], [], [], []
        level.append(0); start.append(0); count.append(n); ijk.append((0, 0, 0)); parent.append(-1)
        first_child.append(-1); nchild.append(0)
        head = 0
        while head < len(level):
            l, s, c = level[head], start[head], count[head]
            if c >= ncrit and l < MAXLEVEL:
                sh = np.uint64(3 * (MAXLEVEL - 1 - l))
                oct_ = ((self.keys[s:s + c] >> sh) & np.uint64(7)).astype(np.int64)
                bounds = np.searchsorted(oct_, np.arange(9))
                first_child[head] = len(level)
                for o in range(8):
                    cs, ce = bounds[o], bounds[o + 1]
                    if ce > cs:
                        i, j, k = ijk[head]
                        ijk.append((2 * i + ((o >> 2) & 1), 2 * j + ((o >> 1) & 1), 2 * k + (o & 1)))
                        level.append(l + 1); start.append(s + cs); count.append(ce - cs)
                        parent.append(head); first_child.append(-1); nchild.append(0)
                        nchild[head] += 1
            head += 1
        self.level = np.array(level, dtype=np.int32)
        self.start = np.array(start, dtype=np.int64)
        self.count = np.array(count, dtype=np.int64)
        self.ijk = np.array(ijk, dtype=np.int64)
        self.parent = np.array(parent, dtype=np.int64)
        self.first_child = np.array(first_child, dtype=np.int64)
        self.nchild = np.array(nchild, dtype=np.int64)
        self.side_l = self.side / (2.0 ** self.level.astype(np.float64))
        self.centre = self.corner[None, :] + (self.ijk.astype(np.float64) + 0.5) * self.side_l[:, None]
        self.rb2 = (self.side_l * self.side_l) * 0.75
        self.is_leaf = self.nchild == 0
        # depth-first pre-order rank
        pre = np.empty(len(level), dtype=np.int64)
        stack, r = [0], 0
        while stack:
            b = stack.pop()
            pre[b] = r
            r += 1
            fc, nc = self.first_child[b], self.nchild[b]
            for c in range(fc + nc - 1, fc - 1, -1):
                if nc:
                    stack.append(c)
        self.preorder = pre
        # leaf of every sorted source point
        self.leaf_of_sorted = np.empty(n, dtype=np.int64)
        for b in np.nonzero(self.is_leaf)[0]:
            self.leaf_of_sorted[self.start[b]:self.start[b] + self.count[b]] = b

    @property
    def n_nodes(self):
        return self.level.size


def interaction_lists(tree: Octree, targets, theta):
    """Per-target M2P and P2P node lists (CSR), each in depth-first pre-order.

    Returns (m2p_ptr, m2p_nodes, p2p_ptr, p2p_nodes).
    """
    x = np.asarray(targets, dtype=np.float64)
    m = x.shape[0]
    th2 = theta * theta
    tgt = np.arange(m, dtype=np.int64)
    node = np.zeros(m, dtype=np.int64)
    m2p_t, m2p_b, p2p_t, p2p_b = [], [], [], []
    while tgt.size:
        c = tree.centre[node]
        dx = x[tgt, 0] - c[:, 0]
        dy = x[tgt, 1] - c[:, 1]
        dz = x[tgt, 2] - c[:, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        acc = tree.rb2[node] < th2 * d2 if theta > 0 else np.zeros(tgt.size, bool)
        m2p_t.append(tgt[acc]); m2p_b.append(node[acc])
        rest = ~acc
        leaf = rest & tree.is_leaf[node]
        p2p_t.append(tgt[leaf]); p2p_b.append(node[leaf])
        op = rest & ~leaf
        t_op, n_op = tgt[op], node[op]
        nc = tree.nchild[n_op]
        tgt = np.repeat(t_op, nc)
        base = np.repeat(tree.first_child[n_op], nc)
        off = np.arange(tgt.size) - np.repeat(np.cumsum(nc) - nc, nc)
        node = base + off

    def csr(ts, bs):
        t = np.concatenate(ts) if ts else np.zeros(0, np.int64)
        b = np.concatenate(bs) if bs else np.zeros(0, np.int64)
        order = np.lexsort((tree.preorder[b], t))
        t, b = t[order], b[order]
        ptr = np.zeros(m + 1, dtype=np.int64)
        np.add.at(ptr, t + 1, 1)
        return np.cumsum(ptr), b

    mp, mb = csr(m2p_t, m2p_b)
    pp, pb = csr(p2p_t, p2p_b)
    return mp, mb, pp, pb


def near_lists(tree: Octree, K, targets, self_panel, cen, L, thres, p2p_ptr, p2p_nodes):
    """Near-singular panel lists (CSR, ascending panel index) and exclusion counts.

    tree: octree over the K*n source points of the source surface, point
    j*K+k being Gauss point k of panel j.  self_panel [m]: panel of the source
    surface that target i sits on (-1 for none).
    Returns (ptr, panels, n_near_excluded, n_self_excluded): panels within
    the near-singular distance that have a point outside the direct-sum leaves
    are excluded and counted; so are targets whose own panel has a point in an
    accepted box.
    """
    x = np.asarray(targets, dtype=np.float64)
    m = x.shape[0]
    npan = cen.shape[0]
    leaf_of_point = np.empty(npan * K, dtype=np.int64)
    leaf_of_point[tree.perm] = tree.leaf_of_sorted
    tl = thres * L
    tl2 = tl * tl
    rows, excl, self_excl = [], 0, 0
    for i in range(m):
        dx = x[i, 0] - cen[:, 0]
        dy = x[i, 1] - cen[:, 1]
        dz = x[i, 2] - cen[:, 2]
        d2 = (dx * dx + dy * dy) + dz * dz
        cand = np.nonzero(d2 < tl2)[0]
        if self_panel[i] >= 0:
            cand = cand[cand != self_panel[i]]
        leaves = set(p2p_nodes[p2p_ptr[i]:p2p_ptr[i + 1]].tolist())
        ok = np.array([all(leaf_of_point[j * K + k] in leaves for k in range(K)) for j in cand],
                      dtype=bool)
        excl += int((~ok).sum()) if cand.size else 0
        rows.append(cand[ok] if cand.size else cand)
        if self_panel[i] >= 0:
            j = self_panel[i]
            if not all(leaf_of_point[j * K + k] in leaves for k in range(K)):
                self_excl += 1
    ptr = np.zeros(m + 1, dtype=np.int64)
    ptr[1:] = np.cumsum([r.size for r in rows])
    panels = np.concatenate(rows) if rows else np.zeros(0, np.int64)
    return ptr, panels.astype(np.int64), excl, self_excl
