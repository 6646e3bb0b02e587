// Device-side data model of one problem: surfaces, octrees, target sets and
// the per-(target set, octree) interaction data of the treecode.
#pragma once

#include "common.cuh"

namespace pb {

struct Params {
    int K = 3, K_fine = 19, N_k = 5;
    double thres = 2.0;
    int P = 6;
    double theta = 0.5;
    int ncrit = 300;
    double tol = 1e-4;
    int restart = 50, max_iter = 1000;
    int precision = PB_FP64;
    bool precond = true;
    int precond_block = 32;  // panels per preconditioner block (1: 2 x 2 self blocks)
    int ncrit_adjoint = 0;   // 0: ncrit
    int p2p_tile = 64;       // targets per P2P work item (above 32: two per lane)
    int m2p_variant = 0;     // 1: FP32 radial M2P with its contraction on the tensor pipe
};

struct Region {
    double eps, kappa;
};

// Geometry of one surface on the device (panels in input order).
struct SurfDev {
    int64_t n = 0, nv = 0;
    int inner = -1, outer = -1;
    int64_t off = 0;                 // first panel in the concatenated panel list
    DevBuf<double> verts;            // nv * 3
    DevBuf<int32_t> tris;            // n * 3
    DevBuf<double> cen, nrm;         // n * 3
    DevBuf<double> area, L;          // n
    DevBuf<double> gy, gwa;          // K Gauss points: n*K*3, n*K (point j*K + k)
};

// Octree over the K * n Gauss points of one surface (the treecode sources).
struct Tree {
    int64_t npts = 0;
    double corner[3] = {0, 0, 0}, side = 1.0, origin[3] = {0, 0, 0};
    int nnodes = 0, nleaves = 0, nlevels = 0;
    std::vector<int> level_off;      // nodes of level l: [level_off[l], level_off[l+1])
    DevBuf<uint64_t> keys;           // sorted Morton keys
    DevBuf<int32_t> perm;            // sorted position -> point index
    DevBuf<int32_t> level, first_child, nchild, parent, node_leaf;
    DevBuf<int64_t> start, count;
    DevBuf<double> centre, rb2;      // centre: nnodes * 3
    DevBuf<float4> cen32;            // (centre - origin) in FP32, r_b^2
    DevBuf<float4> pofs32;           // centre - parent centre, the FP64 difference rounded to FP32 (0 at the root)
    DevBuf<int32_t> leaf_node;       // leaf index (Morton order) -> node
    DevBuf<int32_t> point_leaf;      // point index (input order) -> leaf index
    // sorted source data
    DevBuf<double> ys;               // npts * 3 (absolute, FP64)
    DevBuf<double> was;              // npts weight * area
    DevBuf<int32_t> pids;            // npts owning panel (within the surface)
    DevBuf<float4> pos32;            // (x, y, z relative to origin, weight*area) FP32
    // per-evaluation source strengths
    DevBuf<double> src64;            // npts * 8: x, y, z, s, dx, dy, dz, pid
    DevBuf<float4> srcA32, srcB32;   // (x, y, z, s) and (dx, dy, dz, pid bits)
    DevBuf<float2> phf;              // (phi, dphi) per panel in FP32 (mixed path)
    DevBuf<int4> link;               // per node: (parent, parent's first child, parent's child count, 0)
    DevBuf<int32_t> ucnt;            // per node: children finished in the fused upward pass (0 between passes)
    DevBuf<double> mom64;            // nnodes * 2 * nterms: M then D
    DevBuf<float> mom32;
    DevBuf<float> rmom32;            // moments in radial form (FP32 M2P, P <= kRadialMaxP)
};

// Evaluation points: panel centroids of one surface, or the charges.
struct Targets {
    int64_t n = 0;
    int surface = -1;                // -1: charges
    DevBuf<uint64_t> keys;           // sorted Morton keys of the positions
    DevBuf<double> xs;               // sorted positions n * 3
    DevBuf<int32_t> order;           // sorted position -> input index
    DevBuf<int32_t> rank;            // input index -> sorted position
    DevBuf<int32_t> self_panel;      // sorted position -> own panel (surface targets) or -1
};

// Interaction of one target set with one octree, for one or two kernels.
struct Pair {
    int tgt = 0;                     // index into the problem's target sets
    int tree = 0;                    // source surface
    std::vector<double> kappas;      // distinct kernels (kappa = 0: Laplace)
    DevBuf<int64_t> m2p_ptr, p2p_ptr, near_ptr;
    DevBuf<int32_t> m2p_node, p2p_node, near_panel;
    int64_t n_m2p = 0, n_p2p = 0, n_near = 0, near_excl = 0, self_excl = 0, p2p_pairs = 0;
    DevBuf<unsigned long long> stats;   // list-build counters read back with the list sizes
    int p2p_tile = 32;                  // targets per P2P item (above 32: two per lane)
    // Entry-major work: for every leaf (P2P) / box (M2P) the (sorted target,
    // list entry) pairs that use it, grouped by leaf / box and packed 32 per
    // work item (one warp); every pair writes one partial sum, and a gather
    // adds each target's partials in its own list order.
    DevBuf<int32_t> p2p_inv, m2p_inv;     // target of every grouped (target, entry) pair
    DevBuf<int32_t> p2p_ent, m2p_ent;     // grouped position -> CSR entry (where its record goes)
    DevBuf<int4> p2p_items, m2p_items;    // (leaf | box, grouped start, count <= 32, 0)
    int64_t n_p2p_items = 0, n_m2p_items = 0;
    // partial records, interleaved per entry: (V, K) of every kernel (2 nk
    // values), P2P and M2P records at their CSR entries: each target's records
    // are contiguous, so the gather reads them with coalesced loads and no index
    DevBuf<double> p2p_part, m2p_part64;
    DevBuf<float> p2p_part32, m2p_part32;
    DevBuf<float> dV32, dK32;             // mixed path: near corrections in FP32, kernel-major
    DevBuf<float4> x32;                   // sorted targets relative to the tree origin, FP32
    // near-singular corrections per kernel: dV, dK per near entry; self V per panel
    std::vector<DevBuf<double>> dV, dK, selfV;
    // FP32 path with the own panel's points left in the direct sum (rules without a centroid point):
    // self value minus the K-point own-panel share, per kernel
    bool p2p_self_in = false;
    std::vector<DevBuf<double>> selfV32;
    // outputs per kernel: V then K per sorted target (2 * n)
    std::vector<DevBuf<double>> VK;
};

}  // namespace pb
