// Setup-phase entry points of the octree and interaction-list code (tree.cu).
#pragma once

#include <vector>

#include "model.cuh"

namespace pb {

// Root cube of the points (device: corner x, y, z, side), Morton keys and the
// (key, index) sort, all queued on s.
void morton_sort(const double *d_points, int64_t n, cudaStream_t s, double *cube, DevBuf<uint64_t> &keys,
                 DevBuf<int32_t> &perm);
// Octree over the K Gauss points of every panel of S (point j*K + k).
void build_tree(Tree &T, const SurfDev &S, int K, int ncrit, cudaStream_t s);
// Octree over n points (n * 3, input order) with weights wts (null: 1); point p
// belongs to owner p / K (the Tree's pids).
void build_tree_points(Tree &T, const double *pts, const double *wts, int64_t n, int K, int ncrit, cudaStream_t s);
// Morton-sorted copy of target positions d_x (n * 3, input order).  For a
// surface's target set (surface >= 0) target i sits on panel i / points_per_panel.
void build_targets(Targets &G, const double *d_x, int64_t n, int surface, cudaStream_t s, int points_per_panel = 1);
// M2P / P2P lists, their warp-group unions and the near-singular lists of
// targets G against tree T (built over surface src).  use_self: the targets are
// the panels of the tree's own surface, so each skips its own panel.
void build_lists(Pair &Pr, const Targets &G, const Tree &T, const SurfDev &src, const Params &prm, bool use_self,
                 cudaStream_t s);
// The lists of several pairs, each on its own stream (job.s; its near lists
// on job.helper), their host reads gathered into two waits.  Inputs (tree,
// targets) must be ready on every job's streams; the caller joins the helper
// streams afterwards.
struct ListJob {
    Pair *P;
    const Targets *G;
    const Tree *T;
    const SurfDev *src;
    bool use_self;
    cudaStream_t s;
    cudaStream_t helper = nullptr;   // the near lists run here (null: on s)
};
void build_lists_multi(const std::vector<ListJob> &jobs, const Params &prm);
// The traversal (M2P / P2P lists, direct-sum pair count, entry-major items) alone;
// P2P items hold up to p2p_per_item (32 or 64) (target, leaf) pairs, M2P items 32.
void build_far_lists(Pair &Pr, const Targets &G, const Tree &T, const Params &prm, cudaStream_t s,
                     int p2p_per_item = 32);
// The near-singular lists of targets G against the panels of src (after build_far_lists).
void build_near_lists(Pair &Pr, const Targets &G, const Tree &T, const SurfDev &src, const Params &prm, bool use_self,
                      cudaStream_t s);

}  // namespace pb
