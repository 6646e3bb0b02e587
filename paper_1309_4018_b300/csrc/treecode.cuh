// Evaluation-phase entry points of the treecode (treecode.cu).
#pragma once

#include <utility>
#include <vector>

#include "model.cuh"

namespace pb {

// One contribution cK * K + cV * V of a block sum, read at a target's sorted rank.
struct CombineTerm {
    const double *VK;   // V at [0, ntg), K at [ntg, 2 ntg)
    int64_t ntg;
    double cK, cV;
};
struct CombineRow {
    int nterm;
    CombineTerm term[8];
};

void upload_term_tables();
// Source strengths s_p, d_p of the Gauss points of tree Tr from phi, dphi of its surface.
void compute_strengths(Tree &Tr, const SurfDev &S, const double *phi, const double *dphi, bool mixed, cudaStream_t s);
// P2M at the leaves, then M2M level by level to the root.
void upward_pass(Tree &Tr, int P, bool mixed, cudaStream_t s);
// floats per node of the radial-form moments of order P (FP32 M2P)
size_t radial_floats(int P);
// M2M level by level over moments `mom` (float if mixed, else double) holding
// `stride` values per node; shifts the 2 nterms(P) values at offset `base`.
// M2M of every internal node in one launch (the leaves' moments complete): nval values per node,
// nval / NT moment sets shifted by the same rule.  Needs Tr.ucnt zeroed (the kernel leaves it zeroed).
void m2m_climb(Tree &Tr, int P, bool mixed, void *mom, int nval, cudaStream_t s);
// whether nval values per node fit the one-launch M2M's shared memory
bool climb_fits(int nval, bool mixed);
void m2m_pass(const Tree &Tr, int P, bool mixed, void *mom, int stride, int base, cudaStream_t s);
// Direct-sum partials of every (target, leaf) list entry.
void launch_p2p(const Pair &Pr, const Targets &G, const Tree &Tr, bool use_self, bool mixed, cudaStream_t s);
// Far-field partials of every (target, box) list entry and kernel.
// variant 1: the FP32 radial form's contraction on the tensor pipe where eligible.
void launch_m2p(const Pair &Pr, const Targets &G, const Tree &Tr, int P, bool mixed, cudaStream_t s,
                int variant = 0);
// Pr.VK = each target's partials, plus its near-singular corrections and (use_self)
// its own panel's semi-analytical term, with phi, dphi of the source surface (overwrites).
// phf: FP32 (phi, dphi) of the source surface (the tree's phf after
// compute_strengths), read on the mixed path; may be null without near entries.
void launch_gather(const Pair &Pr, const Targets &G, bool mixed, bool use_self, const double *phi,
                   const double *dphi, const float2 *phf, cudaStream_t s);
// y[i] = half * phi_s[i] (0 if phi_s is null) + sum_terms (cK K + cV V)[rank[i]] for i < n.
// FP32 target positions relative to the tree origin (mixed path).
void targets_to_float(Pair &Pr, const Targets &G, const Tree &Tr, cudaStream_t s);
void launch_combine(int64_t n, const int32_t *rank, const double *phi_s, double half, const CombineRow &row, double *y,
                    cudaStream_t s);
// Rows 0 and 1 of one surface (y: 2 n values, row 0 first), the same sums as two launch_combine calls.
void launch_combine_pair(int64_t n, const int32_t *rank, const double *phi_s, double half, const CombineRow &row0,
                         const CombineRow &row1, double *y, cudaStream_t s);

// Arguments of the FP32 radial-form M2P of one pair (Laplace slot 0, Yukawa slot 1).
struct M2PArgs32 {
    const int4 *items;                     // (box, grouped start, count <= 32, 0)
    const int32_t *inv, *ent;              // grouped pair -> sorted target, list entry
    const float4 *x32, *cen32;             // targets, box centres (FP32, tree-origin relative)
    const float *rmom;                     // radial moments, radial_stride(P) floats per node
    float kappa;                           // Yukawa kernel (slot 1)
    float4 *part;                          // records (VL, KL, VY, KY) per list entry
};
M2PArgs32 m2p_args32(const Pair &Pr, const Tree &Tr);
// The radial-form M2P with its contraction on the tensor pipe (m2p_tc.cu):
// kernel attributes (once per context), eligibility of a pair, launch.
void m2p_tc_prepare();
bool m2p_tc_eligible(const Pair &Pr, int P, bool mixed);
void launch_m2p_tc(const M2PArgs32 &a, int64_t nitems, int P, cudaStream_t s);

// ---------------------------------------------------------------- batched operator
// The direct sums, far-field sums and gathers of several problems' operator
// applications in one persistent launch over a device queue of (pair, phase,
// tile) entries (treecode.cu, batch_operator_kernel); each pair's gathers wait,
// with a bounded number of polls, until its direct and far-field entries are
// done.  Serves mixed-precision pairs of one Laplace and one Yukawa kernel
// with the radial-form M2P whose direct sums keep the own panel's points
// (K = 3): single-surface molecules such as binding triplets and ligand fleets.
struct BatchPairRef {
    const Pair *P;
    const Targets *G;
    const Tree *T;           // source tree (its FP32 densities phf feed the near corrections)
    bool use_self;
    const double *dphi;      // FP64 dphi of the source surface inside the operator's input vector
    int problem;             // index of the problem's active flag
};
struct BatchPlan {
    int P = -1, nproblems = 0, npairs = 0, grid = 0;
    std::vector<std::vector<unsigned char>> seg_args;   // per launch: the pair descriptors (parameter space)
    std::vector<std::pair<int64_t, int64_t>> seg_q;      // per launch: its queue entries (offset, count)
    DevBuf<int4> queue;                // (pair within the launch, phase, first, count)
    DevBuf<unsigned> cnt;              // per launch: [0] next entry, [1 + k] done entries of pair k
    DevBuf<int> active, status;        // per-problem flags; status[0] code, status[1] abort flag
    PinnedBuf<int> active_h, status_h; // host copies: set active_h before a launch, read status_h after it
    long long cap = 0;                 // polls of a waiting gather before it gives up
    unsigned extra = 0;                // added to every pair's count (PB_FAULT=wait)
    cudaEvent_t ev = nullptr;
    BatchPlan() = default;
    BatchPlan(const BatchPlan &) = delete;
    BatchPlan &operator=(const BatchPlan &) = delete;
    ~BatchPlan();
};
bool batch_pair_eligible(const Pair &Pr, const Params &prm, bool use_self);
void batch_plan_build(BatchPlan &bp, const std::vector<BatchPairRef> &pairs, int nproblems, int P, cudaStream_t s);
// One operator application (P2P, M2P, gather) of every pair whose problem has
// its active_h flag set, queued on s; status_h[0] is PB_OK or PB_ETIMEOUT once
// s has been synchronised.
void batch_operator_launch(BatchPlan &bp, cudaStream_t s);

}  // namespace pb
