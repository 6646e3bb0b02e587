// Host-side state of a context and of one problem (shared by the C-ABI in
// api.cu and the adjoint in adjoint.cu).
#pragma once

#include <functional>
#include <memory>
#include <string>
#include <vector>

#include "gmres.cuh"
#include "model.cuh"
#include "precond.cuh"
#include "treecode.cuh"
#include "validate.cuh"

struct pb_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    std::vector<cudaStream_t> pool;   // streams of batched solves (created on first use)
    std::vector<cudaEvent_t> pool_ev;
    int batch_persistent = 0;         // pb_solve_batch: one persistent launch per step for eligible batches
    std::string err;
};

namespace pb {

// Record of a surface built on the device from atoms (surface.cu).
struct SurfGenInfo {
    int shape[3] = {0, 0, 0};    // density grid nodes per axis
    int rounds = 0;              // smoothing rounds used
    int64_t components = 0, raw_nv = 0, raw_nt = 0;
    float ms = 0.0f;
};

struct SurfIn {
    int64_t nv = 0, nt = 0;
    DevBuf<double> v;      // device copy made when the surface is added (or the generated mesh)
    DevBuf<int32_t> t;
    int inner = -1, outer = -1;
    bool generated = false;
    SurfGenInfo gen;
};

// One (pair, kernel) contribution cK * K + cV * V of region `region` to a row
// block or to the reaction potential.
struct Term {
    int pair, kidx;
    double cK, cV;
    int region;
};

struct AdjointState;   // adjoint.cuh

}  // namespace pb

struct pb_problem {
    pb_ctx *ctx = nullptr;
    cudaStream_t stream = nullptr;            // the context stream, or a pool stream inside a batch
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaStream_t side = nullptr;              // the operator's direct sums run here beside the upward pass
    cudaEvent_t evf = nullptr, evj = nullptr; // fork and join of the side stream
    cudaStream_t lists2 = nullptr;            // setup: target sorts and every other pair's list build
    cudaEvent_t ev2a = nullptr, ev2b = nullptr; // setup: joins between the context stream and lists2
    cudaEvent_t ev2c = nullptr;               // setup: the target sorts done (lists2)
    cudaGraphExec_t mv_exec = nullptr;        // captured operator application z1 -> gm.w
    long long mv_kernels = 0;                 // kernels in that graph
    cudaGraphExec_t adj_exec = nullptr;       // captured transposed operator z1 -> gm.w (gradient)
    long long adj_kernels = 0;
    cudaGraphExec_t cyc_exec = nullptr;       // one GMRES cycle's Arnoldi loop as a graph WHILE node (solve)
    long long cyc_kernels = 0;                // kernels per step of that loop
    cudaGraphExec_t adj_cyc_exec = nullptr;   // the same for the adjoint solve
    long long adj_cyc_kernels = 0;
    std::vector<pb::Region> regions;
    std::vector<pb::SurfIn> sin;
    int64_t nc = 0;                         // charges
    int cregion = -1;
    bool is_setup = false;
    pb::Params prm;
    // device data
    std::vector<pb::SurfDev> S;
    std::vector<pb::Tree> T;
    std::vector<pb::Targets> G;               // one per surface, then the charges
    std::vector<pb::Pair> pairs;              // surface-target pairs
    std::vector<pb::Pair> cpairs;             // charge-target pairs
    std::vector<std::vector<pb::Term>> rows;  // per (surface, side)
    std::vector<pb::Term> reac;
    std::vector<bool> need_far;               // per tree: some pair uses its moments
    std::vector<int64_t> off;                 // panel offsets
    int64_t N = 0;
    pb::DevBuf<double> b, x, y, r, xin, yout, z1, z2, minv;
    pb::DevBuf<double> cq_d, cxyz_d, phi_reac, energy;
    pb::DevBuf<int32_t> wind, wind_bad;      // charge-region check: winding numbers, mismatch record
    pb::PinnedBuf<int32_t> wind_bad_h;
    pb::PinnedBuf<pb::MeshCheck> mesh_chk_h;
    pb::PinnedBuf<pb::ValueCheck> val_chk_h;  // outcome of the last pb_add_surface's mesh check
    // cluster block preconditioner (precond_block > 1; else the 2 x 2 self blocks in minv)
    bool use_cluster = false;
    std::vector<pb::ClusterSurface> csurf;
    pb::DevBuf<float> cinv;                    // 128 x 128 floats per block
    pb::DevBuf<int32_t> cerr;                  // a vanished pivot
    pb::PinnedBuf<int32_t> cerr_h;
    pb::Gmres gm;
    double setup_ms = 0.0;
    bool have_solution = false;
    double dG = 0.0;                          // energy of the last solve
    std::shared_ptr<pb::AdjointState> adj;   // built by the first gradient after setup
    ~pb_problem();
};

namespace pb {

// Operator, preconditioner and reaction potential of a set-up problem (api.cu).
struct PhaseEvents {
    cudaEvent_t ev[6];
};
void apply_operator(pb_problem *pb, const double *xd, double *yd, PhaseEvents *ph = nullptr);
void apply_precond(pb_problem *pb, const double *u, double *z);
void reaction(pb_problem *pb, const double *xd);

// Restarted, right-preconditioned GMRES on a problem's Krylov state (scratch
// vectors r, y, z1, z2 of the problem): solves op(x) = b for the 2N-vector x
// (device), starting from x (x_zero: from 0).  precond may be empty.  Several
// jobs advance in lock step, each on its problem's stream: every round queues
// one unit of work per job (a cycle start or one Arnoldi iteration) and the
// host synchronises once per round to read the scalars it decides on.
// graph: when set, the Arnoldi operator is a captured graph z1 -> gm.w launched
// on the given stream (the preconditioned basis vector is first written to z1).
struct KrylovStats {
    int iters = 0, matvecs = 0;
    double rel = 0.0;
};
using DevOp = std::function<void(const double *, double *)>;
struct KrylovJob {
    pb_problem *pb = nullptr;
    DevOp op, precond;
    const double *b = nullptr;
    double *x = nullptr;
    bool x_zero = true;
    std::function<void(cudaStream_t)> graph;
    // cycle: when set, a whole cycle's Arnoldi steps run as one captured graph
    // whose WHILE node the device ends (no host round trip per step); cycle_op
    // enqueues the operator z1 -> gm.w on pb->stream for the capture.
    std::function<void()> cycle_op;
    // prep: when set, the cycle graph's steps start with it (v_j formed, stored
    // and preconditioned into z1 by one launch per surface) and end their
    // Arnoldi step with the loop control in the norm kernel (Gmres::prep_step).
    std::function<void(cudaStream_t)> prep;
    cudaGraphExec_t *cycle_exec = nullptr;
    long long *cycle_kernels = nullptr;
    KrylovStats st;
    // driver state
    int phase = 0, j = 0, act = 0;
    double bnorm = 0.0;
};
// plan: when set, the Arnoldi steps of all jobs advance in lock step and their
// operator applications z1 -> gm.w (every job's pb->z1) run as one batched
// persistent launch per step (the plan's pairs, built for those inputs).
void run_krylov(std::vector<KrylovJob *> &jobs, BatchPlan *plan = nullptr);
// The two ends of one operator application around the pairs' sums: source
// strengths and upward passes (pre); block combination into y (post).
void operator_pre(pb_problem *pb, const double *xd, cudaStream_t s);
void operator_post(pb_problem *pb, const double *xd, double *yd, cudaStream_t s);
KrylovStats run_gmres(pb_problem *pb, const DevOp &op, const DevOp &precond, const double *b, double *x,
                      bool x_zero);
// Operator application as a replayable CUDA graph (captured on first use).
void launch_operator_graph(pb_problem *pb, cudaStream_t s);
// Captures `body` (work on pb->stream) into `exec` on first use, then launches it on s; nk counts its kernels.
void launch_captured(pb_problem *pb, cudaGraphExec_t &exec, long long &nk, const std::function<void()> &body,
                     cudaStream_t s);

}  // namespace pb
