// Transposed treecode operator and the adjoint gradient of the solvation
// energy (adjoint.cu).
#pragma once

#include "problem.cuh"

namespace pb {

// One transposed interaction: the panels of surface `tgt` collect, at their
// Gauss points, the potential and target-normal field of monopoles sitting at
// the collocation points of surface `src` (transpose of a forward surface
// pair) or at the charges (transpose of a forward charge pair).
struct TPair {
    bool charges = false;
    int fwd = -1;              // forward pair (pairs, or cpairs when charges)
    int src = -1;              // source surface (-1: charges)
    int tgt = 0;               // target surface
    int nk = 1;
    double cV[2][2] = {{0.0, 0.0}, {0.0, 0.0}};   // [kernel slot][row side] coefficient of V^T
    double cK[2][2] = {{0.0, 0.0}, {0.0, 0.0}};   // ... of K^T
    int64_t nsrc = 0;
    Pair L;                    // lists, items, partial records, outputs VK per kernel
    DevBuf<double> fold;       // mu_k then nu_k per source (input order): 2 nk x nsrc
    DevBuf<double> src64;      // sorted: x, y, z, mu0, nu0, mu1, nu1, owner
    DevBuf<float4> srcA32, srcB32;   // (x, y, z, mu0), (nu0, mu1, nu1, owner bits)
    DevBuf<double> mom64;      // per node 2 nk nterms(P): mu0, nu0, mu1, nu1 moments
    DevBuf<float> mom32;
    DevBuf<float> rmom32;      // radial-form moments (mixed Laplace + Yukawa pairs)
    DevBuf<int64_t> nt_ptr;    // transposed near list: per target panel its forward entries
    DevBuf<int32_t> nt_ent, nt_src;
};

struct AdjointState {
    std::vector<Tree> TC;          // per surface: octree over the panel centroids
    Tree TQ;                       // octree over the charges
    std::vector<Targets> GP;       // per surface: its Gauss points as targets
    std::vector<DevBuf<double>> gn64;   // sorted target normals, 3 per target
    std::vector<DevBuf<float4>> gn32;
    std::vector<TPair> tp, tq;     // transposed surface pairs, transposed charge pairs
    // FP32 panel data per surface (mixed path of the charge-site sums), relative to the surface's tree origin
    std::vector<DevBuf<float4>> pc32, pn32, gp32;
    DevBuf<double> lam, f, minvT, gacc, dq_d, dxyz_d, part;
};

// out = A^T lam (device 2N vectors, lam in row order, out in unknown order).
void apply_transpose(pb_problem *pb, const double *lam, double *out);
// Gradient of the energy of the current solution (pb_gradient).
void energy_gradient(pb_problem *pb, pb_grad *g);

}  // namespace pb
