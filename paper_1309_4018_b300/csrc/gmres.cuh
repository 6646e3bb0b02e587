// Device GMRES state and vector/energy helpers (gmres.cu).
#pragma once

#include <cmath>
#include <utility>
#include <vector>

#include "common.cuh"

namespace pb {

// Small Krylov state kept on the device (pointers into Gmres buffers).
struct GmresState {
    int m;
    int pend;           // device loop: v_j is still w / ||w|| of the previous step (written by prep_step)
    double *H, *cs, *sn, *g, *y;
    double bnorm, beta, hnext, res_est;
    double steps;       // Arnoldi steps of the current cycle (device loop; next to res_est for one copy)
    int j, maxit;       // device loop: current column, step limit of the cycle
};

// Every step only queues work on the stream; the scalars the host decides on
// (||b||^2, ||r||^2, the residual estimate) are copied into page-locked host
// memory and read with host() after the stream has been synchronised.
struct Gmres {
    int64_t n = 0, ld = 0;
    int m = 0;
    DevBuf<double> V, w, partial, hcol, h2, scal, H, cs, sn, g, y;
    DevBuf<GmresState> st;
    DevBuf<unsigned> count;                                // arrival count of the fused reductions (0 between launches)
    PinnedBuf<double> hs;                                  // 0: ||b||^2, 1: ||r||^2, 2: residual estimate
    PinnedBuf<GmresState> hst;                             // the initial state, copied without a host wait
    void init(int64_t n, int m, cudaStream_t s);
    void norm2_async(const double *x, cudaStream_t s);     // hs[0] = ||x||^2
    void set_bnorm(double bn, cudaStream_t s);
    void start_cycle(const double *r, cudaStream_t s);     // v_0 = r / ||r||; hs[1] = ||r||^2
    double *basis(int j) { return V.p + (int64_t)j * ld; }
    void arnoldi_step(int j, cudaStream_t s);              // needs w = A v_j; hs[2] = residual estimate
    double host(int i) const { return hs.p[i]; }
    void update_solution(int k, double *x, cudaStream_t s);
    // Device-driven Arnoldi loop (one GMRES cycle as a graph WHILE node): the
    // column j lives in the device state.  set_cycle: j = 0, at most maxit
    // steps.  copy_basis: dst = v_j.  arnoldi_step_dev: the step for w = A z
    // (z from v_j), then the loop condition: continue while the residual
    // estimate is >= tol, fewer than maxit steps and j + 1 < m.
    void set_cycle(int maxit, cudaStream_t s);
    void copy_basis(double *dst, cudaStream_t s);
    void arnoldi_step_dev(cudaGraphConditionalHandle h, double tol, cudaStream_t s, bool fused = false);
    // Device loop, fused form: the step's first kernel forms v_j (from w and
    // ||w|| of the previous step when pend, else the stored column), stores
    // it and writes z = M^-1 v_j (minv: 2x2 blocks of the surfaces (offset,
    // panels) given, or null for z = v_j); the loop control then runs in the
    // last block of the norm kernel (arnoldi_step_dev with fused = true).
    void prep_step(const double *minv, const std::vector<std::pair<int64_t, int64_t>> &surfaces, double *z,
                   cudaStream_t s);
    // hs[2] = residual estimate, hs[3] = steps of the cycle (copy queued after the loop)
    void read_cycle_async(cudaStream_t s);
};

// Inverse 2x2 self blocks of one surface's panels: minv = 4 n doubles (m11, m12, m21, m22 per panel).
void block_jacobi_inverse(int64_t n, double cV_in, const double *sa_in, double cV_out, const double *sa_out,
                          double *minv, cudaStream_t s);
// z = M^-1 u for one surface: (z_phi, z_dphi)_i = Minv_i (u_in, u_out)_i.
void block_jacobi_apply(int64_t n, const double *minv, const double *u_in, const double *u_out, double *z_phi,
                        double *z_dphi, cudaStream_t s);
// x = sum_c V[c] y[c] (k basis vectors) written into out.
void basis_combination(const Gmres &G, int k, double *out, cudaStream_t s);

void axpby(double a, const double *x, double b, const double *y, double *out, int64_t n, cudaStream_t s);
// *out = scale * sum_k q_k phi_k (device scalar)
void weighted_sum(const double *q, const double *phi, int64_t n, double scale, double *out, cudaStream_t s);
// rowv[i] = sum_{j != i} q_j / r_ij
void coulomb_rows(const double *xyz, const double *q, int64_t n, double *rowv, cudaStream_t s);

}  // namespace pb
