// Setup-phase geometry and quadrature entry points (geometry.cu).
#pragma once

#include "model.cuh"

namespace pb {

// Symmetric triangle rule: barycentric nodes and weights (weights sum to 1).
struct TriRule {
    int n;
    double l[19][3];
    double w[19];
};
TriRule make_rule(int K);   // K = 1, 3, 7, 19
int rule_slot(int K);       // index of rule K in a table {1, 3, 7, 19}

void upload_rules();
bool valid_rule(int K);
// Centroids, unit normals, areas, L = sqrt(2A), and the K Gauss points of every panel.
void surface_geometry(SurfDev &S, int K, cudaStream_t s);
// dV, dK per near entry of Pr: K_fine-rule minus K-rule values (FP64).
void near_values(const Pair &Pr, const Targets &G, const SurfDev &src, int K, int K_fine, double kappa, double *dV,
                 double *dK, cudaStream_t s);
// The same corrections evaluated in FP32 (mixed path).
// FP32 near-singular corrections of every kernel of the pair (kernel k at offset k * n_near).
void near_values32(const Pair &Pr, const Targets &G, const SurfDev &src, int K, int K_fine, float *dV, float *dK,
                   cudaStream_t s);
// Semi-analytical V_ii of every panel of S (input order).
void self_integrals(const SurfDev &S, int N_k, double kappa, double *out, cudaStream_t s);
// The same for two kernels in one pass (shared geometry).
void self_integrals2(const SurfDev &S, int N_k, double kappa0, double kappa1, double *out0, double *out1,
                     cudaStream_t s);
// out = selfv - the own panel's K-point share of the direct sum at the centroid (1/4pi included);
// valid for rules without a point at the centroid.
void self_minus_kpoint(const SurfDev &S, int K, double kappa, const double *selfv, double *out, cudaStream_t s);
// Its kappa derivative by the same rule.
void self_integrals_dkappa(const SurfDev &S, int N_k, double kappa, double *out, cudaStream_t s);
// b_i = sum_k q_k G(c_i, r_k) / eps for the panels of S (input order); FP64,
// or FP32 with compensated tile sums relative to `origin` when it is not null.
void rhs_rows(const SurfDev &S, int64_t nc, const double *q, const double *xyz, double kappa, double eps, double *b,
              const double *origin, cudaStream_t s);

}  // namespace pb
