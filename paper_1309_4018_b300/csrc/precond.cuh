// Cluster block preconditioner of the right-preconditioned GMRES (precond.cu).
//
// Not in the paper (which solves the collocation system by GMRES, Sec. 2.3):
// the panels of every surface are cut, in the Morton order of their
// centroids, into runs of up to 64; each run's unknowns (phi, dphi per panel)
// and rows (the two sides of the surface per panel) form a block of at most
// 128 x 128 that holds the run's couplings through the surface's own kernels
// (self terms from the semi-analytical rule, the rest from the K-point rule
// without the near-singular refinement), inverted once per setup in FP32 by
// Gauss-Jordan elimination with partial pivoting.  z = M^-1 v is then a block
// product per run with FP64 sums, so that M^-1 is linear to FP64 rounding and
// the solution update x += M^-1 (V y) equals the sum of the preconditioned
// directions.  Right preconditioning leaves the solution unchanged: GMRES
// still drives the true residual of A x = b below the tolerance.
#pragma once

#include <vector>

#include "common.cuh"

namespace pb {

constexpr int kClusterMax = 64;   // panels per block at most

// One surface's part of the preconditioner.
struct ClusterSurface {
    int64_t n = 0, off = 0;     // panels, first panel in the concatenated list
    const int32_t *order = nullptr;   // Morton-sorted position -> panel
    int cb = 64;                // panels per block
    int64_t first = 0;          // its first block in the problem's block list
    int64_t nblocks() const { return (n + cb - 1) / cb; }
};

// The couplings of a run through the surface's own kernel on row side s
// (s = 0 inner, 1 outer): y_s = 1/2 phi + cK[s] K + cV[s] V with the Yukawa
// (or Laplace, kappa = 0) kernel kappa[s] and the self values selfV[s].
struct ClusterRows {
    double cK[2], cV[2], kappa[2];
    const double *selfV[2];
};

struct ClusterGeom {
    const double *cen, *nrm;      // panel centroids and normals (n x 3)
    const double *gy, *gwa;       // K Gauss points per panel (n K x 3) and weight x area (n K)
    int K;
};

// Floats per side of a stored block for runs of cb panels (16, 32, 64 or 128).
int cluster_block_dim(int cb);
// Inverse blocks of one surface into binv (its first block at sf.first;
// cluster_block_dim(cb)^2 floats per block, stored transposed: binv[w][u]
// maps residual entry w to unknown u of the block).  *err is set to 1 where a
// pivot vanished.
void cluster_blocks(const ClusterSurface &sf, const ClusterGeom &g, const ClusterRows &r, float *binv, int *err,
                    cudaStream_t s);
// z = M^-1 u over every surface (u, z: 2 N doubles; may not alias).
void cluster_apply(const std::vector<ClusterSurface> &sfs, const float *binv, const double *u, double *z,
                   cudaStream_t s);

// z = M^-T u (the adjoint solve's right preconditioner).
void cluster_apply_T(const std::vector<ClusterSurface> &sfs, const float *binv, const double *u, double *z,
                     cudaStream_t s);

// Device-loop form (GMRES graph): v_j formed as in Gmres::prep_step (from w
// and ||w|| when st->pend, else column j of V; stored as column j), then z = M^-1 v_j.
struct GmresState;
void cluster_prep(const std::vector<ClusterSurface> &sfs, const float *binv, const GmresState *st, double *V,
                  int64_t ld, const double *w, const double *num_sq, double *z, cudaStream_t s);

}  // namespace pb
