// Gaussian-density molecular surface built on the device (surface.cu).
#pragma once

#include "problem.cuh"

namespace pb {

struct SurfGenParams {
    double spacing = 0.0, beta = 0.5, cutoff = 2.7, radius_offset = 0.0, margin = 4.0, level = 1.0,
           tclamp = 0.02, relax = 0.5, max_step = 0.3;
    int smooth_iters = 5, newton_steps = 3;
};

// Level set rho = level of the atoms' Gaussian density, triangulated by
// marching tetrahedra, outer component kept, smoothed on the level set.
// Host atom arrays; the mesh is left in out.v / out.t (device) and out.gen
// records the grid, components and rounds.  Synchronises s.
void gaussian_surface(const double *xyz, const double *radius, int64_t na, const SurfGenParams &p,
                      cudaStream_t s, SurfIn &out);

}  // namespace pb
