// Checks of the problem description before any boundary-element work.
//
// The paper's surfaces come from MSMS and are closed, consistently oriented
// triangulations with the charges inside the molecule (Sec. 2.2, Sec. 3); the
// boundary-integral equations assume exactly that.  A mesh with a hole, a
// flipped triangle or reversed winding, or a charge outside its region, gives
// a wrong energy without any numerical warning, so these inputs are refused.
#pragma once

#include "common.cuh"

namespace pb {

// PB_EINVAL unless every edge of the mesh is shared by exactly two triangles
// that traverse it in opposite directions (a closed, consistently oriented
// 2-manifold), no triangle repeats a vertex index, and the signed volume
// (1/6) sum v0 . (v1 x v2) is positive: the triangles wind counter-clockwise
// seen from the outer region, so the surface encloses its inner region.
// Host arrays; O(nt) work.
void check_closed_mesh(const double *verts, int64_t nv, const int32_t *tris, int64_t nt);

// Queues on s the winding number of the closed surface (device verts, tris)
// about each of nc points xyz (device): the signed count of the surface's
// crossings by a ray from the point, +1 where the surface's normal points
// along the ray.  It is 1 for a point the surface encloses and 0 outside.
// wind[nc] must be zeroed first; the counts are added to it.
void winding_numbers(const double *verts, const int32_t *tris, int64_t nt, const double *xyz, int64_t nc,
                     int32_t *wind, cudaStream_t s);

// Queues on s: bad[0] = number of points i whose winding numbers
// wind[k * nc + i] differ from expect[k] for some k < nsurf (nsurf <= 8);
// bad[1] = the lowest such i, bad[2] = its surface k.  bad[] is overwritten.
void winding_mismatch(const int32_t *wind, int64_t nc, int nsurf, const int32_t *expect, int32_t *bad,
                      cudaStream_t s);

}  // namespace pb
