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

// Mesh check: every edge of the mesh must be shared by exactly two triangles
// that traverse it in opposite directions (a closed, consistently oriented
// 2-manifold), no triangle may repeat a vertex index, and the signed volume
// (1/6) sum v0 . (v1 x v2) must be positive: the triangles wind
// counter-clockwise seen from the outer region, so the surface encloses its
// inner region.  check_mesh_async queues the check of a device mesh on s and
// copies its outcome to *out (page-locked host memory, valid once s has been
// synchronised); mesh_check_result then fails with PB_EINVAL and a message
// when the mesh is refused.  Work: one thread per directed edge searching
// the triangles at its first vertex.
struct MeshCheck {
    unsigned long long bad;   // all ones: no edge fault; else (code << 60) | (uses << 52) | corner
    double vol6;              // six times the signed volume
};
void check_mesh_async(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, MeshCheck *out,
                      cudaStream_t s);
void mesh_check_result(const MeshCheck &r);

// Check of arrays given by device pointers: bad_value = the lowest i < nx
// with a non-finite x[i], bad_index = the lowest i < ni with idx[i] outside
// [0, lim); all ones where there is none.  Queued on s and copied to *out
// (page-locked host memory, valid once s has been synchronised).
struct ValueCheck {
    unsigned long long bad_value, bad_index;
};
void check_values_async(const double *x, int64_t nx, const int32_t *idx, int64_t ni, int64_t lim, ValueCheck *out,
                        cudaStream_t s);

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
