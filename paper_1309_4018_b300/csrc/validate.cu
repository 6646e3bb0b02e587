// Checks of the problem description: closed, consistently oriented meshes that
// enclose their inner region, and charges inside their region.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "validate.cuh"

namespace pb {

// ---------------------------------------------------------------- meshes (host)

void check_closed_mesh(const double *verts, int64_t nv, const int32_t *tris, int64_t nt) {
    // directed edges bucketed by their lower vertex (counting sort); each
    // undirected edge must occur exactly twice, once in each direction
    std::vector<int64_t> start(nv + 1, 0);
    for (int64_t i = 0; i < nt; ++i) {
        const int32_t *t = tris + 3 * i;
        if (t[0] == t[1] || t[1] == t[2] || t[2] == t[0])
            fail(PB_EINVAL, "triangle " + std::to_string(i) + " repeats a vertex");
        for (int k = 0; k < 3; ++k) ++start[std::min(t[k], t[(k + 1) % 3]) + 1];
    }
    for (int64_t v = 0; v < nv; ++v) start[v + 1] += start[v];
    std::vector<int64_t> fill(start.begin(), start.end() - 1);
    std::vector<int32_t> other(3 * nt);
    std::vector<int8_t> dir(3 * nt);
    for (int64_t i = 0; i < nt; ++i) {
        const int32_t *t = tris + 3 * i;
        for (int k = 0; k < 3; ++k) {
            const int32_t a = t[k], b = t[(k + 1) % 3];
            const int64_t slot = fill[std::min(a, b)]++;
            other[slot] = std::max(a, b);
            dir[slot] = a < b ? 1 : -1;
        }
    }
    for (int64_t v = 0; v < nv; ++v)
        for (int64_t i = start[v]; i < start[v + 1]; ++i) {
            int uses = 0, net = 0;
            for (int64_t j = start[v]; j < start[v + 1]; ++j)
                if (other[j] == other[i]) { ++uses; net += dir[j]; }
            const std::string e = "edge (" + std::to_string(v) + ", " + std::to_string(other[i]) + ")";
            if (uses != 2)
                fail(PB_EINVAL, "surface is not a closed 2-manifold: " + e + " belongs to " +
                                    std::to_string(uses) + " triangle(s), not 2");
            if (net != 0)
                fail(PB_EINVAL, "surface is not consistently oriented: " + e +
                                    " is traversed twice in the same direction");
        }
    double vol6 = 0.0;
    for (int64_t i = 0; i < nt; ++i) {
        const double *a = verts + 3 * (int64_t)tris[3 * i], *b = verts + 3 * (int64_t)tris[3 * i + 1],
                     *c = verts + 3 * (int64_t)tris[3 * i + 2];
        vol6 += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
                a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    if (!(vol6 > 0.0)) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "%.6g", vol6 / 6.0);
        fail(PB_EINVAL, std::string("surface encloses its outer region (signed volume ") + buf +
                            " <= 0): triangles must wind counter-clockwise seen from the outer region");
    }
}

// ---------------------------------------------------------------- winding numbers (device)

namespace {

// The ray from a point p runs along d = (1, kSy, kSz).  In the sheared
// coordinates (y - kSy x, z - kSz x) it is the single point (p_y', p_z'), so a
// triangle is crossed when that point lies inside the triangle's sheared
// projection, ahead of p.  The projected orientation equals n . d, positive
// when the outward normal points along the ray (the ray leaves the enclosed
// region).  The slopes are generic so that the ray meets no edge or vertex of
// a mesh built on a grid or a sphere.
constexpr double kSy = 0.5772156649015329;
constexpr double kSz = 0.3010299956639812;
constexpr int kWindThreads = 128;
constexpr int kWindTile = 512;

struct Sh {
    double y, z;
};

__device__ __forceinline__ Sh shear(const double *v, int32_t i, double *x) {
    const double vx = v[3 * (int64_t)i], vy = v[3 * (int64_t)i + 1], vz = v[3 * (int64_t)i + 2];
    *x = vx;
    return Sh{vy - kSy * vx, vz - kSz * vx};
}

// Edge function of the directed edge u -> w at p, evaluated with the lower
// vertex index first so that the two triangles sharing an edge get exactly
// opposite values (no point is counted by both or by neither).
__device__ __forceinline__ double edge_fn(Sh u, int32_t iu, Sh w, int32_t iw, Sh p) {
    if (iu > iw) {
        const Sh t = u; u = w; w = t;
        return -((w.y - u.y) * (p.z - u.z) - (w.z - u.z) * (p.y - u.y));
    }
    return (w.y - u.y) * (p.z - u.z) - (w.z - u.z) * (p.y - u.y);
}

__device__ int crossing(const double *v, const int32_t *t, int64_t j, double px, Sh p) {
    const int32_t ia = t[3 * j], ib = t[3 * j + 1], ic = t[3 * j + 2];
    double ax, bx, cx;
    const Sh A = shear(v, ia, &ax), B = shear(v, ib, &bx), C = shear(v, ic, &cx);
    const double e0 = edge_fn(B, ib, C, ic, p);   // weight of A
    const double e1 = edge_fn(C, ic, A, ia, p);   // weight of B
    const double e2 = edge_fn(A, ia, B, ib, p);   // weight of C
    const bool pos = e0 > 0.0 && e1 > 0.0 && e2 > 0.0, neg = e0 < 0.0 && e1 < 0.0 && e2 < 0.0;
    if (!pos && !neg) return 0;
    const double o = e0 + e1 + e2;   // twice the projected area, signed
    const double xh = (e0 * ax + e1 * bx + e2 * cx) / o;
    if (!(xh > px)) return 0;
    return pos ? 1 : -1;
}

__global__ void shear_bbox_kernel(const double *v, const int32_t *t, int64_t nt, float4 *bb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    double ylo = 1e300, yhi = -1e300, zlo = 1e300, zhi = -1e300, x;
    for (int k = 0; k < 3; ++k) {
        const Sh s = shear(v, t[3 * i + k], &x);
        ylo = fmin(ylo, s.y); yhi = fmax(yhi, s.y);
        zlo = fmin(zlo, s.z); zhi = fmax(zhi, s.z);
    }
    // rounded outwards: the FP32 box contains the FP64 one
    bb[i] = make_float4(__double2float_rd(ylo), __double2float_ru(yhi), __double2float_rd(zlo),
                        __double2float_ru(zhi));
}

__global__ void __launch_bounds__(kWindThreads) winding_kernel(const double *v, const int32_t *t,
                                                               const float4 *__restrict__ bb, int64_t nt,
                                                               int64_t chunk, const double *xyz, int64_t nc,
                                                               int32_t *wind) {
    __shared__ float4 tile[kWindTile];
    const int64_t i = (int64_t)blockIdx.x * kWindThreads + threadIdx.x;
    const bool act = i < nc;
    double px = 0.0;
    Sh p{0.0, 0.0};
    float ylo = 0.f, yhi = 0.f, zlo = 0.f, zhi = 0.f;
    if (act) {
        px = xyz[3 * i];
        p = Sh{xyz[3 * i + 1] - kSy * px, xyz[3 * i + 2] - kSz * px};
        ylo = __double2float_rd(p.y); yhi = __double2float_ru(p.y);
        zlo = __double2float_rd(p.z); zhi = __double2float_ru(p.z);
    }
    const int64_t t0 = (int64_t)blockIdx.y * chunk, t1 = t0 + chunk < nt ? t0 + chunk : nt;
    int cnt = 0;
    for (int64_t base = t0; base < t1; base += kWindTile) {
        const int m = (int)(t1 - base < kWindTile ? t1 - base : kWindTile);
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += kWindThreads) tile[k] = bb[base + k];
        __syncthreads();
        if (!act) continue;
        for (int k = 0; k < m; ++k) {
            const float4 b = tile[k];
            if (yhi < b.x || ylo > b.y || zhi < b.z || zlo > b.w) continue;
            cnt += crossing(v, t, base + k, px, p);
        }
    }
    if (act && cnt) atomicAdd(&wind[i], cnt);
}

struct Expect8 {
    int32_t v[8];
};

__global__ void __launch_bounds__(1024) winding_mismatch_kernel(const int32_t *wind, int64_t nc, int nsurf,
                                                                Expect8 e, int32_t *bad) {
    __shared__ int nbad;
    __shared__ int first;   // lowest (point * 8 + surface) that mismatches
    if (threadIdx.x == 0) { nbad = 0; first = INT_MAX; }
    __syncthreads();
    for (int64_t i = threadIdx.x; i < nc; i += blockDim.x)
        for (int k = 0; k < nsurf; ++k)
            if (wind[k * nc + i] != e.v[k]) {
                atomicAdd(&nbad, 1);
                atomicMin(&first, (int)(i * 8 + k < INT_MAX ? i * 8 + k : INT_MAX));
                break;
            }
    __syncthreads();
    if (threadIdx.x == 0) {
        bad[0] = nbad;
        bad[1] = nbad ? first / 8 : -1;
        bad[2] = nbad ? first % 8 : -1;
    }
}

}  // namespace

void winding_numbers(const double *verts, const int32_t *tris, int64_t nt, const double *xyz, int64_t nc,
                     int32_t *wind, cudaStream_t s) {
    if (nt == 0 || nc == 0) return;
    TmpBuf<float4> bb(nt, s);
    shear_bbox_kernel<<<div_up(nt, 256), 256, 0, s>>>(verts, tris, nt, bb.p);
    PB_LAUNCH_CHECK();
    const int gx = div_up(nc, kWindThreads);
    // about four blocks per SM over the whole (charges x triangles) product
    const int64_t gy = std::max<int64_t>(1, std::min<int64_t>(div_up(4 * 148, gx), div_up(nt, kWindTile)));
    const int64_t chunk = (nt + gy - 1) / gy;
    winding_kernel<<<dim3(gx, (unsigned)gy), kWindThreads, 0, s>>>(verts, tris, bb.p, nt, chunk, xyz, nc, wind);
    PB_LAUNCH_CHECK();
}

void winding_mismatch(const int32_t *wind, int64_t nc, int nsurf, const int32_t *expect, int32_t *bad,
                      cudaStream_t s) {
    if (nsurf > 8) fail(PB_EINVAL, "internal: more than 8 surfaces in a winding check");
    Expect8 e{};
    for (int k = 0; k < nsurf; ++k) e.v[k] = expect[k];
    winding_mismatch_kernel<<<1, 1024, 0, s>>>(wind, nc, nsurf, e, bad);
    PB_LAUNCH_CHECK();
}

}  // namespace pb
