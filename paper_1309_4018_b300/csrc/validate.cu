// Checks of the problem description: closed, consistently oriented meshes that
// enclose their inner region, and charges inside their region.
#include <algorithm>
#include <climits>
#include <cstdio>

#include "validate.cuh"

namespace pb {

// ---------------------------------------------------------------- meshes (device)

namespace {

// error codes of a mesh check, lowest first reported
constexpr unsigned long long kRepeat = 1, kOpen = 2, kFlip = 3;

__global__ void corner_count_kernel(int64_t n3, const int32_t *__restrict__ tris, int32_t *__restrict__ cnt) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < n3) atomicAdd(&cnt[tris[c]], 1);
}

__global__ void corner_fill_kernel(int64_t n3, const int32_t *__restrict__ tris, const int64_t *__restrict__ off,
                                   int32_t *__restrict__ cur, int32_t *__restrict__ adj) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n3) return;
    const int32_t v = tris[c];
    adj[off[v] + atomicAdd(&cur[v], 1)] = (int32_t)(c / 3);
}

// One thread per directed edge a -> b of triangle i: every other triangle at a
// is searched for b -> a (its partner) and a -> b (a duplicate).  A closed,
// consistently oriented 2-manifold has exactly one partner and no duplicate.
__global__ void edge_check_kernel(int64_t n3, const int32_t *__restrict__ tris, const int64_t *__restrict__ off,
                                  const int32_t *__restrict__ adj, unsigned long long *__restrict__ bad) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n3) return;
    const int64_t i = c / 3;
    const int k = (int)(c - 3 * i);
    const int32_t a = tris[c], b = tris[3 * i + (k == 2 ? 0 : k + 1)];
    unsigned long long code = 0;
    int uses = 1, rev = 0;
    if (a == b) {
        code = kRepeat;
    } else {
        for (int64_t q = off[a]; q < off[a + 1]; ++q) {
            const int32_t j = adj[q];
            if (j == i) continue;
            const int32_t t0 = tris[3 * (int64_t)j], t1 = tris[3 * (int64_t)j + 1], t2 = tris[3 * (int64_t)j + 2];
            const int32_t e[3][2] = {{t0, t1}, {t1, t2}, {t2, t0}};
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                if (e[m][0] == b && e[m][1] == a) { ++uses; ++rev; }
                if (e[m][0] == a && e[m][1] == b) ++uses;
            }
        }
        if (uses != 2) code = kOpen;
        else if (rev != 1) code = kFlip;
    }
    if (code) {
        // code, then the number of triangles on the edge (open case), then the corner
        const unsigned long long rec = (code << 60) | ((unsigned long long)min(uses, 255) << 52) |
                                       (unsigned long long)(c & ((1ull << 52) - 1));
        atomicMin(bad, rec);
    }
}

// Six times the signed volume, sum of a . (b x c): per-block sums in a fixed
// order, then one block adds them (the same result on every run).
constexpr int kVolBlocks = 256, kVolThreads = 256;

__global__ void __launch_bounds__(kVolThreads) volume_partial_kernel(int64_t nt, const double *__restrict__ v,
                                                                     const int32_t *__restrict__ t,
                                                                     double *__restrict__ part) {
    __shared__ double sh[kVolThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kVolThreads + threadIdx.x; i < nt; i += (int64_t)kVolBlocks * kVolThreads) {
        const double *a = v + 3 * (int64_t)t[3 * i], *b = v + 3 * (int64_t)t[3 * i + 1], *c = v + 3 * (int64_t)t[3 * i + 2];
        acc += a[0] * (b[1] * c[2] - b[2] * c[1]) + a[1] * (b[2] * c[0] - b[0] * c[2]) +
               a[2] * (b[0] * c[1] - b[1] * c[0]);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kVolThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kVolBlocks) volume_final_kernel(const double *__restrict__ part,
                                                                  MeshCheck *__restrict__ out,
                                                                  const unsigned long long *__restrict__ bad) {
    __shared__ double sh[kVolBlocks];
    sh[threadIdx.x] = part[threadIdx.x];
    __syncthreads();
    for (int w = kVolBlocks / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out->vol6 = sh[0];
        out->bad = *bad;
    }
}

}  // namespace

__global__ void value_check_kernel(const double *__restrict__ x, int64_t nx, const int32_t *__restrict__ idx,
                                   int64_t ni, int64_t lim, unsigned long long *bad) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nx; i += stride)
        if (!isfinite(x[i])) atomicMin(bad, (unsigned long long)i);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ni; i += stride)
        if (idx[i] < 0 || idx[i] >= lim) atomicMin(bad + 1, (unsigned long long)i);
}

void check_values_async(const double *x, int64_t nx, const int32_t *idx, int64_t ni, int64_t lim, ValueCheck *out,
                        cudaStream_t s) {
    TmpBuf<unsigned long long> bad(2, s);
    PB_CUDA_TRY(cudaMemsetAsync(bad.p, 0xff, 2 * sizeof(unsigned long long), s));
    const int64_t n = nx > ni ? nx : ni;
    if (n > 0) {
        const int64_t want = div_up(n, 256);
        const int blocks = (int)(want < 148 * 8 ? want : 148 * 8);
        value_check_kernel<<<blocks, 256, 0, s>>>(x, nx, idx, ni, lim, bad.p);
        PB_LAUNCH_CHECK();
    }
    PB_CUDA_TRY(cudaMemcpyAsync(out, bad.p, sizeof(ValueCheck), cudaMemcpyDeviceToHost, s));
}

void check_mesh_async(const double *verts, int64_t nv, const int32_t *tris, int64_t nt, MeshCheck *out,
                      cudaStream_t s) {
    const int64_t n3 = 3 * nt;
    TmpBuf<int32_t> cnt(nv, s), cur(nv, s), adj(n3, s);
    TmpBuf<int64_t> off(nv + 1, s);
    TmpBuf<unsigned long long> bad(1, s);
    TmpBuf<double> part(kVolBlocks, s);
    TmpBuf<MeshCheck> res(1, s);
    PB_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, nv * sizeof(int32_t), s));
    PB_CUDA_TRY(cudaMemsetAsync(cur.p, 0, nv * sizeof(int32_t), s));
    PB_CUDA_TRY(cudaMemsetAsync(bad.p, 0xff, sizeof(unsigned long long), s));
    corner_count_kernel<<<div_up(n3, 256), 256, 0, s>>>(n3, tris, cnt.p);
    PB_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(cnt.p, off.p, nv, s);
    corner_fill_kernel<<<div_up(n3, 256), 256, 0, s>>>(n3, tris, off.p, cur.p, adj.p);
    PB_LAUNCH_CHECK();
    edge_check_kernel<<<div_up(n3, 256), 256, 0, s>>>(n3, tris, off.p, adj.p, bad.p);
    PB_LAUNCH_CHECK();
    volume_partial_kernel<<<kVolBlocks, kVolThreads, 0, s>>>(nt, verts, tris, part.p);
    PB_LAUNCH_CHECK();
    volume_final_kernel<<<1, kVolBlocks, 0, s>>>(part.p, res.p, bad.p);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaMemcpyAsync(out, res.p, sizeof(MeshCheck), cudaMemcpyDeviceToHost, s));
}

void mesh_check_result(const MeshCheck &r) {
    if (r.bad != ~0ull) {
        const unsigned long long code = r.bad >> 60, uses = (r.bad >> 52) & 255, c = r.bad & ((1ull << 52) - 1);
        const std::string where = "triangle " + std::to_string(c / 3) + ", corner " + std::to_string(c % 3);
        if (code == kRepeat) fail(PB_EINVAL, "a triangle repeats a vertex (" + where + ")");
        if (code == kOpen)
            fail(PB_EINVAL, "surface is not a closed 2-manifold: an edge belongs to " + std::to_string(uses) +
                                " triangle(s), not 2 (" + where + ")");
        fail(PB_EINVAL, "surface is not consistently oriented: an edge is traversed twice in the same direction (" +
                            where + ")");
    }
    if (!(r.vol6 > 0.0)) {
        char buf[96];
        std::snprintf(buf, sizeof buf, "%.6g", r.vol6 / 6.0);
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
