// Gaussian-density molecular surface built on the device.
//
// The paper takes its solvent-excluded surfaces from MSMS (Sec. 2.2, Sec. 3);
// this library meshes instead the level set rho(x) = level of
//
//   rho(x) = sum_a [|x - x_a| <= cutoff R_a] exp(-beta (|x - x_a|^2 / R_a^2 - 1)),
//
// R_a the atomic radius plus an offset (+2 A for a Stern layer):
//   1. density at the nodes lo + h (i, j, k) of a grid around the atoms, one
//      warp per node summing the atoms of the 27 atom cells around it;
//   2. one vertex on every node edge of the Kuhn split (7 positive directions)
//      whose two ends differ in the test rho >= level, at the zero of the
//      linear interpolant of rho - level (parameter clamped to
//      [tclamp, 1 - tclamp]); vertices are numbered by (lower node, direction),
//      which is ascending (lower node, upper node);
//   3. every grid cube is six positively oriented tetrahedra, each giving 0, 1
//      or 2 triangles; the orientation follows from the parity of the vertex
//      permutation alone, so every normal points from rho >= level to
//      rho < level (into the outer region) with no floating-point test;
//   4. union-find over the vertices; the component of the last vertex (the
//      crossing of largest x index) is the outer surface and is kept;
//   5. smoothing rounds (umbrella step, then Newton projections onto the
//      level set along grad rho); the largest round count that folds no
//      more triangles against grad rho than the unsmoothed mesh is used.
// Every decision that picks an integer (inside test, crossings, components)
// is taken on FP64 values; there are two host synchronisations (the raw
// vertex and triangle counts, then the final counts).
#include <algorithm>
#include <cmath>

#include "surface.cuh"

namespace pb {

namespace {

struct Grid {
    double lo[3], h;
    int n[3];
    int64_t nn;
};

struct Cells {
    double c0[3], cs;
    int nc[3];
    const dvec4 *atoms;       // sorted by cell: x, y, z, 1 / R^2
    const double *rc2;        // same order: (cutoff R)^2
    const float4 *atoms32;    // same order: x - c0, y - c0, z - c0, rejection bound on d^2 (FP32)
    const int64_t *start;     // first atom of every cell; ncell + 1 entries
};

struct Shape {
    double beta, cutoff, level, tclamp, relax, max_step;
    int newton_steps;
};

// The six Kuhn tetrahedra of a cube (corner bit 0: +x, bit 1: +y, bit 2: +z),
// monotone corner paths listed with positive orientation.
__constant__ int8_t kTet[6][4] = {{0, 1, 3, 7}, {0, 1, 7, 5}, {0, 2, 7, 3},
                                  {0, 2, 6, 7}, {0, 4, 5, 7}, {0, 4, 7, 6}};

__device__ __forceinline__ double node_coord(double lo, double h, int i) { return __dadd_rn(lo, __dmul_rn(h, (double)i)); }

__device__ __forceinline__ int64_t corner_offset(const Grid &g, int c) {
    return (int64_t)(c & 1) * g.n[1] * g.n[2] + (int64_t)((c >> 1) & 1) * g.n[2] + ((c >> 2) & 1);
}

// direction number 0..6 of a positive step (dx, dy, dz), ascending in node-id offset
__device__ __forceinline__ int dir_of(int dx, int dy, int dz) { return (dx << 2 | dy << 1 | dz) - 1; }

__device__ __forceinline__ int cell_of(double x, double c0, double cs, int n) {
    double u = floor((x - c0) / cs);
    u = fmin(fmax(u, -2.0), (double)n + 1.0);
    return (int)u;
}

// rho (and grad rho) at p, by one warp: every atom within its cutoff, atoms of
// the 27 cells around p.  The lanes first sweep the candidates with an FP32
// distance test and append the survivors to a per-warp list (buf, kSurvCap
// entries); its bound exceeds (cutoff R)^2 by more than the FP32 rounding of
// the coordinates can move d^2, so the list holds every atom the FP64 test
// keeps.  The lanes then take the listed atoms 32 at a time through the FP64
// test and exponential, so that the FP64 work runs with all lanes busy.  The
// survivors' order is fixed and the butterfly reduction leaves the same bits
// in every lane.
constexpr int kSurvCap = 96;

template <bool GRAD>
__device__ __forceinline__ void eval_survivors(const Cells &C, const Shape &S, double px, double py, double pz,
                                               const int *buf, int n, int lane, double &acc, double &g0, double &g1,
                                               double &g2) {
    const double m2b = -2.0 * S.beta;
    for (int i = lane; i < n; i += 32) {
        const int a = buf[i];
        const dvec4 A = C.atoms[a];
        const double gx = __dsub_rn(px, A.x), gy = __dsub_rn(py, A.y), gz = __dsub_rn(pz, A.z);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(gx, gx), __dmul_rn(gy, gy)), __dmul_rn(gz, gz));
        if (d2 > C.rc2[a]) continue;
        const double e = exp(__dmul_rn(-S.beta, __dsub_rn(__dmul_rn(d2, A.w), 1.0)));
        acc = __dadd_rn(acc, e);
        if (GRAD) {
            const double c = e * m2b * A.w;      // d/dx of the term is c (x - x_a)
            g0 = fma(c, gx, g0);
            g1 = fma(c, gy, g1);
            g2 = fma(c, gz, g2);
        }
    }
}

template <bool GRAD>
__device__ void density_warp(const Cells &C, const Shape &S, double px, double py, double pz, int lane, int *buf,
                             double &rho, double *g) {
    const int q0 = cell_of(px, C.c0[0], C.cs, C.nc[0]);
    const int q1 = cell_of(py, C.c0[1], C.cs, C.nc[1]);
    const int q2 = cell_of(pz, C.c0[2], C.cs, C.nc[2]);
    const int z0 = max(q2 - 1, 0), z1 = min(q2 + 1, C.nc[2] - 1);
    const float fx = (float)(px - C.c0[0]), fy = (float)(py - C.c0[1]), fz = (float)(pz - C.c0[2]);
    double acc = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
    int n = 0;
    if (z0 <= z1)
        for (int ix = max(q0 - 1, 0); ix <= min(q0 + 1, C.nc[0] - 1); ++ix)
            for (int iy = max(q1 - 1, 0); iy <= min(q1 + 1, C.nc[1] - 1); ++iy) {
                const int64_t row = ((int64_t)ix * C.nc[1] + iy) * C.nc[2];
                const int64_t a1 = C.start[row + z1 + 1];
                for (int64_t base = C.start[row + z0]; base < a1; base += 32) {
                    const int64_t a = base + lane;
                    bool keep = false;
                    if (a < a1) {
                        const float4 F = C.atoms32[a];
                        const float dx = fx - F.x, dy = fy - F.y, dz = fz - F.z;
                        keep = dx * dx + dy * dy + dz * dz <= F.w;
                    }
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (keep) buf[n + __popc(m & ((1u << lane) - 1u))] = (int)a;
                    n += __popc(m);
                    if (n > kSurvCap - 32) {
                        __syncwarp();
                        eval_survivors<GRAD>(C, S, px, py, pz, buf, n, lane, acc, g0, g1, g2);
                        __syncwarp();
                        n = 0;
                    }
                }
            }
    __syncwarp();
    eval_survivors<GRAD>(C, S, px, py, pz, buf, n, lane, acc, g0, g1, g2);
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if (GRAD) {
            g0 = __dadd_rn(g0, __shfl_xor_sync(0xffffffffu, g0, o));
            g1 = __dadd_rn(g1, __shfl_xor_sync(0xffffffffu, g1, o));
            g2 = __dadd_rn(g2, __shfl_xor_sync(0xffffffffu, g2, o));
        }
    }
    rho = acc;
    if (GRAD) {
        g[0] = g0;
        g[1] = g1;
        g[2] = g2;
    }
}

// 256-thread blocks, one warp per point; each warp's survivor list in shared memory
constexpr int kWarpsPerBlock = 8;
#define PB_SURV_BUF(name) \
    __shared__ int name##_all[kWarpsPerBlock][kSurvCap]; \
    int *name = name##_all[threadIdx.x >> 5]

// ------------------------------------------------------------------ atoms into cells
__global__ void pack_atoms_kernel(int64_t na, const double *__restrict__ xyz, const double *__restrict__ r,
                                  double offset, Cells C, dvec4 *__restrict__ packed, uint64_t *__restrict__ key,
                                  int32_t *__restrict__ idx) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= na) return;
    const double x = xyz[3 * a], y = xyz[3 * a + 1], z = xyz[3 * a + 2];
    packed[a] = dvec4{x, y, z, r[a] + offset};
    const int cx = min(max(cell_of(x, C.c0[0], C.cs, C.nc[0]), 0), C.nc[0] - 1);
    const int cy = min(max(cell_of(y, C.c0[1], C.cs, C.nc[1]), 0), C.nc[1] - 1);
    const int cz = min(max(cell_of(z, C.c0[2], C.cs, C.nc[2]), 0), C.nc[2] - 1);
    key[a] = ((uint64_t)cx * C.nc[1] + cy) * C.nc[2] + cz;
    idx[a] = (int32_t)a;
}

__global__ void cell_count_kernel(int64_t na, const uint64_t *__restrict__ key, int32_t *__restrict__ cnt) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a < na) atomicAdd(cnt + key[a], 1);
}

// Sorted FP64 atoms (position, 1 / R^2), their cutoff (cutoff R)^2 and their
// FP32 prefilter records.  ecoord bounds the
// FP32 rounding error of a coordinate relative to c0 (query or atom), so
// |d^2_FP32 - d^2| stays below the bound's excess over (cutoff R)^2.
__global__ void gather_atoms_kernel(int64_t na, const int32_t *__restrict__ idx, const dvec4 *__restrict__ in,
                                    Cells C, double cutoff, double ecoord, dvec4 *__restrict__ out,
                                    double *__restrict__ rc2, float4 *__restrict__ out32) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= na) return;
    const dvec4 A = in[idx[a]];
    out[a] = dvec4{A.x, A.y, A.z, 1.0 / __dmul_rn(A.w, A.w)};
    const double rc = __dmul_rn(cutoff, A.w);
    rc2[a] = __dmul_rn(rc, rc);
    const double rp = rc + 8.0 * ecoord;
    out32[a] = make_float4((float)(A.x - C.c0[0]), (float)(A.y - C.c0[1]), (float)(A.z - C.c0[2]),
                           (float)(rp * rp * (1.0 + 1e-5)));
}

// ------------------------------------------------------------------ grid
// One warp per node.
__global__ void density_kernel(Grid g, Cells C, Shape S, double *__restrict__ rho) {
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= g.nn) return;
    const int k = (int)(p % g.n[2]);
    const int64_t ij = p / g.n[2];
    const int j = (int)(ij % g.n[1]), i = (int)(ij / g.n[1]);
    PB_SURV_BUF(buf);
    double r;
    density_warp<false>(C, S, node_coord(g.lo[0], g.h, i), node_coord(g.lo[1], g.h, j), node_coord(g.lo[2], g.h, k),
                        lane, buf, r, nullptr);
    if (lane == 0) rho[p] = r;
}

// Crossing flags of the 7 edges leaving every node, and their count.
__global__ void crossing_kernel(Grid g, double level, const double *__restrict__ rho, uint8_t *__restrict__ flags,
                                int32_t *__restrict__ cnt) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.nn) return;
    const int k = (int)(p % g.n[2]);
    const int64_t ij = p / g.n[2];
    const int j = (int)(ij % g.n[1]), i = (int)(ij / g.n[1]);
    const bool in0 = rho[p] >= level;
    unsigned f = 0;
    for (int c = 1; c < 8; ++c) {
        const int dx = c >> 2, dy = (c >> 1) & 1, dz = c & 1;
        if (i + dx >= g.n[0] || j + dy >= g.n[1] || k + dz >= g.n[2]) continue;
        const int64_t q = p + (int64_t)dx * g.n[1] * g.n[2] + (int64_t)dy * g.n[2] + dz;
        if ((rho[q] >= level) != in0) f |= 1u << dir_of(dx, dy, dz);
    }
    flags[p] = (uint8_t)f;
    cnt[p] = __popc(f);
}

// Triangles of one positively oriented tetrahedron with inside mask m (bit v:
// local vertex v has rho >= level).  For an even permutation (a, b, c, d),
// the triangle through the edges ab, ac, ad faces away from a.
__device__ __forceinline__ int tet_triangles(int m, int8_t e[2][3][2]) {
    const int n = __popc(m);
    if (n == 0 || n == 4) return 0;
    if (n != 2) {
        const int a = n == 1 ? __ffs(m) - 1 : __ffs(~m & 15) - 1;
        const int b = a ^ 1, c = a ^ 2, d = a ^ 3;     // (a, b, c, d) is even
        const int s1 = n == 1 ? c : d, s2 = n == 1 ? d : c;
        e[0][0][0] = a; e[0][0][1] = b;
        e[0][1][0] = a; e[0][1][1] = s1;
        e[0][2][0] = a; e[0][2][1] = s2;
        return 1;
    }
    const int a = __ffs(m) - 1, b = __ffs(m & ~(1 << a)) - 1;
    const int om = ~m & 15;
    int c = __ffs(om) - 1, d = __ffs(om & ~(1 << c)) - 1;
    if (m == 0x5 || m == 0xA) { const int t = c; c = d; d = t; }   // (a, b, c, d) odd otherwise
    e[0][0][0] = a; e[0][0][1] = c;
    e[0][1][0] = a; e[0][1][1] = d;
    e[0][2][0] = b; e[0][2][1] = d;
    e[1][0][0] = a; e[1][0][1] = c;
    e[1][1][0] = b; e[1][1][1] = d;
    e[1][2][0] = b; e[1][2][1] = c;
    return 2;
}

__device__ __forceinline__ void cube_of(const Grid &g, int64_t c, int64_t &p0, unsigned &inside, const double *rho,
                                        double level) {
    const int64_t mz = g.n[2] - 1, my = g.n[1] - 1;
    const int k = (int)(c % mz);
    const int64_t ij = c / mz;
    const int j = (int)(ij % my), i = (int)(ij / my);
    p0 = ((int64_t)i * g.n[1] + j) * g.n[2] + k;
    inside = 0;
    for (int q = 0; q < 8; ++q)
        if (rho[p0 + corner_offset(g, q)] >= level) inside |= 1u << q;
}

__device__ __forceinline__ int tet_mask(int t, unsigned inside) {
    int m = 0;
    for (int v = 0; v < 4; ++v) m |= (int)((inside >> kTet[t][v]) & 1u) << v;
    return m;
}

__global__ void cube_count_kernel(Grid g, int64_t ncube, double level, const double *__restrict__ rho,
                                  int32_t *__restrict__ cnt) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncube) return;
    int64_t p0;
    unsigned inside;
    cube_of(g, c, p0, inside, rho, level);
    int n = 0;
    if (inside != 0 && inside != 0xFF)
        for (int t = 0; t < 6; ++t) {
            const int k = __popc(tet_mask(t, inside));
            n += (k == 2) ? 2 : (k == 1 || k == 3) ? 1 : 0;
        }
    cnt[c] = n;
}

__global__ void vertex_kernel(Grid g, double level, double tclamp, const double *__restrict__ rho,
                              const uint8_t *__restrict__ flags, const int64_t *__restrict__ vbase,
                              double *__restrict__ verts) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.nn) return;
    const unsigned f = flags[p];
    if (!f) return;
    const int k = (int)(p % g.n[2]);
    const int64_t ij = p / g.n[2];
    const int j = (int)(ij % g.n[1]), i = (int)(ij / g.n[1]);
    const double fp = __dsub_rn(rho[p], level);
    const double xp[3] = {node_coord(g.lo[0], g.h, i), node_coord(g.lo[1], g.h, j), node_coord(g.lo[2], g.h, k)};
    int64_t v = vbase[p];
    for (int c = 1; c < 8; ++c) {
        const int dx = c >> 2, dy = (c >> 1) & 1, dz = c & 1;
        if (!(f >> dir_of(dx, dy, dz) & 1u)) continue;
        const int64_t q = p + (int64_t)dx * g.n[1] * g.n[2] + (int64_t)dy * g.n[2] + dz;
        const double fq = __dsub_rn(rho[q], level);
        const double t = fmin(fmax(__ddiv_rn(fp, __dsub_rn(fp, fq)), tclamp), 1.0 - tclamp);
        const double xq[3] = {node_coord(g.lo[0], g.h, i + dx), node_coord(g.lo[1], g.h, j + dy),
                              node_coord(g.lo[2], g.h, k + dz)};
        for (int a = 0; a < 3; ++a) verts[3 * v + a] = __dadd_rn(xp[a], __dmul_rn(t, __dsub_rn(xq[a], xp[a])));
        ++v;   // directions visited in ascending order: c = 1..7 is dir 0..6
    }
}

__global__ void triangle_kernel(Grid g, int64_t ncube, double level, const double *__restrict__ rho,
                                const uint8_t *__restrict__ flags, const int64_t *__restrict__ vbase,
                                const int64_t *__restrict__ tbase, int32_t *__restrict__ tris) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncube || tbase[c + 1] == tbase[c]) return;
    int64_t p0;
    unsigned inside;
    cube_of(g, c, p0, inside, rho, level);
    int64_t m = tbase[c];
    for (int t = 0; t < 6; ++t) {
        int8_t e[2][3][2];
        const int n = tet_triangles(tet_mask(t, inside), e);
        for (int s = 0; s < n; ++s, ++m)
            for (int x = 0; x < 3; ++x) {
                const int u = kTet[t][e[s][x][0]], w = kTet[t][e[s][x][1]];
                const int lower = __popc(u) < __popc(w) ? u : w, delta = u ^ w;
                const int64_t p = p0 + corner_offset(g, lower);
                const int d = dir_of(delta & 1, (delta >> 1) & 1, (delta >> 2) & 1);
                tris[3 * m + x] = (int32_t)(vbase[p] + __popc(flags[p] & ((1u << d) - 1u)));
            }
    }
}

// ------------------------------------------------------------------ components
// Lock-free union-find: links always point to smaller vertex numbers and the
// larger of two roots is hooked under the smaller, so every component ends
// with its smallest vertex as root.  Every loop is bounded; running out sets *err.
constexpr int kUfBudget = 1 << 20;

__device__ __forceinline__ int uf_load(const int32_t *par, int x) { return __ldcg(par + x); }

__device__ int uf_find(int32_t *par, int x, int &budget) {
    while (budget-- > 0) {
        const int p = uf_load(par, x);
        if (p == x) return x;
        const int gp = uf_load(par, p);
        if (gp != p) par[x] = gp;       // path halving: gp is an ancestor of x
        x = gp;
    }
    return -1;
}

__device__ bool uf_unite(int32_t *par, int u, int w, int &budget) {
    while (budget > 0) {
        int ru = uf_find(par, u, budget), rw = uf_find(par, w, budget);
        if (ru < 0 || rw < 0) return false;
        if (ru == rw) return true;
        if (ru < rw) { const int t = ru; ru = rw; rw = t; }
        if (atomicCAS(par + ru, ru, rw) == ru) return true;
        u = ru;
        w = rw;
        --budget;
    }
    return false;
}

__global__ void uf_init_kernel(int64_t nv, int32_t *__restrict__ par) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nv) par[v] = (int32_t)v;
}

__global__ void uf_unite_kernel(int64_t nt, const int32_t *__restrict__ tris, int32_t *par, int *err) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    int budget = kUfBudget;
    const int a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
    if (!uf_unite(par, a, b, budget) || !uf_unite(par, b, c, budget)) atomicExch(err, 1);
}

__global__ void uf_flatten_kernel(int64_t nv, int32_t *par, unsigned long long *ncomp, int *err) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv) return;
    int budget = kUfBudget;
    const int r = uf_find(par, (int)v, budget);
    if (r < 0) { atomicExch(err, 1); return; }
    if (r == v) atomicAdd(ncomp, 1ull);
    par[v] = r;
}

__global__ void keep_kernel(int64_t nv, int64_t nt, const int32_t *__restrict__ par, const int32_t *__restrict__ tris,
                            int32_t *__restrict__ vkeep, int32_t *__restrict__ tkeep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int32_t root = par[nv - 1];
    if (i < nv) vkeep[i] = par[i] == root;
    if (i < nt) tkeep[i] = par[tris[3 * i]] == root;
}

__global__ void compact_vertices_kernel(int64_t nv, const int32_t *__restrict__ vkeep, const int64_t *__restrict__ vnew,
                                        const double *__restrict__ vin, double *__restrict__ vout) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nv || !vkeep[v]) return;
    const int64_t o = vnew[v];
    vout[3 * o] = vin[3 * v];
    vout[3 * o + 1] = vin[3 * v + 1];
    vout[3 * o + 2] = vin[3 * v + 2];
}

__global__ void compact_triangles_kernel(int64_t nt, const int32_t *__restrict__ tkeep, const int64_t *__restrict__ tnew,
                                         const int64_t *__restrict__ vnew, const int32_t *__restrict__ tin,
                                         int32_t *__restrict__ tout) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt || !tkeep[t]) return;
    const int64_t o = tnew[t];
    for (int x = 0; x < 3; ++x) tout[3 * o + x] = (int32_t)vnew[tin[3 * t + x]];
}

// ------------------------------------------------------------------ smoothing
// Neighbours of every kept vertex: the far ends of its outgoing half-edges,
// sorted and made unique (a closed oriented surface lists each edge once per direction).
__global__ void degree_kernel(const int64_t *__restrict__ ntk, const int32_t *__restrict__ tris, int32_t *__restrict__ deg) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *ntk) return;
    for (int x = 0; x < 3; ++x) atomicAdd(deg + tris[3 * t + x], 1);
}

__global__ void halfedge_fill_kernel(const int64_t *__restrict__ ntk, const int32_t *__restrict__ tris,
                                     const int64_t *__restrict__ nstart, int32_t *__restrict__ cursor,
                                     int32_t *__restrict__ nbr) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= *ntk) return;
    for (int x = 0; x < 3; ++x) {
        const int a = tris[3 * t + x], b = tris[3 * t + (x + 1) % 3];
        nbr[nstart[a] + atomicAdd(cursor + a, 1)] = b;
    }
}

__global__ void sort_neighbours_kernel(const int64_t *__restrict__ nvk, const int64_t *__restrict__ nstart,
                                       int32_t *__restrict__ nbr, int32_t *__restrict__ udeg) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= *nvk) return;
    const int64_t s = nstart[v];
    const int n = (int)(nstart[v + 1] - s);
    int32_t *a = nbr + s;
    for (int i = 1; i < n; ++i) {
        const int32_t x = a[i];
        int j = i - 1;
        while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
        a[j + 1] = x;
    }
    int u = 0;
    for (int i = 0; i < n; ++i)
        if (u == 0 || a[i] != a[u - 1]) a[u++] = a[i];
    udeg[v] = u;
}

__global__ void smooth_kernel(const int64_t *__restrict__ nvk, const int64_t *__restrict__ nstart,
                              const int32_t *__restrict__ nbr, const int32_t *__restrict__ udeg, Cells C, Shape S,
                              const double *__restrict__ vin, double *__restrict__ vout) {
    const int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= *nvk) return;
    const int64_t s = nstart[v];
    const int n = udeg[v];
    double sum[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < n; ++i) {
        const int64_t w = nbr[s + i];
        for (int a = 0; a < 3; ++a) sum[a] = __dadd_rn(sum[a], vin[3 * w + a]);
    }
    double x[3];
    for (int a = 0; a < 3; ++a) {
        const double o = vin[3 * v + a];
        x[a] = n > 0 ? __dadd_rn(o, __dmul_rn(S.relax, __dsub_rn(__ddiv_rn(sum[a], (double)n), o))) : o;
    }
    PB_SURV_BUF(buf);
    for (int it = 0; it < S.newton_steps; ++it) {
        double rho, g[3];
        density_warp<true>(C, S, x[0], x[1], x[2], lane, buf, rho, g);
        const double g2 = __dadd_rn(__dadd_rn(__dmul_rn(g[0], g[0]), __dmul_rn(g[1], g[1])), __dmul_rn(g[2], g[2]));
        const double st = g2 > 1e-12 ? __ddiv_rn(__dsub_rn(rho, S.level), g2) : 0.0;
        double dv[3] = {__dmul_rn(st, g[0]), __dmul_rn(st, g[1]), __dmul_rn(st, g[2])};
        const double len = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dv[0], dv[0]), __dmul_rn(dv[1], dv[1])),
                                          __dmul_rn(dv[2], dv[2])));
        const double sc = fmin(1.0, __ddiv_rn(S.max_step, fmax(len, 1e-30)));
        for (int a = 0; a < 3; ++a) x[a] = __dsub_rn(x[a], __dmul_rn(dv[a], sc));
    }
    if (lane < 3) vout[3 * v + lane] = x[lane];
}

// Triangles of round r (0: unsmoothed) whose normal has a non-negative
// component along grad rho at the centroid, counted into folds[r].  A round
// is acceptable when it folds no more triangles than round 0.  Launch order
// R, 0, R - 1, ..., 1: round 0 is skipped when round R folds nothing (then
// R is taken and folds[0] stays 0), a round r < R once a later round is
// acceptable.
__global__ void fold_kernel(const int64_t *__restrict__ ntk, const int32_t *__restrict__ tris,
                            const double *__restrict__ v, Cells C, Shape S, unsigned long long *__restrict__ folds,
                            int r, int R) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= *ntk) return;
    if (r == 0 && folds[R] == 0) return;
    if (r > 0)
        for (int q = r + 1; q <= R; ++q)
            if (folds[q] <= folds[0]) return;
    const double *A = v + 3 * (int64_t)tris[3 * t], *B = v + 3 * (int64_t)tris[3 * t + 1],
                 *Cc = v + 3 * (int64_t)tris[3 * t + 2];
    const double e1[3] = {__dsub_rn(B[0], A[0]), __dsub_rn(B[1], A[1]), __dsub_rn(B[2], A[2])};
    const double e2[3] = {__dsub_rn(Cc[0], A[0]), __dsub_rn(Cc[1], A[1]), __dsub_rn(Cc[2], A[2])};
    const double n[3] = {__dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1])),
                         __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2])),
                         __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]))};
    double c[3];
    for (int a = 0; a < 3; ++a) c[a] = __ddiv_rn(__dadd_rn(__dadd_rn(A[a], B[a]), Cc[a]), 3.0);
    PB_SURV_BUF(buf);
    double rho, g[3];
    density_warp<true>(C, S, c[0], c[1], c[2], lane, buf, rho, g);
    const double dot = __dadd_rn(__dadd_rn(__dmul_rn(n[0], g[0]), __dmul_rn(n[1], g[1])), __dmul_rn(n[2], g[2]));
    if (lane == 0 && dot >= 0.0) atomicAdd(folds + r, 1ull);
}

__device__ __forceinline__ int rounds_used(const unsigned long long *folds, int R) {
    for (int r = R; r >= 1; --r)
        if (folds[r] <= folds[0]) return r;
    return 0;
}

__global__ void select_kernel(const int64_t *__restrict__ nvk, const unsigned long long *__restrict__ folds, int R,
                              int64_t stride, const double *__restrict__ snaps, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 3 * *nvk) return;
    out[i] = snaps[rounds_used(folds, R) * stride + i];
}

__global__ void totals_kernel(const int64_t *a, const int64_t *b, int64_t *out) {
    out[0] = *a;
    out[1] = *b;
}

__global__ void info_kernel(const int64_t *nvk, const int64_t *ntk, const unsigned long long *ncomp, const int *err,
                            const unsigned long long *folds, int R, int64_t *out) {
    out[0] = *nvk;
    out[1] = *ntk;
    out[2] = (int64_t)*ncomp;
    out[3] = *err;
    out[4] = rounds_used(folds, R);
}

}  // namespace

void gaussian_surface(const double *xyz, const double *radius, int64_t na, const SurfGenParams &p, cudaStream_t s,
                      SurfIn &out) {
    if (na < 1 || !xyz || !radius) fail(PB_EINVAL, "no atoms");
    if (!(p.spacing > 0.0) || !(p.beta > 0.0) || !(p.cutoff > 0.0) || !(p.level > 0.0) || !(p.margin >= 0.0) ||
        !(p.tclamp >= 0.0 && p.tclamp < 0.5) || !(p.relax >= 0.0 && p.relax <= 1.0) || !(p.max_step > 0.0) ||
        p.smooth_iters < 0 || p.smooth_iters > 64 || p.newton_steps < 0 || p.newton_steps > 64)
        fail(PB_EINVAL, "bad surface parameters");
    double amin[3] = {INFINITY, INFINITY, INFINITY}, amax[3] = {-INFINITY, -INFINITY, -INFINITY}, rmax = 0.0;
    for (int64_t a = 0; a < na; ++a) {
        for (int d = 0; d < 3; ++d) {
            const double x = xyz[3 * a + d];
            if (!std::isfinite(x)) fail(PB_EINVAL, "non-finite atom position");
            amin[d] = std::min(amin[d], x);
            amax[d] = std::max(amax[d], x);
        }
        const double r = radius[a] + p.radius_offset;
        if (!(r > 0.0) || !std::isfinite(r)) fail(PB_EINVAL, "atom radius plus offset must be positive");
        rmax = std::max(rmax, r);
    }
    Grid g;
    g.h = p.spacing;
    g.nn = 1;
    for (int d = 0; d < 3; ++d) {
        g.lo[d] = amin[d] - rmax - p.margin;
        const double hi = amax[d] + rmax + p.margin;
        const double n = std::ceil((hi - g.lo[d]) / p.spacing) + 1.0;
        if (n > 4096.0) fail(PB_EINVAL, "surface grid too large (more than 4096 nodes along an axis)");
        g.n[d] = (int)n;
        g.nn *= g.n[d];
    }
    if (g.nn > ((int64_t)1 << 31) - 1) fail(PB_EINVAL, "surface grid too large");
    const int64_t ncube = (int64_t)(g.n[0] - 1) * (g.n[1] - 1) * (g.n[2] - 1);
    // atom cells: edge >= the largest cutoff radius, at most 256 cells per axis
    Cells C;
    double ext = 0.0;
    for (int d = 0; d < 3; ++d) ext = std::max(ext, amax[d] - amin[d]);
    C.cs = std::max(p.cutoff * rmax * (1.0 + 1e-12), ext / 255.0);
    int64_t ncell = 1;
    for (int d = 0; d < 3; ++d) {
        C.c0[d] = amin[d];
        C.nc[d] = (int)std::floor((amax[d] - amin[d]) / C.cs) + 1;
        ncell *= C.nc[d];
    }
    Shape S{p.beta, p.cutoff, p.level, p.tclamp, p.relax, p.max_step, p.newton_steps};
    // largest |coordinate - c0| of any atom or query point (grid nodes, vertices, centroids), and
    // the FP32 rounding bound of such a coordinate (two roundings)
    double reach = 0.0;
    for (int d = 0; d < 3; ++d)
        reach = std::max(reach, std::fabs(g.lo[d] - C.c0[d]) + g.h * (g.n[d] - 1) + p.spacing);
    const double ecoord = (reach + 1.0) * std::ldexp(1.0, -22);

    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PB_CUDA_TRY(cudaEventCreate(&e0));
    PB_CUDA_TRY(cudaEventCreate(&e1));
    struct EvGuard {
        cudaEvent_t a, b;
        ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evg{e0, e1};
    PB_CUDA_TRY(cudaEventRecord(e0, s));

    // 1. atoms by cell, density at the nodes
    TmpBuf<double> axyz(3 * na, s), arad(na, s);
    PB_CUDA_TRY(cudaMemcpyAsync(axyz.p, xyz, 3 * na * sizeof(double), cudaMemcpyHostToDevice, s));
    PB_CUDA_TRY(cudaMemcpyAsync(arad.p, radius, na * sizeof(double), cudaMemcpyHostToDevice, s));
    TmpBuf<dvec4> packed(na, s), sorted(na, s);
    TmpBuf<float4> sorted32(na, s);
    TmpBuf<double> rc2(na, s);
    TmpBuf<uint64_t> key(na, s);
    TmpBuf<int32_t> idx(na, s), ccount(ncell, s);
    TmpBuf<int64_t> cstart(ncell + 1, s);
    pack_atoms_kernel<<<div_up(na, 256), 256, 0, s>>>(na, axyz.p, arad.p, p.radius_offset, C, packed.p, key.p, idx.p);
    PB_LAUNCH_CHECK();
    sort_key_index(key.p, idx.p, na, s);
    PB_CUDA_TRY(cudaMemsetAsync(ccount.p, 0, ncell * sizeof(int32_t), s));
    cell_count_kernel<<<div_up(na, 256), 256, 0, s>>>(na, key.p, ccount.p);
    PB_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(ccount.p, cstart.p, ncell, s);
    gather_atoms_kernel<<<div_up(na, 256), 256, 0, s>>>(na, idx.p, packed.p, C, p.cutoff, ecoord, sorted.p, rc2.p,
                                                         sorted32.p);
    PB_LAUNCH_CHECK();
    C.atoms = sorted.p;
    C.rc2 = rc2.p;
    C.atoms32 = sorted32.p;
    C.start = cstart.p;
    TmpBuf<double> rho(g.nn, s);
    density_kernel<<<div_up(g.nn * 32, 256), 256, 0, s>>>(g, C, S, rho.p);
    PB_LAUNCH_CHECK();

    // 2-3. crossings, vertices, triangles
    TmpBuf<uint8_t> flags(g.nn, s);
    TmpBuf<int32_t> vcnt(g.nn, s), tcnt(ncube, s);
    TmpBuf<int64_t> vbase(g.nn + 1, s), tbase(ncube + 1, s), tot(2, s);
    crossing_kernel<<<div_up(g.nn, 256), 256, 0, s>>>(g, p.level, rho.p, flags.p, vcnt.p);
    PB_LAUNCH_CHECK();
    cube_count_kernel<<<div_up(ncube, 256), 256, 0, s>>>(g, ncube, p.level, rho.p, tcnt.p);
    PB_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(vcnt.p, vbase.p, g.nn, s);
    exclusive_scan_i32_to_i64(tcnt.p, tbase.p, ncube, s);
    totals_kernel<<<1, 1, 0, s>>>(vbase.p + g.nn, tbase.p + ncube, tot.p);
    PB_LAUNCH_CHECK();
    PinnedBuf<int64_t> hs;
    hs.alloc(8);
    PB_CUDA_TRY(cudaMemcpyAsync(hs.p, tot.p, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t nv = hs.p[0], nt = hs.p[1];
    if (nt < 1) fail(PB_EINVAL, "the density has no level-set crossing on the surface grid");
    if (3 * nt > ((int64_t)1 << 31) - 1 || nv > ((int64_t)1 << 31) - 1) fail(PB_EINVAL, "surface too large");
    TmpBuf<double> vraw(3 * nv, s);
    TmpBuf<int32_t> traw(3 * nt, s);
    vertex_kernel<<<div_up(g.nn, 256), 256, 0, s>>>(g, p.level, p.tclamp, rho.p, flags.p, vbase.p, vraw.p);
    PB_LAUNCH_CHECK();
    triangle_kernel<<<div_up(ncube, 256), 256, 0, s>>>(g, ncube, p.level, rho.p, flags.p, vbase.p, tbase.p, traw.p);
    PB_LAUNCH_CHECK();

    // 4. outer component
    TmpBuf<int32_t> par(nv, s), vkeep(nv, s), tkeep(nt, s);
    TmpBuf<int64_t> vnew(nv + 1, s), tnew(nt + 1, s);
    TmpBuf<unsigned long long> counters(2 + 65, s);     // components, unused, folds[0..64]
    TmpBuf<int> err(1, s);
    PB_CUDA_TRY(cudaMemsetAsync(counters.p, 0, (2 + 65) * sizeof(unsigned long long), s));
    PB_CUDA_TRY(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    uf_init_kernel<<<div_up(nv, 256), 256, 0, s>>>(nv, par.p);
    PB_LAUNCH_CHECK();
    uf_unite_kernel<<<div_up(nt, 256), 256, 0, s>>>(nt, traw.p, par.p, err.p);
    PB_LAUNCH_CHECK();
    uf_flatten_kernel<<<div_up(nv, 256), 256, 0, s>>>(nv, par.p, counters.p, err.p);
    PB_LAUNCH_CHECK();
    keep_kernel<<<div_up(std::max(nv, nt), 256), 256, 0, s>>>(nv, nt, par.p, traw.p, vkeep.p, tkeep.p);
    PB_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(vkeep.p, vnew.p, nv, s);
    exclusive_scan_i32_to_i64(tkeep.p, tnew.p, nt, s);
    const int R = p.smooth_iters;
    const int64_t stride = 3 * nv;
    TmpBuf<double> snaps((R + 1) * stride, s);
    out.t.alloc(3 * nt);
    out.v.alloc(3 * nv);
    compact_vertices_kernel<<<div_up(nv, 256), 256, 0, s>>>(nv, vkeep.p, vnew.p, vraw.p, snaps.p);
    PB_LAUNCH_CHECK();
    compact_triangles_kernel<<<div_up(nt, 256), 256, 0, s>>>(nt, tkeep.p, tnew.p, vnew.p, traw.p, out.t.p);
    PB_LAUNCH_CHECK();
    const int64_t *nvk = vnew.p + nv, *ntk = tnew.p + nt;
    unsigned long long *folds = counters.p + 2;

    // 5. smoothing rounds, each checked for folds
    if (R > 0) {
        TmpBuf<int32_t> deg(nv, s), cursor(nv, s), udeg(nv, s), nbr(3 * nt, s);
        TmpBuf<int64_t> nstart(nv + 1, s);
        PB_CUDA_TRY(cudaMemsetAsync(deg.p, 0, nv * sizeof(int32_t), s));
        PB_CUDA_TRY(cudaMemsetAsync(cursor.p, 0, nv * sizeof(int32_t), s));
        degree_kernel<<<div_up(nt, 256), 256, 0, s>>>(ntk, out.t.p, deg.p);
        PB_LAUNCH_CHECK();
        exclusive_scan_i32_to_i64(deg.p, nstart.p, nv, s);
        halfedge_fill_kernel<<<div_up(nt, 256), 256, 0, s>>>(ntk, out.t.p, nstart.p, cursor.p, nbr.p);
        PB_LAUNCH_CHECK();
        sort_neighbours_kernel<<<div_up(nv, 256), 256, 0, s>>>(nvk, nstart.p, nbr.p, udeg.p);
        PB_LAUNCH_CHECK();
        for (int r = 1; r <= R; ++r) {
            smooth_kernel<<<div_up(nv * 32, 256), 256, 0, s>>>(nvk, nstart.p, nbr.p, udeg.p, C, S,
                                                              snaps.p + (r - 1) * stride, snaps.p + r * stride);
            PB_LAUNCH_CHECK();
        }
        for (int k = 0; k <= R; ++k) {
            const int r = k == 0 ? R : k == 1 ? 0 : R + 1 - k;     // R, 0, R - 1, ..., 1
            fold_kernel<<<div_up(nt * 32, 256), 256, 0, s>>>(ntk, out.t.p, snaps.p + r * stride, C, S, folds, r, R);
            PB_LAUNCH_CHECK();
        }
    }
    select_kernel<<<div_up(3 * nv, 256), 256, 0, s>>>(nvk, folds, R, stride, snaps.p, out.v.p);
    PB_LAUNCH_CHECK();
    TmpBuf<int64_t> info(5, s);
    info_kernel<<<1, 1, 0, s>>>(nvk, ntk, counters.p, err.p, folds, R, info.p);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaMemcpyAsync(hs.p, info.p, 5 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaEventRecord(e1, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    if (hs.p[3]) fail(PB_ETIMEOUT, "surface component labelling ran out of its step budget");
    out.nv = hs.p[0];
    out.nt = hs.p[1];
    out.v.n = 3 * out.nv;
    out.t.n = 3 * out.nt;
    out.generated = true;
    for (int d = 0; d < 3; ++d) out.gen.shape[d] = g.n[d];
    out.gen.components = hs.p[2];
    out.gen.rounds = (int)hs.p[4];
    out.gen.raw_nv = nv;
    out.gen.raw_nt = nt;
    PB_CUDA_TRY(cudaEventElapsedTime(&out.gen.ms, e0, e1));
}

}  // namespace pb
