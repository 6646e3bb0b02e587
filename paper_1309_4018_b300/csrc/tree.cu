// Octree construction and per-target interaction lists (Sec. 2.3, Eq. MAC).
//
// Integer decisions (Morton keys, splits, MAC, near-singular test) use FP64
// arithmetic written with explicit round-to-nearest intrinsics, so no multiply
// is fused with an add and the results are reproducible bit for bit:
//   root cube   centre = (lo + hi) / 2, side = max extent * (1 + 2^-20)
//   key         q_a = min(2^21 - 1, floor((p_a - corner_a) * (2^21 / side))),
//               bits interleaved with x the most significant of each triple
//   split       a box with >= ncrit sources below level 21 splits into its
//               non-empty octants; nodes numbered breadth first
//   MAC         accept when (side_l^2 * 0.75) < theta^2 ((dx^2 + dy^2) + dz^2),
//               box centre corner + (i + 0.5) side_l (Eq. MAC, r_b the half diagonal)
//   near        |x_i - c_j|^2 < (thres L_j)^2, L_j = sqrt(2 A_j), for panels whose
//               Gauss points all lie in the target's direct-sum leaves
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <optional>

#include <cooperative_groups.h>

#include "model.cuh"
#include "tree.cuh"

namespace cg = cooperative_groups;

namespace pb {

namespace {

// Per-block min/max of a strided slice (min and max are exact: any order gives the same box).
__global__ void bbox_blocks_kernel(const double *__restrict__ p, int64_t n, double *__restrict__ part) {
    __shared__ double sm[6][8];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int a = 0; a < 3; ++a) {
            const double v = p[3 * i + a];
            lo[a] = fmin(lo[a], v);
            hi[a] = fmax(hi[a], v);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) { sm[a][warp] = lo[a]; sm[3 + a][warp] = hi[a]; }
    __syncthreads();
    if (threadIdx.x == 0)
        for (int a = 0; a < 3; ++a) {
            double l = sm[a][0], h = sm[3 + a][0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { l = fmin(l, sm[a][w]); h = fmax(h, sm[3 + a][w]); }
            part[6 * blockIdx.x + a] = l;
            part[6 * blockIdx.x + 3 + a] = h;
        }
}

// Root cube from the block boxes: cube = (corner x, y, z, side), with
//   centre = (lo + hi) / 2, side = max extent * (1 + 2^-20) (1 if that is 0 or
//   not finite), corner = centre - side / 2,
// each operation rounded on its own (no fused multiply-add).
__global__ void cube_final_kernel(const double *__restrict__ part, int nb, double *__restrict__ cube) {
    // one warp: lanes take the block boxes in turn, then a butterfly (min and max are exact)
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = threadIdx.x; b < nb; b += 32)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], part[6 * b + a]);
            hi[a] = fmax(hi[a], part[6 * b + 3 + a]);
        }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    if (threadIdx.x != 0) return;
    double centre[3], ext[3];
    for (int a = 0; a < 3; ++a) {
        centre[a] = __dmul_rn(__dadd_rn(lo[a], hi[a]), 0.5);
        ext[a] = __dsub_rn(hi[a], lo[a]);
    }
    const double m01 = ext[0] < ext[1] ? ext[1] : ext[0];
    const double m = m01 < ext[2] ? ext[2] : m01;
    double side = __dmul_rn(m, 1.0 + 0x1p-20);
    if (side == 0.0 || !isfinite(side)) side = 1.0;
    const double half = __dmul_rn(side, 0.5);
    for (int a = 0; a < 3; ++a) cube[a] = __dsub_rn(centre[a], half);
    cube[3] = side;
}

// The tree origin (the root cube's centre) as the host forms it: corner + 0.5 side.
__device__ __forceinline__ double cube_origin(const double *cube, int a) {
    return __dadd_rn(cube[a], __dmul_rn(0.5, cube[3]));
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

__global__ void morton_kernel(const double *__restrict__ p, int64_t n, const double *__restrict__ cube,
                              uint64_t *__restrict__ keys, int32_t *__restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c[3] = {cube[0], cube[1], cube[2]};
    const double scale = __ddiv_rn(2097152.0, cube[3]);
    uint64_t q[3];
    for (int a = 0; a < 3; ++a) {
        double f = floor(__dmul_rn(__dsub_rn(p[3 * i + a], c[a]), scale));
        f = fmin(fmax(f, 0.0), 2097151.0);
        q[a] = (uint64_t)f;
    }
    keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    idx[i] = (int32_t)i;
}

// The whole octree below the root in one cooperative launch, level by level
// (a host round trip per level cost more than the levels themselves), with a
// grid-wide barrier between the phases of a level:
//   A  per (node, octant o = 1..8) of a node with >= ncrit points above the
//      deepest level: the first of the node's sorted keys whose octant digit
//      is >= o (binary search), into bnd[9 t + o];
//   B  (block 0) child counts (non-empty octants) and their exclusive scan in
//      node order: the children are numbered breadth first, octants in order
//      within a node;
//   C  per node: the children written.
// info: [0] nodes, [1] levels, [2] 1 if maxn nodes were not enough, [3 + l]
// first node of level l (levels + 1 entries).  Writes beyond maxn are skipped.
constexpr int kLevelThreads = 256;

__global__ void __launch_bounds__(kLevelThreads) build_levels_kernel(
    int64_t n, int ncrit, int maxn, const uint64_t *__restrict__ keys, int64_t *__restrict__ start,
    int64_t *__restrict__ count, int32_t *__restrict__ level, int32_t *__restrict__ first_child,
    int32_t *__restrict__ nchild, int32_t *__restrict__ parent, int64_t *__restrict__ ijk, int32_t *__restrict__ bnd,
    int32_t *__restrict__ cscan, int32_t *__restrict__ info) {
    cg::grid_group grid = cg::this_grid();
    __shared__ int wsum[kLevelThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t gtid = (int64_t)blockIdx.x * kLevelThreads + tid, gsize = (int64_t)gridDim.x * kLevelThreads;
    if (gtid == 0) {
        start[0] = 0; count[0] = n; level[0] = 0; first_child[0] = -1; nchild[0] = 0; parent[0] = -1;
        ijk[0] = 0; ijk[1] = 0; ijk[2] = 0;
        info[3] = 0;
        info[2] = 0;
    }
    grid.sync();
    int lb = 0, le = 1, lvl = 0;
    while (true) {
        const int nb = le - lb;
        const int sh = 3 * (kMaxLevel - 1 - lvl);
        // A: octant bounds of the nodes that split
        for (int64_t g = gtid; g < (int64_t)nb * 8; g += gsize) {
            const int t = (int)(g >> 3), o = (int)(g & 7) + 1;
            const int64_t c = count[lb + t];
            if (!(c >= ncrit && lvl < kMaxLevel)) continue;
            const int64_t s0 = start[lb + t];
            int64_t lo = 0, hi = c;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int d = (int)((keys[s0 + mid] >> sh) & 7ull);
                if (d < o) lo = mid + 1; else hi = mid;
            }
            bnd[9 * t + o] = (int32_t)lo;
            if (o == 1) bnd[9 * t] = 0;
        }
        grid.sync();
        // B: child counts and their scan (block 0)
        if (blockIdx.x == 0) {
            if (tid == 0) info[3 + lvl + 1] = le;
            int carry = 0;
            for (int c0 = 0; c0 < nb; c0 += kLevelThreads) {
                const int t = c0 + tid;
                int nc = 0;
                if (t < nb) {
                    const int64_t c = count[lb + t];
                    if (c >= ncrit && lvl < kMaxLevel)
                        for (int o = 0; o < 8; ++o) nc += bnd[9 * t + o + 1] > bnd[9 * t + o];
                    nchild[lb + t] = nc;
                }
                int incl = nc;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) wsum[warp] = incl;
                __syncthreads();
                int before = 0, total = 0;
                for (int w = 0; w < kLevelThreads / 32; ++w) {
                    if (w < warp) before += wsum[w];
                    total += wsum[w];
                }
                if (t < nb) cscan[t] = carry + before + incl - nc;
                carry += total;
                __syncthreads();
            }
            if (tid == 0) cscan[nb] = carry;
        }
        grid.sync();
        // C: the children
        const int nnew = cscan[nb];
        const bool over = (int64_t)le + nnew > maxn;
        for (int64_t t = gtid; t < nb; t += gsize) {
            const int b = lb + (int)t;
            const int nc = nchild[b];
            if (nc == 0) {
                first_child[b] = -1;
                continue;
            }
            int ch = le + cscan[t];
            first_child[b] = ch;
            const int64_t s0 = start[b];
            for (int o = 0; o < 8; ++o) {
                const int64_t cs = bnd[9 * t + o], ce = bnd[9 * t + o + 1];
                if (ce <= cs) continue;
                if (ch < maxn) {
                    start[ch] = s0 + cs;
                    count[ch] = ce - cs;
                    level[ch] = lvl + 1;
                    parent[ch] = b;
                    nchild[ch] = 0;
                    first_child[ch] = -1;
                    ijk[3 * ch + 0] = 2 * ijk[3 * b + 0] + ((o >> 2) & 1);
                    ijk[3 * ch + 1] = 2 * ijk[3 * b + 1] + ((o >> 1) & 1);
                    ijk[3 * ch + 2] = 2 * ijk[3 * b + 2] + (o & 1);
                }
                ++ch;
            }
        }
        grid.sync();
        if (nnew == 0 || over) {
            if (gtid == 0) {
                info[0] = le;
                info[1] = lvl + 1;
                info[2] = over ? 1 : 0;
            }
            return;
        }
        lb = le;
        le += nnew;
        ++lvl;
    }
}

__global__ void node_geom_kernel(const int32_t *__restrict__ info, const int32_t *__restrict__ level,
                                 const int64_t *__restrict__ ijk, const double *__restrict__ cube,
                                 double *__restrict__ centre, double *__restrict__ rb2) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= info[0]) return;
    const double sl = ldexp(cube[3], -level[b]);
    const double c[3] = {cube[0], cube[1], cube[2]};
    for (int a = 0; a < 3; ++a)
        centre[3 * b + a] = __dadd_rn(c[a], __dmul_rn(__dadd_rn((double)ijk[3 * b + a], 0.5), sl));
    rb2[b] = __dmul_rn(__dmul_rn(sl, sl), 0.75);
}

// Per node: (parent, the parent's first child, the parent's child count, 0);
// (-1, 0, 0, 0) at the root.  One record per level of the upward climb.
__global__ void link_kernel(const int32_t *__restrict__ info, const int32_t *__restrict__ parent,
                            const int32_t *__restrict__ first_child, const int32_t *__restrict__ nchild,
                            int4 *__restrict__ link) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= info[0]) return;
    const int p = parent[i];
    link[i] = p >= 0 ? make_int4(p, first_child[p], nchild[p], 0) : make_int4(-1, 0, 0, 0);
}

__global__ void centre32_kernel(const int32_t *__restrict__ info, const double *__restrict__ centre,
                                const double *__restrict__ rb2, const double *__restrict__ cube,
                                float4 *__restrict__ cen32) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= info[0]) return;
    const double ox = cube_origin(cube, 0), oy = cube_origin(cube, 1), oz = cube_origin(cube, 2);
    cen32[b] = make_float4((float)(centre[3 * b] - ox), (float)(centre[3 * b + 1] - oy), (float)(centre[3 * b + 2] - oz),
                           (float)rb2[b]);
}

__global__ void parent_offset_kernel(const int32_t *__restrict__ info, const int32_t *__restrict__ parent,
                                     const double *__restrict__ centre, float4 *__restrict__ pofs32) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= info[0]) return;
    const int p = parent[b];
    pofs32[b] = p < 0 ? make_float4(0.f, 0.f, 0.f, 0.f)
                      : make_float4((float)(centre[3 * b] - centre[3 * p]), (float)(centre[3 * b + 1] - centre[3 * p + 1]),
                                    (float)(centre[3 * b + 2] - centre[3 * p + 2]), 0.f);
}

__global__ void leaf_flag_kernel(const int32_t *__restrict__ info, const int32_t *__restrict__ nchild,
                                 const int64_t *__restrict__ start, int32_t *__restrict__ head /*npts*/) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= info[0]) return;
    if (nchild[b] == 0) head[start[b]] = 1;
}

__global__ void leaf_index_kernel(const int32_t *__restrict__ info, const int32_t *__restrict__ nchild,
                                  const int64_t *__restrict__ start, const int64_t *__restrict__ hscan,
                                  int32_t *__restrict__ node_leaf, int32_t *__restrict__ leaf_node) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= info[0]) return;
    if (nchild[b] != 0) { node_leaf[b] = -1; return; }
    const int li = (int)hscan[start[b]];
    node_leaf[b] = li;
    leaf_node[li] = b;
}

// The leaf of sorted point q is the number of leaf starts at or before q, less one.
__global__ void point_leaf_kernel(int64_t n, const int64_t *__restrict__ hscan, const int32_t *__restrict__ perm,
                                  int32_t *__restrict__ point_leaf) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) point_leaf[perm[q]] = (int32_t)(hscan[q + 1] - 1);
}

__global__ void gather_sources_kernel(int64_t n, int K, const int32_t *__restrict__ perm, const double *__restrict__ gy,
                                      const double *__restrict__ gwa, const double *__restrict__ cube,
                                      double *__restrict__ ys, double *__restrict__ was, int32_t *__restrict__ pids,
                                      float4 *__restrict__ pos32) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const double ox = cube_origin(cube, 0), oy = cube_origin(cube, 1), oz = cube_origin(cube, 2);
    const int p = perm[q];
    const double x = gy[3 * p], y = gy[3 * p + 1], z = gy[3 * p + 2];
    const double w = gwa ? gwa[p] : 1.0;
    ys[3 * q] = x; ys[3 * q + 1] = y; ys[3 * q + 2] = z;
    was[q] = w;
    pids[q] = p / K;
    pos32[q] = make_float4((float)(x - ox), (float)(y - oy), (float)(z - oz), (float)w);
}

__global__ void gather_targets_kernel(int64_t n, const int32_t *__restrict__ order, const double *__restrict__ x,
                                      double *__restrict__ xs, int32_t *__restrict__ selfp, int32_t *__restrict__ rank,
                                      int self_div) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = order[q];
    rank[i] = (int32_t)q;
    xs[3 * q] = x[3 * i]; xs[3 * q + 1] = x[3 * i + 1]; xs[3 * q + 2] = x[3 * i + 2];
    selfp[q] = self_div > 0 ? i / self_div : -1;
}

// ---------------------------------------------------------------- traversal (Eq. MAC)
constexpr int kStack = 192;

// The MAC decision is the exact FP64 test below.  An FP32 estimate decides
// first when it is clearly on one side: with coordinates relative to the tree
// origin, |f32 - f| <= 8 eps32 R theta / r_b * (theta^2 d^2 + r_b^2) for
// f = theta^2 d^2 - r_b^2 and R the largest coordinate, so for theta <= 1 and
// r_b > R / 1024 a margin of 1e-3 (theta^2 d^2 + r_b^2) can never flip it.
template <bool FILL>
__global__ void traverse_kernel(int64_t ntg, const double *__restrict__ xs, const double *__restrict__ centre,
                                const double *__restrict__ rb2, const float4 *__restrict__ cen32,
                                const int32_t *__restrict__ first_child, const int32_t *__restrict__ nchild,
                                double theta2, int direct, double ox, double oy, double oz,
                                int32_t *__restrict__ m2p_cnt, int32_t *__restrict__ p2p_cnt,
                                const int64_t *__restrict__ m2p_ptr, const int64_t *__restrict__ p2p_ptr,
                                int32_t *__restrict__ m2p_node, int32_t *__restrict__ p2p_node,
                                unsigned long long *__restrict__ err, int nsplit) {
    // nsplit > 1: thread (i, c) traverses only the subtree of the root's child c
    // (the root itself, when accepted or a leaf, belongs to c = 0); counts and
    // offsets are per (i, c), and a target's list is their concatenation in c
    // order, which is its depth-first pre-order.
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid >= ntg * nsplit) return;
    const int64_t i = tid / nsplit;
    const int csub = nsplit > 1 ? (int)(tid % nsplit) : -1;
    const double x = xs[3 * i], y = xs[3 * i + 1], z = xs[3 * i + 2];
    const float fx = (float)(x - ox), fy = (float)(y - oy), fz = (float)(z - oz);
    const float th2f = (float)theta2;
    const bool pref = theta2 <= 1.0;
    const float tmax = fmaxf(fabsf(fx), fmaxf(fabsf(fy), fabsf(fz)));
    int stack[kStack];
    int sp = 0;
    stack[sp++] = 0;
    int nm = 0, np = 0;
    int64_t mo = FILL ? m2p_ptr[tid] : 0, po = FILL ? p2p_ptr[tid] : 0;
    while (sp > 0) {
        const int b = stack[--sp];
        bool accept = false;
        if (!direct) {
            int dec = -1;
            if (pref) {
                const float4 c = cen32[b];
                const float R = fmaxf(tmax, fmaxf(fabsf(c.x), fmaxf(fabsf(c.y), fabsf(c.z))));
                if (c.w > R * R * 9.5367431640625e-7f) {   // r_b > R / 1024
                    const float dx = fx - c.x, dy = fy - c.y, dz = fz - c.z;
                    const float rhs = th2f * (dx * dx + dy * dy + dz * dz);
                    const float marg = 1e-3f * (rhs + c.w);
                    if (rhs - c.w > marg) dec = 1;
                    else if (c.w - rhs > marg) dec = 0;
                }
            }
            if (dec < 0) {
                const double dx = __dsub_rn(x, centre[3 * b]);
                const double dy = __dsub_rn(y, centre[3 * b + 1]);
                const double dz = __dsub_rn(z, centre[3 * b + 2]);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                accept = rb2[b] < __dmul_rn(theta2, d2);
            } else {
                accept = dec == 1;
            }
        }
        const bool mine = b != 0 || csub <= 0;   // the root's own entry goes to c = 0
        if (accept) {
            if (mine) {
                if (FILL) m2p_node[mo + nm] = b;
                ++nm;
            }
        } else if (nchild[b] == 0) {
            if (mine) {
                if (FILL) p2p_node[po + np] = b;
                ++np;
            }
        } else if (b == 0 && csub >= 0) {
            if (csub < nchild[0]) stack[sp++] = first_child[0] + csub;
        } else {
            const int fc = first_child[b], nc = nchild[b];
            // cannot happen below 22 levels (at most 7 pending siblings per level);
            // counting and filling stop at the same node, so the lists stay consistent
            if (sp + nc > kStack) { atomicExch(err, 1ull); break; }
            for (int c = fc + nc - 1; c >= fc; --c) stack[sp++] = c;
        }
    }
    if (!FILL) { m2p_cnt[tid] = nm; p2p_cnt[tid] = np; }
}

// ptr[i] = off[i * nsplit], i = 0 .. m (per-target offsets from per-(target, subtree) ones).
__global__ void take_every_kernel(int64_t m, int nsplit, const int64_t *__restrict__ off, int64_t *__restrict__ ptr) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= m) ptr[i] = off[i * nsplit];
}

// ---------------------------------------------------------------- entry-major grouping
// key(e) = leaf index of a P2P entry (remap = node_leaf) or node id of an M2P entry.
// owner[e] = the target whose list holds entry e (one warp per target).
__global__ void owner_kernel(int64_t m, const int64_t *__restrict__ ptr, int32_t *__restrict__ owner) {
    const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= m) return;
    const int lane = threadIdx.x & 31;
    for (int64_t e = ptr[t] + lane; e < ptr[t + 1]; e += 32) owner[e] = (int32_t)t;
}

// Lanes holding the same key (neighbouring Morton-sorted targets share most
// boxes) add once per group: one atomic per distinct key per warp.
__global__ void inv_count_kernel(int64_t nent, const int32_t *__restrict__ ent, const int32_t *__restrict__ remap,
                                 int32_t *__restrict__ cnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = e < nent;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const int key = remap ? remap[ent[e]] : ent[e];
    const unsigned grp = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    if (lane == __ffs(grp) - 1) atomicAdd(&cnt[key], __popc(grp));
}

// The order of the pairs inside one key's group does not matter: every pair
// writes its own partial record, and the gather reads them back in list
// order.  by_entry: the record of grouped position p goes to its list entry
// (map[p] = entry; the gather then reads each target's records contiguously);
// otherwise it stays at p and map[entry] = p tells the gather where.
__global__ void inv_fill_kernel(int64_t nent, const int32_t *__restrict__ owner, const int32_t *__restrict__ ent,
                                const int32_t *__restrict__ remap, const int64_t *__restrict__ off,
                                int32_t *__restrict__ cursor, int by_entry, int32_t *__restrict__ inv,
                                int32_t *__restrict__ map) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = e < nent;
    const unsigned act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const int key = remap ? remap[ent[e]] : ent[e];
    const unsigned grp = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&cursor[key], __popc(grp));
    base = __shfl_sync(grp, base, leader);
    const int64_t p = off[key] + base + __popc(grp & ((1u << lane) - 1u));
    inv[p] = owner[e];
    if (by_entry) map[p] = (int32_t)e;
    else map[e] = (int32_t)p;
}

// The same grouping with per-block histograms in shared memory (few keys):
// every block counts its contiguous chunk of entries by key with shared
// atomics, a per-key pass turns the block counts into each block's starting
// offset, and every block then places its entries from those offsets.  The
// global atomics of the kernels above, up to one per entry on a few thousand
// popular keys, become shared ones.
constexpr int kHistKeys = 12000;   // keys per shared-memory histogram (48 KB)

__global__ void hist_count_kernel(int64_t nent, int64_t chunk, const int32_t *__restrict__ ent,
                                  const int32_t *__restrict__ remap, int nkeys, int32_t *__restrict__ hb) {
    extern __shared__ int32_t hist[];
    for (int k = threadIdx.x; k < nkeys; k += blockDim.x) hist[k] = 0;
    __syncthreads();
    const int64_t e0 = (int64_t)blockIdx.x * chunk, e1 = min(nent, e0 + chunk);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int key = remap ? remap[ent[e]] : ent[e];
        atomicAdd(&hist[key], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nkeys; k += blockDim.x) hb[(int64_t)blockIdx.x * nkeys + k] = hist[k];
}

// hb[b][k] <- sum_{b' < b} hb[b'][k] (each block's start within key k); cnt[k] = the total.
// One warp per key: 64 blocks' counts loaded at once, scanned with shuffles.
__device__ __forceinline__ int32_t warp_inclusive_scan(int32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__global__ void hist_scan_kernel(int nkeys, int nb, int32_t *__restrict__ hb, int32_t *__restrict__ cnt) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k >= nkeys) return;
    int32_t run = 0;
    for (int b0 = 0; b0 < nb; b0 += 64) {
        const int ba = b0 + lane, bb = b0 + 32 + lane;
        const int32_t ca = ba < nb ? hb[(int64_t)ba * nkeys + k] : 0;
        const int32_t cb = bb < nb ? hb[(int64_t)bb * nkeys + k] : 0;
        const int32_t xa = warp_inclusive_scan(ca, lane), xb = warp_inclusive_scan(cb, lane);
        const int32_t ta = __shfl_sync(0xffffffffu, xa, 31), tb = __shfl_sync(0xffffffffu, xb, 31);
        if (ba < nb) hb[(int64_t)ba * nkeys + k] = run + xa - ca;
        if (bb < nb) hb[(int64_t)bb * nkeys + k] = run + ta + xb - cb;
        run += ta + tb;
    }
    if (lane == 0) cnt[k] = run;
}

__global__ void hist_fill_kernel(int64_t nent, int64_t chunk, const int32_t *__restrict__ owner,
                                 const int32_t *__restrict__ ent, const int32_t *__restrict__ remap,
                                 const int64_t *__restrict__ off, const int32_t *__restrict__ hb, int nkeys,
                                 int by_entry, int32_t *__restrict__ inv, int32_t *__restrict__ map) {
    extern __shared__ int32_t cur[];
    for (int k = threadIdx.x; k < nkeys; k += blockDim.x) cur[k] = hb[(int64_t)blockIdx.x * nkeys + k];
    __syncthreads();
    const int64_t e0 = (int64_t)blockIdx.x * chunk, e1 = min(nent, e0 + chunk);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int key = remap ? remap[ent[e]] : ent[e];
        const int64_t p = off[key] + atomicAdd(&cur[key], 1);
        inv[p] = owner[e];
        if (by_entry) map[p] = (int32_t)e;
        else map[e] = (int32_t)p;
    }
}

__global__ void item_count_kernel(int nkeys, const int64_t *__restrict__ off, int per, int32_t *__restrict__ nitems) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    nitems[k] = (int)((off[k + 1] - off[k] + per - 1) / per);
}

// The items of key k: (k, first grouped entry, entries <= per, 0), one warp per key.
__global__ void item_fill_kernel(int nkeys, const int64_t *__restrict__ off, const int64_t *__restrict__ ioff, int per,
                                 int4 *__restrict__ items) {
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= nkeys) return;
    const int lane = threadIdx.x & 31;
    const int64_t c = off[k + 1] - off[k];
    for (int64_t w = lane; per * w < c; w += 32)
        items[ioff[k] + w] = make_int4((int)k, (int)(off[k] + per * w), (int)(c - per * w < per ? c - per * w : per), 0);
}

// P2P items in descending order of cost (sources of the leaf x targets), by
// buckets of width `step`: the expensive items start first and the cheap
// ones fill the last wave.  Only the launch order changes; every item writes
// its own records, so results do not depend on it.
__global__ void item_bucket_kernel(int64_t n, const int4 *__restrict__ items, const int32_t *__restrict__ leaf_node,
                                   const int64_t *__restrict__ count, int nb, int step, int32_t *__restrict__ bucket,
                                   int32_t *__restrict__ bcnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int4 it = items[i];
    const int64_t cost = count[leaf_node[it.x]] * it.z;
    const int64_t q = cost / step;
    const int b = nb - 1 - (int)(q < nb - 1 ? q : nb - 1);
    bucket[i] = b;
    atomicAdd(bcnt + b, 1);
}

__global__ void item_scatter_kernel(int64_t n, const int4 *__restrict__ in, const int32_t *__restrict__ bucket,
                                    const int64_t *__restrict__ boff, int32_t *__restrict__ cursor,
                                    int4 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int b = bucket[i];
    out[boff[b] + atomicAdd(cursor + b, 1)] = in[i];
}

// ---------------------------------------------------------------- near-singular lists
__device__ __forceinline__ bool in_sorted(const int32_t *__restrict__ a, int64_t n, int v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < n && a[lo] == v;
}

__device__ __forceinline__ bool is_near(double x, double y, double z, const double *__restrict__ cen,
                                        const double *__restrict__ L, double thres, int j) {
    const double dx = __dsub_rn(x, cen[3 * j]);
    const double dy = __dsub_rn(y, cen[3 * j + 1]);
    const double dz = __dsub_rn(z, cen[3 * j + 2]);
    const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    const double tl = __dmul_rn(thres, L[j]);
    return d2 < __dmul_rn(tl, tl);
}

// One warp per target: lanes walk the points of the target's direct-sum
// leaves.  An FP32 distance test with a safety margin only prefilters; the
// decision is the exact FP64 test above.  The fill pass writes the accepted
// panels in any order and then sorts them ascending (deterministic result).
constexpr int kNearCap = 256;   // row capacity of the one-pass mode

// MODE 0: counts; 1: fills the CSR list (after the counts' scan); 2: counts
// and writes the panels to a row of kNearCap entries per target (compacted
// and sorted by near_compact_kernel; a longer row sets *overflow).
template <int MODE>
__global__ void __launch_bounds__(128) near_kernel(
    int64_t ntg, int K, const double *__restrict__ xs, const int32_t *__restrict__ selfp, int use_self,
    const int64_t *__restrict__ p2p_ptr, const int32_t *__restrict__ p2p_leafidx, const int32_t *__restrict__ leaf_node,
    const int64_t *__restrict__ start, const int64_t *__restrict__ count, const int32_t *__restrict__ perm,
    const int32_t *__restrict__ pids, const int32_t *__restrict__ point_leaf, const double *__restrict__ cen,
    const double *__restrict__ L, const float4 *__restrict__ ppan32, double ox, double oy, double oz, double thres,
    int32_t *__restrict__ ncount, int32_t *__restrict__ excl, int32_t *__restrict__ self_excl,
    const int64_t *__restrict__ near_ptr, int32_t *__restrict__ near_panel, const int64_t *__restrict__ m2p_ptr,
    const int32_t *__restrict__ m2p_node, const float4 *__restrict__ cen32, double reach, int32_t *__restrict__ rows,
    int32_t *__restrict__ overflow) {
    constexpr bool FILL = MODE == 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float freach = (float)reach;
    const int64_t i = (int64_t)blockIdx.x * 4 + warp;
    if (i >= ntg) return;
    const double x = xs[3 * i], y = xs[3 * i + 1], z = xs[3 * i + 2];
    const float fx = (float)(x - ox), fy = (float)(y - oy), fz = (float)(z - oz);
    const int me = use_self ? selfp[i] : -1;
    const int64_t l0 = p2p_ptr[i], l1 = p2p_ptr[i + 1];
    const int32_t *lst = p2p_leafidx + l0;
    const int64_t nl = l1 - l0;
    int cnt = 0, ex = 0;
    const int64_t o = FILL ? near_ptr[i] : 0;
    for (int64_t e = 0; e < nl; ++e) {
        const int b = leaf_node[lst[e]];
        // a leaf farther than reach + r_b holds no point of a near panel (FP32 with margin)
        const float4 bc = cen32[b];
        const float bx = fx - bc.x, by = fy - bc.y, bz = fz - bc.z;
        const float rr = freach + sqrtf(bc.w);
        if (bx * bx + by * by + bz * bz > rr * rr * 1.0001f + 1e-3f) continue;
        const int64_t q0 = start[b], q1 = start[b] + count[b];
        for (int64_t qb = q0; qb < q1; qb += 32) {
            const int64_t q = qb + lane;
            bool acc = false, exc = false;
            int j = -1;
            if (q < q1) {
                // the point's panel (centroid, near radius) in point order: one coalesced load
                const float4 pc = ppan32[q];
                const float dx = fx - pc.x, dy = fy - pc.y, dz = fz - pc.z;
                const float d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < pc.w) j = pids[q];
                if (d2 < pc.w && j != me && is_near(x, y, z, cen, L, thres, j)) {
                    const int k = perm[q] - j * K;
                    // handle panel j once, at its lowest-numbered point inside the direct leaves
                    bool first = true;
                    for (int kk = 0; kk < k; ++kk)
                        if (in_sorted(lst, nl, point_leaf[j * K + kk])) { first = false; break; }
                    if (first) {
                        // points 0..k-1 lie outside the direct leaves when k > 0
                        bool all = k == 0;
                        for (int kk = k + 1; all && kk < K; ++kk)
                            if (!in_sorted(lst, nl, point_leaf[j * K + kk])) all = false;
                        acc = all;
                        exc = !all;
                    }
                }
            }
            const uint32_t ba = __ballot_sync(0xffffffffu, acc);
            if (FILL && acc) near_panel[o + cnt + __popc(ba & ((1u << lane) - 1u))] = j;
            if (MODE == 2 && acc) {
                const int at = cnt + __popc(ba & ((1u << lane) - 1u));
                if (at < kNearCap) rows[i * kNearCap + at] = j;
            }
            cnt += __popc(ba);
            ex += __popc(__ballot_sync(0xffffffffu, exc));
        }
    }
    if (FILL) {
        __syncwarp();
        if (lane == 0) {  // ascending panel order
            int32_t *a = near_panel + o;
            for (int u = 1; u < cnt; ++u) {
                int v = a[u], w = u - 1;
                while (w >= 0 && a[w] > v) { a[w + 1] = a[w]; --w; }
                a[w + 1] = v;
            }
        }
        return;
    }
    // near panels lying wholly in accepted boxes: only boxes that can hold a
    // point within `reach` (>= thres L_j + panel radius) of the target are
    // scanned; lanes test the boxes in turn (FP32 with margin)
    for (int64_t eb = m2p_ptr[i]; eb < m2p_ptr[i + 1]; eb += 32) {
        const int64_t e = eb + lane;
        bool hit = false;
        int bsel = -1;
        if (e < m2p_ptr[i + 1]) {
            bsel = m2p_node[e];
            const float4 bc = cen32[bsel];
            const float bx = fx - bc.x, by = fy - bc.y, bz = fz - bc.z;
            const float rr = freach + sqrtf(bc.w);
            hit = bx * bx + by * by + bz * bz <= rr * rr * 1.0001f + 1e-3f;
        }
        uint32_t hits = __ballot_sync(0xffffffffu, hit);
        while (hits) {
            const int src = __ffs(hits) - 1;
            hits &= hits - 1;
            const int b = __shfl_sync(0xffffffffu, bsel, src);
            const int64_t q0 = start[b], q1 = start[b] + count[b];
            for (int64_t qb = q0; qb < q1; qb += 32) {
                const int64_t q = qb + lane;
                bool exc = false;
                if (q < q1) {
                    const float4 pc = ppan32[q];
                    const float dx = fx - pc.x, dy = fy - pc.y, dz = fz - pc.z;
                    const int j = dx * dx + dy * dy + dz * dz < pc.w ? pids[q] : -1;
                    if (j >= 0 && perm[q] == j * K && j != me && is_near(x, y, z, cen, L, thres, j)) {
                        bool any = false;
                        for (int kk = 0; kk < K && !any; ++kk) any = in_sorted(lst, nl, point_leaf[j * K + kk]);
                        exc = !any;
                    }
                }
                ex += __popc(__ballot_sync(0xffffffffu, exc));
            }
        }
    }
    if (lane == 0) {
        ncount[i] = cnt;
        excl[i] = ex;
        if (MODE == 2 && cnt > kNearCap) atomicExch(overflow, 1);
        int se = 0;
        if (me >= 0)
            for (int kk = 0; kk < K; ++kk)
                if (!in_sorted(lst, nl, point_leaf[me * K + kk])) se = 1;
        self_excl[i] = se;
    }
}

// FP32 copy of the panel centroids (relative to the tree origin) and a
// conservative FP32 bound of the squared near-singular radius.
__global__ void pan32_kernel(int64_t n, const double *__restrict__ cen, const double *__restrict__ L, double thres,
                             double ox, double oy, double oz, float4 *__restrict__ pan32) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double tl = thres * L[j];
    pan32[j] = make_float4((float)(cen[3 * j] - ox), (float)(cen[3 * j + 1] - oy), (float)(cen[3 * j + 2] - oz),
                           (float)(tl * tl * (1.0 + 1e-3) + 1e-3));
}

// The panel record of every source point, in the tree's point order.
__global__ void point_pan32_kernel(int64_t npts, const int32_t *__restrict__ pids, const float4 *__restrict__ pan32,
                                   float4 *__restrict__ ppan32) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < npts) ppan32[q] = pan32[pids[q]];
}

// max_j (thres L_j + max_v |v - c_j|) over the panels of a surface; the
// non-negative doubles are combined with an integer atomic max of their bits.
__global__ void reach_kernel(int64_t n, const double *__restrict__ v, const int32_t *__restrict__ t,
                             const double *__restrict__ cen, const double *__restrict__ L, double thres,
                             unsigned long long *__restrict__ out) {
    double m = 0.0, h = 0.0;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        double r = 0.0;
        for (int c = 0; c < 3; ++c) {
            const int a = t[3 * j + c];
            const double dx = v[3 * a] - cen[3 * j], dy = v[3 * a + 1] - cen[3 * j + 1], dz = v[3 * a + 2] - cen[3 * j + 2];
            r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
        }
        m = fmax(m, thres * L[j] + r);
        h = fmax(h, thres * L[j]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        h = fmax(h, __shfl_xor_sync(0xffffffffu, h, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(m * (1.0 + 1e-12) + 1e-12));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(h * (1.0 + 1e-12) + 1e-12));
    }
}

// ---------------------------------------------------------------- near lists through a cell grid
// Panel centroids binned in a uniform grid of cells at least as wide as the
// largest near-singular radius thres L_j: every panel near a target lies in
// one of the 27 cells around the target's cell.  The decision is the same
// exact FP64 test as in near_kernel, so the lists are the same.
struct NearGrid {
    double corner[3];
    double inv_cell;
    int n[3];
};

__device__ __forceinline__ int grid_axis(double v, double c, double inv, int n) {
    const double f = floor((v - c) * inv);
    return f < -2.0 ? -2 : (f > (double)(n + 1) ? n + 1 : (int)f);
}

__global__ void cell_count_kernel(int64_t n, const double *__restrict__ cen, NearGrid g, int32_t *__restrict__ cellof,
                                  int32_t *__restrict__ cnt) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int c[3];
    for (int a = 0; a < 3; ++a) c[a] = min(max(grid_axis(cen[3 * j + a], g.corner[a], g.inv_cell, g.n[a]), 0), g.n[a] - 1);
    const int flat = (c[0] * g.n[1] + c[1]) * g.n[2] + c[2];
    cellof[j] = flat;
    atomicAdd(cnt + flat, 1);
}

// Panel ids, FP32 records (centroid, near radius bound) and FP64 (centroid,
// L) in cell order.
__global__ void cell_fill_kernel(int64_t n, const int32_t *__restrict__ cellof, const int64_t *__restrict__ off,
                                 int32_t *__restrict__ cursor, const float4 *__restrict__ pan32,
                                 const double *__restrict__ cen, const double *__restrict__ L, double thres,
                                 int32_t *__restrict__ order, float4 *__restrict__ cpan, dvec4 *__restrict__ cgeo,
                                 float *__restrict__ cr2) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int c = cellof[j];
    const int64_t q = off[c] + atomicAdd(cursor + c, 1);
    order[q] = (int32_t)j;
    cpan[q] = pan32[j];
    cgeo[q] = dvec4{cen[3 * j], cen[3 * j + 1], cen[3 * j + 2], L[j]};
    const double tl = __dmul_rn(thres, L[j]);
    cr2[q] = (float)__dmul_rn(tl, tl);
}

// One warp per target.  The panels of the 27 cells around the target form one
// list (the cells' ranges loaded one per lane, their offsets by a warp scan)
// that the lanes walk 32 entries at a time, whatever the cells' sizes: the
// FP32 record (prefilter) and the panel id, then the FP64 centroid and L of
// the exact test, all in cell order; the target's direct-sum leaf list is
// staged in shared memory for the membership tests of the near panels' points.  The
// decision is the same FP64 test as is_near.  Near panels whose points all
// lie in the target's direct-sum leaves go to its row (any order;
// near_compact_kernel sorts), the others are counted as excluded.  Outputs as
// near_kernel<2>.
constexpr int kNearLeafStage = 128;   // direct-sum leaves staged per warp

__device__ __forceinline__ bool in_sorted_shared(const int32_t *a, int n, int v) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo < n && a[lo] == v;
}

__global__ void __launch_bounds__(128) near_grid_kernel(
    int64_t ntg, int K, const double *__restrict__ xs, const int32_t *__restrict__ selfp, int use_self,
    const int64_t *__restrict__ p2p_ptr, const int32_t *__restrict__ p2p_leafidx, const int32_t *__restrict__ point_leaf,
    double ox, double oy, double oz, double thres, NearGrid g, const int64_t *__restrict__ off,
    const int32_t *__restrict__ order, const float4 *__restrict__ cpan, const dvec4 *__restrict__ cgeo,
    const float *__restrict__ cr2, double side, int32_t *__restrict__ ncount, int32_t *__restrict__ excl,
    int32_t *__restrict__ self_excl, int32_t *__restrict__ rows, int32_t *__restrict__ overflow) {
    __shared__ int32_t sleaf[4][kNearLeafStage];
    __shared__ int32_t scell[4][27];
    __shared__ int64_t sbase[4][27];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + warp;
    if (i >= ntg) return;
    const double x = xs[3 * i], y = xs[3 * i + 1], z = xs[3 * i + 2];
    const float fx = (float)(x - ox), fy = (float)(y - oy), fz = (float)(z - oz);
    // bound on the FP32 coordinate differences' error (the panels lie in the
    // root cube, |c - o| <= side / 2 per axis)
    const float ecoord = (float)(0x1p-23 * (fmax(fabs(x - ox), fmax(fabs(y - oy), fabs(z - oz))) + side));
    const int me = use_self ? selfp[i] : -1;
    const int64_t l0 = p2p_ptr[i];
    const int64_t nl = p2p_ptr[i + 1] - l0;
    const bool staged = nl <= kNearLeafStage;
    if (staged)
        for (int u = lane; u < nl; u += 32) sleaf[warp][u] = p2p_leafidx[l0 + u];
    __syncwarp();
    auto member = [&](int leaf) {
        return staged ? in_sorted_shared(sleaf[warp], (int)nl, leaf) : in_sorted(p2p_leafidx + l0, nl, leaf);
    };
    const int cx = grid_axis(x, g.corner[0], g.inv_cell, g.n[0]);
    const int cy = grid_axis(y, g.corner[1], g.inv_cell, g.n[1]);
    const int cz = grid_axis(z, g.corner[2], g.inv_cell, g.n[2]);
    // the 27 cells' panels as one list: lane k < 27 holds cell k's range, a
    // warp scan of the counts gives every cell's first position in the list
    int64_t cs = 0;
    int cn = 0;
    if (lane < 27) {
        const int ax = cx - 1 + lane / 9, ay = cy - 1 + (lane / 3) % 3, az = cz - 1 + lane % 3;
        if (ax >= 0 && ax < g.n[0] && ay >= 0 && ay < g.n[1] && az >= 0 && az < g.n[2]) {
            const int c = (ax * g.n[1] + ay) * g.n[2] + az;
            cs = off[c];
            cn = (int)(off[c + 1] - cs);
        }
    }
    int pre = cn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, pre, o);
        if (lane >= o) pre += v;
    }
    const int total = __shfl_sync(0xffffffffu, pre, 31);
    if (lane < 27) {
        scell[warp][lane] = pre - cn;   // first list position of cell `lane`
        sbase[warp][lane] = cs - (pre - cn);
    }
    __syncwarp();
    const double tt = thres;
    int cnt = 0, ex = 0;
    int32_t *row = rows + i * kNearCap;
    for (int ub = 0; ub < total; ub += 32) {
        const int u = ub + lane;
        bool acc = false, exc = false;
        int j = -1;
        if (u < total) {
            // the last cell whose first position is <= u
            int lo = 0, hi = 26;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (scell[warp][mid] <= u) lo = mid; else hi = mid - 1;
            }
            const int64_t q = sbase[warp][lo] + u;
            const float4 pc = cpan[q];
            j = order[q];
            const float dx = fx - pc.x, dy = fy - pc.y, dz = fz - pc.z;
            const float d2f = dx * dx + dy * dy + dz * dz;
            if (d2f < pc.w && j != me) {
                // is_near: in FP32 where the error bound leaves no doubt (|d2f - d2| and
                // |r2f - r2| within err), else by the FP64 test with the panel's
                // centroid and L from its cell-ordered copy
                const float r2f = cr2[q];
                const float err = 1e-4f * (d2f + r2f) + ecoord * (4.f * sqrtf(d2f) + 10.f * ecoord);
                bool nearp;
                if (d2f + err < r2f) {
                    nearp = true;
                } else if (d2f - err > r2f) {
                    nearp = false;
                } else {
                    const dvec4 cg = cgeo[q];
                    const double ddx = __dsub_rn(x, cg.x), ddy = __dsub_rn(y, cg.y), ddz = __dsub_rn(z, cg.z);
                    const double d2 =
                        __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
                    const double tl = __dmul_rn(tt, cg.w);
                    nearp = d2 < __dmul_rn(tl, tl);
                }
                if (nearp) {
                    bool all = true;
                    for (int kk = 0; kk < K && all; ++kk) all = member(point_leaf[(int64_t)j * K + kk]);
                    acc = all;
                    exc = !all;
                }
            }
        }
        const uint32_t ba = __ballot_sync(0xffffffffu, acc);
        if (acc) {
            const int at = cnt + __popc(ba & ((1u << lane) - 1u));
            if (at < kNearCap) row[at] = j;
        }
        cnt += __popc(ba);
        ex += __popc(__ballot_sync(0xffffffffu, exc));
    }
    if (lane == 0) {
        ncount[i] = cnt;
        excl[i] = ex;
        if (cnt > kNearCap) atomicExch(overflow, 1);
        int se = 0;
        if (me >= 0)
            for (int kk = 0; kk < K; ++kk)
                if (!member(point_leaf[(int64_t)me * K + kk])) se = 1;
        self_excl[i] = se;
    }
}

// Copies every target's row into the CSR list in ascending order (insertion sort).
__global__ void near_compact_kernel(int64_t ntg, const int32_t *__restrict__ rows, const int64_t *__restrict__ ptr,
                                    int32_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ntg) return;
    const int32_t *row = rows + i * kNearCap;
    int32_t *a = out + ptr[i];
    const int n = (int)(ptr[i + 1] - ptr[i]);
    for (int u = 0; u < n; ++u) {
        const int v = row[u];
        int w = u - 1;
        while (w >= 0 && a[w] > v) { a[w + 1] = a[w]; --w; }
        a[w + 1] = v;
    }
}

__global__ void node_to_leaf_kernel(int64_t n, const int32_t *__restrict__ nodes, const int32_t *__restrict__ node_leaf,
                                    int32_t *__restrict__ out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < n) out[e] = node_leaf[nodes[e]];
}

__global__ void sum_i32_kernel(const int32_t *__restrict__ a, int64_t n, unsigned long long *out) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned long long)a[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void p2p_pairs_kernel(int64_t ntg, const int64_t *__restrict__ ptr, const int32_t *__restrict__ nodes,
                                 const int64_t *__restrict__ count, unsigned long long *out) {
    unsigned long long s = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ntg; i += (int64_t)gridDim.x * blockDim.x)
        for (int64_t e = ptr[i]; e < ptr[i + 1]; ++e) s += (unsigned long long)count[nodes[e]];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

void root_cube_from(const double *d_points, int64_t n, cudaStream_t s, double *cube) {
    const int nb = (int)std::min<int64_t>(592, std::max<int64_t>(1, (n + 1023) / 1024));
    TmpBuf<double> part(6 * nb, s);
    bbox_blocks_kernel<<<nb, 256, 0, s>>>(d_points, n, part.p);
    PB_LAUNCH_CHECK();
    cube_final_kernel<<<1, 32, 0, s>>>(part.p, nb, cube);
    PB_LAUNCH_CHECK();
}

}  // namespace

void morton_sort(const double *d_points, int64_t n, cudaStream_t s, double *cube, DevBuf<uint64_t> &keys,
                 DevBuf<int32_t> &perm) {
    root_cube_from(d_points, n, s, cube);
    keys.alloc(n);
    perm.alloc(n);
    if (n) {
        morton_kernel<<<div_up(n, 256), 256, 0, s>>>(d_points, n, cube, keys.p, perm.p);
        PB_LAUNCH_CHECK();
        sort_key_index(keys.p, perm.p, n, s);
    }
}

void build_tree(Tree &T, const SurfDev &S, int K, int ncrit, cudaStream_t s) {
    build_tree_points(T, S.gy.p, S.gwa.p, S.n * K, K, ncrit, s);
}

// Everything on the device, one host read at the end: the root cube, the
// sort, the levels (one block), node geometry, leaves and sorted sources are
// sized by the node bound maxn, and the kernels read the node count from info.
void build_tree_points(Tree &T, const double *pts, const double *wts, int64_t n, int K, int ncrit, cudaStream_t s) {
    T.npts = n;
    constexpr int kInfo = 32;
    TmpBuf<double> cube(4, s);
    TmpBuf<int32_t> info(kInfo, s);
    morton_sort(pts, n, s, cube.p, T.keys, T.perm);
    // node bound: every level holds disjoint nodes, each split node >= ncrit points
    const int64_t maxn = std::min<int64_t>((int64_t)1 + 8LL * (kMaxLevel + 1) * (n / std::max(1, ncrit) + 1),
                                           2 * n + 64);
    T.level.alloc(maxn); T.first_child.alloc(maxn); T.nchild.alloc(maxn); T.parent.alloc(maxn);
    T.start.alloc(maxn); T.count.alloc(maxn);
    TmpBuf<int64_t> ijk(3 * maxn, s);
    {
        // at most maxn nodes on a level: bounds of 9 per node, scan of maxn + 1
        TmpBuf<int32_t> bnd(9 * maxn, s), cscan(maxn + 1, s);
        int per_sm = 0;
        PB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, build_levels_kernel, kLevelThreads, 0));
        int nsm = 0, dev = 0;
        PB_CUDA_TRY(cudaGetDevice(&dev));
        PB_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        const int grid = std::max(1, std::min(nsm * std::min(per_sm, 2), div_up(maxn * 8, kLevelThreads)));
        int64_t a_n = n;
        int a_ncrit = ncrit, a_maxn = (int)maxn;
        const uint64_t *a_keys = T.keys.p;
        int64_t *a_start = T.start.p, *a_count = T.count.p, *a_ijk = ijk.p;
        int32_t *a_level = T.level.p, *a_fc = T.first_child.p, *a_nch = T.nchild.p, *a_par = T.parent.p,
                *a_bnd = bnd.p, *a_cs = cscan.p, *a_info = info.p;
        void *args[] = {&a_n, &a_ncrit, &a_maxn, &a_keys, &a_start, &a_count, &a_level, &a_fc, &a_nch, &a_par,
                        &a_ijk, &a_bnd, &a_cs, &a_info};
        PB_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)build_levels_kernel, grid, kLevelThreads, args, 0, s));
        PB_LAUNCH_CHECK();
    }
    const int gn = div_up(maxn, 128);
    T.centre.alloc(3 * (size_t)maxn);
    T.rb2.alloc(maxn);
    node_geom_kernel<<<gn, 128, 0, s>>>(info.p, T.level.p, ijk.p, cube.p, T.centre.p, T.rb2.p);
    PB_LAUNCH_CHECK();
    T.link.alloc(maxn);
    link_kernel<<<gn, 128, 0, s>>>(info.p, T.parent.p, T.first_child.p, T.nchild.p, T.link.p);
    PB_LAUNCH_CHECK();
    T.cen32.alloc(maxn);
    centre32_kernel<<<gn, 128, 0, s>>>(info.p, T.centre.p, T.rb2.p, cube.p, T.cen32.p);
    PB_LAUNCH_CHECK();
    T.pofs32.alloc(maxn);
    parent_offset_kernel<<<gn, 128, 0, s>>>(info.p, T.parent.p, T.centre.p, T.pofs32.p);
    PB_LAUNCH_CHECK();
    // leaves in Morton order (= depth-first pre-order)
    TmpBuf<int32_t> head(std::max<int64_t>(1, n), s);
    TmpBuf<int64_t> hscan(n + 1, s);
    if (n) PB_CUDA_TRY(cudaMemsetAsync(head.p, 0, n * sizeof(int32_t), s));
    leaf_flag_kernel<<<gn, 128, 0, s>>>(info.p, T.nchild.p, T.start.p, head.p);
    PB_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(head.p, hscan.p, n, s);
    T.node_leaf.alloc(maxn);
    T.leaf_node.alloc(maxn);
    T.point_leaf.alloc(std::max<int64_t>(1, n));
    leaf_index_kernel<<<gn, 128, 0, s>>>(info.p, T.nchild.p, T.start.p, hscan.p, T.node_leaf.p, T.leaf_node.p);
    PB_LAUNCH_CHECK();
    if (n) {
        point_leaf_kernel<<<div_up(n, 256), 256, 0, s>>>(n, hscan.p, T.perm.p, T.point_leaf.p);
        PB_LAUNCH_CHECK();
    }
    // sorted source geometry
    T.ys.alloc(3 * n); T.was.alloc(n); T.pids.alloc(n); T.pos32.alloc(n);
    if (n) {
        gather_sources_kernel<<<div_up(n, 256), 256, 0, s>>>(n, K, T.perm.p, pts, wts, cube.p, T.ys.p, T.was.p,
                                                             T.pids.p, T.pos32.p);
        PB_LAUNCH_CHECK();
    }
    T.src64.alloc(8 * n); T.srcA32.alloc(n); T.srcB32.alloc(n);
    HostReads rd(s);
    const double *hc = rd.add(cube.p, 4);
    const int32_t *hi = rd.add(info.p, kInfo);
    const int64_t *hl = rd.add(hscan.p + n);
    rd.wait();
    if (hi[2]) fail(PB_ENOMEM, "octree node capacity exceeded");
    for (int a = 0; a < 3; ++a) T.corner[a] = hc[a];
    T.side = hc[3];
    for (int a = 0; a < 3; ++a) T.origin[a] = T.corner[a] + 0.5 * T.side;
    T.nnodes = hi[0];
    T.nlevels = hi[1];
    T.level_off.assign(hi + 3, hi + 3 + T.nlevels + 1);
    T.nleaves = (int)*hl;
    // the arrays keep their bound-sized blocks; their counts become the tree's
    for (auto *b : {&T.level, &T.first_child, &T.nchild, &T.parent, &T.node_leaf}) b->alloc(T.nnodes);
    T.start.alloc(T.nnodes); T.count.alloc(T.nnodes);
    T.centre.alloc(3 * (size_t)T.nnodes); T.rb2.alloc(T.nnodes);
    T.link.alloc(T.nnodes); T.cen32.alloc(T.nnodes); T.pofs32.alloc(T.nnodes);
    T.leaf_node.alloc(std::max(1, T.nleaves));
}

void build_targets(Targets &G, const double *d_x, int64_t n, int surface, cudaStream_t s, int points_per_panel) {
    G.n = n;
    G.surface = surface;
    TmpBuf<double> cube(4, s);
    morton_sort(d_x, n, s, cube.p, G.keys, G.order);
    G.xs.alloc(3 * n);
    G.self_panel.alloc(n);
    G.rank.alloc(n);
    if (n) {
        gather_targets_kernel<<<div_up(n, 256), 256, 0, s>>>(n, G.order.p, d_x, G.xs.p, G.self_panel.p, G.rank.p,
                                                             surface >= 0 ? points_per_panel : 0);
        PB_LAUNCH_CHECK();
    }
}

namespace {

// Entry-major grouping of one list kind (P2P or M2P) across the phases of a list build.
struct Grouping {
    int nkeys = 0;
    int per = 32;
    std::optional<TmpBuf<int64_t>> off, ioff;   // per key: first grouped entry, first item
};

// inv / pos: the list entries regrouped by key (box or leaf), and the per-key
// item offsets; the item count is ioff[nkeys] (read by the caller).
void group_count(int64_t m, const int64_t *ptr, const int32_t *ent, const int32_t *remap, int nkeys, int64_t nent,
                 int per, int by_entry, DevBuf<int32_t> &inv, DevBuf<int32_t> &pos, Grouping &gr, cudaStream_t s) {
    gr.nkeys = nkeys;
    gr.per = per;
    gr.off.emplace(nkeys + 1, s);
    gr.ioff.emplace(nkeys + 1, s);
    TmpBuf<int32_t> cnt(std::max(1, nkeys), s), cursor(std::max(1, nkeys), s), nit(std::max(1, nkeys), s);
    PB_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * std::max(1, nkeys), s));
    PB_CUDA_TRY(cudaMemsetAsync(cursor.p, 0, sizeof(int32_t) * std::max(1, nkeys), s));
    inv.alloc(std::max<int64_t>(1, nent));
    pos.alloc(std::max<int64_t>(1, nent));
    TmpBuf<int32_t> owner(std::max<int64_t>(1, nent), s);
    const bool hist = nkeys <= kHistKeys && nent > 0;
    const int nb = hist ? (int)std::min<int64_t>(296, div_up(nent, 2048)) : 0;
    const int64_t chunk = hist ? (nent + nb - 1) / nb : 0;
    TmpBuf<int32_t> hb(hist ? (size_t)nb * nkeys : 0, s);
    const size_t hshm = (size_t)nkeys * sizeof(int32_t);
    if (m && nent) {
        owner_kernel<<<div_up(m * 32, 256), 256, 0, s>>>(m, ptr, owner.p);
        PB_LAUNCH_CHECK();
        if (hist) {
            hist_count_kernel<<<nb, 256, hshm, s>>>(nent, chunk, ent, remap, nkeys, hb.p);
            PB_LAUNCH_CHECK();
            hist_scan_kernel<<<div_up(nkeys, 4), 128, 0, s>>>(nkeys, nb, hb.p, cnt.p);
            PB_LAUNCH_CHECK();
        } else {
            inv_count_kernel<<<div_up(nent, 256), 256, 0, s>>>(nent, ent, remap, cnt.p);
            PB_LAUNCH_CHECK();
        }
    }
    exclusive_scan_i32_to_i64(cnt.p, gr.off->p, nkeys, s);
    if (m && nent) {
        if (hist)
            hist_fill_kernel<<<nb, 256, hshm, s>>>(nent, chunk, owner.p, ent, remap, gr.off->p, hb.p, nkeys, by_entry,
                                                   inv.p, pos.p);
        else
            inv_fill_kernel<<<div_up(nent, 256), 256, 0, s>>>(nent, owner.p, ent, remap, gr.off->p, cursor.p, by_entry,
                                                              inv.p, pos.p);
        PB_LAUNCH_CHECK();
    }
    item_count_kernel<<<div_up(nkeys, 128), 128, 0, s>>>(nkeys, gr.off->p, per, nit.p);
    PB_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(nit.p, gr.ioff->p, nkeys, s);
}

void group_fill(Grouping &gr, int64_t nitems, DevBuf<int4> &items, cudaStream_t s) {
    items.alloc(std::max<int64_t>(1, nitems));
    item_fill_kernel<<<div_up((int64_t)gr.nkeys * 32, 256), 256, 0, s>>>(gr.nkeys, gr.off->p, gr.ioff->p, gr.per,
                                                                         items.p);
    PB_LAUNCH_CHECK();
}

// P2P items in buckets of similar source-leaf size (the larger leaves first
// keep the direct-sum warps of one wave alike), stable within a bucket.
void bucket_p2p_items(Pair &Pr, const Tree &T, int ncrit, int p2p_per_item, cudaStream_t s) {
    if (Pr.n_p2p_items <= 1) return;
    constexpr int nb = 64;
    const int step = std::max(1, ncrit * p2p_per_item / nb);
    const int64_t ni = Pr.n_p2p_items;
    TmpBuf<int32_t> bucket(ni, s), bcnt(nb, s), cursor(nb, s);
    TmpBuf<int64_t> boff(nb + 1, s);
    TmpBuf<int4> sorted(ni, s);
    PB_CUDA_TRY(cudaMemsetAsync(bcnt.p, 0, nb * sizeof(int32_t), s));
    PB_CUDA_TRY(cudaMemsetAsync(cursor.p, 0, nb * sizeof(int32_t), s));
    item_bucket_kernel<<<div_up(ni, 256), 256, 0, s>>>(ni, Pr.p2p_items.p, T.leaf_node.p, T.count.p, nb, step,
                                                       bucket.p, bcnt.p);
    PB_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(bcnt.p, boff.p, nb, s);
    item_scatter_kernel<<<div_up(ni, 256), 256, 0, s>>>(ni, Pr.p2p_items.p, bucket.p, boff.p, cursor.p, sorted.p);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaMemcpyAsync(Pr.p2p_items.p, sorted.p, ni * sizeof(int4), cudaMemcpyDeviceToDevice, s));
}

// State of one pair's list build between its two host reads.
struct ListBuild {
    static constexpr int nsplit = 8;   // a target walks the root's eight subtrees as eight threads
    std::optional<TmpBuf<int64_t>> mo, po;             // per (target, subtree) list offsets
    std::optional<TmpBuf<unsigned long long>> reach;   // source panels: largest near radius bits, largest h
    Grouping gp, gm;
    std::optional<TmpBuf<int32_t>> pleaf, rows, ovf;
    std::optional<TmpBuf<float4>> pan32;
};

// Phase 1: list lengths per (target, subtree) and their offsets; the source
// panels' near-field reach.
void far_count(Pair &Pr, const Targets &G, const Tree &T, const SurfDev *src, const Params &prm, ListBuild &lb,
               cudaStream_t s) {
    const int64_t m = G.n, ms = m * ListBuild::nsplit;
    Pr.stats.alloc(4);
    PB_CUDA_TRY(cudaMemsetAsync(Pr.stats.p, 0, 4 * sizeof(unsigned long long), s));
    TmpBuf<int32_t> mc(ms, s), pc(ms, s);
    lb.mo.emplace(ms + 1, s);
    lb.po.emplace(ms + 1, s);
    Pr.m2p_ptr.alloc(m + 1);
    Pr.p2p_ptr.alloc(m + 1);
    if (m) {
        traverse_kernel<false><<<div_up(ms, 128), 128, 0, s>>>(
            m, G.xs.p, T.centre.p, T.rb2.p, T.cen32.p, T.first_child.p, T.nchild.p, prm.theta * prm.theta,
            prm.theta <= 0.0, T.origin[0], T.origin[1], T.origin[2], mc.p, pc.p, nullptr, nullptr, nullptr, nullptr,
            Pr.stats.p, ListBuild::nsplit);
        PB_LAUNCH_CHECK();
    }
    exclusive_scan_i32_to_i64(mc.p, lb.mo->p, ms, s);
    exclusive_scan_i32_to_i64(pc.p, lb.po->p, ms, s);
    take_every_kernel<<<div_up(m + 1, 256), 256, 0, s>>>(m, ListBuild::nsplit, lb.mo->p, Pr.m2p_ptr.p);
    PB_LAUNCH_CHECK();
    take_every_kernel<<<div_up(m + 1, 256), 256, 0, s>>>(m, ListBuild::nsplit, lb.po->p, Pr.p2p_ptr.p);
    PB_LAUNCH_CHECK();
    if (src) {
        lb.reach.emplace(2, s);
        PB_CUDA_TRY(cudaMemsetAsync(lb.reach->p, 0, 2 * sizeof(unsigned long long), s));
        reach_kernel<<<std::min<int64_t>(592, div_up(src->n, 256)), 256, 0, s>>>(
            src->n, src->verts.p, src->tris.p, src->cen.p, src->L.p, prm.thres, lb.reach->p);
        PB_LAUNCH_CHECK();
    }
}

// Phase 2 (Pr.n_m2p, Pr.n_p2p known): the lists, the direct-sum pair count and
// the first half of both groupings.
void far_fill(Pair &Pr, const Targets &G, const Tree &T, const Params &prm, int p2p_per_item, ListBuild &lb,
              cudaStream_t s, cudaEvent_t lists_done = nullptr) {
    const int64_t m = G.n, ms = m * ListBuild::nsplit;
    Pr.m2p_node.alloc(std::max<int64_t>(1, Pr.n_m2p));
    Pr.p2p_node.alloc(std::max<int64_t>(1, Pr.n_p2p));
    if (m) {
        traverse_kernel<true><<<div_up(ms, 128), 128, 0, s>>>(
            m, G.xs.p, T.centre.p, T.rb2.p, T.cen32.p, T.first_child.p, T.nchild.p, prm.theta * prm.theta,
            prm.theta <= 0.0, T.origin[0], T.origin[1], T.origin[2], nullptr, nullptr, lb.mo->p, lb.po->p,
            Pr.m2p_node.p, Pr.p2p_node.p, Pr.stats.p, ListBuild::nsplit);
        PB_LAUNCH_CHECK();
        p2p_pairs_kernel<<<std::min<int64_t>(1024, div_up(m, 256)), 256, 0, s>>>(m, Pr.p2p_ptr.p, Pr.p2p_node.p,
                                                                                T.count.p, Pr.stats.p + 1);
        PB_LAUNCH_CHECK();
    }
    if (lists_done) PB_CUDA_TRY(cudaEventRecord(lists_done, s));   // the near lists may start
    group_count(m, Pr.p2p_ptr.p, Pr.p2p_node.p, T.node_leaf.p, T.nleaves, Pr.n_p2p, p2p_per_item, 1, Pr.p2p_inv,
                Pr.p2p_ent, lb.gp, s);
    group_count(m, Pr.m2p_ptr.p, Pr.m2p_node.p, nullptr, T.nnodes, Pr.n_m2p, 32, 1, Pr.m2p_inv, Pr.m2p_ent, lb.gm, s);
}

// Phase 2, near part (reach known): the cell grid of the source panels and one
// pass of near_grid_kernel (counts, rows of up to kNearCap panels), the CSR
// offsets and the excluded-panel counts.
void near_count(Pair &Pr, const Targets &G, const Tree &T, const SurfDev &src, const Params &prm, bool use_self,
                double hmax, ListBuild &lb, cudaStream_t s) {
    const int64_t m = G.n;
    lb.pleaf.emplace(std::max<int64_t>(1, Pr.n_p2p), s);
    if (Pr.n_p2p) {
        node_to_leaf_kernel<<<div_up(Pr.n_p2p, 256), 256, 0, s>>>(Pr.n_p2p, Pr.p2p_node.p, T.node_leaf.p,
                                                                   lb.pleaf->p);
        PB_LAUNCH_CHECK();
    }
    TmpBuf<int32_t> nc(std::max<int64_t>(1, m), s), ex(std::max<int64_t>(1, m), s), se(std::max<int64_t>(1, m), s);
    lb.pan32.emplace(std::max<int64_t>(1, src.n), s);
    pan32_kernel<<<div_up(src.n, 256), 256, 0, s>>>(src.n, src.cen.p, src.L.p, prm.thres, T.origin[0], T.origin[1],
                                                     T.origin[2], lb.pan32->p);
    PB_LAUNCH_CHECK();
    // cell grid over the tree's root cube (it holds every centroid): cells at
    // least as wide as the largest near radius, at most about two per panel
    NearGrid g{};
    {
        const double cmin = hmax * 1.001 + 1e-9;
        int na = (int)std::max(1.0, std::floor(T.side / cmin));
        while ((double)na * na * na > 2.0 * (double)src.n + 64.0 && na > 1) --na;
        const double cell = std::max(cmin, T.side / na);
        for (int a = 0; a < 3; ++a) {
            g.corner[a] = T.corner[a];
            g.n[a] = na;
        }
        g.inv_cell = 1.0 / cell;
    }
    const int64_t ncell = (int64_t)g.n[0] * g.n[1] * g.n[2];
    TmpBuf<int32_t> cellof(std::max<int64_t>(1, src.n), s), ccnt(ncell, s), ccur(ncell, s),
        corder(std::max<int64_t>(1, src.n), s);
    TmpBuf<float4> cpan(std::max<int64_t>(1, src.n), s);
    TmpBuf<dvec4> cgeo(std::max<int64_t>(1, src.n), s);
    TmpBuf<float> cr2(std::max<int64_t>(1, src.n), s);
    TmpBuf<int64_t> coff(ncell + 1, s);
    PB_CUDA_TRY(cudaMemsetAsync(ccnt.p, 0, ncell * sizeof(int32_t), s));
    PB_CUDA_TRY(cudaMemsetAsync(ccur.p, 0, ncell * sizeof(int32_t), s));
    if (src.n) {
        cell_count_kernel<<<div_up(src.n, 256), 256, 0, s>>>(src.n, src.cen.p, g, cellof.p, ccnt.p);
        PB_LAUNCH_CHECK();
    }
    exclusive_scan_i32_to_i64(ccnt.p, coff.p, ncell, s);
    if (src.n) {
        cell_fill_kernel<<<div_up(src.n, 256), 256, 0, s>>>(src.n, cellof.p, coff.p, ccur.p, lb.pan32->p, src.cen.p,
                                                            src.L.p, prm.thres, corder.p, cpan.p, cgeo.p, cr2.p);
        PB_LAUNCH_CHECK();
    }
    Pr.near_ptr.alloc(m + 1);
    lb.ovf.emplace(1, s);
    PB_CUDA_TRY(cudaMemsetAsync(lb.ovf->p, 0, 4, s));
    if (m) {
        lb.rows.emplace((size_t)m * kNearCap, s);
        near_grid_kernel<<<div_up(m, 4), 128, 0, s>>>(m, prm.K, G.xs.p, G.self_panel.p, (int)use_self, Pr.p2p_ptr.p,
                                                       lb.pleaf->p, T.point_leaf.p, T.origin[0], T.origin[1],
                                                       T.origin[2], prm.thres, g, coff.p, corder.p, cpan.p, cgeo.p,
                                                       cr2.p, T.side, nc.p, ex.p, se.p, lb.rows->p, lb.ovf->p);
        PB_LAUNCH_CHECK();
        sum_i32_kernel<<<std::min<int64_t>(1024, div_up(m, 256)), 256, 0, s>>>(ex.p, m, Pr.stats.p + 2);
        PB_LAUNCH_CHECK();
        sum_i32_kernel<<<std::min<int64_t>(1024, div_up(m, 256)), 256, 0, s>>>(se.p, m, Pr.stats.p + 3);
        PB_LAUNCH_CHECK();
    }
    exclusive_scan_i32_to_i64(nc.p, Pr.near_ptr.p, m, s);
}

// Phase 3 (n_near and the row overflow flag known): the near lists in CSR form,
// compacted from the rows or, where some target has more than kNearCap near
// panels, filled by a second pass.
void near_fill(Pair &Pr, const Targets &G, const Tree &T, const SurfDev &src, const Params &prm, bool use_self,
               double reach, bool overflow, ListBuild &lb, cudaStream_t s) {
    const int64_t m = G.n;
    Pr.near_panel.alloc(std::max<int64_t>(1, Pr.n_near));
    if (!m) return;
    if (!overflow) {
        near_compact_kernel<<<div_up(m, 128), 128, 0, s>>>(m, lb.rows->p, Pr.near_ptr.p, Pr.near_panel.p);
        PB_LAUNCH_CHECK();
        return;
    }
    TmpBuf<float4> ppan32(std::max<int64_t>(1, T.npts), s);
    if (T.npts) {
        point_pan32_kernel<<<div_up(T.npts, 256), 256, 0, s>>>(T.npts, T.pids.p, lb.pan32->p, ppan32.p);
        PB_LAUNCH_CHECK();
    }
    near_kernel<1><<<div_up(m, 4), 128, 0, s>>>(m, prm.K, G.xs.p, G.self_panel.p, (int)use_self, Pr.p2p_ptr.p,
                                                lb.pleaf->p, T.leaf_node.p, T.start.p, T.count.p, T.perm.p, T.pids.p,
                                                T.point_leaf.p, src.cen.p, src.L.p, ppan32.p, T.origin[0],
                                                T.origin[1], T.origin[2], prm.thres, nullptr, nullptr, nullptr,
                                                Pr.near_ptr.p, Pr.near_panel.p, Pr.m2p_ptr.p, Pr.m2p_node.p,
                                                T.cen32.p, reach, nullptr, nullptr);
    PB_LAUNCH_CHECK();
}

// stats: [0] traversal stack overflow, [1] direct-sum pairs, [2] near panels
// excluded (outside the direct-sum leaves), [3] own panels excluded.
void apply_list_stats(Pair &Pr, const unsigned long long *h) {
    if (h[0]) fail(PB_EINVAL, "octree traversal stack overflow");
    Pr.p2p_pairs = (int64_t)h[1];
    Pr.near_excl = (int64_t)h[2];
    Pr.self_excl = (int64_t)h[3];
}

void read_far_counts(Pair &Pr, ListBuild &lb, int64_t m, double *reach, double *hmax, cudaStream_t s) {
    HostReads rd(s);
    const int64_t *hm = rd.add(Pr.m2p_ptr.p + m);
    const int64_t *hp = rd.add(Pr.p2p_ptr.p + m);
    const unsigned long long *hr = lb.reach ? rd.add(lb.reach->p, 2) : nullptr;
    rd.wait();
    Pr.n_m2p = *hm;
    Pr.n_p2p = *hp;
    if (hr) {
        std::memcpy(reach, &hr[0], sizeof(double));
        std::memcpy(hmax, &hr[1], sizeof(double));
    }
}

}  // namespace

void build_lists(Pair &Pr, const Targets &G, const Tree &T, const SurfDev &src, const Params &prm, bool use_self,
                 cudaStream_t s) {
    std::vector<ListJob> jobs{ListJob{&Pr, &G, &T, &src, use_self, s}};
    build_lists_multi(jobs, prm);
}

// Every pair's list build in three phases on its own stream; the host reads
// of a phase (list lengths and near-field reach; item counts, near-list
// length, overflow flag and counters) are one wait over all the streams.
void build_lists_multi(const std::vector<ListJob> &jobs, const Params &prm) {
    const size_t nj = jobs.size();
    if (!nj) return;
    std::vector<std::unique_ptr<ListBuild>> lbs;
    for (size_t j = 0; j < nj; ++j) lbs.emplace_back(new ListBuild());
    std::vector<double> reach(nj, 0.0), hmax(nj, 0.0);
    for (size_t j = 0; j < nj; ++j) {
        const ListJob &jb = jobs[j];
        // the FP64 direct sum takes one target per lane: at most 32 per item
        jb.P->p2p_tile = prm.precision == PB_MIXED ? prm.p2p_tile : std::min(prm.p2p_tile, 32);
        far_count(*jb.P, *jb.G, *jb.T, jb.src, prm, *lbs[j], jb.s);
    }
    {
        HostReads rd(jobs[0].s);
        std::vector<const int64_t *> hm(nj), hp(nj);
        std::vector<const unsigned long long *> hr(nj);
        for (size_t j = 0; j < nj; ++j) {
            const ListJob &jb = jobs[j];
            hm[j] = rd.add_on(jb.s, jb.P->m2p_ptr.p + jb.G->n);
            hp[j] = rd.add_on(jb.s, jb.P->p2p_ptr.p + jb.G->n);
            hr[j] = rd.add_on(jb.s, lbs[j]->reach->p, 2);
        }
        rd.wait();
        for (size_t j = 0; j < nj; ++j) {
            jobs[j].P->n_m2p = *hm[j];
            jobs[j].P->n_p2p = *hp[j];
            std::memcpy(&reach[j], &hr[j][0], sizeof(double));
            std::memcpy(&hmax[j], &hr[j][1], sizeof(double));
        }
    }
    // the near lists of a pair on its helper stream, beside its list grouping
    struct Events {
        std::vector<cudaEvent_t> e;
        ~Events() {
            for (cudaEvent_t x : e) cudaEventDestroy(x);
        }
    } ev;
    for (size_t j = 0; j < 2 * nj; ++j) {
        cudaEvent_t x = nullptr;
        PB_CUDA_TRY(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        ev.e.push_back(x);
    }
    for (size_t j = 0; j < nj; ++j) {
        const ListJob &jb = jobs[j];
        const cudaStream_t hs = jb.helper ? jb.helper : jb.s;
        far_fill(*jb.P, *jb.G, *jb.T, prm, jb.P->p2p_tile, *lbs[j], jb.s, hs != jb.s ? ev.e[2 * j] : nullptr);
        if (hs != jb.s) PB_CUDA_TRY(cudaStreamWaitEvent(hs, ev.e[2 * j], 0));
        near_count(*jb.P, *jb.G, *jb.T, *jb.src, prm, jb.use_self, hmax[j], *lbs[j], hs);
        if (hs != jb.s) {
            PB_CUDA_TRY(cudaEventRecord(ev.e[2 * j + 1], hs));
            PB_CUDA_TRY(cudaStreamWaitEvent(jb.s, ev.e[2 * j + 1], 0));
        }
    }
    std::vector<int32_t> ovf(nj, 0);
    {
        HostReads rd(jobs[0].s);
        std::vector<const int64_t *> hpi(nj), hmi(nj), hnn(nj);
        std::vector<const int32_t *> hov(nj);
        std::vector<const unsigned long long *> hst(nj);
        for (size_t j = 0; j < nj; ++j) {
            const ListJob &jb = jobs[j];
            ListBuild &lb = *lbs[j];
            hpi[j] = rd.add_on(jb.s, lb.gp.ioff->p + lb.gp.nkeys);
            hmi[j] = rd.add_on(jb.s, lb.gm.ioff->p + lb.gm.nkeys);
            hov[j] = rd.add_on(jb.s, lb.ovf->p);
            hnn[j] = rd.add_on(jb.s, jb.P->near_ptr.p + jb.G->n);
            hst[j] = rd.add_on(jb.s, jb.P->stats.p, 4);
        }
        rd.wait();
        for (size_t j = 0; j < nj; ++j) {
            Pair &Pr = *jobs[j].P;
            apply_list_stats(Pr, hst[j]);
            Pr.n_p2p_items = *hpi[j];
            Pr.n_m2p_items = *hmi[j];
            Pr.n_near = jobs[j].G->n ? *hnn[j] : 0;
            ovf[j] = *hov[j];
        }
    }
    for (size_t j = 0; j < nj; ++j) {
        const ListJob &jb = jobs[j];
        Pair &Pr = *jb.P;
        ListBuild &lb = *lbs[j];
        group_fill(lb.gp, Pr.n_p2p_items, Pr.p2p_items, jb.s);
        bucket_p2p_items(Pr, *jb.T, prm.ncrit, Pr.p2p_tile, jb.s);
        group_fill(lb.gm, Pr.n_m2p_items, Pr.m2p_items, jb.s);
        near_fill(Pr, *jb.G, *jb.T, *jb.src, prm, jb.use_self, reach[j], ovf[j] != 0, lb,
                  jb.helper ? jb.helper : jb.s);
    }
    // the temporaries go back on their own streams, in reverse order of creation
    while (!lbs.empty()) lbs.pop_back();
}

void build_far_lists(Pair &Pr, const Targets &G, const Tree &T, const Params &prm, cudaStream_t s, int p2p_per_item) {
    const int64_t m = G.n;
    ListBuild lb;
    double reach = 0.0, hmax = 0.0;
    Pr.p2p_tile = p2p_per_item;
    far_count(Pr, G, T, nullptr, prm, lb, s);
    read_far_counts(Pr, lb, m, &reach, &hmax, s);
    far_fill(Pr, G, T, prm, p2p_per_item, lb, s);
    HostReads rd(s);
    const int64_t *hpi = rd.add(lb.gp.ioff->p + lb.gp.nkeys);
    const int64_t *hmi = rd.add(lb.gm.ioff->p + lb.gm.nkeys);
    const unsigned long long *hst = rd.add(Pr.stats.p, 4);
    rd.wait();
    apply_list_stats(Pr, hst);
    Pr.n_p2p_items = *hpi;
    Pr.n_m2p_items = *hmi;
    group_fill(lb.gp, Pr.n_p2p_items, Pr.p2p_items, s);
    bucket_p2p_items(Pr, T, prm.ncrit, p2p_per_item, s);
    group_fill(lb.gm, Pr.n_m2p_items, Pr.m2p_items, s);
}

}  // namespace pb
