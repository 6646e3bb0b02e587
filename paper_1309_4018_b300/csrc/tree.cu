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

#include "model.cuh"
#include "tree.cuh"

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

__global__ void bbox_final_kernel(const double *__restrict__ part, int nb, double *__restrict__ out) {
    if (threadIdx.x != 0) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], part[6 * b + a]);
            hi[a] = fmax(hi[a], part[6 * b + 3 + a]);
        }
    for (int a = 0; a < 3; ++a) { out[a] = lo[a]; out[3 + a] = hi[a]; }
}

__device__ __forceinline__ uint64_t spread3(uint64_t v) {
    uint64_t r = 0;
    for (int b = 0; b < 21; ++b) r |= ((v >> b) & 1ull) << (3 * b);
    return r;
}

__global__ void morton_kernel(const double *__restrict__ p, int64_t n, double cx, double cy, double cz,
                              double scale, uint64_t *__restrict__ keys, int32_t *__restrict__ idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double c[3] = {cx, cy, cz};
    uint64_t q[3];
    for (int a = 0; a < 3; ++a) {
        double f = floor(__dmul_rn(__dsub_rn(p[3 * i + a], c[a]), scale));
        f = fmin(fmax(f, 0.0), 2097151.0);
        q[a] = (uint64_t)f;
    }
    keys[i] = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    idx[i] = (int32_t)i;
}

// For every node of one level: count the non-empty octants of the nodes that split.
// Eight threads per node (consecutive lanes), thread o (1..8) finding the first
// position of the node's keys whose octant digit is >= o by binary search; the
// node's child count is the number of non-empty octants (a ballot over the
// eight lanes).  Nodes of fewer than ncrit points, or at the deepest level,
// do not split.
__global__ void split_count_kernel(int lvl, int nb, int nodes_begin, const int64_t *__restrict__ start,
                                   const int64_t *__restrict__ count, const uint64_t *__restrict__ keys, int ncrit,
                                   int32_t *__restrict__ nchild, int32_t *__restrict__ child_bounds /*nodes*9*/) {
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int t = (int)(gt >> 3), o = (int)(gt & 7) + 1;
    const bool act = t < nb;
    const int b = nodes_begin + t;
    int64_t c = 0, lo = 0;
    bool split = false;
    if (act) {
        c = count[b];
        split = c >= ncrit && lvl < kMaxLevel;
        if (split) {
            const int64_t s = start[b];
            const int sh = 3 * (kMaxLevel - 1 - lvl);
            int64_t hi = c;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int d = (int)((keys[s + mid] >> sh) & 7ull);
                if (d < o) lo = mid + 1; else hi = mid;
            }
        }
    }
    const int64_t up = __shfl_up_sync(0xffffffffu, lo, 1);
    const int64_t prev = o == 1 ? 0 : up;
    const unsigned nonempty = __ballot_sync(0xffffffffu, split && lo > prev);
    if (!act) return;
    if (split) {
        child_bounds[9 * t + o] = (int32_t)lo;
        if (o == 1) child_bounds[9 * t] = 0;
    }
    if (o == 1) nchild[b] = split ? __popc((nonempty >> (lane & ~7)) & 0xffu) : 0;
}

__global__ void split_write_kernel(int lvl, int nb, int nodes_begin, int nodes_end, const int64_t *__restrict__ cscan,
                                   const int32_t *__restrict__ child_bounds, int64_t *__restrict__ start,
                                   int64_t *__restrict__ count, int32_t *__restrict__ level,
                                   int32_t *__restrict__ first_child, int32_t *__restrict__ nchild,
                                   int32_t *__restrict__ parent, int64_t *__restrict__ ijk /*nodes*3*/) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nb) return;
    const int b = nodes_begin + t;
    const int nc = nchild[b];
    if (nc == 0) { first_child[b] = -1; return; }
    int c = nodes_end + (int)cscan[t];
    first_child[b] = c;
    const int64_t s = start[b];
    for (int o = 0; o < 8; ++o) {
        const int64_t cs = child_bounds[9 * t + o], ce = child_bounds[9 * t + o + 1];
        if (ce > cs) {
            start[c] = s + cs;
            count[c] = ce - cs;
            level[c] = lvl + 1;
            parent[c] = b;
            nchild[c] = 0;
            first_child[c] = -1;
            ijk[3 * c + 0] = 2 * ijk[3 * b + 0] + ((o >> 2) & 1);
            ijk[3 * c + 1] = 2 * ijk[3 * b + 1] + ((o >> 1) & 1);
            ijk[3 * c + 2] = 2 * ijk[3 * b + 2] + (o & 1);
            ++c;
        }
    }
}

__global__ void node_geom_kernel(int nnodes, const int32_t *__restrict__ level, const int64_t *__restrict__ ijk,
                                 double cx, double cy, double cz, double side, double *__restrict__ centre,
                                 double *__restrict__ rb2) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnodes) return;
    const double sl = ldexp(side, -level[b]);
    const double c[3] = {cx, cy, cz};
    for (int a = 0; a < 3; ++a)
        centre[3 * b + a] = __dadd_rn(c[a], __dmul_rn(__dadd_rn((double)ijk[3 * b + a], 0.5), sl));
    rb2[b] = __dmul_rn(__dmul_rn(sl, sl), 0.75);
}

// Per node: (parent, the parent's first child, the parent's child count, 0);
// (-1, 0, 0, 0) at the root.  One record per level of the upward climb.
__global__ void link_kernel(int nnodes, const int32_t *__restrict__ parent, const int32_t *__restrict__ first_child,
                            const int32_t *__restrict__ nchild, int4 *__restrict__ link) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nnodes) return;
    const int p = parent[i];
    link[i] = p >= 0 ? make_int4(p, first_child[p], nchild[p], 0) : make_int4(-1, 0, 0, 0);
}

__global__ void centre32_kernel(int nnodes, const double *__restrict__ centre, const double *__restrict__ rb2,
                                double ox, double oy, double oz, float4 *__restrict__ cen32) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnodes) return;
    cen32[b] = make_float4((float)(centre[3 * b] - ox), (float)(centre[3 * b + 1] - oy), (float)(centre[3 * b + 2] - oz),
                           (float)rb2[b]);
}

__global__ void leaf_flag_kernel(int nnodes, const int32_t *__restrict__ nchild, const int64_t *__restrict__ start,
                                 int32_t *__restrict__ head /*npts*/) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnodes) return;
    if (nchild[b] == 0) head[start[b]] = 1;
}

__global__ void leaf_index_kernel(int nnodes, const int32_t *__restrict__ nchild, const int64_t *__restrict__ start,
                                  const int64_t *__restrict__ count, const int64_t *__restrict__ hscan,
                                  const int32_t *__restrict__ perm, int32_t *__restrict__ node_leaf,
                                  int32_t *__restrict__ leaf_node, int32_t *__restrict__ point_leaf) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nnodes) return;
    if (nchild[b] != 0) { node_leaf[b] = -1; return; }
    const int li = (int)hscan[start[b]];
    node_leaf[b] = li;
    leaf_node[li] = b;
    for (int64_t q = start[b]; q < start[b] + count[b]; ++q) point_leaf[perm[q]] = li;
}

__global__ void gather_sources_kernel(int64_t n, int K, const int32_t *__restrict__ perm, const double *__restrict__ gy,
                                      const double *__restrict__ gwa, double ox, double oy, double oz,
                                      double *__restrict__ ys, double *__restrict__ was, int32_t *__restrict__ pids,
                                      float4 *__restrict__ pos32) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
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
                                int32_t *__restrict__ err, int nsplit) {
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
            if (sp + nc > kStack) { atomicExch(err, 1); return; }
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
__global__ void owner_kernel(int64_t m, const int64_t *__restrict__ ptr, int32_t *__restrict__ owner) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    for (int64_t e = ptr[t]; e < ptr[t + 1]; ++e) owner[e] = (int32_t)t;
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

__global__ void item_fill_kernel(int nkeys, const int64_t *__restrict__ off, const int64_t *__restrict__ ioff, int per,
                                 int4 *__restrict__ items) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    const int64_t c = off[k + 1] - off[k];
    for (int64_t w = 0; per * w < c; ++w)
        items[ioff[k] + w] = make_int4(k, (int)(off[k] + per * w), (int)(c - per * w < per ? c - per * w : per), 0);
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
                                 const double *__restrict__ cen, const double *__restrict__ L,
                                 int32_t *__restrict__ order, float4 *__restrict__ cpan, dvec4 *__restrict__ cgeo) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int c = cellof[j];
    const int64_t q = off[c] + atomicAdd(cursor + c, 1);
    order[q] = (int32_t)j;
    cpan[q] = pan32[j];
    cgeo[q] = dvec4{cen[3 * j], cen[3 * j + 1], cen[3 * j + 2], L[j]};
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
    int32_t *__restrict__ ncount, int32_t *__restrict__ excl, int32_t *__restrict__ self_excl,
    int32_t *__restrict__ rows, int32_t *__restrict__ overflow) {
    __shared__ int32_t sleaf[4][kNearLeafStage];
    __shared__ int32_t scell[4][27];
    __shared__ int64_t sbase[4][27];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * 4 + warp;
    if (i >= ntg) return;
    const double x = xs[3 * i], y = xs[3 * i + 1], z = xs[3 * i + 2];
    const float fx = (float)(x - ox), fy = (float)(y - oy), fz = (float)(z - oz);
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
            if (dx * dx + dy * dy + dz * dz < pc.w && j != me) {
                // is_near with the panel's centroid and L from its cell-ordered copy
                const dvec4 cg = cgeo[q];
                const double ddx = __dsub_rn(x, cg.x), ddy = __dsub_rn(y, cg.y), ddz = __dsub_rn(z, cg.z);
                const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
                const double tl = __dmul_rn(tt, cg.w);
                if (d2 < __dmul_rn(tl, tl)) {
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

int64_t device_sum_i32(const int32_t *a, int64_t n, cudaStream_t s) {
    TmpBuf<unsigned long long> d(1, s);
    PB_CUDA_TRY(cudaMemsetAsync(d.p, 0, sizeof(unsigned long long), s));
    if (n > 0) {
        sum_i32_kernel<<<std::min<int64_t>(1024, div_up(n, 256)), 256, 0, s>>>(a, n, d.p);
        PB_LAUNCH_CHECK();
    }
    unsigned long long h = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&h, d.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    return (int64_t)h;
}

void root_cube_from(const double *d_points, int64_t n, cudaStream_t s, double corner[3], double &side) {
    TmpBuf<double> bb(6, s);
    const int nb = (int)std::min<int64_t>(256, std::max<int64_t>(1, (n + 4095) / 4096));
    TmpBuf<double> part(6 * nb, s);
    bbox_blocks_kernel<<<nb, 256, 0, s>>>(d_points, n, part.p);
    PB_LAUNCH_CHECK();
    bbox_final_kernel<<<1, 32, 0, s>>>(part.p, nb, bb.p);
    PB_LAUNCH_CHECK();
    double h[6];
    PB_CUDA_TRY(cudaMemcpyAsync(h, bb.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    // plain IEEE double arithmetic, one operation per statement (the host is
    // compiled without contraction)
    double centre[3], ext[3];
    for (int a = 0; a < 3; ++a) {
        centre[a] = (h[a] + h[3 + a]) * 0.5;
        ext[a] = h[3 + a] - h[a];
    }
    const double m = std::max(std::max(ext[0], ext[1]), ext[2]);
    side = m * (1.0 + 0x1p-20);
    if (side == 0.0 || !std::isfinite(side)) side = 1.0;
    for (int a = 0; a < 3; ++a) {
        const double half = side * 0.5;
        corner[a] = centre[a] - half;
    }
}

}  // namespace

int64_t read_i64(const int64_t *d, cudaStream_t s) {
    int64_t h = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    return h;
}

void morton_sort(const double *d_points, int64_t n, cudaStream_t s, double corner[3], double &side,
                 DevBuf<uint64_t> &keys, DevBuf<int32_t> &perm) {
    root_cube_from(d_points, n, s, corner, side);
    keys.alloc(n);
    perm.alloc(n);
    const double scale = 2097152.0 / side;
    if (n) {
        morton_kernel<<<div_up(n, 256), 256, 0, s>>>(d_points, n, corner[0], corner[1], corner[2], scale, keys.p, perm.p);
        PB_LAUNCH_CHECK();
        sort_key_index(keys.p, perm.p, n, s);
    }
}

void build_tree(Tree &T, const SurfDev &S, int K, int ncrit, cudaStream_t s) {
    build_tree_points(T, S.gy.p, S.gwa.p, S.n * K, K, ncrit, s);
}

void build_tree_points(Tree &T, const double *pts, const double *wts, int64_t n, int K, int ncrit, cudaStream_t s) {
    T.npts = n;
    morton_sort(pts, n, s, T.corner, T.side, T.keys, T.perm);
    for (int a = 0; a < 3; ++a) T.origin[a] = T.corner[a] + 0.5 * T.side;
    // level-by-level splitting; capacity bound: every level holds disjoint nodes
    const int64_t maxn = std::min<int64_t>((int64_t)1 + 8LL * (kMaxLevel + 1) * (n / std::max(1, ncrit) + 1),
                                           2 * n + 64);
    T.level.alloc(maxn); T.first_child.alloc(maxn); T.nchild.alloc(maxn); T.parent.alloc(maxn);
    T.start.alloc(maxn); T.count.alloc(maxn);
    TmpBuf<int64_t> ijk(3 * maxn, s);
    {
        int32_t l0 = 0, fc = -1, nc = 0, par = -1;
        int64_t st = 0, ct = n, z3[3] = {0, 0, 0};
        PB_CUDA_TRY(cudaMemcpyAsync(T.level.p, &l0, 4, cudaMemcpyHostToDevice, s));
        PB_CUDA_TRY(cudaMemcpyAsync(T.first_child.p, &fc, 4, cudaMemcpyHostToDevice, s));
        PB_CUDA_TRY(cudaMemcpyAsync(T.nchild.p, &nc, 4, cudaMemcpyHostToDevice, s));
        PB_CUDA_TRY(cudaMemcpyAsync(T.parent.p, &par, 4, cudaMemcpyHostToDevice, s));
        PB_CUDA_TRY(cudaMemcpyAsync(T.start.p, &st, 8, cudaMemcpyHostToDevice, s));
        PB_CUDA_TRY(cudaMemcpyAsync(T.count.p, &ct, 8, cudaMemcpyHostToDevice, s));
        PB_CUDA_TRY(cudaMemcpyAsync(ijk.p, z3, 24, cudaMemcpyHostToDevice, s));
        PB_CUDA_TRY(cudaStreamSynchronize(s));
    }
    T.level_off.assign(1, 0);
    int lb = 0, le = 1, lvl = 0;
    while (true) {
        T.level_off.push_back(le);
        const int nb = le - lb;
        TmpBuf<int32_t> bounds((size_t)nb * 9, s);
        TmpBuf<int64_t> cscan(nb + 1, s);
        split_count_kernel<<<div_up((int64_t)nb * 8, 128), 128, 0, s>>>(lvl, nb, lb, T.start.p, T.count.p, T.keys.p,
                                                                         ncrit, T.nchild.p, bounds.p);
        PB_LAUNCH_CHECK();
        exclusive_scan_i32_to_i64(T.nchild.p + lb, cscan.p, nb, s);
        const int64_t nnew = read_i64(cscan.p + nb, s);
        if (le + nnew > maxn) fail(PB_ENOMEM, "octree node capacity exceeded");
        split_write_kernel<<<div_up(nb, 128), 128, 0, s>>>(lvl, nb, lb, le, cscan.p, bounds.p, T.start.p, T.count.p,
                                                           T.level.p, T.first_child.p, T.nchild.p, T.parent.p, ijk.p);
        PB_LAUNCH_CHECK();
        if (nnew == 0) break;
        lb = le;
        le = le + (int)nnew;
        ++lvl;
    }
    T.nnodes = le;
    T.nlevels = lvl + 1;
    T.centre.alloc(3 * (size_t)T.nnodes);
    T.rb2.alloc(T.nnodes);
    node_geom_kernel<<<div_up(T.nnodes, 128), 128, 0, s>>>(T.nnodes, T.level.p, ijk.p, T.corner[0], T.corner[1],
                                                           T.corner[2], T.side, T.centre.p, T.rb2.p);
    PB_LAUNCH_CHECK();
    T.link.alloc(T.nnodes);
    link_kernel<<<div_up(T.nnodes, 128), 128, 0, s>>>(T.nnodes, T.parent.p, T.first_child.p, T.nchild.p, T.link.p);
    PB_LAUNCH_CHECK();
    T.cen32.alloc(T.nnodes);
    centre32_kernel<<<div_up(T.nnodes, 128), 128, 0, s>>>(T.nnodes, T.centre.p, T.rb2.p, T.origin[0], T.origin[1],
                                                          T.origin[2], T.cen32.p);
    PB_LAUNCH_CHECK();
    // leaves in Morton order (= depth-first pre-order)
    TmpBuf<int32_t> head(n, s);
    TmpBuf<int64_t> hscan(n + 1, s);
    PB_CUDA_TRY(cudaMemsetAsync(head.p, 0, n * sizeof(int32_t), s));
    leaf_flag_kernel<<<div_up(T.nnodes, 128), 128, 0, s>>>(T.nnodes, T.nchild.p, T.start.p, head.p);
    PB_LAUNCH_CHECK();
    exclusive_scan_i32_to_i64(head.p, hscan.p, n, s);
    T.nleaves = (int)read_i64(hscan.p + n, s);
    T.node_leaf.alloc(T.nnodes);
    T.leaf_node.alloc(T.nleaves);
    T.point_leaf.alloc(n);
    leaf_index_kernel<<<div_up(T.nnodes, 128), 128, 0, s>>>(T.nnodes, T.nchild.p, T.start.p, T.count.p, hscan.p,
                                                            T.perm.p, T.node_leaf.p, T.leaf_node.p, T.point_leaf.p);
    PB_LAUNCH_CHECK();
    // sorted source geometry
    T.ys.alloc(3 * n); T.was.alloc(n); T.pids.alloc(n); T.pos32.alloc(n);
    gather_sources_kernel<<<div_up(n, 256), 256, 0, s>>>(n, K, T.perm.p, pts, wts, T.origin[0], T.origin[1],
                                                         T.origin[2], T.ys.p, T.was.p, T.pids.p, T.pos32.p);
    PB_LAUNCH_CHECK();
    T.src64.alloc(8 * n); T.srcA32.alloc(n); T.srcB32.alloc(n);
}

void build_targets(Targets &G, const double *d_x, int64_t n, int surface, cudaStream_t s, int points_per_panel) {
    G.n = n;
    G.surface = surface;
    double corner[3], side;
    morton_sort(d_x, n, s, corner, side, G.keys, G.order);
    G.xs.alloc(3 * n);
    G.self_panel.alloc(n);
    G.rank.alloc(n);
    if (n) {
        gather_targets_kernel<<<div_up(n, 256), 256, 0, s>>>(n, G.order.p, d_x, G.xs.p, G.self_panel.p, G.rank.p,
                                                             surface >= 0 ? points_per_panel : 0);
        PB_LAUNCH_CHECK();
    }
    PB_CUDA_TRY(cudaStreamSynchronize(s));
}

void build_lists(Pair &Pr, const Targets &G, const Tree &T, const SurfDev &src, const Params &prm, bool use_self,
                 cudaStream_t s) {
    build_far_lists(Pr, G, T, prm, s, prm.p2p_tile);
    build_near_lists(Pr, G, T, src, prm, use_self, s);
}

void build_far_lists(Pair &Pr, const Targets &G, const Tree &T, const Params &prm, cudaStream_t s, int p2p_per_item) {
    const int64_t m = G.n;
    // every target traverses the root's eight subtrees as eight threads (eight times
    // the parallelism for the charges, shorter serial walks for the panels)
    const int nsplit = 8;
    const int64_t ms = m * nsplit;
    TmpBuf<int32_t> mc(ms, s), pc(ms, s), err(1, s);
    TmpBuf<int64_t> mo(nsplit > 1 ? ms + 1 : 0, s), po(nsplit > 1 ? ms + 1 : 0, s);
    PB_CUDA_TRY(cudaMemsetAsync(err.p, 0, 4, s));
    const double theta2 = prm.theta * prm.theta;
    const int direct = prm.theta <= 0.0;
    Pr.m2p_ptr.alloc(m + 1);
    Pr.p2p_ptr.alloc(m + 1);
    if (m) {
        traverse_kernel<false><<<div_up(ms, 128), 128, 0, s>>>(m, G.xs.p, T.centre.p, T.rb2.p, T.cen32.p,
                                                               T.first_child.p, T.nchild.p, theta2, direct, T.origin[0],
                                                               T.origin[1], T.origin[2], mc.p, pc.p, nullptr, nullptr,
                                                               nullptr, nullptr, err.p, nsplit);
        PB_LAUNCH_CHECK();
    }
    int64_t *moff = Pr.m2p_ptr.p, *poff = Pr.p2p_ptr.p;
    if (nsplit > 1) {
        exclusive_scan_i32_to_i64(mc.p, mo.p, ms, s);
        exclusive_scan_i32_to_i64(pc.p, po.p, ms, s);
        take_every_kernel<<<div_up(m + 1, 256), 256, 0, s>>>(m, nsplit, mo.p, Pr.m2p_ptr.p);
        PB_LAUNCH_CHECK();
        take_every_kernel<<<div_up(m + 1, 256), 256, 0, s>>>(m, nsplit, po.p, Pr.p2p_ptr.p);
        PB_LAUNCH_CHECK();
        moff = mo.p;
        poff = po.p;
    } else {
        exclusive_scan_i32_to_i64(mc.p, Pr.m2p_ptr.p, m, s);
        exclusive_scan_i32_to_i64(pc.p, Pr.p2p_ptr.p, m, s);
    }
    Pr.n_m2p = read_i64(Pr.m2p_ptr.p + m, s);
    Pr.n_p2p = read_i64(Pr.p2p_ptr.p + m, s);
    Pr.m2p_node.alloc(std::max<int64_t>(1, Pr.n_m2p));
    Pr.p2p_node.alloc(std::max<int64_t>(1, Pr.n_p2p));
    if (m) {
        traverse_kernel<true><<<div_up(ms, 128), 128, 0, s>>>(m, G.xs.p, T.centre.p, T.rb2.p, T.cen32.p,
                                                              T.first_child.p, T.nchild.p, theta2, direct, T.origin[0],
                                                              T.origin[1], T.origin[2], nullptr, nullptr, moff, poff,
                                                              Pr.m2p_node.p, Pr.p2p_node.p, err.p, nsplit);
        PB_LAUNCH_CHECK();
    }
    int herr = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&herr, err.p, 4, cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr) fail(PB_EINVAL, "octree traversal stack overflow");
    // direct-sum pair count
    {
        TmpBuf<unsigned long long> d(1, s);
        PB_CUDA_TRY(cudaMemsetAsync(d.p, 0, 8, s));
        if (m) {
            p2p_pairs_kernel<<<std::min<int64_t>(1024, div_up(m, 256)), 256, 0, s>>>(m, Pr.p2p_ptr.p, Pr.p2p_node.p,
                                                                                    T.count.p, d.p);
            PB_LAUNCH_CHECK();
        }
        unsigned long long h = 0;
        PB_CUDA_TRY(cudaMemcpyAsync(&h, d.p, 8, cudaMemcpyDeviceToHost, s));
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        Pr.p2p_pairs = (int64_t)h;
    }
    // entry-major grouping of the lists
    auto group = [&](const int64_t *ptr, const int32_t *ent, const int32_t *remap, int nkeys, int64_t nent, int per,
                     int by_entry,
                     DevBuf<int32_t> &inv, DevBuf<int32_t> &pos, DevBuf<int4> &items, int64_t &nitems) {
        TmpBuf<int32_t> cnt(std::max(1, nkeys), s), cursor(std::max(1, nkeys), s), nit(std::max(1, nkeys), s);
        TmpBuf<int64_t> off(nkeys + 1, s), ioff(nkeys + 1, s);
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
            owner_kernel<<<div_up(m, 128), 128, 0, s>>>(m, ptr, owner.p);
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
        exclusive_scan_i32_to_i64(cnt.p, off.p, nkeys, s);
        if (m && nent) {
            if (hist)
                hist_fill_kernel<<<nb, 256, hshm, s>>>(nent, chunk, owner.p, ent, remap, off.p, hb.p, nkeys, by_entry,
                                                       inv.p, pos.p);
            else
                inv_fill_kernel<<<div_up(nent, 256), 256, 0, s>>>(nent, owner.p, ent, remap, off.p, cursor.p, by_entry,
                                                                  inv.p, pos.p);
            PB_LAUNCH_CHECK();
        }
        item_count_kernel<<<div_up(nkeys, 128), 128, 0, s>>>(nkeys, off.p, per, nit.p);
        PB_LAUNCH_CHECK();
        exclusive_scan_i32_to_i64(nit.p, ioff.p, nkeys, s);
        nitems = read_i64(ioff.p + nkeys, s);
        items.alloc(std::max<int64_t>(1, nitems));
        item_fill_kernel<<<div_up(nkeys, 128), 128, 0, s>>>(nkeys, off.p, ioff.p, per, items.p);
        PB_LAUNCH_CHECK();
    };
    group(Pr.p2p_ptr.p, Pr.p2p_node.p, T.node_leaf.p, T.nleaves, Pr.n_p2p, p2p_per_item, 1, Pr.p2p_inv, Pr.p2p_ent,
          Pr.p2p_items,
          Pr.n_p2p_items);
    if (Pr.n_p2p_items > 1) {
        constexpr int nb = 64;
        const int step = std::max(1, prm.ncrit * p2p_per_item / nb);
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
    group(Pr.m2p_ptr.p, Pr.m2p_node.p, nullptr, T.nnodes, Pr.n_m2p, 32, 1, Pr.m2p_inv, Pr.m2p_ent, Pr.m2p_items,
          Pr.n_m2p_items);
}

void build_near_lists(Pair &Pr, const Targets &G, const Tree &T, const SurfDev &src, const Params &prm, bool use_self,
                      cudaStream_t s) {
    const int64_t m = G.n;
    // P2P leaf indices per target (ascending = pre-order)
    TmpBuf<int32_t> pleaf(std::max<int64_t>(1, Pr.n_p2p), s);
    if (Pr.n_p2p) {
        node_to_leaf_kernel<<<div_up(Pr.n_p2p, 256), 256, 0, s>>>(Pr.n_p2p, Pr.p2p_node.p, T.node_leaf.p, pleaf.p);
        PB_LAUNCH_CHECK();
    }
    // near-singular lists
    TmpBuf<int32_t> nc(m, s), ex(m, s), se(m, s);
    TmpBuf<unsigned long long> reach_d(2, s);
    PB_CUDA_TRY(cudaMemsetAsync(reach_d.p, 0, 2 * sizeof(unsigned long long), s));
    reach_kernel<<<std::min<int64_t>(592, div_up(src.n, 256)), 256, 0, s>>>(src.n, src.verts.p, src.tris.p, src.cen.p,
                                                                           src.L.p, prm.thres, reach_d.p);
    PB_LAUNCH_CHECK();
    unsigned long long rbits[2] = {0, 0};
    PB_CUDA_TRY(cudaMemcpyAsync(rbits, reach_d.p, sizeof(rbits), cudaMemcpyDeviceToHost, s));
    TmpBuf<float4> pan32(std::max<int64_t>(1, src.n), s);
    pan32_kernel<<<div_up(src.n, 256), 256, 0, s>>>(src.n, src.cen.p, src.L.p, prm.thres, T.origin[0], T.origin[1],
                                                     T.origin[2], pan32.p);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    double reach = 0.0, hmax = 0.0;
    std::memcpy(&reach, &rbits[0], sizeof(reach));
    std::memcpy(&hmax, &rbits[1], sizeof(hmax));
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
    TmpBuf<int64_t> coff(ncell + 1, s);
    PB_CUDA_TRY(cudaMemsetAsync(ccnt.p, 0, ncell * sizeof(int32_t), s));
    PB_CUDA_TRY(cudaMemsetAsync(ccur.p, 0, ncell * sizeof(int32_t), s));
    if (src.n) {
        cell_count_kernel<<<div_up(src.n, 256), 256, 0, s>>>(src.n, src.cen.p, g, cellof.p, ccnt.p);
        PB_LAUNCH_CHECK();
    }
    exclusive_scan_i32_to_i64(ccnt.p, coff.p, ncell, s);
    if (src.n) {
        cell_fill_kernel<<<div_up(src.n, 256), 256, 0, s>>>(src.n, cellof.p, coff.p, ccur.p, pan32.p, src.cen.p,
                                                            src.L.p, corder.p, cpan.p, cgeo.p);
        PB_LAUNCH_CHECK();
    }
    Pr.near_ptr.alloc(m + 1);
    bool done = false;
    if (m) {
        // one pass: counts and a row of panels per target
        TmpBuf<int32_t> rows((size_t)m * kNearCap, s), ovf(1, s);
        PB_CUDA_TRY(cudaMemsetAsync(ovf.p, 0, 4, s));
        near_grid_kernel<<<div_up(m, 4), 128, 0, s>>>(m, prm.K, G.xs.p, G.self_panel.p, (int)use_self, Pr.p2p_ptr.p,
                                                       pleaf.p, T.point_leaf.p, T.origin[0], T.origin[1],
                                                       T.origin[2], prm.thres, g, coff.p, corder.p, cpan.p, cgeo.p,
                                                       nc.p, ex.p, se.p, rows.p, ovf.p);
        PB_LAUNCH_CHECK();
        int hov = 0;
        PB_CUDA_TRY(cudaMemcpyAsync(&hov, ovf.p, 4, cudaMemcpyDeviceToHost, s));
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        exclusive_scan_i32_to_i64(nc.p, Pr.near_ptr.p, m, s);
        Pr.n_near = read_i64(Pr.near_ptr.p + m, s);
        Pr.near_panel.alloc(std::max<int64_t>(1, Pr.n_near));
        if (!hov) {
            near_compact_kernel<<<div_up(m, 128), 128, 0, s>>>(m, rows.p, Pr.near_ptr.p, Pr.near_panel.p);
            PB_LAUNCH_CHECK();
            done = true;
        }
    } else {
        exclusive_scan_i32_to_i64(nc.p, Pr.near_ptr.p, m, s);
        Pr.n_near = 0;
        Pr.near_panel.alloc(1);
        done = true;
    }
    Pr.near_excl = device_sum_i32(ex.p, m, s);
    Pr.self_excl = device_sum_i32(se.p, m, s);
    if (!done) {
        // some target has more than kNearCap near panels: fill the CSR list in a second pass
        TmpBuf<float4> ppan32(std::max<int64_t>(1, T.npts), s);
        if (T.npts) {
            point_pan32_kernel<<<div_up(T.npts, 256), 256, 0, s>>>(T.npts, T.pids.p, pan32.p, ppan32.p);
            PB_LAUNCH_CHECK();
        }
        near_kernel<1><<<div_up(m, 4), 128, 0, s>>>(m, prm.K, G.xs.p, G.self_panel.p, (int)use_self, Pr.p2p_ptr.p,
                                                    pleaf.p, T.leaf_node.p, T.start.p, T.count.p, T.perm.p, T.pids.p,
                                                    T.point_leaf.p, src.cen.p, src.L.p, ppan32.p, T.origin[0],
                                                    T.origin[1], T.origin[2], prm.thres, nullptr, nullptr, nullptr,
                                                    Pr.near_ptr.p, Pr.near_panel.p, Pr.m2p_ptr.p, Pr.m2p_node.p,
                                                    T.cen32.p, reach, nullptr, nullptr);
        PB_LAUNCH_CHECK();
    }
    PB_CUDA_TRY(cudaStreamSynchronize(s));
}

}  // namespace pb
