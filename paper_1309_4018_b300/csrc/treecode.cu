// Treecode evaluation kernels: one application of the BEM operator (Sec. 2.3,
// Eqs. nbody, taylor, multexp, MAC; "Treecode-accelerated BEM").
//
// Sources are the Gauss points y_p of the panels of one surface, with
// single-layer strength s_p = w_p A_j dphi_j and double-layer dipole
// d_p = w_p A_j phi_j n_j.  For a target x and kernel G (Laplace 1/(4 pi r) or
// Yukawa exp(-kappa r)/(4 pi r)) every block sum is split into
//   V(x) = sum_p s_p G(x, y_p)            K(x) = sum_p d_p . grad_y G(x, y_p)
// evaluated by direct summation over the leaves that fail the MAC (P2P) and
// by the Taylor expansion sum_k a^k M^k, sum_k a^k D^k over the accepted boxes
// (M2P), with M^k = sum_p s_p (y_p - y_c)^k and
// D^k = sum_p sum_l d_{p,l} k_l (y_p - y_c)^(k - e_l) (P2M at the leaves,
// M2M shifts towards the root).
//
// The Taylor coefficients a^k = (1/k!) D_y^k G(x, y_c) follow from the
// recurrences (u = y_c - x, r = |u|, n = |k|; b^k the coefficients of
// exp(-kappa r); both start from a^0 = exp(-kappa r)/r, b^0 = exp(-kappa r)):
//   n r^2 a^k = -(2n-1) sum_j u_j a^(k-e_j) - (n-1) sum_j a^(k-2e_j)
//               - kappa (sum_j u_j b^(k-e_j) + sum_j b^(k-2e_j))
//   n b^k     = -kappa (sum_j u_j a^(k-e_j) + sum_j a^(k-2e_j))
// obtained by taking Taylor coefficients of r^2 d_j G = -u_j (G + kappa H),
// d_j H = -kappa u_j G (H = exp(-kappa r)); with kappa = 0 this is the Laplace
// recurrence of Duan & Krasny, with kappa > 0 the screened-Coulomb form of
// Li, Johnston & Krasny that the paper cites.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <type_traits>

#include "treecode.cuh"
#include "radial.cuh"

namespace pb {

namespace {

__constant__ int c_terms[3 * kMaxTerms1];   // (k1, k2, k3) of every term up to order kMaxP + 1, graded order
__constant__ double c_binom[13][13];
__constant__ float c_binom32[13][13];   // the same integers in FP32 (exact)


__host__ __device__ constexpr int term_index(int k1, int k2, int k3) {
    // graded by n = |k|, then k1 descending, then k2 descending
    return (k1 + k2 + k3) * (k1 + k2 + k3 + 1) * (k1 + k2 + k3 + 2) / 6 + (k2 + k3) * (k2 + k3 + 1) / 2 + k3;
}

// ---------------------------------------------------------------- source strengths
__global__ void strengths64_kernel(int64_t n, const double *__restrict__ ys, const double *__restrict__ was,
                                   const int32_t *__restrict__ pids, const double *__restrict__ nrm,
                                   const double *__restrict__ phi, const double *__restrict__ dphi,
                                   double *__restrict__ src) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int j = pids[q];
    const double w = was[q];
    const double f = w * phi[j];
    double *o = src + 8 * q;
    o[0] = ys[3 * q]; o[1] = ys[3 * q + 1]; o[2] = ys[3 * q + 2];
    o[3] = w * dphi[j];
    o[4] = f * nrm[3 * j]; o[5] = f * nrm[3 * j + 1]; o[6] = f * nrm[3 * j + 2];
    o[7] = (double)j;
}

// Also the FP32 copy (phi, dphi) of the ns panel densities (threads q < ns).
__global__ void strengths32_kernel(int64_t n, const float4 *__restrict__ pos, const double *__restrict__ was,
                                   const int32_t *__restrict__ pids, const double *__restrict__ nrm,
                                   const double *__restrict__ phi, const double *__restrict__ dphi,
                                   float4 *__restrict__ A, float4 *__restrict__ B, int64_t ns,
                                   float2 *__restrict__ phf) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < ns) phf[q] = make_float2((float)phi[q], (float)dphi[q]);
    if (q >= n) return;
    const int j = pids[q];
    const double w = was[q];
    const double f = w * phi[j];
    const float4 p = pos[q];
    A[q] = make_float4(p.x, p.y, p.z, (float)(w * dphi[j]));
    B[q] = make_float4((float)(f * nrm[3 * j]), (float)(f * nrm[3 * j + 1]), (float)(f * nrm[3 * j + 2]),
                       __int_as_float(j));
}

// FP32 copies of (phi, dphi) per panel, read by the mixed-precision gather's
// near-field terms (one conversion per panel instead of one per near entry).
// ---------------------------------------------------------------- P2M (leaves)
template <typename T>
struct SrcView;

template <>
struct SrcView<double> {
    const double *src;
    __device__ void get(int64_t q, const double c[3], double &x, double &y, double &z, double &s, double &dx,
                        double &dy, double &dz) const {
        const double *o = src + 8 * q;
        x = o[0] - c[0]; y = o[1] - c[1]; z = o[2] - c[2];
        s = o[3]; dx = o[4]; dy = o[5]; dz = o[6];
    }
};

template <>
struct SrcView<float> {
    const float4 *A, *B;
    __device__ void get(int64_t q, const float c[3], float &x, float &y, float &z, float &s, float &dx, float &dy,
                        float &dz) const {
        const float4 a = A[q], b = B[q];
        x = a.x - c[0]; y = a.y - c[1]; z = a.z - c[2];
        s = a.w; dx = b.x; dy = b.y; dz = b.z;
    }
};

constexpr int kP2MChunk = 128;

// Four consecutive shared-memory values as one (float) or two (double) 16-byte loads.
template <typename T>
struct Quad {
    T x, y, z, w;
};
__device__ __forceinline__ Quad<float> ld4(const float *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Quad<double> ld4(const double *p) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    return {a.x, a.y, b.x, b.y};
}

// ---------------------------------------------------------------- M2M (one level, bottom-up)
// M_parent^k = sum_children sum_{l <= k} C(k, l) (y_child - y_parent)^(k-l) M_child^l;
// the dipole moments D shift with the same rule.  The shift factorises by
// axis, so it is applied as three one-dimensional passes (z, then y, then x),
// each output term summing at most P + 1 inputs; a term with |k| <= P only
// reads terms with |l| <= |k|, so the truncated set is closed under the
// passes.  One block per node of the level; the children (contiguous node
// ids) are shifted in parallel in shared memory and added in child order.
constexpr size_t kClimbMaxShared = 220 * 1024;   // dynamic shared memory of the one-launch M2M (227 KB less the static arrays)
constexpr int kM2MMaxShared = 2 * 8 * 2 * 455 * 8 + 3 * 455 * 4;

// Shift the children's moments (src: 8 x nval, child-major, nval = sets x NT;
// the rows of absent children zero) to the parent's centre and add them in
// child order into out[0, nval).  hs[c][ax] = (child c - parent)_ax, sbin =
// binomials.  Each thread owns outputs r (one term k of one set) and, per
// pass, walks the inputs of k along the axis once for all eight children:
// e = 0 .. k_ax with l = k_ax - e, coefficient C(k_ax, l) h^e, the power
// h^e carried in a register (1, h, h h, ... as a running product) and the
// input's index stepped down from k by additions.  No per-child branch, so
// the eight loads of an input are issued together; the last pass adds the
// children's shifted values and stores the sum.  Two barriers; src and dst
// are overwritten.
template <typename T>
__device__ __forceinline__ void shift_children(int NT, int nval, const int *__restrict__ sterm,
                                               const T (*sbin)[kMaxP + 1], const T (*hs)[3], T *src, T *dst,
                                               T *__restrict__ out) {
#pragma unroll
    for (int ax = 2; ax >= 0; --ax) {
        T hh[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) hh[c] = hs[c][ax];
        for (int r = threadIdx.x; r < nval; r += blockDim.x) {
            const int set = r / NT, k = r - set * NT;
            const int k1 = sterm[3 * k], k2 = sterm[3 * k + 1], k3 = sterm[3 * k + 2];
            const int kax = ax == 0 ? k1 : ax == 1 ? k2 : k3;
            // index of k with k_ax = l: T3(n0 + l) + T2(m0 + dm l) + c0 + dc l
            // (T3(n) = n(n+1)(n+2)/6, T2(m) = m(m+1)/2), equal to k at l = k_ax
            const int n = k1 + k2 + k3, n0 = n - kax, m = k2 + k3;
            const int dm = ax == 0 ? 0 : 1, dc = ax == 2 ? 1 : 0;
            int t3 = n * (n + 1) * (n + 2) / 6, w3 = n * (n + 1) / 2;
            int t2 = m * (m + 1) / 2, w2 = m, cc = k3;
            const T *sc = src + set * NT;
            T acc[8], v[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) { acc[c] = 0; v[c] = 1; }
            for (int e = 0; e <= kax; ++e) {
                const int l = kax - e;
                const int li = t3 + t2 + cc;
                t3 -= w3; w3 -= n0 + l;
                t2 -= dm * w2; w2 -= dm;
                cc -= dc;
                const T b = sbin[kax][l];
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    acc[c] += b * v[c] * sc[c * nval + li];
                    v[c] *= hh[c];
                }
            }
            if (ax > 0) {
#pragma unroll
                for (int c = 0; c < 8; ++c) dst[c * nval + r] = acc[c];
            } else {
                T sum = 0;
#pragma unroll
                for (int c = 0; c < 8; ++c) sum += acc[c];
                out[r] = sum;
            }
        }
        if (ax > 0) {
            __syncthreads();
            T *tmp = src; src = dst; dst = tmp;
        }
    }
}

// Each node holds `stride` values; one launch shifts the 2 NT values at
// offset `base` (one (M, D) or two monopole sets).
template <typename T>
__global__ void __launch_bounds__(256) m2m_kernel(int nodes_begin, const int32_t *__restrict__ first_child,
                                                  const int32_t *__restrict__ nchild,
                                                  const double *__restrict__ centre, int P, int NT, int stride,
                                                  int base, T *__restrict__ mom) {
    extern __shared__ __align__(16) unsigned char m2m_smem[];
    T *buf0 = reinterpret_cast<T *>(m2m_smem);          // nc x 2NT
    T *buf1 = buf0 + 8 * 2 * NT;                        // nc x 2NT
    int *sterm = reinterpret_cast<int *>(buf1 + 8 * 2 * NT);
    __shared__ T hs[8][3];
    __shared__ T sbin[kMaxP + 1][kMaxP + 1];
    const int b = nodes_begin + blockIdx.x;
    const int nc = nchild[b];
    if (nc == 0) return;
    const int fc = first_child[b];
    for (int i = threadIdx.x; i < 8 * 2 * NT; i += blockDim.x) {
        const int c = i / (2 * NT), r = i - c * 2 * NT;
        buf0[i] = c < nc ? mom[(int64_t)(fc + c) * stride + base + r] : T(0);
    }
    for (int i = threadIdx.x; i < 3 * NT; i += blockDim.x) sterm[i] = c_terms[i];
    for (int i = threadIdx.x; i < 8 * 3; i += blockDim.x) {
        const int c = i / 3, ax = i - 3 * c;
        hs[c][ax] = c < nc ? (T)(centre[3 * (fc + c) + ax] - centre[3 * b + ax]) : T(0);
    }
    for (int i = threadIdx.x; i < (P + 1) * (P + 1); i += blockDim.x) {
        const int n = i / (P + 1), k = i - n * (P + 1);
        sbin[n][k] = sizeof(T) == 4 ? (T)c_binom32[n][k] : (T)c_binom[n][k];
    }
    __syncthreads();
    shift_children<T>(NT, 2 * NT, sterm, sbin, hs, buf0, buf1, mom + (int64_t)b * stride + base);
}

// ---------------------------------------------------------------- P2P, FP32 (mixed precision)
// Leaf-major work items (below): every leaf's sources are staged 32 at a time
// in shared memory and broadcast to the lanes of a warp, each lane owning one
// target that sums over the leaf.  FP32 partial sums of each 32-source chunk
// are added into (hi, lo) FP32 pairs with Neumaier's compensated summation.
struct KSet {
    float kap[2];
};

// Single-instruction special-function unit approximations (PTX rsqrt.approx,
// ex2.approx, flush-to-zero): relative error ~2^-22, below the FP32 rounding
// of the sums they feed.
__device__ __forceinline__ float fast_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float fast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void comp_add(float &hi, float &lo, float v) {
    const float t = hi + v;
    lo += (fabsf(hi) >= fabsf(v)) ? ((hi - t) + v) : ((v - t) + hi);
    hi = t;
}

// Leaf-major: one warp per work item = one leaf and up to 32 (target, entry)
// pairs that sum over it.  The leaf's sources are staged 32 at a time in
// shared memory and broadcast; every lane owns one target.  FP32 partial sums
// per 32-source chunk go into compensated (hi, lo) pairs; the pair's result is
// the FP32 sum hi + lo, rounded once into an FP32 float2 record (one value per
// row kernel) at its list entry.
// MASK: skip the target's own panel (needed when a rule point sits at the
// centroid); without it the own points stay in and the self value is corrected.
struct P2PArgs32 {
    const int4 *items;                     // (leaf, grouped start, count <= 32, 0)
    const int32_t *inv, *sent;             // grouped pair -> sorted target, list entry
    const float4 *x32;                     // sorted targets (FP32, tree-origin relative)
    const int32_t *selfp;
    int use_self;
    const int32_t *leaf_node;
    const int64_t *start, *count;
    const float4 *A, *B;                   // sorted sources (x, y, z, s) and (d, panel)
    KSet ks;
    float *part;                           // records, 2 NK floats per list entry
};

// The work item `item` on the calling warp; sA, sB: the warp's 32-source staging.
template <int NK, bool Y0, bool Y1, bool MASK>
__device__ __forceinline__ void p2p32_item(const P2PArgs32 &g, int64_t item, int lane, float4 *sA, float4 *sB) {
    const int4 it = g.items[item];
    const bool valid = lane < it.z;
    const int64_t slot = (int64_t)it.y + lane;
    float tx = 0.f, ty = 0.f, tz = 0.f;
    int me = -1;
    if (valid) {
        const int t = g.inv[slot];
        const float4 x = g.x32[t];
        tx = x.x;
        ty = x.y;
        tz = x.z;
        if (MASK && g.use_self) me = g.selfp[t];
    }
    const float k0 = g.ks.kap[0], k1 = g.ks.kap[1];
    const float l2e0 = -k0 * 1.4426950408889634f, l2e1 = -k1 * 1.4426950408889634f;
    float hi[2 * NK], lo[2 * NK];
#pragma unroll
    for (int a = 0; a < 2 * NK; ++a) { hi[a] = 0.f; lo[a] = 0.f; }
    const int node = g.leaf_node[it.x];
    const int64_t s0 = g.start[node];
    const int cnt = (int)g.count[node];
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int m = min(32, cnt - c0);
        if (lane < m) {
            sA[lane] = g.A[s0 + c0 + lane];
            sB[lane] = g.B[s0 + c0 + lane];
        }
        __syncwarp();
        if (valid) {
            float p[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const float4 a = sA[j];
                const float4 b = sB[j];
                const float dx = tx - a.x, dy = ty - a.y, dz = tz - a.z;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float inv = (MASK && __float_as_int(b.w) == me) ? 0.f : fast_rsqrt(r2);
                const float sv = a.w * inv;
                const float rd = fmaf(dx, b.x, fmaf(dy, b.y, dz * b.z));
                const float kv = rd * (inv * inv * inv);
                if (!Y0) {
                    p[0] += sv;
                    p[1] += kv;
                } else {
                    const float rho = r2 * inv;
                    const float ex = fast_ex2(l2e0 * rho);
                    p[0] = fmaf(sv, ex, p[0]);
                    p[1] = fmaf(kv * ex, fmaf(k0, rho, 1.f), p[1]);
                }
                if (NK == 2) {
                    if (!Y1) {
                        p[2] += sv;
                        p[3] += kv;
                    } else {
                        const float rho = r2 * inv;
                        const float ex = fast_ex2(l2e1 * rho);
                        p[2] = fmaf(sv, ex, p[2]);
                        p[3] = fmaf(kv * ex, fmaf(k1, rho, 1.f), p[3]);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 2 * NK; ++a) comp_add(hi[a], lo[a], p[a]);
        }
        __syncwarp();
    }
    if (valid) {
        // interleaved record of the entry: (V0, K0[, V1, K1]), the compensated pair rounded once
        float2 *rec = reinterpret_cast<float2 *>(g.part + (int64_t)2 * NK * g.sent[slot]);
#pragma unroll
        for (int a = 0; a < NK; ++a) rec[a] = make_float2(hi[2 * a] + lo[2 * a], hi[2 * a + 1] + lo[2 * a + 1]);
    }
}

// One target's pair contribution with a staged source (a, b): Laplace or
// Yukawa potential and normal derivative of each kernel, added to p.
template <int NK, bool Y0, bool Y1, bool MASK>
__device__ __forceinline__ void p2p32_pair(float tx, float ty, float tz, int me, const float4 &a, const float4 &b,
                                           float k0, float k1, float l2e0, float l2e1, float p[4]) {
    const float dx = tx - a.x, dy = ty - a.y, dz = tz - a.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float inv = (MASK && __float_as_int(b.w) == me) ? 0.f : fast_rsqrt(r2);
    const float sv = a.w * inv;
    const float rd = fmaf(dx, b.x, fmaf(dy, b.y, dz * b.z));
    const float kv = rd * (inv * inv * inv);
    if (!Y0) {
        p[0] += sv;
        p[1] += kv;
    } else {
        const float rho = r2 * inv;
        const float ex = fast_ex2(l2e0 * rho);
        p[0] = fmaf(sv, ex, p[0]);
        p[1] = fmaf(kv * ex, fmaf(k0, rho, 1.f), p[1]);
    }
    if (NK == 2) {
        if (!Y1) {
            p[2] += sv;
            p[3] += kv;
        } else {
            const float rho = r2 * inv;
            const float ex = fast_ex2(l2e1 * rho);
            p[2] = fmaf(sv, ex, p[2]);
            p[3] = fmaf(kv * ex, fmaf(k1, rho, 1.f), p[3]);
        }
    }
}

// Packed FP32 pairs (f32x2: two lanes' worth of one FP32 operation in one
// instruction on sm_100-family parts).  The FMA pipe takes a pair instruction
// in two cycles, so the FP32 rate is unchanged, but the issue slot between
// them is free for the MUFU, shared-memory and integer instructions: the
// two-targets-per-lane P2P issues about 15 instead of 28 instructions per pair.
// Each is the IEEE round-to-nearest operation of its scalar form.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p f2_make(float lo, float hi) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ float f2_lo(f2p v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return lo;
}
__device__ __forceinline__ float f2_hi(f2p v) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
    return hi;
}
__device__ __forceinline__ f2p f2_sub(f2p a, f2p b) {
    f2p d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p f2_add(f2p a, f2p b) {
    f2p d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p f2_mul(f2p a, f2p b) {
    f2p d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2p f2_fma(f2p a, f2p b, f2p c) {
    f2p d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// The pair contributions of one staged source to two targets (tX.. hold the
// two targets' coordinates), the same operations in the same order as
// p2p32_pair, two at a time.  a*, b* hold the source's values twice.
template <int NK, bool Y0, bool Y1, bool MASK>
__device__ __forceinline__ void p2p32_pair2(f2p tX, f2p tY, f2p tZ, int me0, int me1, f2p aX, f2p aY, f2p aZ,
                                            f2p aW, f2p bX, f2p bY, f2p bZ, int pid, f2p k0, f2p k1, f2p l2e0,
                                            f2p l2e1, f2p one, f2p p[4]) {
    const f2p dX = f2_sub(tX, aX), dY = f2_sub(tY, aY), dZ = f2_sub(tZ, aZ);
    const f2p R2 = f2_fma(dX, dX, f2_fma(dY, dY, f2_mul(dZ, dZ)));
    const float i0 = (MASK && pid == me0) ? 0.f : fast_rsqrt(f2_lo(R2));
    const float i1 = (MASK && pid == me1) ? 0.f : fast_rsqrt(f2_hi(R2));
    const f2p INV = f2_make(i0, i1);
    const f2p SV = f2_mul(aW, INV);
    const f2p RD = f2_fma(dX, bX, f2_fma(dY, bY, f2_mul(dZ, bZ)));
    const f2p KV = f2_mul(RD, f2_mul(f2_mul(INV, INV), INV));
    if (!Y0) {
        p[0] = f2_add(p[0], SV);
        p[1] = f2_add(p[1], KV);
    } else {
        const f2p RHO = f2_mul(R2, INV);
        const f2p ARG = f2_mul(l2e0, RHO);
        const f2p EX = f2_make(fast_ex2(f2_lo(ARG)), fast_ex2(f2_hi(ARG)));
        p[0] = f2_fma(SV, EX, p[0]);
        p[1] = f2_fma(f2_mul(KV, EX), f2_fma(k0, RHO, one), p[1]);
    }
    if (NK == 2) {
        if (!Y1) {
            p[2] = f2_add(p[2], SV);
            p[3] = f2_add(p[3], KV);
        } else {
            const f2p RHO = f2_mul(R2, INV);
            const f2p ARG = f2_mul(l2e1, RHO);
            const f2p EX = f2_make(fast_ex2(f2_lo(ARG)), fast_ex2(f2_hi(ARG)));
            p[2] = f2_fma(SV, EX, p[2]);
            p[3] = f2_fma(f2_mul(KV, EX), f2_fma(k1, RHO, one), p[3]);
        }
    }
}

// A work item of up to 64 targets: every lane sums the staged sources for
// targets `lane` and `lane + 32`, so each staged source is read once for two
// pairs.  Same arithmetic per pair, same order over the sources, same records
// as p2p32_item.
template <int NK, bool Y0, bool Y1, bool MASK>
__device__ __forceinline__ void p2p32x2_item(const P2PArgs32 &g, int64_t item, int lane, float4 *sA, float4 *sB) {
    const int4 it = g.items[item];
    float tx[2] = {0.f, 0.f}, ty[2] = {0.f, 0.f}, tz[2] = {0.f, 0.f};
    int me[2] = {-1, -1};
    bool valid[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        valid[h] = lane + 32 * h < it.z;
        if (valid[h]) {
            const int t = g.inv[(int64_t)it.y + lane + 32 * h];
            const float4 x = g.x32[t];
            tx[h] = x.x;
            ty[h] = x.y;
            tz[h] = x.z;
            if (MASK && g.use_self) me[h] = g.selfp[t];
        }
    }
    const bool two = it.z > 32;   // warp-uniform
    const float k0 = g.ks.kap[0], k1 = g.ks.kap[1];
    const float l2e0 = -k0 * 1.4426950408889634f, l2e1 = -k1 * 1.4426950408889634f;
    float hi[2][2 * NK], lo[2][2 * NK];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int a = 0; a < 2 * NK; ++a) { hi[h][a] = 0.f; lo[h][a] = 0.f; }
    const int node = g.leaf_node[it.x];
    const int64_t s0 = g.start[node];
    const int cnt = (int)g.count[node];
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int m = min(32, cnt - c0);
        if (lane < m) {
            sA[lane] = g.A[s0 + c0 + lane];
            sB[lane] = g.B[s0 + c0 + lane];
        }
        __syncwarp();
        float p0[4] = {0.f, 0.f, 0.f, 0.f}, p1[4] = {0.f, 0.f, 0.f, 0.f};
        if (two) {
            // both targets in packed pairs (lo: target lane, hi: target lane + 32)
            const f2p tX = f2_make(tx[0], tx[1]), tY = f2_make(ty[0], ty[1]), tZ = f2_make(tz[0], tz[1]);
            const f2p K0 = f2_make(k0, k0), K1 = f2_make(k1, k1), L0 = f2_make(l2e0, l2e0),
                      L1 = f2_make(l2e1, l2e1), ONE = f2_make(1.f, 1.f);
            f2p pp[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const float4 a = sA[j];
                const float4 b = sB[j];
                p2p32_pair2<NK, Y0, Y1, MASK>(tX, tY, tZ, me[0], me[1], f2_make(a.x, a.x), f2_make(a.y, a.y),
                                              f2_make(a.z, a.z), f2_make(a.w, a.w), f2_make(b.x, b.x),
                                              f2_make(b.y, b.y), f2_make(b.z, b.z), __float_as_int(b.w), K0, K1, L0,
                                              L1, ONE, pp);
            }
#pragma unroll
            for (int v = 0; v < 2 * NK; ++v) {
                p0[v] = f2_lo(pp[v]);
                p1[v] = f2_hi(pp[v]);
            }
        } else if (valid[0]) {
#pragma unroll 4
            for (int j = 0; j < m; ++j)
                p2p32_pair<NK, Y0, Y1, MASK>(tx[0], ty[0], tz[0], me[0], sA[j], sB[j], k0, k1, l2e0, l2e1, p0);
        }
#pragma unroll
        for (int a = 0; a < 2 * NK; ++a) {
            comp_add(hi[0][a], lo[0][a], p0[a]);
            comp_add(hi[1][a], lo[1][a], p1[a]);
        }
        __syncwarp();
    }
#pragma unroll
    for (int h = 0; h < 2; ++h)
        if (valid[h]) {
            float2 *rec =
                reinterpret_cast<float2 *>(g.part + (int64_t)2 * NK * g.sent[(int64_t)it.y + lane + 32 * h]);
#pragma unroll
            for (int a = 0; a < NK; ++a)
                rec[a] = make_float2(hi[h][2 * a] + lo[h][2 * a], hi[h][2 * a + 1] + lo[h][2 * a + 1]);
        }
}

template <int NK, bool Y0, bool Y1, bool MASK>
__global__ void __launch_bounds__(128) p2p32x2_kernel(int64_t nitems, P2PArgs32 g) {
    __shared__ float4 sA[4][32], sB[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 4 + warp;
    if (item >= nitems) return;
    p2p32x2_item<NK, Y0, Y1, MASK>(g, item, lane, sA[warp], sB[warp]);
}

template <int NK, bool Y0, bool Y1, bool MASK>
__global__ void __launch_bounds__(128) p2p32_kernel(int64_t nitems, P2PArgs32 g) {
    __shared__ float4 sA[4][32], sB[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 4 + warp;
    if (item >= nitems) return;
    p2p32_item<NK, Y0, Y1, MASK>(g, item, lane, sA[warp], sB[warp]);
}

// ---------------------------------------------------------------- P2P, FP64
template <int NK, bool Y0, bool Y1>
__global__ void __launch_bounds__(128) p2p64_kernel(int64_t nitems, const int4 *__restrict__ items,
                                                    const int32_t *__restrict__ inv,
                                                    const int32_t *__restrict__ sent,
                                                    const double *__restrict__ xs, const int32_t *__restrict__ selfp,
                                                    int use_self, const int32_t *__restrict__ leaf_node,
                                                    const int64_t *__restrict__ start, const int64_t *__restrict__ count,
                                                    const double *__restrict__ src, double kap0, double kap1,
                                                    double *__restrict__ part) {
    __shared__ dvec4 sA[4][32], sB[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 4 + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    const bool valid = lane < it.z;
    const int64_t slot = (int64_t)it.y + lane;
    double tx = 0, ty = 0, tz = 0;
    int me = -1;
    if (valid) {
        const int t = inv[slot];
        tx = xs[3 * t]; ty = xs[3 * t + 1]; tz = xs[3 * t + 2];
        if (use_self) me = selfp[t];
    }
    double acc[4] = {0, 0, 0, 0};
    const dvec4 *src4 = reinterpret_cast<const dvec4 *>(src);
    const int node = leaf_node[it.x];
    const int64_t s0 = start[node];
    const int cnt = (int)count[node];
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int m = min(32, cnt - c0);
        if (lane < m) {
            sA[warp][lane] = src4[2 * (s0 + c0 + lane)];
            sB[warp][lane] = src4[2 * (s0 + c0 + lane) + 1];
        }
        __syncwarp();
        if (valid) {
            for (int j = 0; j < m; ++j) {
                const dvec4 a = sA[warp][j];
                const dvec4 b = sB[warp][j];
                if ((int)b.w == me) continue;
                const double dx = tx - a.x, dy = ty - a.y, dz = tz - a.z;
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double rho = sqrt(r2);
                const double inv = 1.0 / rho;
                const double sv = a.w * inv;
                const double rd = dx * b.x + dy * b.y + dz * b.z;
                const double kv = rd * inv * inv * inv;
                if (!Y0) {
                    acc[0] += sv;
                    acc[1] += kv;
                } else {
                    const double ex = exp(-kap0 * rho);
                    acc[0] += sv * ex;
                    acc[1] += kv * ex * (1.0 + kap0 * rho);
                }
                if (NK == 2) {
                    if (!Y1) {
                        acc[2] += sv;
                        acc[3] += kv;
                    } else {
                        const double ex = exp(-kap1 * rho);
                        acc[2] += sv * ex;
                        acc[3] += kv * ex * (1.0 + kap1 * rho);
                    }
                }
            }
        }
        __syncwarp();
    }
    if (valid) {
        double2 *rec = reinterpret_cast<double2 *>(part + (int64_t)2 * NK * sent[slot]);
#pragma unroll
        for (int a = 0; a < NK; ++a) rec[a] = make_double2(acc[2 * a], acc[2 * a + 1]);
    }
}

// ---------------------------------------------------------------- M2P
// a^k and contraction with the box moments, fully unrolled for a fixed order P
// so that every coefficient index is a compile-time constant.
template <int P, bool YUK, typename T>
__device__ __forceinline__ void m2p_eval(T ux, T uy, T uz, T kappa, const T *__restrict__ mom, T &V, T &K) {
    constexpr int NT = (P + 1) * (P + 2) * (P + 3) / 6;
    T a[NT];
    T b[YUK ? NT : 1];
    const T r2 = ux * ux + uy * uy + uz * uz;
    T rinv;
    if constexpr (sizeof(T) == 4) rinv = rsqrtf(r2); else rinv = rsqrt(r2);
    const T ir2 = rinv * rinv;
    T e0 = (T)1;
    if (YUK) {
        if constexpr (sizeof(T) == 4) e0 = __expf(-kappa * r2 * rinv); else e0 = exp(-kappa * r2 * rinv);
    }
    a[0] = e0 * rinv;
    if (YUK) b[0] = e0;
    V = a[0] * mom[0];
    K = a[0] * mom[NT];
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        // the order's constants folded with -1/r^2
        const T C1 = -(T)(2 * n - 1) / (T)n * ir2, C2 = -(T)(n - 1) / (T)n * ir2;
        const T kn = kappa / (T)n, KN = -kn * ir2;
#pragma unroll
        for (int k1 = n; k1 >= 0; --k1) {
#pragma unroll
            for (int k2 = n - k1; k2 >= 0; --k2) {
                const int k3 = n - k1 - k2;
                const int i = term_index(k1, k2, k3);
                T s1 = 0, s2 = 0, t1 = 0, t2 = 0;
                if (k1 >= 1) { s1 += ux * a[term_index(k1 - 1, k2, k3)]; if (YUK) t1 += ux * b[term_index(k1 - 1, k2, k3)]; }
                if (k2 >= 1) { s1 += uy * a[term_index(k1, k2 - 1, k3)]; if (YUK) t1 += uy * b[term_index(k1, k2 - 1, k3)]; }
                if (k3 >= 1) { s1 += uz * a[term_index(k1, k2, k3 - 1)]; if (YUK) t1 += uz * b[term_index(k1, k2, k3 - 1)]; }
                if (k1 >= 2) { s2 += a[term_index(k1 - 2, k2, k3)]; if (YUK) t2 += b[term_index(k1 - 2, k2, k3)]; }
                if (k2 >= 2) { s2 += a[term_index(k1, k2 - 2, k3)]; if (YUK) t2 += b[term_index(k1, k2 - 2, k3)]; }
                if (k3 >= 2) { s2 += a[term_index(k1, k2, k3 - 2)]; if (YUK) t2 += b[term_index(k1, k2, k3 - 2)]; }
                T ai = C1 * s1 + C2 * s2;
                if (YUK) ai += KN * (t1 + t2);
                a[i] = ai;
                if (YUK) b[i] = -kn * (s1 + s2);
                V += a[i] * mom[i];
                K += a[i] * mom[NT + i];
            }
        }
    }
}

// Runtime-order variant for orders without a compiled specialisation (local arrays).
template <bool YUK, typename T>
__device__ void m2p_eval_rt(int P, T ux, T uy, T uz, T kappa, const T *__restrict__ mom, T &V, T &K) {
    const int NT = (P + 1) * (P + 2) * (P + 3) / 6;
    T a[455];
    T b[YUK ? 455 : 1];
    const T r2 = ux * ux + uy * uy + uz * uz;
    const T r = sqrt(r2);
    const T ir2 = (T)1 / r2;
    const T e0 = YUK ? (T)exp(-kappa * r) : (T)1;
    a[0] = e0 / r;
    if (YUK) b[0] = e0;
    V = a[0] * mom[0];
    K = a[0] * mom[NT];
    for (int i = 1; i < NT; ++i) {
        const int k1 = c_terms[3 * i], k2 = c_terms[3 * i + 1], k3 = c_terms[3 * i + 2];
        const int n = k1 + k2 + k3;
        T s1 = 0, s2 = 0, t1 = 0, t2 = 0;
        if (k1 >= 1) { s1 += ux * a[term_index(k1 - 1, k2, k3)]; if (YUK) t1 += ux * b[term_index(k1 - 1, k2, k3)]; }
        if (k2 >= 1) { s1 += uy * a[term_index(k1, k2 - 1, k3)]; if (YUK) t1 += uy * b[term_index(k1, k2 - 1, k3)]; }
        if (k3 >= 1) { s1 += uz * a[term_index(k1, k2, k3 - 1)]; if (YUK) t1 += uz * b[term_index(k1, k2, k3 - 1)]; }
        if (k1 >= 2) { s2 += a[term_index(k1 - 2, k2, k3)]; if (YUK) t2 += b[term_index(k1 - 2, k2, k3)]; }
        if (k2 >= 2) { s2 += a[term_index(k1, k2 - 2, k3)]; if (YUK) t2 += b[term_index(k1, k2 - 2, k3)]; }
        if (k3 >= 2) { s2 += a[term_index(k1, k2, k3 - 2)]; if (YUK) t2 += b[term_index(k1, k2, k3 - 2)]; }
        T ai = ((T)(2 * n - 1) * s1 + (T)(n - 1) * s2) / (T)n;
        if (YUK) ai += kappa / (T)n * (t1 + t2);
        a[i] = -ai * ir2;
        if (YUK) b[i] = -kappa / (T)n * (s1 + s2);
        V += a[i] * mom[i];
        K += a[i] * mom[NT + i];
    }
}

// Box-major: one warp per work item = one accepted box and up to 32
// (target, entry) pairs that use it; the box's moments and centre are the
// same for every lane, each lane runs the recurrences for its own target and
// stores (V, K) at the pair's list entry.
template <int P, bool YUK, typename T>
__global__ void __launch_bounds__(128) m2p_kernel(int64_t nitems, const int4 *__restrict__ items,
                                                  const int32_t *__restrict__ inv,
                                                  const int32_t *__restrict__ ent, int Prt,
                                                  const double *__restrict__ xs, const float4 *__restrict__ x32,
                                                  const double *__restrict__ centre, const float4 *__restrict__ cen32,
                                                  const T *__restrict__ mom, double kappa, int kslot, int nk,
                                                  T *__restrict__ part) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 4 + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    if (lane >= it.z) return;
    const int64_t slot = (int64_t)it.y + lane;
    const int t = inv[slot];
    const int b = it.x;
    const int Pe = P >= 0 ? P : Prt;
    const int NT = (Pe + 1) * (Pe + 2) * (Pe + 3) / 6;
    T ux, uy, uz;
    if constexpr (sizeof(T) == 4) {
        const float4 c = cen32[b];
        const float4 x = x32[t];
        ux = c.x - x.x;
        uy = c.y - x.y;
        uz = c.z - x.z;
    } else {
        ux = centre[3 * b] - xs[3 * t];
        uy = centre[3 * b + 1] - xs[3 * t + 1];
        uz = centre[3 * b + 2] - xs[3 * t + 2];
    }
    T V, K;
    if constexpr (P >= 0) m2p_eval<(P >= 0 ? P : 0), YUK, T>(ux, uy, uz, (T)kappa, mom + (int64_t)b * 2 * NT, V, K);
    else m2p_eval_rt<YUK, T>(Prt, ux, uy, uz, (T)kappa, mom + (int64_t)b * 2 * NT, V, K);
    // interleaved record of the entry: (V, K) of every kernel
    T *rec = part + (int64_t)2 * nk * ent[slot] + 2 * kslot;
    rec[0] = V;
    rec[1] = K;
}

// ---------------------------------------------------------------- M2P in radial form (FP32)
// (the regrouping and its tables: radial.cuh)

// One thread per (node, output pair): (N^M_r, N^D_r) of the node; the padding pairs are zeroed.
template <int P>
__global__ void radial_moments_kernel(int nnodes, const float *__restrict__ mom, float *__restrict__ rmom) {
    constexpr int NT = (P + 1) * (P + 2) * (P + 3) / 6, NR = radial_terms(P), NP = radial_stride(P) / 2;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nnodes * NP) return;
    const int64_t b = t / NP;
    const int r = (int)(t % NP);
    float sm = 0.f, sd = 0.f;
    if (r < NR) {
        const RadialTable<P> &T = g_radial<P>;
        const float *M = mom + b * 2 * NT, *D = M + NT;
        for (int q = T.start[r]; q < T.start[r + 1]; ++q) {
            const float w = T.w[q];
            const int k = T.k[q];
            sm = fmaf(w, M[k], sm);
            sd = fmaf(w, D[k], sd);
        }
    }
    reinterpret_cast<float2 *>(rmom)[b * NP + r] = make_float2(sm, sd);
}

// The radial-form M2P sums of NTG targets against one box's staged radial
// moments R: every moment pair is read from shared memory once for all NTG
// targets.  u = box centre - target; out = (VL, KL, VY, KY) per target.  The
// arithmetic per target is that of the one-target form, in the same order.
// The monopole and dipole sums of one radial index n share their monomial, so
// they run as one packed FP32 pair (SM_n, SD_n) += (m, m) (N^M, N^D), with the
// staged moment pair as the second operand; the closing sums pair (V, K) of
// each kernel the same way.  Every half is the scalar fma of the unpacked form.
template <int P, int NTG>
__device__ __forceinline__ void m2p_ly_eval(const float4 *R, const float (&ux)[NTG], const float (&uy)[NTG],
                                            const float (&uz)[NTG], float kappa, float4 (&out)[NTG]) {
    float px[NTG][P + 1], py[NTG][P + 1], pz[NTG][P + 1];
    f2p S[NTG][P + 1];     // (SM_n, SD_n)
#pragma unroll
    for (int t = 0; t < NTG; ++t) {
        px[t][0] = py[t][0] = pz[t][0] = 1.f;
#pragma unroll
        for (int i = 1; i <= P; ++i) {
            px[t][i] = px[t][i - 1] * ux[t];
            py[t][i] = py[t][i - 1] * uy[t];
            pz[t][i] = pz[t][i - 1] * uz[t];
        }
#pragma unroll
        for (int n = 0; n <= P; ++n) S[t][n] = 0ull;
    }
    const ulonglong2 *R2 = reinterpret_cast<const ulonglong2 *>(R);
    ulonglong2 cur = make_ulonglong2(0ull, 0ull);
    int o = 0;
#pragma unroll
    for (int a1 = 0; a1 <= P; ++a1)
#pragma unroll
        for (int a2 = 0; a2 <= P - a1; ++a2) {
            float base[NTG];
#pragma unroll
            for (int t = 0; t < NTG; ++t) base[t] = px[t][a1] * py[t][a2];
#pragma unroll
            for (int a3 = 0; a3 <= P - a1 - a2; ++a3) {
                f2p mono[NTG];
#pragma unroll
                for (int t = 0; t < NTG; ++t) {
                    const float m = base[t] * pz[t][a3];
                    mono[t] = f2_make(m, m);
                }
                const int a = a1 + a2 + a3;
#pragma unroll
                for (int n = a; 2 * n <= a + P; ++n) {
                    if ((o & 3) == 0) cur = R2[o >> 2];
                    const f2p nmd = (o & 3) == 0 ? cur.x : cur.y;
#pragma unroll
                    for (int t = 0; t < NTG; ++t) S[t][n] = f2_fma(mono[t], nmd, S[t][n]);
                    o += 2;
                }
            }
        }
#pragma unroll
    for (int t = 0; t < NTG; ++t) {
        const float r2 = fmaf(ux[t], ux[t], fmaf(uy[t], uy[t], uz[t] * uz[t]));
        const float rinv = rsqrtf(r2), ir2 = rinv * rinv;
        float FL[P + 1], FY[P + 1];
        FL[0] = rinv;
#pragma unroll
        for (int n = 0; n < P; ++n) FL[n + 1] = (-(float)(2 * n + 1) * ir2) * FL[n];
        const float rho = r2 * rinv;
        const float e = __expf(-kappa * rho);
        FY[0] = e * rinv;
        if (P >= 1) FY[1] = -fmaf(kappa, rho, 1.f) * FY[0] * ir2;
        const float k2 = kappa * kappa;
#pragma unroll
        for (int n = 1; n < P; ++n) FY[n + 1] = fmaf(k2, FY[n - 1], -(float)(2 * n + 1) * FY[n]) * ir2;
        f2p L = 0ull, Y = 0ull;     // (VL, KL), (VY, KY)
#pragma unroll
        for (int n = 0; n <= P; ++n) {
            L = f2_fma(f2_make(FL[n], FL[n]), S[t][n], L);
            Y = f2_fma(f2_make(FY[n], FY[n]), S[t][n], Y);
        }
        out[t] = make_float4(f2_lo(L), f2_hi(L), f2_lo(Y), f2_hi(Y));
    }
}

// Box-major M2P for a pair whose two kernels are Laplace (slot 0) and Yukawa
// (slot 1), one record (VL, KL, VY, KY) per (target, box).  A warp takes NI
// consecutive (box, up to 32 targets) items and stages the box's radial
// moments in shared memory with coalesced loads; every lane reads them as
// broadcasts.  When the NI items are all the same box's groups of targets
// (the usual case: a box's items are consecutive and all but the last hold
// 32 targets), every lane evaluates one target of each, so each moment pair
// is read once for NI targets; otherwise the items are evaluated one after
// the other.  Lanes past the last item's count evaluate their first target
// again and store it once.  Seven blocks per SM (72 registers; at P = 6 the
// packed evaluation spills 12 bytes outside its loops): 90 -> 86 us at P = 6
// against the unbounded 80 registers and six blocks.  A persistent form, each
// warp walking its tasks with the next box's moments copied by cp.async and
// the next targets' indices loaded one and two tasks ahead, was slower (103
// against 92 us: 96 registers, 17 resident warps per SM, 13% more
// instructions), so the short warps stay.

// The NI items i0.. on the calling warp; sR: the warp's staging of one box's radial moments.
template <int P, int NI>
__device__ __forceinline__ void m2p_ly32x_task(const M2PArgs32 &g, int64_t nitems, int64_t i0, int lane, float4 *sR) {
    constexpr int NQ = radial_stride(P) / 4;     // float4 per box
    int4 it[NI];
    bool same = true;
#pragma unroll
    for (int k = 0; k < NI; ++k) {
        it[k] = i0 + k < nitems ? g.items[i0 + k] : make_int4(-1, 0, 0, 0);
        same = same && it[k].x == it[0].x;
    }
    const float4 *R = sR;
    auto stage = [&](int b) {
        const float4 *src = reinterpret_cast<const float4 *>(g.rmom + (int64_t)b * radial_stride(P));
        __syncwarp();
        for (int q = lane; q < NQ; q += 32) sR[q] = src[q];
        __syncwarp();
    };
    stage(it[0].x);
    if (same) {
        const float4 c = g.cen32[it[0].x];
        int64_t sl[NI];
        float ux[NI], uy[NI], uz[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) {
            sl[k] = lane < it[k].z ? (int64_t)it[k].y + lane : (int64_t)it[0].y + lane;
            const float4 x = g.x32[g.inv[sl[k]]];
            ux[k] = c.x - x.x; uy[k] = c.y - x.y; uz[k] = c.z - x.z;
        }
        float4 out[NI];
        m2p_ly_eval<P, NI>(R, ux, uy, uz, g.kappa, out);
#pragma unroll
        for (int k = 0; k < NI; ++k)
            if (lane < it[k].z) g.part[g.ent[sl[k]]] = out[k];
    } else {
#pragma unroll 1
        for (int k = 0; k < NI; ++k) {
            if (it[k].x < 0) break;
            if (k > 0) stage(it[k].x);
            if (lane < it[k].z) {
                const int64_t slot = (int64_t)it[k].y + lane;
                const float4 c = g.cen32[it[k].x];
                const float4 x = g.x32[g.inv[slot]];
                const float ux[1] = {c.x - x.x}, uy[1] = {c.y - x.y}, uz[1] = {c.z - x.z};
                float4 out[1];
                m2p_ly_eval<P, 1>(R, ux, uy, uz, g.kappa, out);
                g.part[g.ent[slot]] = out[0];
            }
        }
    }
}

template <int P, int NI>
__global__ void __launch_bounds__(128, 7) m2p_ly32x_kernel(int64_t nitems, M2PArgs32 g) {
    constexpr int NQ = radial_stride(P) / 4;
    __shared__ float4 sR[4][NQ];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = ((int64_t)blockIdx.x * 4 + warp) * NI;
    if (i0 >= nitems) return;
    m2p_ly32x_task<P, NI>(g, nitems, i0, lane, sR[warp]);
}

// One warp per target: V and K of every kernel = its P2P and M2P partials
// (FP64 sums) plus the near-singular corrections and the self term, times
// 1/(4 pi) for the treecode part.  Lanes take the list entries in turn and a
// fixed butterfly combines them, so the result does not depend on scheduling.
struct NearArgs {
    const int64_t *ptr;
    const int32_t *panel;
    const double *dV[2], *dK[2], *selfV[2];
    const int32_t *selfp;
    int use_self;
    const double *phi, *dphi;
};

struct NearArgs32 {
    const int64_t *ptr;
    const int32_t *panel;
    const float *dV[2], *dK[2];
    const double *selfV[2];
    const int32_t *selfp;
    int use_self;
    const float2 *phf;      // (phi, dphi) of the source surface in FP32
    const double *dphi;     // FP64 dphi for the self term
};

template <typename TM, int NK>
__global__ void __launch_bounds__(128) gather_kernel(int64_t ntg, const int64_t *__restrict__ p2p_ptr,
                                                     const double *__restrict__ p2p_part,
                                                     const int64_t *__restrict__ m2p_ptr,
                                                     const TM *__restrict__ m2p_part, NearArgs nr,
                                                     double *__restrict__ VK0, double *__restrict__ VK1) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 4 + warp;
    if (t >= ntg) return;
    double acc[2 * NK], far[2 * NK];
#pragma unroll
    for (int a = 0; a < 2 * NK; ++a) { acc[a] = 0.0; far[a] = 0.0; }
    for (int64_t e = p2p_ptr[t] + lane; e < p2p_ptr[t + 1]; e += 32) {
        const double2 *rec = reinterpret_cast<const double2 *>(p2p_part + (int64_t)2 * NK * e);
#pragma unroll
        for (int a = 0; a < NK; ++a) {
            const double2 v = rec[a];
            acc[2 * a] += v.x;
            acc[2 * a + 1] += v.y;
        }
    }
    if (m2p_part)
        for (int64_t e = m2p_ptr[t] + lane; e < m2p_ptr[t + 1]; e += 32) {
            const TM *rec = m2p_part + (int64_t)2 * NK * e;
#pragma unroll
            for (int a = 0; a < 2 * NK; ++a) far[a] += (double)rec[a];
        }
#pragma unroll
    for (int a = 0; a < 2 * NK; ++a) acc[a] = (acc[a] + far[a]) * kInv4Pi;
    for (int64_t e = nr.ptr[t] + lane; e < nr.ptr[t + 1]; e += 32) {
        const int j = nr.panel[e];
        const double ph = nr.phi[j], dph = nr.dphi[j];
#pragma unroll
        for (int a = 0; a < NK; ++a) {
            acc[2 * a] += nr.dV[a][e] * dph;
            acc[2 * a + 1] += nr.dK[a][e] * ph;
        }
    }
#pragma unroll
    for (int a = 0; a < 2 * NK; ++a)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[a] += __shfl_xor_sync(0xffffffffu, acc[a], o);
    if (lane == 0) {
        if (nr.use_self) {
            const int me = nr.selfp[t];
#pragma unroll
            for (int a = 0; a < NK; ++a) acc[2 * a] += nr.selfV[a][me] * nr.dphi[me];
        }
        VK0[t] = acc[0];
        VK0[ntg + t] = acc[1];
        if (NK == 2) {
            VK1[t] = acc[2 % (2 * NK)];
            VK1[ntg + t] = acc[3 % (2 * NK)];
        }
    }
}

// Mixed precision: the same gather entirely in FP32, every sum compensated
// (TwoSum into (hi, lo) pairs, pairs combined by a fixed butterfly): the FP64
// pipe of the B300 is too narrow for ~10^3 conversions and adds per target.
__device__ __forceinline__ void two_add(float &hi, float &lo, float v) {
    const float s = hi + v;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (v - bb);
    hi = s;
}

struct GatherArgs32 {
    const int64_t *p2p_ptr;                // per sorted target: its P2P list entries
    const float *p2p_part;                 // P2P records at the list entries
    const int64_t *m2p_ptr;
    const float *m2p_part;                 // M2P records at the list entries (null: no far field)
    NearArgs32 nr;
    double *VK0, *VK1;                     // outputs of kernel 0 and 1: V at [0, ntg), K at [ntg, 2 ntg)
};

// Target t on W consecutive lanes of the calling warp (the whole warp, or
// one half with W = 16, the other half taking the next target); lane is the
// lane within the group.  valid = false: the group has no target (the last
// half-warp of an odd count) and only joins the shuffles.
template <int NK, int W = 32, int UM = 4>
__device__ __forceinline__ void gather32_target(const GatherArgs32 &g, int64_t ntg, int64_t t, int lane,
                                                bool valid = true) {
    float hi[2 * NK], lo[2 * NK], nh[2 * NK], nl[2 * NK];
#pragma unroll
    for (int a = 0; a < 2 * NK; ++a) { hi[a] = 0.f; lo[a] = 0.f; nh[a] = 0.f; nl[a] = 0.f; }
    // records as one 16-byte (two kernels) or 8-byte load each, every
    // target's P2P and M2P records contiguous (written at their list entries).
    // The list bounds, then the first four P2P and four M2P records and two
    // near entries of every lane, then the densities of those near panels,
    // are each issued as one round of independent loads (three dependent
    // rounds in all); longer lists continue in loops.  Every lane adds its
    // P2P, then M2P, then near values, each in list order.
    using Rec = typename std::conditional<NK == 2, float4, float2>::type;
    auto add_rec = [&](const Rec &r) {
        two_add(hi[0], lo[0], r.x);
        two_add(hi[1], lo[1], r.y);
        if constexpr (NK == 2) {
            two_add(hi[2 % (2 * NK)], lo[2 % (2 * NK)], r.z);
            two_add(hi[3 % (2 * NK)], lo[3 % (2 * NK)], r.w);
        }
    };
    const Rec *pp = reinterpret_cast<const Rec *>(g.p2p_part);
    const Rec *mp = reinterpret_cast<const Rec *>(g.m2p_part);
    const int64_t tt = valid ? t : 0;
    const int64_t pb = g.p2p_ptr[tt] + lane, pe = valid ? g.p2p_ptr[tt + 1] : 0;
    const int64_t mb = g.m2p_part ? g.m2p_ptr[tt] + lane : 0, me = g.m2p_part && valid ? g.m2p_ptr[tt + 1] : 0;
    const int64_t nb = g.nr.ptr[tt] + lane, ne = valid ? g.nr.ptr[tt + 1] : 0;
    const int sp = g.nr.use_self && lane < 2 * NK ? g.nr.selfp[tt] : 0;
    // first load round
    Rec rp[4], rm[4];
    int jn[2];
    float dv[2][NK], dk[2][NK];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (pb + W * u < pe) rp[u] = pp[pb + W * u];
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (mb + W * u < me) rm[u] = mp[mb + W * u];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
        const int64_t e = nb + W * u;
        jn[u] = e < ne ? g.nr.panel[e] : -1;
#pragma unroll
        for (int a = 0; a < NK; ++a) {
            dv[u][a] = e < ne ? g.nr.dV[a][e] : 0.f;
            dk[u][a] = e < ne ? g.nr.dK[a][e] : 0.f;
        }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (pb + W * u < pe) add_rec(rp[u]);
    // second load round: the densities of the near panels
    float2 pd[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) pd[u] = jn[u] >= 0 ? g.nr.phf[jn[u]] : make_float2(0.f, 0.f);
    double sv = 0.0, sd = 0.0;
    if (g.nr.use_self && lane < 2 * NK && (lane & 1) == 0) {
        sv = g.nr.selfV[lane >> 1][sp];
        sd = g.nr.dphi[sp];
    }
    // P2P beyond four entries per lane
    for (int64_t e = pb + 4 * W; e < pe; e += 4 * W) {
        Rec r[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e + W * u < pe) r[u] = pp[e + W * u];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (e + W * u < pe) add_rec(r[u]);
    }
    // M2P
#pragma unroll
    for (int u = 0; u < 4; ++u)
        if (mb + W * u < me) add_rec(rm[u]);
    for (int64_t e = mb + 4 * W; e < me; e += UM * W) {
        Rec r[UM];
#pragma unroll
        for (int u = 0; u < UM; ++u)
            if (e + W * u < me) r[u] = mp[e + W * u];
#pragma unroll
        for (int u = 0; u < UM; ++u)
            if (e + W * u < me) add_rec(r[u]);
    }
    // near-singular corrections
#pragma unroll
    for (int u = 0; u < 2; ++u)
        if (jn[u] >= 0) {
#pragma unroll
            for (int a = 0; a < NK; ++a) {
                two_add(nh[2 * a], nl[2 * a], dv[u][a] * pd[u].y);
                two_add(nh[2 * a + 1], nl[2 * a + 1], dk[u][a] * pd[u].x);
            }
        }
    for (int64_t e = nb + 2 * W; e < ne; e += W) {
        const int j = g.nr.panel[e];
        const float2 pdj = g.nr.phf[j];
#pragma unroll
        for (int a = 0; a < NK; ++a) {
            two_add(nh[2 * a], nl[2 * a], g.nr.dV[a][e] * pdj.y);
            two_add(nh[2 * a + 1], nl[2 * a + 1], g.nr.dK[a][e] * pdj.x);
        }
    }
#pragma unroll
    for (int a = 0; a < 2 * NK; ++a)
#pragma unroll
        for (int o = W / 2; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, hi[a], o), ol = __shfl_xor_sync(0xffffffffu, lo[a], o);
            const float ph = __shfl_xor_sync(0xffffffffu, nh[a], o), pl = __shfl_xor_sync(0xffffffffu, nl[a], o);
            two_add(hi[a], lo[a], oh);
            lo[a] += ol;
            two_add(nh[a], nl[a], ph);
            nl[a] += pl;
        }
    // FP64 epilogue: lane a finishes value a (V0, K0[, V1, K1]) - the B300 FP64
    // pipe is narrow, so one lane doing all of them dominated the kernel
    float vh = hi[0], vl = lo[0], wh = nh[0], wl = nl[0];
#pragma unroll
    for (int a = 1; a < 2 * NK; ++a)
        if (lane == a) { vh = hi[a]; vl = lo[a]; wh = nh[a]; wl = nl[a]; }
    if (lane < 2 * NK && valid) {
        double out = ((double)vh + (double)vl) * kInv4Pi + ((double)wh + (double)wl);
        const int a = lane;
        if (g.nr.use_self && (a & 1) == 0) out += sv * sd;
        double *dst = (a >> 1) == 0 ? g.VK0 : g.VK1;
        dst[(a & 1) ? ntg + t : t] = out;
    }
}

// Four targets per warp, eight lanes each: a target's records are few per
// lane either way (~150 over 32 lanes), and its closing butterfly (four
// values, each a compensated pair, for far and near) and FP64 epilogue cost
// the same per warp whatever the width, so eight lanes serve four targets
// with them (gather 49 -> 32 us against one target per warp; 37 us with 16
// lanes, 34 with 4).
constexpr int kGatherLanes = 8;

// UM: M2P records per lane in flight in the loop after the first round (eight:
// a target's ~134 records over eight lanes take two rounds instead of four;
// 32.6 -> 30.7 us).
template <int NK, int UM = 4>
__global__ void __launch_bounds__(128) gather32_kernel(int64_t ntg, GatherArgs32 g) {
    constexpr int W = kGatherLanes;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t0 = (32 / W) * ((int64_t)blockIdx.x * 4 + warp);
    if (t0 >= ntg) return;
    const int64_t t = t0 + lane / W;
    gather32_target<NK, W, UM>(g, ntg, t, lane % W, t < ntg);
}

// ---------------------------------------------------------------- near field and combine
// Both block rows of one surface in one launch: element i < 2 n is entry i - s n of row s.
__global__ void combine_pair_kernel(int64_t n, const int32_t *__restrict__ rank, const double *__restrict__ phi_s,
                                    double half, CombineRow row0, CombineRow row1, double *__restrict__ y) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * n) return;
    const bool second = e >= n;
    const int64_t i = second ? e - n : e;
    const CombineRow &row = second ? row1 : row0;
    const int r = rank[i];
    double v = phi_s ? half * phi_s[i] : 0.0;
    for (int k = 0; k < row.nterm; ++k) {
        const CombineTerm &tm = row.term[k];
        v += tm.cK * tm.VK[tm.ntg + r] + tm.cV * tm.VK[r];
    }
    y[e] = v;
}

__global__ void combine_kernel(int64_t n, const int32_t *__restrict__ rank, const double *__restrict__ phi_s,
                               double half, CombineRow row, double *__restrict__ y) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int r = rank[i];
    double v = phi_s ? half * phi_s[i] : 0.0;
    for (int k = 0; k < row.nterm; ++k) {
        const CombineTerm &tm = row.term[k];
        v += tm.cK * tm.VK[tm.ntg + r] + tm.cV * tm.VK[r];
    }
    y[i] = v;
}

template <typename T>
void launch_m2p_typed(int P, bool yuk, const Pair &Pr, const double *xs, const double o[3], const Tree &Tr,
                      const T *mom, double kappa, int kslot, int nk, T *part, cudaStream_t s) {
    const int64_t ni = Pr.n_m2p_items;
    const unsigned grid = (unsigned)((ni + 3) / 4);
#define PB_M2P_ARGS \
    ni, Pr.m2p_items.p, Pr.m2p_inv.p, Pr.m2p_ent.p, P, xs, Pr.x32.p, Tr.centre.p, Tr.cen32.p, mom, kappa, kslot, nk, \
        part
#define PB_M2P_CASE(PP)                                                                                  \
    case PP:                                                                                             \
        if (yuk) m2p_kernel<PP, true, T><<<grid, 128, 0, s>>>(PB_M2P_ARGS);                              \
        else m2p_kernel<PP, false, T><<<grid, 128, 0, s>>>(PB_M2P_ARGS);                                 \
        break;
    switch (P) {
        PB_M2P_CASE(0)
        PB_M2P_CASE(1)
        PB_M2P_CASE(2)
        PB_M2P_CASE(3)
        PB_M2P_CASE(4)
        PB_M2P_CASE(5)
        PB_M2P_CASE(6)
        PB_M2P_CASE(7)
        PB_M2P_CASE(8)
        default:
            if (yuk) m2p_kernel<-1, true, T><<<grid, 128, 0, s>>>(PB_M2P_ARGS);
            else m2p_kernel<-1, false, T><<<grid, 128, 0, s>>>(PB_M2P_ARGS);
    }
#undef PB_M2P_CASE
#undef PB_M2P_ARGS
    PB_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- fused upward pass
// P2M and every M2M level in one launch: one block per leaf computes the
// leaf's moments; then the block that finishes last among a node's children
// (an atomic count per node, each child announcing itself after a memory
// fence) shifts the children into the parent, and so on to the root.  No
// block waits for another; each node is computed exactly once, from its
// children in child order, so the moments equal the level-by-level ones.
template <typename T>
__device__ __forceinline__ T ld_cg(const T *p) { return __ldcg(p); }

// Climb from a node whose moments are complete towards the root: after each
// node the block announces it to the parent (a barrier, a fence by thread 0,
// then an atomic count); the block that brings a parent's count to its number
// of children shifts the children's moments into it (three one-axis passes in
// shared memory, children added in child order) and continues from there.
// Every node holds `nval` values: nval / NT sets of NT moments, each shifted
// by the same rule.  No block waits for another.  link[i] = (parent, the
// parent's first child, the parent's child count, 0), (-1, 0, 0, 0) at the
// root; `up` = the starting node's record, read by thread 0 ahead of time (as is each next
// level's record), so a level costs the fence, the atomic and one round of
// loads.  buf0, buf1: 8 * nval values each.
template <typename T>
__device__ void climb_m2m(int4 up, int NT, int nval, const double *__restrict__ centre,
                          const float4 *__restrict__ pofs32,
                          const int4 *__restrict__ link, int32_t *__restrict__ ucnt, T *__restrict__ mom, T *buf0,
                          T *buf1, T (*hs)[3], T (*sbin)[kMaxP + 1], const int *sterm, int4 &s_next) {
    while (true) {
        __syncthreads();   // the block's moment stores of `node` are issued
        if (threadIdx.x == 0) {
            int4 nx = make_int4(-1, 0, 0, 0);
            if (up.x >= 0) {
                __threadfence();   // cumulative over the barrier: the block's stores before the announcement
                if (atomicAdd(&ucnt[up.x], 1) == up.z - 1) {
                    ucnt[up.x] = 0;
                    __threadfence();   // the siblings' stores before this block's reads
                    nx = up;
                    up = link[up.x];   // consumed one level up
                }
            }
            s_next = nx;
        }
        __syncthreads();
        const int4 nx = s_next;
        const int b = nx.x;
        if (b < 0) return;
        const int fc = nx.y, nc = nx.z;
        // the centre offsets are loaded first so that their latency overlaps the moments'
        T h = 0;
        const int hc = threadIdx.x / 3, hax = threadIdx.x - 3 * hc;
        if (threadIdx.x < 3 * nc) {
            if (sizeof(T) == 4) {   // the FP64 difference rounded to FP32, formed at the tree build
                const float4 o = pofs32[fc + hc];
                h = (T)(hax == 0 ? o.x : hax == 1 ? o.y : o.z);
            } else {
                h = (T)(centre[3 * (fc + hc) + hax] - centre[3 * b + hax]);
            }
        }
        // absent children: zero rows (and zero offsets)
        for (int i = nc * nval + threadIdx.x; i < 8 * nval; i += blockDim.x) buf0[i] = 0;
        // the children are consecutive nodes; eight loads per thread in flight at once
        const T *cm = mom + (int64_t)fc * nval;
        const int tot = nc * nval;
        for (int i0 = threadIdx.x; i0 < tot; i0 += 8 * blockDim.x) {
            T v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * blockDim.x;
                v[u] = i < tot ? ld_cg(cm + i) : T(0);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < tot) buf0[i] = v[u];
            }
        }
        if (threadIdx.x < 24) hs[hc][hax] = h;
        __syncthreads();
        shift_children<T>(NT, nval, sterm, sbin, hs, buf0, buf1, mom + (int64_t)b * nval);
    }
}

// M2M of every internal node by the climb alone (the leaves' moments already
// computed): one block per leaf, nval values per node.
template <typename T>
__global__ void __launch_bounds__(256) climb_kernel(int nleaves, const int32_t *__restrict__ leaf_node,
                                                    const double *__restrict__ centre,
                                                    const float4 *__restrict__ pofs32, int P, int NT, int nval,
                                                    const int4 *__restrict__ link, int32_t *__restrict__ ucnt,
                                                    T *__restrict__ mom) {
    extern __shared__ __align__(16) unsigned char up_smem[];
    int *sterm = reinterpret_cast<int *>(up_smem);
    T *region = reinterpret_cast<T *>(up_smem + ((3 * 455 * sizeof(int) + 31) / 32) * 32);
    __shared__ T hs[8][3];
    __shared__ T sbin[kMaxP + 1][kMaxP + 1];
    __shared__ int4 s_next;
    const int node = leaf_node[blockIdx.x];
    int4 up = make_int4(-1, 0, 0, 0);
    if (threadIdx.x == 0) up = link[node];
    for (int i = threadIdx.x; i < 3 * NT; i += blockDim.x) sterm[i] = c_terms[i];
    for (int i = threadIdx.x; i < (P + 1) * (P + 1); i += blockDim.x) {
        const int n = i / (P + 1), k = i - n * (P + 1);
        sbin[n][k] = sizeof(T) == 4 ? (T)c_binom32[n][k] : (T)c_binom[n][k];
    }
    climb_m2m<T>(up, NT, nval, centre, pofs32, link, ucnt, mom, region, region + 8 * nval, hs, sbin, sterm, s_next);
}

template <typename T>
__global__ void __launch_bounds__(256) upward_kernel(int nleaves, const int32_t *__restrict__ leaf_node,
                                                     const int64_t *__restrict__ start,
                                                     const int64_t *__restrict__ count,
                                                     const double *__restrict__ centre,
                                                     const float4 *__restrict__ pofs32, double ox, double oy,
                                                     double oz, SrcView<T> sv, int P, int NT,
                                                     const int4 *__restrict__ link, int32_t *__restrict__ ucnt,
                                                     T *__restrict__ mom) {
    constexpr int CH = sizeof(T) == 4 ? kP2MChunk : kP2MChunk / 2;
    extern __shared__ __align__(16) unsigned char up_smem[];
    int *sterm = reinterpret_cast<int *>(up_smem);
    T *region = reinterpret_cast<T *>(up_smem + ((3 * 455 * sizeof(int) + 31) / 32) * 32);
    __shared__ T hs[8][3];
    __shared__ T sbin[kMaxP + 1][kMaxP + 1];
    __shared__ int4 s_next;
    for (int i = threadIdx.x; i < 3 * NT; i += blockDim.x) sterm[i] = c_terms[i];
    for (int i = threadIdx.x; i < (P + 1) * (P + 1); i += blockDim.x) {
        const int n = i / (P + 1), k = i - n * (P + 1);
        sbin[n][k] = sizeof(T) == 4 ? (T)c_binom32[n][k] : (T)c_binom[n][k];
    }
    // ---- P2M of this block's leaf (the 4-source quad scheme of p2m_kernel)
    // power rows padded by 4 values: threads owning different terms read
    // different rows at the same column without bank conflicts
    constexpr int CP = CH + 4;
    T(*pw)[kMaxP + 1][CP] = reinterpret_cast<T(*)[kMaxP + 1][CP]>(region);
    T(*sd)[CH] = reinterpret_cast<T(*)[CH]>(region + 3 * (kMaxP + 1) * CP);
    T(*part)[2][128] = reinterpret_cast<T(*)[2][128]>(region + 3 * (kMaxP + 1) * CP + 4 * CH);
    const int node = leaf_node[blockIdx.x];
    int4 up = make_int4(-1, 0, 0, 0);
    if (threadIdx.x == 0) up = link[node];   // used after the P2M
    {
        const int64_t s0 = start[node], cnt = count[node];
        T c[3];
        if (sizeof(T) == 8) {
            c[0] = (T)centre[3 * node]; c[1] = (T)centre[3 * node + 1]; c[2] = (T)centre[3 * node + 2];
        } else {
            c[0] = (T)(centre[3 * node] - ox); c[1] = (T)(centre[3 * node + 1] - oy);
            c[2] = (T)(centre[3 * node + 2] - oz);
        }
        const int G = NT <= 85 ? 3 : NT <= 128 ? 2 : 1;
        const int g = G > 1 ? threadIdx.x / NT : 0;
        int kk[2] = {G > 1 ? (int)(threadIdx.x % NT) : (int)threadIdx.x, (int)threadIdx.x + 256};
        const int nk = G > 1 ? (g < G ? 1 : 0) : (kk[1] < NT ? 2 : (kk[0] < NT ? 1 : 0));
        T accM[2] = {0, 0}, accD[2] = {0, 0};
        for (int64_t c0 = 0; c0 < cnt; c0 += CH) {
            const int m = (int)(cnt - c0 < CH ? cnt - c0 : CH);
            const int m4 = (m + 3) >> 2;
            __syncthreads();
            if (threadIdx.x < 4 * m4) {
                const int j = threadIdx.x;
                T x = 0, y = 0, z = 0, st = 0, dx = 0, dy = 0, dz = 0;
                if (j < m) sv.get(s0 + c0 + j, c, x, y, z, st, dx, dy, dz);
                T px = 1, py = 1, pz = 1;
                for (int e = 0; e <= P; ++e) {
                    pw[0][e][j] = px; pw[1][e][j] = py; pw[2][e][j] = pz;
                    px *= x; py *= y; pz *= z;
                }
                sd[0][j] = st; sd[1][j] = dx; sd[2][j] = dy; sd[3][j] = dz;
            }
            __syncthreads();
            for (int r = 0; r < nk; ++r) {
                const int k = kk[r];
                const int k1 = sterm[3 * k], k2 = sterm[3 * k + 1], k3 = sterm[3 * k + 2];
                T aM = accM[r], aD = accD[r];
                for (int q = g; q < m4; q += G) {
                    const int j = 4 * q;
                    const Quad<T> p1 = ld4(&pw[0][k1][j]), p2 = ld4(&pw[1][k2][j]), p3 = ld4(&pw[2][k3][j]);
                    const Quad<T> sq = ld4(&sd[0][j]);
                    const Quad<T> m12 = {p1.x * p2.x, p1.y * p2.y, p1.z * p2.z, p1.w * p2.w};
                    aM += sq.x * (m12.x * p3.x) + sq.y * (m12.y * p3.y) + sq.z * (m12.z * p3.z) + sq.w * (m12.w * p3.w);
                    if (k1) {
                        const Quad<T> q1 = ld4(&pw[0][k1 - 1][j]), d = ld4(&sd[1][j]);
                        aD += (T)k1 * (d.x * q1.x * p2.x * p3.x + d.y * q1.y * p2.y * p3.y + d.z * q1.z * p2.z * p3.z +
                                       d.w * q1.w * p2.w * p3.w);
                    }
                    if (k2) {
                        const Quad<T> q2 = ld4(&pw[1][k2 - 1][j]), d = ld4(&sd[2][j]);
                        aD += (T)k2 * (d.x * p1.x * q2.x * p3.x + d.y * p1.y * q2.y * p3.y + d.z * p1.z * q2.z * p3.z +
                                       d.w * p1.w * q2.w * p3.w);
                    }
                    if (k3) {
                        const Quad<T> q3 = ld4(&pw[2][k3 - 1][j]), d = ld4(&sd[3][j]);
                        aD += (T)k3 * (d.x * m12.x * q3.x + d.y * m12.y * q3.y + d.z * m12.z * q3.z +
                                       d.w * m12.w * q3.w);
                    }
                }
                accM[r] = aM;
                accD[r] = aD;
            }
        }
        if (G > 1) {
            __syncthreads();
            if (nk && g > 0) {
                part[g - 1][0][kk[0]] = accM[0];
                part[g - 1][1][kk[0]] = accD[0];
            }
            __syncthreads();
            if (nk && g == 0) {
                T aM = accM[0], aD = accD[0];
                for (int h = 1; h < G; ++h) {
                    aM += part[h - 1][0][kk[0]];
                    aD += part[h - 1][1][kk[0]];
                }
                mom[(int64_t)node * 2 * NT + kk[0]] = aM;
                mom[(int64_t)node * 2 * NT + NT + kk[0]] = aD;
            }
        } else {
            for (int r = 0; r < nk; ++r) {
                mom[(int64_t)node * 2 * NT + kk[r]] = accM[r];
                mom[(int64_t)node * 2 * NT + NT + kk[r]] = accD[r];
            }
        }
    }
    // ---- climb: the last child to finish computes the parent
    climb_m2m<T>(up, NT, 2 * NT, centre, pofs32, link, ucnt, mom, region, region + 8 * 2 * NT, hs, sbin, sterm,
                 s_next);
}

size_t upward_smem(int NT, size_t elem) {
    const size_t CH = elem == 4 ? kP2MChunk : kP2MChunk / 2;
    const size_t p2m = (3 * (kMaxP + 1) * (CH + 4) + 4 * CH + 2 * 2 * 128) * elem;
    const size_t m2m = (size_t)2 * 8 * 2 * NT * elem;
    return (3 * 455 * sizeof(int) + 31) / 32 * 32 + std::max(p2m, m2m);
}

// ---------------------------------------------------------------- batched operator: one persistent launch
// Several problems' treecode sums in one launch.  A device queue holds
// (pair, phase, first, count) entries: phase 0 = P2P work items, 1 = M2P
// tasks (two box items each), 2 = gathers of consecutive sorted targets.
// Warps take entries in queue order from one counter, so an entry is only
// ever held by a running warp.  P2P and M2P entries never wait; a gather
// entry waits until every P2P and M2P entry of its pair is done (the pair's
// counter reaches `need`).  Those entries come earlier in the queue and are
// held by warps that finish them without waiting, so every wait ends; the
// wait is still bounded: after `cap` polls (or once another warp gave up) the
// warp records PB_ETIMEOUT in status[0], raises the abort flag status[1] and
// skips the entry.  A pair's records are published by a fence of every lane
// before the warp counts the entry done; the waiting warp fences after the
// counter has reached `need`.
struct BatchPair {
    P2PArgs32 p2p;
    M2PArgs32 m2p;
    GatherArgs32 ga;
    int64_t n_m2p_items, ntg;
    int problem;          // index of the problem's active flag
    unsigned need;        // P2P and M2P entries of the pair
    int p2p_two;          // P2P items of up to 64 targets, two per lane
};

// The pair descriptors travel in the launch's parameter space (up to
// kMaxBatchPairs pairs per launch): every field is a warp-uniform constant
// load that the item code can re-read instead of keeping it in a register.
constexpr int kMaxBatchPairs = 30000 / (int)sizeof(BatchPair);
struct BatchArgs {
    BatchPair p[kMaxBatchPairs];
};

template <int P>
__global__ void __launch_bounds__(128, 6) batch_operator_kernel(const __grid_constant__ BatchArgs args,
                                                                const int4 *__restrict__ queue, int64_t nq,
                                                                const int *__restrict__ active,
                                                                unsigned *__restrict__ cnt, int *__restrict__ status,
                                                                long long cap, unsigned extra) {
    constexpr int NQ = radial_stride(P) / 4;
    constexpr int W = NQ > 64 ? NQ : 64;
    __shared__ float4 sh[4][W];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float4 *ws = sh[warp];
    while (true) {
        unsigned k = 0;
        if (lane == 0) k = atomicAdd(cnt, 1u);
        k = __shfl_sync(0xffffffffu, k, 0);
        if ((int64_t)k >= nq) return;
        const int4 e = queue[k];
        const BatchPair &bp = args.p[e.x];
        if (!active[bp.problem]) continue;
        if (e.y == 2) {
            int ok = 1;
            if (lane == 0) {
                const unsigned want = bp.need + extra;
                const volatile unsigned *d = cnt + 1 + e.x;
                const volatile int *abort_flag = status + 1;
                for (long long it = 0; *d < want; ++it) {
                    if (*abort_flag || it >= cap) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(128);
                }
                if (!ok) {
                    atomicExch(status, PB_ETIMEOUT);
                    atomicExch(status + 1, 1);
                }
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) continue;
            __threadfence();
            for (int u0 = 0; u0 < e.w; u0 += 32 / kGatherLanes) {   // the standalone gather's lane groups
                const int u = u0 + lane / kGatherLanes;
                gather32_target<2, kGatherLanes>(bp.ga, bp.ntg, (int64_t)e.z + u, lane % kGatherLanes, u < e.w);
            }
            continue;
        }
        if (e.y == 0) {
            if (bp.p2p_two)
                for (int u = 0; u < e.w; ++u)
                    p2p32x2_item<2, false, true, false>(bp.p2p, (int64_t)e.z + u, lane, ws, ws + 32);
            else
                for (int u = 0; u < e.w; ++u)
                    p2p32_item<2, false, true, false>(bp.p2p, (int64_t)e.z + u, lane, ws, ws + 32);
        } else {
            for (int u = 0; u < e.w; ++u) m2p_ly32x_task<P, 2>(bp.m2p, bp.n_m2p_items, (int64_t)e.z + 2 * u, lane, ws);
        }
        __threadfence();
        __syncwarp();
        if (lane == 0) atomicAdd(cnt + 1 + e.x, 1u);
    }
}

}  // namespace

void upload_term_tables() {
    PB_CUDA_TRY(cudaFuncSetAttribute(upward_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)upward_smem(455, 8)));
    PB_CUDA_TRY(cudaFuncSetAttribute(upward_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)upward_smem(455, 4)));
    PB_CUDA_TRY(cudaFuncSetAttribute(climb_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kClimbMaxShared));
    PB_CUDA_TRY(cudaFuncSetAttribute(climb_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)kClimbMaxShared));
    PB_CUDA_TRY(cudaFuncSetAttribute(m2m_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, kM2MMaxShared));
    PB_CUDA_TRY(cudaFuncSetAttribute(m2m_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, kM2MMaxShared));
    m2p_tc_prepare();
    int terms[3 * kMaxTerms1];
    int i = 0;
    for (int n = 0; n <= kMaxP + 1; ++n)
        for (int k1 = n; k1 >= 0; --k1)
            for (int k2 = n - k1; k2 >= 0; --k2) {
                const int k3 = n - k1 - k2;
                if (term_index(k1, k2, k3) != i) fail(PB_ECUDA, "term table layout");
                terms[3 * i] = k1; terms[3 * i + 1] = k2; terms[3 * i + 2] = k3;
                ++i;
            }
    PB_CUDA_TRY(cudaMemcpyToSymbol(c_terms, terms, sizeof(terms)));
    double bin[13][13] = {};
    for (int n = 0; n <= 12; ++n) {
        bin[n][0] = 1.0;
        for (int k = 1; k <= n; ++k) bin[n][k] = bin[n][k - 1] * (n - k + 1) / k;
    }
    PB_CUDA_TRY(cudaMemcpyToSymbol(c_binom, bin, sizeof(bin)));
    float bin32[13][13];
    for (int n = 0; n <= 12; ++n)
        for (int k = 0; k <= 12; ++k) bin32[n][k] = (float)bin[n][k];
    PB_CUDA_TRY(cudaMemcpyToSymbol(c_binom32, bin32, sizeof(bin32)));
}

void compute_strengths(Tree &Tr, const SurfDev &S, const double *phi, const double *dphi, bool mixed, cudaStream_t s) {
    const int64_t n = Tr.npts;
    if (!n) return;
    if (mixed) {
        Tr.phf.alloc(S.n);
        strengths32_kernel<<<div_up(std::max<int64_t>(n, S.n), 256), 256, 0, s>>>(
            n, Tr.pos32.p, Tr.was.p, Tr.pids.p, S.nrm.p, phi, dphi, Tr.srcA32.p, Tr.srcB32.p, S.n, Tr.phf.p);
    } else {
        strengths64_kernel<<<div_up(n, 256), 256, 0, s>>>(n, Tr.ys.p, Tr.was.p, Tr.pids.p, S.nrm.p, phi, dphi,
                                                          Tr.src64.p);
    }
    PB_LAUNCH_CHECK();
}

size_t radial_floats(int P) { return (size_t)radial_stride(P); }

void upward_pass(Tree &Tr, int P, bool mixed, cudaStream_t s) {
    const int NT = nterms(P);
    if (Tr.ucnt.n != (size_t)Tr.nnodes) {
        Tr.ucnt.alloc(Tr.nnodes);
        Tr.ucnt.zero(s);
    }
    if (mixed) {
        Tr.mom32.alloc((size_t)Tr.nnodes * 2 * NT);
        SrcView<float> sv{Tr.srcA32.p, Tr.srcB32.p};
        upward_kernel<float><<<Tr.nleaves, 256, upward_smem(NT, 4), s>>>(
            Tr.nleaves, Tr.leaf_node.p, Tr.start.p, Tr.count.p, Tr.centre.p, Tr.pofs32.p, Tr.origin[0], Tr.origin[1],
            Tr.origin[2],
            sv, P, NT, Tr.link.p, Tr.ucnt.p, Tr.mom32.p);
        if (P <= kRadialMaxP) {
            PB_LAUNCH_CHECK();
            Tr.rmom32.alloc((size_t)Tr.nnodes * radial_stride(P));
            const unsigned g = (unsigned)div_up((int64_t)Tr.nnodes * (radial_stride(P) / 2), 128);
#define PB_RAD(PP) \
    case PP: radial_moments_kernel<PP><<<g, 128, 0, s>>>(Tr.nnodes, Tr.mom32.p, Tr.rmom32.p); break;
            switch (P) { PB_RAD(0) PB_RAD(1) PB_RAD(2) PB_RAD(3) PB_RAD(4) PB_RAD(5) PB_RAD(6) PB_RAD(7) PB_RAD(8) }
#undef PB_RAD
        }
    } else {
        Tr.mom64.alloc((size_t)Tr.nnodes * 2 * NT);
        SrcView<double> sv{Tr.src64.p};
        upward_kernel<double><<<Tr.nleaves, 256, upward_smem(NT, 8), s>>>(
            Tr.nleaves, Tr.leaf_node.p, Tr.start.p, Tr.count.p, Tr.centre.p, Tr.pofs32.p, Tr.origin[0], Tr.origin[1],
            Tr.origin[2],
            sv, P, NT, Tr.link.p, Tr.ucnt.p, Tr.mom64.p);
    }
    PB_LAUNCH_CHECK();
}

size_t climb_smem(int nval, bool mixed) {
    return (3 * 455 * sizeof(int) + 31) / 32 * 32 + (size_t)2 * 8 * nval * (mixed ? sizeof(float) : sizeof(double));
}

bool climb_fits(int nval, bool mixed) { return climb_smem(nval, mixed) <= kClimbMaxShared; }

void m2m_climb(Tree &Tr, int P, bool mixed, void *mom, int nval, cudaStream_t s) {
    const int NT = nterms(P);
    if (Tr.ucnt.n != (size_t)Tr.nnodes) {
        Tr.ucnt.alloc(Tr.nnodes);
        Tr.ucnt.zero(s);
    }
    const size_t shm = climb_smem(nval, mixed);
    if (shm > kClimbMaxShared) fail(PB_EINVAL, "internal: moment sets too large for the one-launch M2M");
    if (mixed)
        climb_kernel<float><<<Tr.nleaves, 256, shm, s>>>(Tr.nleaves, Tr.leaf_node.p, Tr.centre.p, Tr.pofs32.p, P, NT, nval,
                                                         Tr.link.p, Tr.ucnt.p, (float *)mom);
    else
        climb_kernel<double><<<Tr.nleaves, 256, shm, s>>>(Tr.nleaves, Tr.leaf_node.p, Tr.centre.p, Tr.pofs32.p, P, NT, nval,
                                                          Tr.link.p, Tr.ucnt.p, (double *)mom);
    PB_LAUNCH_CHECK();
}

void m2m_pass(const Tree &Tr, int P, bool mixed, void *mom, int stride, int base, cudaStream_t s) {
    const int NT = nterms(P);
    const size_t shm = (size_t)2 * 8 * 2 * NT * (mixed ? sizeof(float) : sizeof(double)) + 3 * NT * sizeof(int);
    for (int l = Tr.nlevels - 2; l >= 0; --l) {
        const int b0 = Tr.level_off[l], nb = Tr.level_off[l + 1] - b0;
        if (mixed)
            m2m_kernel<float><<<nb, 256, shm, s>>>(b0, Tr.first_child.p, Tr.nchild.p, Tr.centre.p, P, NT, stride, base,
                                                   (float *)mom);
        else
            m2m_kernel<double><<<nb, 256, shm, s>>>(b0, Tr.first_child.p, Tr.nchild.p, Tr.centre.p, P, NT, stride,
                                                    base, (double *)mom);
        PB_LAUNCH_CHECK();
    }
}

P2PArgs32 p2p_args32(const Pair &Pr, const Targets &G, const Tree &Tr, bool use_self) {
    const int nk = (int)Pr.kappas.size();
    P2PArgs32 a{};
    a.items = Pr.p2p_items.p;
    a.inv = Pr.p2p_inv.p;
    a.sent = Pr.p2p_ent.p;
    a.x32 = Pr.x32.p;
    a.selfp = G.self_panel.p;
    a.use_self = use_self ? 1 : 0;
    a.leaf_node = Tr.leaf_node.p;
    a.start = Tr.start.p;
    a.count = Tr.count.p;
    a.A = Tr.srcA32.p;
    a.B = Tr.srcB32.p;
    a.ks = KSet{{(float)Pr.kappas[0], nk > 1 ? (float)Pr.kappas[1] : 0.f}};
    a.part = Pr.p2p_part32.p;
    return a;
}

void launch_p2p(const Pair &Pr, const Targets &G, const Tree &Tr, bool use_self, bool mixed, cudaStream_t s) {
    const int64_t ni = Pr.n_p2p_items;
    if (!ni) return;
    const unsigned grid = (unsigned)((ni + 3) / 4);
    const int nk = (int)Pr.kappas.size();
    const double k0 = Pr.kappas[0], k1 = nk > 1 ? Pr.kappas[1] : 0.0;
    const bool y0 = k0 != 0.0, y1 = k1 != 0.0;
    const int32_t *sp = G.self_panel.p;
    const int us = use_self ? 1 : 0;
    if (mixed) {
        const bool mask = use_self && !Pr.p2p_self_in;
        const P2PArgs32 ga = p2p_args32(Pr, G, Tr, use_self);
#define PB_P2P32M(NK, A, B, M)                                                        \
    do {                                                                              \
        if (Pr.p2p_tile > 32) p2p32x2_kernel<NK, A, B, M><<<grid, 128, 0, s>>>(ni, ga); \
        else p2p32_kernel<NK, A, B, M><<<grid, 128, 0, s>>>(ni, ga);                    \
    } while (0)
#define PB_P2P32(NK, A, B) do { if (mask) PB_P2P32M(NK, A, B, true); else PB_P2P32M(NK, A, B, false); } while (0)
        if (nk == 1) { if (y0) PB_P2P32(1, true, false); else PB_P2P32(1, false, false); }
        else if (!y0 && y1) PB_P2P32(2, false, true);
        else if (y0 && !y1) PB_P2P32(2, true, false);
        else if (y0 && y1) PB_P2P32(2, true, true);
        else PB_P2P32(2, false, false);
#undef PB_P2P32
#undef PB_P2P32M
    } else {
#define PB_P2P64(NK, A, B)                                                                                       \
    p2p64_kernel<NK, A, B><<<grid, 128, 0, s>>>(ni, Pr.p2p_items.p, Pr.p2p_inv.p, Pr.p2p_ent.p, G.xs.p, sp, us,   \
                                                Tr.leaf_node.p, Tr.start.p, Tr.count.p, Tr.src64.p, k0, k1,      \
                                                Pr.p2p_part.p)
        if (nk == 1) { if (y0) PB_P2P64(1, true, false); else PB_P2P64(1, false, false); }
        else if (!y0 && y1) PB_P2P64(2, false, true);
        else if (y0 && !y1) PB_P2P64(2, true, false);
        else if (y0 && y1) PB_P2P64(2, true, true);
        else PB_P2P64(2, false, false);
#undef PB_P2P64
    }
    PB_LAUNCH_CHECK();
}

M2PArgs32 m2p_args32(const Pair &Pr, const Tree &Tr) {
    M2PArgs32 a{};
    a.items = Pr.m2p_items.p;
    a.inv = Pr.m2p_inv.p;
    a.ent = Pr.m2p_ent.p;
    a.x32 = Pr.x32.p;
    a.cen32 = Tr.cen32.p;
    a.rmom = Tr.rmom32.p;
    a.kappa = Pr.kappas.size() > 1 ? (float)Pr.kappas[1] : 0.f;
    a.part = reinterpret_cast<float4 *>(Pr.m2p_part32.p);
    return a;
}

void launch_m2p(const Pair &Pr, const Targets &G, const Tree &Tr, int P, bool mixed, cudaStream_t s, int variant) {
    if (Pr.n_m2p_items == 0) return;
    if (variant == 1 && m2p_tc_eligible(Pr, P, mixed)) {
        launch_m2p_tc(m2p_args32(Pr, Tr), Pr.n_m2p_items, P, s);
        return;
    }
    if (mixed && Pr.kappas.size() == 2 && Pr.kappas[0] == 0.0 && Pr.kappas[1] != 0.0 && P <= kRadialMaxP) {
        const int64_t ni = Pr.n_m2p_items;
        constexpr int NI = 2;   // items per warp (three or four: 99 us against 90 at P = 6, fewer warps per SM)
        const unsigned grid = (unsigned)((ni + 4 * NI - 1) / (4 * NI));
        const M2PArgs32 ga = m2p_args32(Pr, Tr);
#define PB_LY(PP)                                                            \
    case PP:                                                                 \
        m2p_ly32x_kernel<PP, NI><<<grid, 128, 0, s>>>(ni, ga);               \
        break;
        switch (P) {
            PB_LY(0) PB_LY(1) PB_LY(2) PB_LY(3) PB_LY(4) PB_LY(5) PB_LY(6) PB_LY(7) PB_LY(8)
        }
#undef PB_LY
        PB_LAUNCH_CHECK();
        return;
    }
    for (size_t k = 0; k < Pr.kappas.size(); ++k) {
        const double kap = Pr.kappas[k];
        const int nk = (int)Pr.kappas.size();
        if (mixed) {
            launch_m2p_typed<float>(P, kap != 0.0, Pr, G.xs.p, Tr.origin, Tr, Tr.mom32.p, kap, (int)k, nk,
                                    Pr.m2p_part32.p, s);
        } else {
            const double zero[3] = {0.0, 0.0, 0.0};
            launch_m2p_typed<double>(P, kap != 0.0, Pr, G.xs.p, zero, Tr, Tr.mom64.p, kap, (int)k, nk,
                                     Pr.m2p_part64.p, s);
        }
    }
}

GatherArgs32 gather_args32(const Pair &Pr, const Targets &G, bool use_self, const double *dphi, const float2 *phf) {
    const int nk = (int)Pr.kappas.size();
    NearArgs32 nr{};
    nr.ptr = Pr.near_ptr.p;
    nr.panel = Pr.near_panel.p;
    for (int k = 0; k < nk; ++k) {
        nr.dV[k] = Pr.dV32.p + (int64_t)k * Pr.n_near;
        nr.dK[k] = Pr.dK32.p + (int64_t)k * Pr.n_near;
        nr.selfV[k] = use_self ? (Pr.p2p_self_in ? Pr.selfV32[k].p : Pr.selfV[k].p) : nullptr;
    }
    nr.selfp = G.self_panel.p;
    nr.use_self = use_self ? 1 : 0;
    nr.phf = phf;
    nr.dphi = dphi;
    if (Pr.n_near > 0 && !phf) fail(PB_EINVAL, "internal: FP32 densities missing");
    return GatherArgs32{Pr.p2p_ptr.p, Pr.p2p_part32.p, Pr.m2p_ptr.p, Pr.n_m2p_items > 0 ? Pr.m2p_part32.p : nullptr,
                        nr, Pr.VK[0].p, nk > 1 ? Pr.VK[1].p : nullptr};
}

void launch_gather(const Pair &Pr, const Targets &G, bool mixed, bool use_self, const double *phi,
                   const double *dphi, const float2 *phf, cudaStream_t s) {
    const int64_t ntg = G.n;
    if (!ntg) return;
    const int nk = (int)Pr.kappas.size();
    const bool far = Pr.n_m2p_items > 0;
    double *V0 = Pr.VK[0].p, *V1 = nk > 1 ? Pr.VK[1].p : nullptr;
    const unsigned grid = (unsigned)((ntg + 3) / 4);
    if (mixed) {
        const GatherArgs32 ga = gather_args32(Pr, G, use_self, dphi, phf);
        constexpr int TPB = 4 * (32 / kGatherLanes);   // targets per block
        const unsigned g8 = (unsigned)((ntg + TPB - 1) / TPB);
        if (nk == 1) gather32_kernel<1><<<g8, 128, 0, s>>>(ntg, ga);
        else gather32_kernel<2, 8><<<g8, 128, 0, s>>>(ntg, ga);
    } else {
        NearArgs nr{};
        nr.ptr = Pr.near_ptr.p;
        nr.panel = Pr.near_panel.p;
        for (int k = 0; k < nk; ++k) {
            nr.dV[k] = Pr.dV[k].p;
            nr.dK[k] = Pr.dK[k].p;
            nr.selfV[k] = use_self ? Pr.selfV[k].p : nullptr;
        }
        nr.selfp = G.self_panel.p;
        nr.use_self = use_self ? 1 : 0;
        nr.phi = phi;
        nr.dphi = dphi;
        const double *mp = far ? Pr.m2p_part64.p : nullptr;
        if (nk == 1)
            gather_kernel<double, 1><<<grid, 128, 0, s>>>(ntg, Pr.p2p_ptr.p, Pr.p2p_part.p, Pr.m2p_ptr.p, mp,
                                                          nr, V0, V1);
        else
            gather_kernel<double, 2><<<grid, 128, 0, s>>>(ntg, Pr.p2p_ptr.p, Pr.p2p_part.p, Pr.m2p_ptr.p, mp,
                                                          nr, V0, V1);
    }
    PB_LAUNCH_CHECK();
}

__global__ void targets32_kernel(int64_t n, const double *__restrict__ xs, double ox, double oy, double oz,
                                 float4 *__restrict__ x32) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x32[i] = make_float4((float)(xs[3 * i] - ox), (float)(xs[3 * i + 1] - oy), (float)(xs[3 * i + 2] - oz), 0.f);
}

void targets_to_float(Pair &Pr, const Targets &G, const Tree &Tr, cudaStream_t s) {
    Pr.x32.alloc(std::max<int64_t>(1, G.n));
    if (!G.n) return;
    targets32_kernel<<<div_up(G.n, 256), 256, 0, s>>>(G.n, G.xs.p, Tr.origin[0], Tr.origin[1], Tr.origin[2], Pr.x32.p);
    PB_LAUNCH_CHECK();
}

void launch_combine_pair(int64_t n, const int32_t *rank, const double *phi_s, double half, const CombineRow &row0,
                         const CombineRow &row1, double *y, cudaStream_t s) {
    if (!n) return;
    combine_pair_kernel<<<div_up(2 * n, 256), 256, 0, s>>>(n, rank, phi_s, half, row0, row1, y);
    PB_LAUNCH_CHECK();
}

void launch_combine(int64_t n, const int32_t *rank, const double *phi_s, double half, const CombineRow &row, double *y,
                    cudaStream_t s) {
    if (!n) return;
    combine_kernel<<<div_up(n, 256), 256, 0, s>>>(n, rank, phi_s, half, row, y);
    PB_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- batched operator (host)
namespace {

constexpr int kBatchPer = 8;   // work items (P2P), two-item tasks (M2P) or targets (gather) per queue entry

// PB_FAULT=wait (read when the library is loaded): every gather of a batched
// operator application waits for one entry more than its pair has, so the
// bounded wait runs out (test of the timeout path; nothing else changes).
bool fault_wait() {
    const char *e = std::getenv("PB_FAULT");
    return e && std::strcmp(e, "wait") == 0;
}
const bool g_fault_wait = fault_wait();

template <int P>
int batch_grid() {
    int nsm = 0, dev = 0, per = 0;
    PB_CUDA_TRY(cudaGetDevice(&dev));
    PB_CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    PB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, batch_operator_kernel<P>, 128, 0));
    return std::max(1, nsm * std::max(1, per));
}

}  // namespace

BatchPlan::~BatchPlan() {
    if (ev) cudaEventDestroy(ev);
}

bool batch_pair_eligible(const Pair &Pr, const Params &prm, bool use_self) {
    return prm.precision == PB_MIXED && Pr.kappas.size() == 2 && Pr.kappas[0] == 0.0 && Pr.kappas[1] != 0.0 &&
           prm.P >= 0 && prm.P <= kRadialMaxP && !(use_self && !Pr.p2p_self_in);
}

void batch_plan_build(BatchPlan &bp, const std::vector<BatchPairRef> &prs, int nproblems, int P, cudaStream_t s) {
    if (P < 0 || P > kRadialMaxP) fail(PB_EINVAL, "internal: batched operator needs the radial-form M2P");
    bp.P = P;
    bp.nproblems = nproblems;
    bp.npairs = (int)prs.size();
    bp.seg_args.clear();
    bp.seg_q.clear();
    std::vector<int4> q;
    // segments of at most kMaxBatchPairs pairs, one launch each
    for (size_t p0 = 0; p0 < prs.size(); p0 += kMaxBatchPairs) {
        const size_t p1 = std::min(prs.size(), p0 + (size_t)kMaxBatchPairs);
        std::vector<unsigned char> bytes(sizeof(BatchArgs), 0);
        BatchArgs &args = *reinterpret_cast<BatchArgs *>(bytes.data());
        const int64_t q0 = (int64_t)q.size();
        auto gathers = [&](int k) {
            const int64_t n = args.p[k].ntg;
            for (int64_t t = 0; t < n; t += kBatchPer)
                q.push_back(make_int4(k, 2, (int)t, (int)std::min<int64_t>(kBatchPer, n - t)));
        };
        for (size_t k = 0; k < p1 - p0; ++k) {
            const BatchPairRef &r = prs[p0 + k];
            const Pair &Pr = *r.P;
            if (Pr.n_p2p_items >= INT32_MAX || Pr.n_m2p_items >= INT32_MAX || r.G->n >= INT32_MAX)
                fail(PB_EINVAL, "internal: batched operator pair too large");
            BatchPair &b = args.p[k];
            b.p2p = p2p_args32(Pr, *r.G, *r.T, r.use_self);
            b.p2p_two = Pr.p2p_tile > 32 ? 1 : 0;
            b.m2p = m2p_args32(Pr, *r.T);
            b.ga = gather_args32(Pr, *r.G, r.use_self, r.dphi, r.T->phf.p);
            b.n_m2p_items = Pr.n_m2p_items;
            b.ntg = r.G->n;
            b.problem = r.problem;
            const size_t e0 = q.size();
            for (int64_t i = 0; i < Pr.n_p2p_items; i += kBatchPer)
                q.push_back(make_int4((int)k, 0, (int)i, (int)std::min<int64_t>(kBatchPer, Pr.n_p2p_items - i)));
            const int64_t ntask = (Pr.n_m2p_items + 1) / 2;
            for (int64_t t = 0; t < ntask; t += kBatchPer)
                q.push_back(make_int4((int)k, 1, (int)(2 * t), (int)std::min<int64_t>(kBatchPer, ntask - t)));
            b.need = (unsigned)(q.size() - e0);
            // a pair's gathers follow the next pair's direct and far-field entries
            if (k > 0) gathers((int)k - 1);
        }
        gathers((int)(p1 - p0) - 1);
        bp.seg_args.push_back(std::move(bytes));
        bp.seg_q.emplace_back(q0, (int64_t)q.size() - q0);
    }
    bp.queue.alloc(std::max<size_t>(1, q.size()));
    if (!q.empty()) bp.queue.upload(q.data(), q.size(), s);
    bp.cnt.alloc(std::max<size_t>(1, bp.seg_args.size()) * (1 + kMaxBatchPairs));
    bp.active.alloc(std::max(1, nproblems));
    bp.status.alloc(2);
    bp.active_h.alloc(std::max(1, nproblems));
    bp.status_h.alloc(2);
    for (int i = 0; i < nproblems; ++i) bp.active_h.p[i] = 0;
    bp.status_h.p[0] = PB_OK;
    bp.status_h.p[1] = 0;
    bp.extra = g_fault_wait ? 1u : 0u;
    bp.cap = g_fault_wait ? (1ll << 12) : (1ll << 24);   // polls 128 ns apart: ~0.5 ms / ~2 s
    if (!bp.ev) PB_CUDA_TRY(cudaEventCreateWithFlags(&bp.ev, cudaEventDisableTiming));
    switch (P) {
#define PB_BG(PP) case PP: bp.grid = batch_grid<PP>(); break;
        PB_BG(0) PB_BG(1) PB_BG(2) PB_BG(3) PB_BG(4) PB_BG(5) PB_BG(6) PB_BG(7) PB_BG(8)
#undef PB_BG
    }
}

void batch_operator_launch(BatchPlan &bp, cudaStream_t s) {
    PB_CUDA_TRY(cudaMemcpyAsync(bp.active.p, bp.active_h.p, sizeof(int) * std::max(1, bp.nproblems),
                                cudaMemcpyHostToDevice, s));
    PB_CUDA_TRY(cudaMemsetAsync(bp.cnt.p, 0, sizeof(unsigned) * bp.cnt.n, s));
    PB_CUDA_TRY(cudaMemsetAsync(bp.status.p, 0, 2 * sizeof(int), s));
    for (size_t g = 0; g < bp.seg_args.size(); ++g) {
        const BatchArgs &args = *reinterpret_cast<const BatchArgs *>(bp.seg_args[g].data());
        const int4 *queue = bp.queue.p + bp.seg_q[g].first;
        const int64_t nq = bp.seg_q[g].second;
        unsigned *cnt = bp.cnt.p + g * (1 + kMaxBatchPairs);
        switch (bp.P) {
#define PB_BL(PP)                                                                                                 \
    case PP:                                                                                                      \
        batch_operator_kernel<PP><<<bp.grid, 128, 0, s>>>(args, queue, nq, bp.active.p, cnt, bp.status.p,         \
                                                          bp.cap, bp.extra);                                      \
        break;
            PB_BL(0) PB_BL(1) PB_BL(2) PB_BL(3) PB_BL(4) PB_BL(5) PB_BL(6) PB_BL(7) PB_BL(8)
#undef PB_BL
        }
        PB_LAUNCH_CHECK();
    }
    PB_CUDA_TRY(cudaMemcpyAsync(bp.status_h.p, bp.status.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
}

}  // namespace pb
