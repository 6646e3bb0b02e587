// Adjoint of the treecode BEM operator and the gradient of the solvation
// energy (Eq. solv) with respect to the charges, their positions, and the
// permittivity and inverse Debye length of every region.
//
// With the operator A (Eq. matrix, multi-surface form), b = B q (Eq. matel,
// Q) and the reaction-potential map phi_reac = Rm x (Eq. reac_integral),
//   E = c0 q^T Rm x,  A x = b,  c0 = C/2 * 4 pi,
// and the adjoint A^T lambda = c0 Rm^T q,
//   dE/dq_k = c0 (Rm x)_k + (B^T lambda)_k
//   dE/dr_k = c0 q_k grad (Rm x)_k + q_k lambda^T grad_k B
//   dE/dp   = c0 q^T (dRm/dp) x + lambda^T (db/dp - (dA/dp) x).
//
// Transposed treecode.  A block V (entries sum_q w_q A_j G(x_i, y_jq)) and K
// (sum_q w_q A_j n_j . grad_y G(x_i, y_jq)) transpose to
//   (V^T mu)_j = sum_q w_q A_j phi_mu(y_jq),   phi_mu(y) = sum_i mu_i G(x_i, y)
//   (K^T nu)_j = sum_q w_q A_j n_j . grad phi_nu(y_jq),
// so the transposed product is a treecode whose sources are the collocation
// points x_i (monopoles mu_i, nu_i: the row weights lambda folded with each
// block's coefficients) and whose targets are the Gauss points y_jq.  Direct
// sums run over the leaves that fail the MAC; the far field of a box with
// monopole moments M^k = sum_i mu_i (x_i - x_c)^k is sum_k a^k(u) M^k with
// u = x_c - y and the coefficients a^k of the forward treecode, and its
// target-normal derivative is
//   n . grad_y phi = -sum_{1 <= |m| <= P} a^m sum_l n_l m_l N^(m - e_l),
// truncated like the forward double layer (whose dipole moments pair order-P
// coefficients with order-(P-1) source monomials).  The near-singular and
// self corrections of the forward operator enter transposed.
//
// Kernel derivatives (r = x - y, rho = |r|, e = exp(-kappa rho), all / 4 pi):
//   dG/dkappa = -e,  d(n . grad_y G)/dkappa = -kappa (r . n) e / rho,
//   grad_x G_L = -r / rho^3,  grad_x (n . grad_y G_L) = n / rho^3 - 3 (r . n) r / rho^5.
// The kappa derivative of the far field differentiates the coefficient
// recurrence (a, b -> da/dkappa, db/dkappa) alongside it.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "adjoint.cuh"
#include "geometry.cuh"
#include "tree.cuh"
#include "treecode.cuh"
#include "radial.cuh"

namespace pb {

namespace {

constexpr double kC0 = 0.5 * kKjPerMol * 4.0 * kPi;

__constant__ int c_aterms[3 * kMaxTerms1];
__constant__ TriRule c_arules[4];

__host__ __device__ constexpr int tindex(int k1, int k2, int k3) {
    // graded by n = |k|, then k1 descending, then k2 descending (the forward layout)
    return (k1 + k2 + k3) * (k1 + k2 + k3 + 1) * (k1 + k2 + k3 + 2) / 6 + (k2 + k3) * (k2 + k3 + 1) / 2 + k3;
}

// ---------------------------------------------------------------- targets and strengths
__global__ void gnormals_kernel(int64_t n, int K, const int32_t *__restrict__ order, const double *__restrict__ nrm,
                                double *__restrict__ n64, float4 *__restrict__ n32) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int j = order[q] / K;
    const double a = nrm[3 * j], b = nrm[3 * j + 1], c = nrm[3 * j + 2];
    n64[3 * q] = a; n64[3 * q + 1] = b; n64[3 * q + 2] = c;
    n32[q] = make_float4((float)a, (float)b, (float)c, 0.f);
}

struct FoldCoef {
    double cV[2][2], cK[2][2];
};

// mu_k = sum_side cV[k][side] u_side, nu_k = sum_side cK[k][side] u_side per source.
__global__ void fold_kernel(int64_t n, int nk, FoldCoef fc, const double *__restrict__ u0,
                            const double *__restrict__ u1, double *__restrict__ fold) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = u0[i], b = u1 ? u1[i] : 0.0;
    for (int k = 0; k < nk; ++k) {
        fold[(2 * k) * n + i] = fc.cV[k][0] * a + fc.cV[k][1] * b;
        fold[(2 * k + 1) * n + i] = fc.cK[k][0] * a + fc.cK[k][1] * b;
    }
}

__global__ void tstrengths64_kernel(int64_t n, const double *__restrict__ ys, const int32_t *__restrict__ pids,
                                    const double *__restrict__ fold, int64_t nsrc, int nk, double *__restrict__ src) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = pids[q];
    double *o = src + 8 * q;
    o[0] = ys[3 * q]; o[1] = ys[3 * q + 1]; o[2] = ys[3 * q + 2];
    o[3] = fold[i];
    o[4] = fold[nsrc + i];
    o[5] = nk > 1 ? fold[2 * nsrc + i] : 0.0;
    o[6] = nk > 1 ? fold[3 * nsrc + i] : 0.0;
    o[7] = (double)i;
}

__global__ void tstrengths32_kernel(int64_t n, const float4 *__restrict__ pos, const int32_t *__restrict__ pids,
                                    const double *__restrict__ fold, int64_t nsrc, int nk, float4 *__restrict__ A,
                                    float4 *__restrict__ B) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int i = pids[q];
    const float4 p = pos[q];
    A[q] = make_float4(p.x, p.y, p.z, (float)fold[i]);
    B[q] = make_float4((float)fold[nsrc + i], nk > 1 ? (float)fold[2 * nsrc + i] : 0.f,
                       nk > 1 ? (float)fold[3 * nsrc + i] : 0.f, __int_as_float(i));
}

// ---------------------------------------------------------------- P2M of monopole sets
template <typename T>
struct TSrc;

template <>
struct TSrc<double> {
    const double *src;
    __device__ void get(int64_t q, const double c[3], double &x, double &y, double &z, double s[4]) const {
        const double *o = src + 8 * q;
        x = o[0] - c[0]; y = o[1] - c[1]; z = o[2] - c[2];
        s[0] = o[3]; s[1] = o[4]; s[2] = o[5]; s[3] = o[6];
    }
};

template <>
struct TSrc<float> {
    const float4 *A, *B;
    __device__ void get(int64_t q, const float c[3], float &x, float &y, float &z, float s[4]) const {
        const float4 a = A[q], b = B[q];
        x = a.x - c[0]; y = a.y - c[1]; z = a.z - c[2];
        s[0] = a.w; s[1] = b.x; s[2] = b.y; s[3] = b.z;
    }
};

// One block per leaf; NS (2 or 4) monopole moment sets M^k = sum_i s_i (x_i - x_c)^k,
// stored per node as NS consecutive runs of NT terms.
template <typename T>
__global__ void __launch_bounds__(128) p2m_mono_kernel(int nleaves, const int32_t *__restrict__ leaf_node,
                                                       const int64_t *__restrict__ start,
                                                       const int64_t *__restrict__ count,
                                                       const double *__restrict__ centre, double ox, double oy,
                                                       double oz, TSrc<T> sv, int P, int NT, int NS,
                                                       T *__restrict__ mom) {
    constexpr int CH = sizeof(T) == 4 ? 128 : 64;
    __shared__ T pw[3][kMaxP + 1][CH];
    __shared__ T sd[4][CH];
    __shared__ int sterm[3 * 455];
    const int node = leaf_node[blockIdx.x];
    const int64_t s0 = start[node], cnt = count[node];
    T c[3];
    if (sizeof(T) == 8) {
        c[0] = (T)centre[3 * node]; c[1] = (T)centre[3 * node + 1]; c[2] = (T)centre[3 * node + 2];
    } else {
        c[0] = (T)(centre[3 * node] - ox); c[1] = (T)(centre[3 * node + 1] - oy); c[2] = (T)(centre[3 * node + 2] - oz);
    }
    for (int i = threadIdx.x; i < 3 * NT; i += blockDim.x) sterm[i] = c_aterms[i];
    T acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[r][t] = 0;
    for (int64_t c0 = 0; c0 < cnt; c0 += CH) {
        const int m = (int)(cnt - c0 < CH ? cnt - c0 : CH);
        __syncthreads();
        if (threadIdx.x < m) {
            T x, y, z, st[4];
            sv.get(s0 + c0 + threadIdx.x, c, x, y, z, st);
            T px = 1, py = 1, pz = 1;
            for (int e = 0; e <= P; ++e) {
                pw[0][e][threadIdx.x] = px; pw[1][e][threadIdx.x] = py; pw[2][e][threadIdx.x] = pz;
                px *= x; py *= y; pz *= z;
            }
#pragma unroll
            for (int t = 0; t < 4; ++t) sd[t][threadIdx.x] = st[t];
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int k = threadIdx.x + 128 * r;
            if (k >= NT) break;
            const int k1 = sterm[3 * k], k2 = sterm[3 * k + 1], k3 = sterm[3 * k + 2];
            for (int j = 0; j < m; ++j) {
                const T p = pw[0][k1][j] * pw[1][k2][j] * pw[2][k3][j];
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (t < NS) acc[r][t] += sd[t][j] * p;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int k = threadIdx.x + 128 * r;
        if (k >= NT) break;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (t < NS) mom[(int64_t)node * NS * NT + t * NT + k] = acc[r][t];
    }
}

// ---------------------------------------------------------------- transposed P2P
// Leaf-major like the forward P2P: one warp per (leaf, up to 32 targets) item,
// sources staged in shared memory; every lane owns one Gauss-point target with
// its panel normal n.  Per pair (d = source - target): V += mu / rho,
// K += nu (d . n) / rho^3, times exp(-kappa rho) and (1 + kappa rho) exp(-kappa rho)
// for a Yukawa kernel.
struct TKSet {
    float kap[2];
};

// Single-instruction PTX approximations (flush-to-zero), as in the forward P2P.
__device__ __forceinline__ float tfast_rsqrt(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float tfast_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void tcomp_add(float &hi, float &lo, float v) {
    const float t = hi + v;
    lo += (fabsf(hi) >= fabsf(v)) ? ((hi - t) + v) : ((v - t) + hi);
    hi = t;
}

template <int NK, bool Y0, bool Y1>
__global__ void __launch_bounds__(128) p2pT32_kernel(int64_t nitems, const int4 *__restrict__ items,
                                                     const int32_t *__restrict__ inv,
                                                     const int32_t *__restrict__ sent, const float4 *__restrict__ x32,
                                                     const float4 *__restrict__ n32, const int32_t *__restrict__ selfp,
                                                     int use_self, const int32_t *__restrict__ leaf_node,
                                                     const int64_t *__restrict__ start,
                                                     const int64_t *__restrict__ count, const float4 *__restrict__ A,
                                                     const float4 *__restrict__ B, TKSet ks, float *__restrict__ part) {
    __shared__ float4 sA[4][32], sB[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 4 + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    const bool valid = lane < it.z;
    const int64_t slot = (int64_t)it.y + lane;
    float tx = 0.f, ty = 0.f, tz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f;
    int me = -1;
    if (valid) {
        const int t = inv[slot];
        const float4 x = x32[t];
        const float4 nn = n32[t];
        tx = x.x; ty = x.y; tz = x.z;
        nx = nn.x; ny = nn.y; nz = nn.z;
        if (use_self) me = selfp[t];
    }
    const float k0 = ks.kap[0], k1 = ks.kap[1];
    const float l2e0 = -k0 * 1.4426950408889634f, l2e1 = -k1 * 1.4426950408889634f;
    float hi[2 * NK], lo[2 * NK];
#pragma unroll
    for (int a = 0; a < 2 * NK; ++a) { hi[a] = 0.f; lo[a] = 0.f; }
    const int node = leaf_node[it.x];
    const int64_t s0 = start[node];
    const int cnt = (int)count[node];
    for (int c0 = 0; c0 < cnt; c0 += 32) {
        const int m = min(32, cnt - c0);
        if (lane < m) {
            sA[warp][lane] = A[s0 + c0 + lane];
            sB[warp][lane] = B[s0 + c0 + lane];
        }
        __syncwarp();
        if (valid) {
            float p[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
            for (int j = 0; j < m; ++j) {
                const float4 a = sA[warp][j];
                const float4 b = sB[warp][j];
                const float dx = a.x - tx, dy = a.y - ty, dz = a.z - tz;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                const float iv = (__float_as_int(b.w) == me) ? 0.f : tfast_rsqrt(r2);
                const float rn = fmaf(dx, nx, fmaf(dy, ny, dz * nz));
                const float i3 = iv * iv * iv;
                if (!Y0) {
                    p[0] = fmaf(a.w, iv, p[0]);
                    p[1] = fmaf(b.x * rn, i3, p[1]);
                } else {
                    const float rho = r2 * iv;
                    const float ex = tfast_ex2(l2e0 * rho);
                    p[0] = fmaf(a.w * iv, ex, p[0]);
                    p[1] = fmaf(b.x * rn * i3 * ex, fmaf(k0, rho, 1.f), p[1]);
                }
                if (NK == 2) {
                    if (!Y1) {
                        p[2] = fmaf(b.y, iv, p[2]);
                        p[3] = fmaf(b.z * rn, i3, p[3]);
                    } else {
                        const float rho = r2 * iv;
                        const float ex = tfast_ex2(l2e1 * rho);
                        p[2] = fmaf(b.y * iv, ex, p[2]);
                        p[3] = fmaf(b.z * rn * i3 * ex, fmaf(k1, rho, 1.f), p[3]);
                    }
                }
            }
#pragma unroll
            for (int a = 0; a < 2 * NK; ++a) tcomp_add(hi[a], lo[a], p[a]);
        }
        __syncwarp();
    }
    if (valid) {
        float2 *rec = reinterpret_cast<float2 *>(part + (int64_t)2 * NK * sent[slot]);
#pragma unroll
        for (int a = 0; a < NK; ++a) rec[a] = make_float2(hi[2 * a] + lo[2 * a], hi[2 * a + 1] + lo[2 * a + 1]);
    }
}

template <int NK, bool Y0, bool Y1>
__global__ void __launch_bounds__(128) p2pT64_kernel(int64_t nitems, const int4 *__restrict__ items,
                                                     const int32_t *__restrict__ inv,
                                                     const int32_t *__restrict__ sent, const double *__restrict__ xs,
                                                     const double *__restrict__ n64, const int32_t *__restrict__ selfp,
                                                     int use_self, const int32_t *__restrict__ leaf_node,
                                                     const int64_t *__restrict__ start,
                                                     const int64_t *__restrict__ count, const double *__restrict__ src,
                                                     double kap0, double kap1, double *__restrict__ part) {
    __shared__ dvec4 sA[4][32], sB[4][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 4 + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    const bool valid = lane < it.z;
    const int64_t slot = (int64_t)it.y + lane;
    double tx = 0, ty = 0, tz = 0, nx = 0, ny = 0, nz = 0;
    int me = -1;
    if (valid) {
        const int t = inv[slot];
        tx = xs[3 * t]; ty = xs[3 * t + 1]; tz = xs[3 * t + 2];
        nx = n64[3 * t]; ny = n64[3 * t + 1]; nz = n64[3 * t + 2];
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
                const double dx = a.x - tx, dy = a.y - ty, dz = a.z - tz;
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double rho = sqrt(r2);
                const double iv = 1.0 / rho;
                const double rn = dx * nx + dy * ny + dz * nz;
                const double i3 = iv * iv * iv;
                if (!Y0) {
                    acc[0] += a.w * iv;
                    acc[1] += b.x * rn * i3;
                } else {
                    const double ex = exp(-kap0 * rho);
                    acc[0] += a.w * iv * ex;
                    acc[1] += b.x * rn * i3 * ex * (1.0 + kap0 * rho);
                }
                if (NK == 2) {
                    if (!Y1) {
                        acc[2] += b.y * iv;
                        acc[3] += b.z * rn * i3;
                    } else {
                        const double ex = exp(-kap1 * rho);
                        acc[2] += b.y * iv * ex;
                        acc[3] += b.z * rn * i3 * ex * (1.0 + kap1 * rho);
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

// ---------------------------------------------------------------- transposed M2P
// V = sum_{|k| <= P} a^k M^k and K = -sum_{1 <= |m| <= P} a^m sum_l n_l m_l N^(m - e_l)
// with the forward recurrences for a^k (and b^k, the coefficients of exp(-kappa r)).
template <int P, bool YUK, typename T>
__device__ __forceinline__ void m2pT_eval(T ux, T uy, T uz, T nx, T ny, T nz, T kappa, const T *__restrict__ mM,
                                          const T *__restrict__ mN, T &V, T &K) {
    constexpr int NT1 = (P + 1) * (P + 2) * (P + 3) / 6;
    T a[NT1];
    T b[YUK ? NT1 : 1];
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
    V = a[0] * mM[0];
    K = 0;
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        const T c1 = (T)(2 * n - 1) / (T)n, c2 = (T)(n - 1) / (T)n;
        const T kn = kappa / (T)n;
#pragma unroll
        for (int k1 = n; k1 >= 0; --k1) {
#pragma unroll
            for (int k2 = n - k1; k2 >= 0; --k2) {
                const int k3 = n - k1 - k2;
                const int i = tindex(k1, k2, k3);
                T s1 = 0, s2 = 0, t1 = 0, t2 = 0;
                if (k1 >= 1) { s1 += ux * a[tindex(k1 - 1, k2, k3)]; if (YUK) t1 += ux * b[tindex(k1 - 1, k2, k3)]; }
                if (k2 >= 1) { s1 += uy * a[tindex(k1, k2 - 1, k3)]; if (YUK) t1 += uy * b[tindex(k1, k2 - 1, k3)]; }
                if (k3 >= 1) { s1 += uz * a[tindex(k1, k2, k3 - 1)]; if (YUK) t1 += uz * b[tindex(k1, k2, k3 - 1)]; }
                if (k1 >= 2) { s2 += a[tindex(k1 - 2, k2, k3)]; if (YUK) t2 += b[tindex(k1 - 2, k2, k3)]; }
                if (k2 >= 2) { s2 += a[tindex(k1, k2 - 2, k3)]; if (YUK) t2 += b[tindex(k1, k2 - 2, k3)]; }
                if (k3 >= 2) { s2 += a[tindex(k1, k2, k3 - 2)]; if (YUK) t2 += b[tindex(k1, k2, k3 - 2)]; }
                T ai = c1 * s1 + c2 * s2;
                if (YUK) ai += kn * (t1 + t2);
                a[i] = -ai * ir2;
                if (YUK) b[i] = -kn * (s1 + s2);
                V += a[i] * mM[i];
                T g = 0;
                if (k1 >= 1) g += nx * (T)k1 * mN[tindex(k1 - 1, k2, k3)];
                if (k2 >= 1) g += ny * (T)k2 * mN[tindex(k1, k2 - 1, k3)];
                if (k3 >= 1) g += nz * (T)k3 * mN[tindex(k1, k2, k3 - 1)];
                K -= a[i] * g;
            }
        }
    }
}

template <bool YUK, typename T>
__device__ void m2pT_eval_rt(int P, T ux, T uy, T uz, T nx, T ny, T nz, T kappa, const T *__restrict__ mM,
                             const T *__restrict__ mN, T &V, T &K) {
    const int NT1 = (P + 1) * (P + 2) * (P + 3) / 6;
    T a[455];
    T b[YUK ? 455 : 1];
    const T r2 = ux * ux + uy * uy + uz * uz;
    const T r = sqrt(r2);
    const T ir2 = (T)1 / r2;
    const T e0 = YUK ? (T)exp(-kappa * r) : (T)1;
    a[0] = e0 / r;
    if (YUK) b[0] = e0;
    V = a[0] * mM[0];
    K = 0;
    for (int i = 1; i < NT1; ++i) {
        const int k1 = c_aterms[3 * i], k2 = c_aterms[3 * i + 1], k3 = c_aterms[3 * i + 2];
        const int n = k1 + k2 + k3;
        T s1 = 0, s2 = 0, t1 = 0, t2 = 0;
        if (k1 >= 1) { s1 += ux * a[tindex(k1 - 1, k2, k3)]; if (YUK) t1 += ux * b[tindex(k1 - 1, k2, k3)]; }
        if (k2 >= 1) { s1 += uy * a[tindex(k1, k2 - 1, k3)]; if (YUK) t1 += uy * b[tindex(k1, k2 - 1, k3)]; }
        if (k3 >= 1) { s1 += uz * a[tindex(k1, k2, k3 - 1)]; if (YUK) t1 += uz * b[tindex(k1, k2, k3 - 1)]; }
        if (k1 >= 2) { s2 += a[tindex(k1 - 2, k2, k3)]; if (YUK) t2 += b[tindex(k1 - 2, k2, k3)]; }
        if (k2 >= 2) { s2 += a[tindex(k1, k2 - 2, k3)]; if (YUK) t2 += b[tindex(k1, k2 - 2, k3)]; }
        if (k3 >= 2) { s2 += a[tindex(k1, k2, k3 - 2)]; if (YUK) t2 += b[tindex(k1, k2, k3 - 2)]; }
        T ai = ((T)(2 * n - 1) * s1 + (T)(n - 1) * s2) / (T)n;
        if (YUK) ai += kappa / (T)n * (t1 + t2);
        a[i] = -ai * ir2;
        if (YUK) b[i] = -kappa / (T)n * (s1 + s2);
        V += a[i] * mM[i];
        T g = 0;
        if (k1 >= 1) g += nx * (T)k1 * mN[tindex(k1 - 1, k2, k3)];
        if (k2 >= 1) g += ny * (T)k2 * mN[tindex(k1, k2 - 1, k3)];
        if (k3 >= 1) g += nz * (T)k3 * mN[tindex(k1, k2, k3 - 1)];
        K -= a[i] * g;
    }
}

// Box-major: one warp per (box, up to 32 targets) item.
template <int P, bool YUK, typename T>
__global__ void __launch_bounds__(128) m2pT_kernel(int64_t nitems, const int4 *__restrict__ items,
                                                   const int32_t *__restrict__ inv,
                                                   const int32_t *__restrict__ ent, int Prt,
                                                   const double *__restrict__ xs, const float4 *__restrict__ x32,
                                                   const double *__restrict__ n64, const float4 *__restrict__ n32,
                                                   const double *__restrict__ centre,
                                                   const float4 *__restrict__ cen32, const T *__restrict__ mom,
                                                   int64_t stride, double kappa, int kslot, int nk,
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
    T ux, uy, uz, nx, ny, nz;
    if constexpr (sizeof(T) == 4) {
        const float4 c = cen32[b];
        const float4 x = x32[t];
        const float4 nn = n32[t];
        ux = c.x - x.x; uy = c.y - x.y; uz = c.z - x.z;
        nx = nn.x; ny = nn.y; nz = nn.z;
    } else {
        ux = centre[3 * b] - xs[3 * t];
        uy = centre[3 * b + 1] - xs[3 * t + 1];
        uz = centre[3 * b + 2] - xs[3 * t + 2];
        nx = n64[3 * t]; ny = n64[3 * t + 1]; nz = n64[3 * t + 2];
    }
    const T *mM = mom + (int64_t)b * stride + (int64_t)2 * kslot * NT;
    T V, K;
    if constexpr (P >= 0) m2pT_eval<(P >= 0 ? P : 0), YUK, T>(ux, uy, uz, nx, ny, nz, (T)kappa, mM, mM + NT, V, K);
    else m2pT_eval_rt<YUK, T>(Prt, ux, uy, uz, nx, ny, nz, (T)kappa, mM, mM + NT, V, K);
    T *rec = part + (int64_t)2 * nk * ent[slot] + 2 * kslot;
    rec[0] = V;
    rec[1] = K;
}

bool radial_pair(const TPair &tp, const Params &prm);
size_t radialT_floats_per_node(int P);

// ---------------------------------------------------------------- transposed M2P in radial form (FP32)
// For a pair whose kernels are Laplace (slot 0) and Yukawa (slot 1), both
// transposed sums in one pass.  With u = y_c - x and the radial expansion
// of radial.cuh, the monopole potential of the box is
//   Phi_mu(x) = sum_{alpha, n} u^alpha F_n N^mu_{alpha,n}          (order P),
// and the target-normal field of the nu monopoles (expansion of order P - 1) is
//   n . grad_x Phi_nu = -sum_{alpha, m} N^nu_{alpha,m} [ (n . grad u^alpha) F_m + (n . u) u^alpha F_{m+1} ],
// since grad_x u^alpha = -grad_u u^alpha and grad_x F_m(|u|) = -u F_{m+1}.
// Per node the radial moments are [mu_0 (order P), nu_0 (order P - 1),
// mu_1 (order P), nu_1 (order P - 1)], padded to 16 bytes.
__host__ __device__ constexpr int radialT_floats(int P) { return 2 * (radial_terms(P) + radial_terms(P - 1)); }
__host__ __device__ constexpr int radialT_stride(int P) { return (radialT_floats(P) + 3) / 4 * 4; }

template <int Q>
__device__ __forceinline__ float radial_apply(int r, const float *__restrict__ M) {
    const RadialTable<Q> &T = g_radial<Q>;
    float v = 0.f;
    for (int q = T.start[r]; q < T.start[r + 1]; ++q) v = fmaf(T.w[q], M[T.k[q]], v);
    return v;
}

// One thread per (node, output).  mom: per node 4 monopole sets of NT(P) terms (mu_0, nu_0, mu_1, nu_1).
template <int P>
__global__ void radialT_moments_kernel(int nnodes, const float *__restrict__ mom, float *__restrict__ rmom) {
    constexpr int NT = (P + 1) * (P + 2) * (P + 3) / 6, A = radial_terms(P), B = radial_terms(P - 1);
    constexpr int ST = radialT_stride(P);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nnodes * ST) return;
    const int64_t b = t / ST;
    const int r = (int)(t % ST);
    const float *M = mom + b * 4 * NT;
    float v = 0.f;
    if (r < A) v = radial_apply<P>(r, M);
    else if (r < A + B) v = radial_apply<P - 1>(r - A, M + NT);
    else if (r < 2 * A + B) v = radial_apply<P>(r - A - B, M + 2 * NT);
    else if (r < 2 * A + 2 * B) v = radial_apply<P - 1>(r - 2 * A - B, M + 3 * NT);
    rmom[t] = v;
}

template <int P>
__global__ void __launch_bounds__(128) m2pT_ly32_kernel(int64_t nitems, const int4 *__restrict__ items,
                                                        const int32_t *__restrict__ inv,
                                                        const int32_t *__restrict__ ent, const float4 *__restrict__ x32,
                                                        const float4 *__restrict__ n32, const float4 *__restrict__ cen32,
                                                        const float *__restrict__ rmom, float kappa,
                                                        float4 *__restrict__ part) {
    constexpr int A = radial_terms(P), B = radial_terms(P - 1), NQ = radialT_stride(P) / 4;
    __shared__ float4 sR[4][NQ];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 4 + warp;
    if (item >= nitems) return;
    const int4 it = items[item];
    const int b = it.x;
    {
        const float4 *src = reinterpret_cast<const float4 *>(rmom + (int64_t)b * radialT_stride(P));
        for (int q = lane; q < NQ; q += 32) sR[warp][q] = src[q];
        __syncwarp();
    }
    if (lane >= it.z) return;
    const int64_t slot = (int64_t)it.y + lane;
    const int t = inv[slot];
    const float4 c = cen32[b], x = x32[t], nn = n32[t];
    const float ux = c.x - x.x, uy = c.y - x.y, uz = c.z - x.z;
    const float r2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float rinv = rsqrtf(r2), ir2 = rinv * rinv;
    float FL[P + 1], FY[P + 1];
    FL[0] = rinv;
#pragma unroll
    for (int n = 0; n < P; ++n) FL[n + 1] = (-(float)(2 * n + 1) * ir2) * FL[n];
    const float rho = r2 * rinv;
    const float e = __expf(-kappa * rho);
    FY[0] = e * rinv;
    FY[1] = -fmaf(kappa, rho, 1.f) * FY[0] * ir2;
    const float k2 = kappa * kappa;
#pragma unroll
    for (int n = 1; n < P; ++n) FY[n + 1] = fmaf(k2, FY[n - 1], -(float)(2 * n + 1) * FY[n]) * ir2;
    float px[P + 1], py[P + 1], pz[P + 1], dx[P + 1], dy[P + 1], dz[P + 1];
    px[0] = py[0] = pz[0] = 1.f;
    dx[0] = dy[0] = dz[0] = 0.f;
#pragma unroll
    for (int i = 1; i <= P; ++i) {
        dx[i] = (float)i * nn.x * px[i - 1];
        dy[i] = (float)i * nn.y * py[i - 1];
        dz[i] = (float)i * nn.z * pz[i - 1];
        px[i] = px[i - 1] * ux;
        py[i] = py[i - 1] * uy;
        pz[i] = pz[i - 1] * uz;
    }
    float SL[P + 1], SY[P + 1], GL[P], HL[P], GY[P], HY[P];
#pragma unroll
    for (int n = 0; n <= P; ++n) { SL[n] = 0.f; SY[n] = 0.f; }
#pragma unroll
    for (int n = 0; n < P; ++n) { GL[n] = 0.f; HL[n] = 0.f; GY[n] = 0.f; HY[n] = 0.f; }
    const float *R = reinterpret_cast<const float *>(sR[warp]);
    int om = 0, on = 0;
#pragma unroll
    for (int a1 = 0; a1 <= P; ++a1)
#pragma unroll
        for (int a2 = 0; a2 <= P - a1; ++a2) {
            const float base = px[a1] * py[a2];
            const float dbase = fmaf(dx[a1], py[a2], px[a1] * dy[a2]);
#pragma unroll
            for (int a3 = 0; a3 <= P - a1 - a2; ++a3) {
                const int a = a1 + a2 + a3;
                const float mono = base * pz[a3];
#pragma unroll
                for (int n = a; 2 * n <= a + P; ++n, ++om) {
                    SL[n] = fmaf(mono, R[om], SL[n]);
                    SY[n] = fmaf(mono, R[A + B + om], SY[n]);
                }
                if (a <= P - 1) {
                    const float dmono = fmaf(dbase, pz[a3], base * dz[a3]);
#pragma unroll
                    for (int m = a; 2 * m <= a + P - 1; ++m, ++on) {
                        const float wl = R[A + on], wy = R[2 * A + B + on];
                        GL[m] = fmaf(dmono, wl, GL[m]);
                        HL[m] = fmaf(mono, wl, HL[m]);
                        GY[m] = fmaf(dmono, wy, GY[m]);
                        HY[m] = fmaf(mono, wy, HY[m]);
                    }
                }
            }
        }
    const float nu = fmaf(nn.x, ux, fmaf(nn.y, uy, nn.z * uz));
    float VL = 0.f, VY = 0.f, KL = 0.f, KY = 0.f;
#pragma unroll
    for (int n = 0; n <= P; ++n) {
        VL = fmaf(FL[n], SL[n], VL);
        VY = fmaf(FY[n], SY[n], VY);
    }
#pragma unroll
    for (int m = 0; m < P; ++m) {
        KL = fmaf(FL[m], GL[m], fmaf(nu * FL[m + 1], HL[m], KL));
        KY = fmaf(FY[m], GY[m], fmaf(nu * FY[m + 1], HY[m], KY));
    }
    part[ent[slot]] = make_float4(VL, -KL, VY, -KY);
}

// ---------------------------------------------------------------- transposed near list
__global__ void near_owner_kernel(int64_t m, const int64_t *__restrict__ ptr, int32_t *__restrict__ owner) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    for (int64_t e = ptr[t]; e < ptr[t + 1]; ++e) owner[e] = (int32_t)t;
}

__global__ void near_keys_kernel(int64_t n, const int32_t *__restrict__ panel, uint64_t *__restrict__ keys,
                                 int32_t *__restrict__ idx, int32_t *__restrict__ cnt) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    keys[e] = ((uint64_t)(uint32_t)panel[e] << 32) | (uint64_t)e;
    idx[e] = (int32_t)e;
    atomicAdd(&cnt[panel[e]], 1);
}

__global__ void near_fill_kernel(int64_t n, const int32_t *__restrict__ idx, const int32_t *__restrict__ owner,
                                 const int32_t *__restrict__ order, int32_t *__restrict__ ent,
                                 int32_t *__restrict__ srcs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const int f = idx[e];
    ent[e] = f;
    srcs[e] = order[owner[f]];
}

// ---------------------------------------------------------------- transposed combine
struct TCombPair {
    const double *VK[2];
    int64_t ntg;
    int nk;
    const int32_t *rank;
    const int64_t *nt_ptr;
    const int32_t *nt_ent, *nt_src;
    const double *dV64[2], *dK64[2];
    const float *dV32[2], *dK32[2];
    const double *fold;
    int64_t nsrc;
    const double *selfV[2];
};
struct TComb {
    int np;
    TCombPair p[8];
};

// Per panel j of the target surface: out_phi = 1/2 (h0 + h1) + sum over pairs of
// the quadrature sum of K^T at its Gauss points + transposed near terms;
// out_dphi = the same for V^T plus the transposed self term.
__global__ void tcombine_kernel(int64_t n, int K, const double *__restrict__ wa, TComb tc,
                                const double *__restrict__ h0, const double *__restrict__ h1,
                                double *__restrict__ out_phi, double *__restrict__ out_dphi) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double ph = h0 ? 0.5 * (h0[j] + h1[j]) : 0.0;
    double dp = 0.0;
    for (int a = 0; a < tc.np; ++a) {
        const TCombPair &P = tc.p[a];
        for (int q = 0; q < K; ++q) {
            const int64_t pt = j * K + q;
            const int r = P.rank[pt];
            const double w = wa[pt];
            for (int k = 0; k < P.nk; ++k) {
                dp += w * P.VK[k][r];
                ph += w * P.VK[k][P.ntg + r];
            }
        }
        for (int64_t e = P.nt_ptr[j]; e < P.nt_ptr[j + 1]; ++e) {
            const int f = P.nt_ent[e], i = P.nt_src[e];
            for (int k = 0; k < P.nk; ++k) {
                const double mu = P.fold[(2 * k) * P.nsrc + i], nu = P.fold[(2 * k + 1) * P.nsrc + i];
                if (P.dV64[0]) {
                    dp += P.dV64[k][f] * mu;
                    ph += P.dK64[k][f] * nu;
                } else {
                    dp += (double)P.dV32[k][f] * mu;
                    ph += (double)P.dK32[k][f] * nu;
                }
            }
        }
        if (P.selfV[0])
            for (int k = 0; k < P.nk; ++k) dp += P.selfV[k][j] * P.fold[(2 * k) * P.nsrc + j];
    }
    out_phi[j] = ph;
    out_dphi[j] = dp;
}

__global__ void transpose_minv_kernel(int64_t n, const double *__restrict__ m, double *__restrict__ mt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    mt[4 * i] = m[4 * i];
    mt[4 * i + 1] = m[4 * i + 2];
    mt[4 * i + 2] = m[4 * i + 1];
    mt[4 * i + 3] = m[4 * i + 3];
}

// ---------------------------------------------------------------- gradient pieces
// Deterministic dot products: out[0] += scale * sum_i u_i (ca va[r_i] + cb vb[r_i]),
// r_i = rank[i] (identity if rank is null), vb optional.
constexpr int kDotBlocks = 256;

__global__ void __launch_bounds__(256) rdot_partial_kernel(int64_t n, const double *__restrict__ u,
                                                           const int32_t *__restrict__ rank,
                                                           const double *__restrict__ va, double ca,
                                                           const double *__restrict__ vb, double cb,
                                                           double *__restrict__ partial) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = rank ? rank[i] : i;
        double v = ca * va[r];
        if (vb) v += cb * vb[r];
        acc += u[i] * v;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void rdot_final_kernel(const double *__restrict__ partial, int nb, double scale, double *__restrict__ out) {
    __shared__ double sh[256];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partial[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] += scale * sh[0];
}

// Sources of B^T lambda: the collocation points of the rows of the charged
// region with their adjoint weights, packed (x, y, z, w).
__global__ void pack_colloc_kernel(int64_t n, const double *__restrict__ cen, const double *__restrict__ w,
                                   dvec4 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = dvec4{cen[3 * i], cen[3 * i + 1], cen[3 * i + 2], w[i]};
}

// Per charge k and source chunk: P = sum w G(x_i, r_k), F = sum w grad_r G,
// D = sum w dG/dkappa (SoA partials [chunk][5][nc], without 1/(4 pi)).
__global__ void __launch_bounds__(128) colloc_kernel(int64_t nc, const double *__restrict__ xyz, int64_t m,
                                                     const dvec4 *__restrict__ src, double kappa, int64_t chunk,
                                                     double *__restrict__ part) {
    __shared__ dvec4 tile[128];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.y * chunk, b1 = min(m, b0 + chunk);
    double rx = 0, ry = 0, rz = 0;
    if (k < nc) { rx = xyz[3 * k]; ry = xyz[3 * k + 1]; rz = xyz[3 * k + 2]; }
    double P = 0, Fx = 0, Fy = 0, Fz = 0, D = 0;
    for (int64_t c0 = b0; c0 < b1; c0 += 128) {
        __syncthreads();
        if (c0 + threadIdx.x < b1) tile[threadIdx.x] = src[c0 + threadIdx.x];
        __syncthreads();
        const int cnt = (int)min((int64_t)128, b1 - c0);
        if (k < nc)
            for (int j = 0; j < cnt; ++j) {
                const dvec4 s = tile[j];
                const double dx = s.x - rx, dy = s.y - ry, dz = s.z - rz;
                const double r2 = dx * dx + dy * dy + dz * dz;
                const double rho = sqrt(r2);
                const double e = kappa == 0.0 ? 1.0 : exp(-kappa * rho);
                const double g = s.w * e / rho;
                P += g;
                const double f = g * (1.0 + kappa * rho) / r2;
                Fx += f * dx; Fy += f * dy; Fz += f * dz;
                D -= s.w * e;
            }
    }
    if (k < nc) {
        double *o = part + (int64_t)blockIdx.y * 5 * nc;
        o[k] = P; o[nc + k] = Fx; o[2 * nc + k] = Fy; o[3 * nc + k] = Fz; o[4 * nc + k] = D;
    }
}

// out[c * nc + k] (+)= sum over chunks of part[chunk][c][k], fixed order.
__global__ void sum_parts_kernel(int64_t nc, int width, int nparts, const double *__restrict__ part, double scale,
                                 int accumulate, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nc * width) return;
    double s = 0.0;
    for (int p = 0; p < nparts; ++p) s += part[(int64_t)p * width * nc + i];
    out[i] = (accumulate ? out[i] : 0.0) + scale * s;
}

// Laplace field at the charges of one surface's layer potentials,
// grad_r [cV V dphi + cK K phi], with the forward rule choice (K_fine points
// when |r - c_j| < thres L_j).  Partials [chunk][3][nc] without 1/(4 pi).
__device__ __forceinline__ void field_point(const double r[3], const double y[3], const double n[3], double wv,
                                            double wk, double F[3]) {
    const double dx = r[0] - y[0], dy = r[1] - y[1], dz = r[2] - y[2];
    const double r2 = dx * dx + dy * dy + dz * dz;
    const double rho = sqrt(r2);
    const double i3 = 1.0 / (r2 * rho);
    const double rn = dx * n[0] + dy * n[1] + dz * n[2];
    const double c3 = 3.0 * rn * i3 / r2;
    F[0] += -wv * dx * i3 + wk * (n[0] * i3 - c3 * dx);
    F[1] += -wv * dy * i3 + wk * (n[1] * i3 - c3 * dy);
    F[2] += -wv * dz * i3 + wk * (n[2] * i3 - c3 * dz);
}

__global__ void __launch_bounds__(128) reac_field_kernel(int64_t nc, const double *__restrict__ xyz, int64_t npan,
                                                         int K, int slotF, const double *__restrict__ gy,
                                                         const double *__restrict__ gwa,
                                                         const double *__restrict__ cen,
                                                         const double *__restrict__ nrm, const double *__restrict__ L,
                                                         const double *__restrict__ area,
                                                         const double *__restrict__ verts,
                                                         const int32_t *__restrict__ tris, double thres, double cK,
                                                         double cV, const double *__restrict__ phi,
                                                         const double *__restrict__ dphi, int64_t chunk,
                                                         double *__restrict__ part) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(npan, j0 + chunk);
    const double r[3] = {xyz[3 * k], xyz[3 * k + 1], xyz[3 * k + 2]};
    double F[3] = {0.0, 0.0, 0.0};
    for (int64_t j = j0; j < j1; ++j) {
        const double n[3] = {nrm[3 * j], nrm[3 * j + 1], nrm[3 * j + 2]};
        const double sv = cV * dphi[j], sk = cK * phi[j];
        const double dx = r[0] - cen[3 * j], dy = r[1] - cen[3 * j + 1], dz = r[2] - cen[3 * j + 2];
        const double tl = thres * L[j];
        if (dx * dx + dy * dy + dz * dz < tl * tl) {
            const TriRule &R = c_arules[slotF];
            const int a = tris[3 * j], b = tris[3 * j + 1], c = tris[3 * j + 2];
            for (int q = 0; q < R.n; ++q) {
                double y[3];
                for (int d = 0; d < 3; ++d)
                    y[d] = R.l[q][0] * verts[3 * a + d] + R.l[q][1] * verts[3 * b + d] + R.l[q][2] * verts[3 * c + d];
                const double w = R.w[q] * area[j];
                field_point(r, y, n, w * sv, w * sk, F);
            }
        } else {
            for (int q = 0; q < K; ++q) {
                const int64_t p = j * K + q;
                const double y[3] = {gy[3 * p], gy[3 * p + 1], gy[3 * p + 2]};
                field_point(r, y, n, gwa[p] * sv, gwa[p] * sk, F);
            }
        }
    }
    double *o = part + (int64_t)blockIdx.y * 3 * nc;
    o[k] = F[0]; o[nc + k] = F[1]; o[2 * nc + k] = F[2];
}

__global__ void assemble_charges_kernel(int64_t nc, double c0, double inv_eps, const double *__restrict__ q,
                                        const double *__restrict__ phi_reac, const double *__restrict__ col,
                                        const double *__restrict__ fld, double *__restrict__ dq,
                                        double *__restrict__ dxyz) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    dq[k] = c0 * phi_reac[k] + col[k] * inv_eps;
    for (int d = 0; d < 3; ++d) dxyz[3 * k + d] = q[k] * (c0 * fld[d * nc + k] + col[(1 + d) * nc + k] * inv_eps);
}

// ---------------------------------------------------------------- kappa derivative of a forward block
// The forward recurrence and its kappa derivative side by side:
//   n r^2 da^k = -(2n-1) sum u_j da^(k-e_j) - (n-1) sum da^(k-2e_j)
//                - (sum u_j b^(k-e_j) + sum b^(k-2e_j)) - kappa (sum u_j db^(k-e_j) + sum db^(k-2e_j))
//   n db^k     = -(sum u_j a^(k-e_j) + sum a^(k-2e_j)) - kappa (sum u_j da^(k-e_j) + sum da^(k-2e_j))
// from da^0 = -exp(-kappa r), db^0 = -r exp(-kappa r).
#define PB_DK_STEP(I, K1, K2, K3, NN)                                                                         \
    {                                                                                                         \
        const T c1 = (T)(2 * (NN) - 1) / (T)(NN), c2 = (T)((NN) - 1) / (T)(NN), kn = kappa / (T)(NN),          \
                in = (T)1 / (T)(NN);                                                                          \
        T s1 = 0, s2 = 0, t1 = 0, t2 = 0, ds1 = 0, ds2 = 0, dt1 = 0, dt2 = 0;                                 \
        if ((K1) >= 1) { const int j = tindex((K1) - 1, K2, K3); s1 += ux * a[j]; t1 += ux * b[j]; ds1 += ux * da[j]; dt1 += ux * db[j]; } \
        if ((K2) >= 1) { const int j = tindex(K1, (K2) - 1, K3); s1 += uy * a[j]; t1 += uy * b[j]; ds1 += uy * da[j]; dt1 += uy * db[j]; } \
        if ((K3) >= 1) { const int j = tindex(K1, K2, (K3) - 1); s1 += uz * a[j]; t1 += uz * b[j]; ds1 += uz * da[j]; dt1 += uz * db[j]; } \
        if ((K1) >= 2) { const int j = tindex((K1) - 2, K2, K3); s2 += a[j]; t2 += b[j]; ds2 += da[j]; dt2 += db[j]; } \
        if ((K2) >= 2) { const int j = tindex(K1, (K2) - 2, K3); s2 += a[j]; t2 += b[j]; ds2 += da[j]; dt2 += db[j]; } \
        if ((K3) >= 2) { const int j = tindex(K1, K2, (K3) - 2); s2 += a[j]; t2 += b[j]; ds2 += da[j]; dt2 += db[j]; } \
        a[I] = -(c1 * s1 + c2 * s2 + kn * (t1 + t2)) * ir2;                                                   \
        da[I] = -(c1 * ds1 + c2 * ds2 + in * (t1 + t2) + kn * (dt1 + dt2)) * ir2;                             \
        b[I] = -kn * (s1 + s2);                                                                               \
        db[I] = -in * (s1 + s2) - kn * (ds1 + ds2);                                                           \
        dV += da[I] * mM[I];                                                                                  \
        dK += da[I] * mD[I];                                                                                  \
    }

template <int P, typename T>
__device__ __forceinline__ void m2p_dkappa_eval(T ux, T uy, T uz, T kappa, const T *__restrict__ mM,
                                                const T *__restrict__ mD, T &dV, T &dK) {
    constexpr int NT = (P + 1) * (P + 2) * (P + 3) / 6;
    T a[NT], b[NT], da[NT], db[NT];
    const T r2 = ux * ux + uy * uy + uz * uz;
    const T r = sqrt(r2);
    const T ir2 = (T)1 / r2;
    const T e0 = exp(-kappa * r);
    a[0] = e0 / r;
    b[0] = e0;
    da[0] = -e0;
    db[0] = -r * e0;
    dV = da[0] * mM[0];
    dK = da[0] * mD[0];
#pragma unroll
    for (int n = 1; n <= P; ++n)
#pragma unroll
        for (int k1 = n; k1 >= 0; --k1)
#pragma unroll
            for (int k2 = n - k1; k2 >= 0; --k2) PB_DK_STEP(tindex(k1, k2, n - k1 - k2), k1, k2, n - k1 - k2, n)
}

__device__ void m2p_dkappa_eval_rt(int P, double ux, double uy, double uz, double kappa, const double *__restrict__ mM,
                                   const double *__restrict__ mD, double &dV, double &dK) {
    using T = double;
    const int NT = (P + 1) * (P + 2) * (P + 3) / 6;
    double a[455], b[455], da[455], db[455];
    const double r2 = ux * ux + uy * uy + uz * uz;
    const double r = sqrt(r2);
    const double ir2 = 1.0 / r2;
    const double e0 = exp(-kappa * r);
    a[0] = e0 / r;
    b[0] = e0;
    da[0] = -e0;
    db[0] = -r * e0;
    dV = da[0] * mM[0];
    dK = da[0] * mD[0];
    for (int i = 1; i < NT; ++i) {
        const int k1 = c_aterms[3 * i], k2 = c_aterms[3 * i + 1], k3 = c_aterms[3 * i + 2];
        PB_DK_STEP(i, k1, k2, k3, k1 + k2 + k3)
    }
}
#undef PB_DK_STEP

__device__ void panel_rule_dkappa(const double x[3], const double *__restrict__ v, const int32_t *__restrict__ t,
                                  int j, const double n[3], double area, const TriRule &R, double kappa, double &dV,
                                  double &dK) {
    const int a = t[3 * j], b = t[3 * j + 1], c = t[3 * j + 2];
    double sv = 0.0, sk = 0.0;
    for (int k = 0; k < R.n; ++k) {
        double r[3];
        for (int d = 0; d < 3; ++d)
            r[d] = x[d] - (R.l[k][0] * v[3 * a + d] + R.l[k][1] * v[3 * b + d] + R.l[k][2] * v[3 * c + d]);
        const double rho = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        const double rn = r[0] * n[0] + r[1] * n[1] + r[2] * n[2];
        const double e = exp(-kappa * rho);
        const double w = R.w[k] * area;
        sv -= w * e;
        sk -= w * kappa * rn * e / rho;
    }
    dV = sv * kInv4Pi;
    dK = sk * kInv4Pi;
}

struct DkArgs {
    int64_t ntg;
    const double *xs;
    const int32_t *selfp;
    int use_self;
    const int64_t *p2p_ptr;
    const int32_t *p2p_node;
    const int64_t *start, *count;
    const double *src64;
    const int64_t *m2p_ptr;
    const int32_t *m2p_node;
    const double *centre;
    const double *mom;
    int NT, Prt;
    const int64_t *near_ptr;
    const int32_t *near_panel;
    const double *verts;
    const int32_t *tris;
    const double *nrm, *area;
    int slotK, slotF;
    double kappa;
    const double *phi, *dphi, *dself;
};

// One warp per sorted target of a forward pair: d/dkappa of its V and K sums
// (direct leaves, expansions, near-singular and self corrections), FP64.
template <int P>
__global__ void __launch_bounds__(128) dkappa_kernel(DkArgs g, double *__restrict__ outV, double *__restrict__ outK) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 4 + warp;
    if (t >= g.ntg) return;
    const double x[3] = {g.xs[3 * t], g.xs[3 * t + 1], g.xs[3 * t + 2]};
    const int me = g.use_self ? g.selfp[t] : -1;
    const double kap = g.kappa;
    double fV = 0.0, fK = 0.0, nV = 0.0, nK = 0.0;
    for (int64_t e = g.p2p_ptr[t]; e < g.p2p_ptr[t + 1]; ++e) {
        const int node = g.p2p_node[e];
        const int64_t q0 = g.start[node], q1 = q0 + g.count[node];
        for (int64_t q = q0 + lane; q < q1; q += 32) {
            const double *o = g.src64 + 8 * q;
            if ((int)o[7] == me) continue;
            const double rx = x[0] - o[0], ry = x[1] - o[1], rz = x[2] - o[2];
            const double rho = sqrt(rx * rx + ry * ry + rz * rz);
            const double ex = exp(-kap * rho);
            fV -= o[3] * ex;
            fK -= kap * (rx * o[4] + ry * o[5] + rz * o[6]) * ex / rho;
        }
    }
    for (int64_t e = g.m2p_ptr[t] + lane; e < g.m2p_ptr[t + 1]; e += 32) {
        const int b = g.m2p_node[e];
        const double *mM = g.mom + (int64_t)b * 2 * g.NT;
        double dv, dk;
        const double ux = g.centre[3 * b] - x[0], uy = g.centre[3 * b + 1] - x[1], uz = g.centre[3 * b + 2] - x[2];
        if constexpr (P >= 0) m2p_dkappa_eval<(P >= 0 ? P : 0), double>(ux, uy, uz, kap, mM, mM + g.NT, dv, dk);
        else m2p_dkappa_eval_rt(g.Prt, ux, uy, uz, kap, mM, mM + g.NT, dv, dk);
        fV += dv;
        fK += dk;
    }
    for (int64_t e = g.near_ptr[t] + lane; e < g.near_ptr[t + 1]; e += 32) {
        const int j = g.near_panel[e];
        const double n[3] = {g.nrm[3 * j], g.nrm[3 * j + 1], g.nrm[3 * j + 2]};
        double vf, kf, vk, kk;
        panel_rule_dkappa(x, g.verts, g.tris, j, n, g.area[j], c_arules[g.slotF], kap, vf, kf);
        panel_rule_dkappa(x, g.verts, g.tris, j, n, g.area[j], c_arules[g.slotK], kap, vk, kk);
        nV += (vf - vk) * g.dphi[j];
        nK += (kf - kk) * g.phi[j];
    }
    double V = fV * kInv4Pi + nV, Kv = fK * kInv4Pi + nK;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        V += __shfl_xor_sync(0xffffffffu, V, o);
        Kv += __shfl_xor_sync(0xffffffffu, Kv, o);
    }
    if (lane == 0) {
        if (g.use_self) V += g.dself[me] * g.dphi[me];
        outV[t] = V;
        outK[t] = Kv;
    }
}

// FP32 form of the same (mixed path): the forward FP32 sources (x, y, z, s),
// (d, pid) and moments of the current solution, targets relative to the tree
// origin; each lane's FP32 sums are combined in FP64.  The near-singular
// corrections use panel-relative FP32 coordinates.
struct Dk32Args {
    int64_t ntg;
    const float4 *x32;
    const int32_t *selfp;
    int use_self;
    const int64_t *p2p_ptr;
    const int32_t *p2p_node;
    const int64_t *start, *count;
    const float4 *A, *B;
    const int64_t *m2p_ptr;
    const int32_t *m2p_node;
    const float4 *cen32;
    const float *mom;
    int NT;
    const int64_t *near_ptr;
    const int32_t *near_panel;
    const double *xs, *verts;
    const int32_t *tris;
    const double *nrm, *area;
    int slotK, slotF;
    float kappa;
    const double *phi, *dphi, *dself;
};

__device__ void panel_rule_dkappa32(const float xr[3], const float e1[3], const float e2[3], const float n[3],
                                    float area, const TriRule &R, float kappa, float &dV, float &dK) {
    float sv = 0.f, sk = 0.f;
    for (int k = 0; k < R.n; ++k) {
        const float l1 = (float)R.l[k][1], l2 = (float)R.l[k][2];
        const float rx = xr[0] - (l1 * e1[0] + l2 * e2[0]);
        const float ry = xr[1] - (l1 * e1[1] + l2 * e2[1]);
        const float rz = xr[2] - (l1 * e1[2] + l2 * e2[2]);
        const float rho = sqrtf(rx * rx + ry * ry + rz * rz);
        const float rn = rx * n[0] + ry * n[1] + rz * n[2];
        const float e = __expf(-kappa * rho);
        const float w = (float)R.w[k] * area;
        sv -= w * e;
        sk -= w * kappa * rn * e / rho;
    }
    dV = sv * (float)kInv4Pi;
    dK = sk * (float)kInv4Pi;
}

template <int P>
__global__ void __launch_bounds__(128) dkappa32_kernel(Dk32Args g, double *__restrict__ outV,
                                                       double *__restrict__ outK) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t t = (int64_t)blockIdx.x * 4 + warp;
    if (t >= g.ntg) return;
    const float4 xt = g.x32[t];
    const int me = g.use_self ? g.selfp[t] : -1;
    const float kap = g.kappa;
    const float l2e = -kap * 1.4426950408889634f;
    double fV = 0.0, fK = 0.0, nV = 0.0, nK = 0.0;
    for (int64_t e = g.p2p_ptr[t]; e < g.p2p_ptr[t + 1]; ++e) {
        const int node = g.p2p_node[e];
        const int64_t q0 = g.start[node], q1 = q0 + g.count[node];
        float pv = 0.f, pk = 0.f;
        for (int64_t q = q0 + lane; q < q1; q += 32) {
            const float4 a = g.A[q], b = g.B[q];
            if (__float_as_int(b.w) == me) continue;
            const float rx = xt.x - a.x, ry = xt.y - a.y, rz = xt.z - a.z;
            const float r2 = rx * rx + ry * ry + rz * rz;
            const float iv = rsqrtf(r2);
            const float ex = exp2f(l2e * r2 * iv);
            pv -= a.w * ex;
            pk -= kap * (rx * b.x + ry * b.y + rz * b.z) * ex * iv;
        }
        fV += pv;
        fK += pk;
    }
    for (int64_t e = g.m2p_ptr[t] + lane; e < g.m2p_ptr[t + 1]; e += 32) {
        const int b = g.m2p_node[e];
        const float4 c = g.cen32[b];
        const float *mM = g.mom + (int64_t)b * 2 * g.NT;
        float dv, dk;
        m2p_dkappa_eval<P, float>(c.x - xt.x, c.y - xt.y, c.z - xt.z, kap, mM, mM + g.NT, dv, dk);
        fV += dv;
        fK += dk;
    }
    for (int64_t e = g.near_ptr[t] + lane; e < g.near_ptr[t + 1]; e += 32) {
        const int j = g.near_panel[e];
        const int a = g.tris[3 * j], b = g.tris[3 * j + 1], c = g.tris[3 * j + 2];
        float xr[3], e1[3], e2[3], n[3];
        for (int d = 0; d < 3; ++d) {
            xr[d] = (float)(g.xs[3 * t + d] - g.verts[3 * a + d]);
            e1[d] = (float)(g.verts[3 * b + d] - g.verts[3 * a + d]);
            e2[d] = (float)(g.verts[3 * c + d] - g.verts[3 * a + d]);
            n[d] = (float)g.nrm[3 * j + d];
        }
        float vf, kf, vk, kk;
        panel_rule_dkappa32(xr, e1, e2, n, (float)g.area[j], c_arules[g.slotF], kap, vf, kf);
        panel_rule_dkappa32(xr, e1, e2, n, (float)g.area[j], c_arules[g.slotK], kap, vk, kk);
        nV += (double)(vf - vk) * g.dphi[j];
        nK += (double)(kf - kk) * g.phi[j];
    }
    double V = fV * kInv4Pi + nV, Kv = fK * kInv4Pi + nK;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        V += __shfl_xor_sync(0xffffffffu, V, o);
        Kv += __shfl_xor_sync(0xffffffffu, Kv, o);
    }
    if (lane == 0) {
        if (g.use_self) V += g.dself[me] * g.dphi[me];
        outV[t] = V;
        outK[t] = Kv;
    }
}

// FP32 forms of the charge-site sums (mixed path), coordinates relative to an
// origin near the molecule; every chunk's FP32 sum is combined in FP64.
// Panel data: (centroid - o, (thres L)^2 padded) and the unit normal; Gauss
// points (y - o, w A) in input order.
__global__ void pack_panels32_kernel(int64_t n, int K, const double *__restrict__ cen, const double *__restrict__ L,
                                     const double *__restrict__ nrm, const double *__restrict__ gy,
                                     const double *__restrict__ gwa, double thres, double ox, double oy, double oz,
                                     float4 *__restrict__ pc, float4 *__restrict__ pn, float4 *__restrict__ gp) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const double tl = thres * L[j];
    pc[j] = make_float4((float)(cen[3 * j] - ox), (float)(cen[3 * j + 1] - oy), (float)(cen[3 * j + 2] - oz),
                        (float)(tl * tl * (1.0 + 1e-3) + 1e-3));
    pn[j] = make_float4((float)nrm[3 * j], (float)nrm[3 * j + 1], (float)nrm[3 * j + 2], 0.f);
    for (int q = 0; q < K; ++q) {
        const int64_t p = j * K + q;
        gp[p] = make_float4((float)(gy[3 * p] - ox), (float)(gy[3 * p + 1] - oy), (float)(gy[3 * p + 2] - oz),
                            (float)gwa[p]);
    }
}

__device__ __forceinline__ void field_point32(const float r[3], const float4 &y, const float4 &n, float wv, float wk,
                                              float F[3]) {
    const float dx = r[0] - y.x, dy = r[1] - y.y, dz = r[2] - y.z;
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float iv = rsqrtf(r2);
    const float i3 = iv * iv * iv;
    const float rn = dx * n.x + dy * n.y + dz * n.z;
    const float c3 = 3.f * rn * i3 * iv * iv;
    F[0] += -wv * dx * i3 + wk * (n.x * i3 - c3 * dx);
    F[1] += -wv * dy * i3 + wk * (n.y * i3 - c3 * dy);
    F[2] += -wv * dz * i3 + wk * (n.z * i3 - c3 * dz);
}

__global__ void __launch_bounds__(128) reac_field32_kernel(int64_t nc, const double *__restrict__ xyz, double ox,
                                                           double oy, double oz, int64_t npan, int K, int slotF,
                                                           const float4 *__restrict__ pc,
                                                           const float4 *__restrict__ pn,
                                                           const float4 *__restrict__ gp, const double *__restrict__ cen,
                                                           const double *__restrict__ L,
                                                           const double *__restrict__ area,
                                                           const double *__restrict__ verts,
                                                           const int32_t *__restrict__ tris, double thres, float cK,
                                                           float cV, const float2 *__restrict__ phf, int64_t chunk,
                                                           double *__restrict__ part) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nc) return;
    const int64_t j0 = (int64_t)blockIdx.y * chunk, j1 = min(npan, j0 + chunk);
    const double rd[3] = {xyz[3 * k], xyz[3 * k + 1], xyz[3 * k + 2]};
    const float r[3] = {(float)(rd[0] - ox), (float)(rd[1] - oy), (float)(rd[2] - oz)};
    float F[3] = {0.f, 0.f, 0.f};
    for (int64_t j = j0; j < j1; ++j) {
        const float4 c = pc[j];
        const float4 n = pn[j];
        const float2 pd = phf[j];
        const float sv = cV * pd.y, sk = cK * pd.x;
        const float dx = r[0] - c.x, dy = r[1] - c.y, dz = r[2] - c.z;
        bool near = false;
        if (dx * dx + dy * dy + dz * dz < c.w) {
            const double ex = rd[0] - cen[3 * j], ey = rd[1] - cen[3 * j + 1], ez = rd[2] - cen[3 * j + 2];
            const double tl = thres * L[j];
            near = ex * ex + ey * ey + ez * ez < tl * tl;
        }
        if (near) {
            const TriRule &R = c_arules[slotF];
            const int a = tris[3 * j], b = tris[3 * j + 1], cc = tris[3 * j + 2];
            for (int q = 0; q < R.n; ++q) {
                float4 y;
                y.x = (float)(R.l[q][0] * verts[3 * a] + R.l[q][1] * verts[3 * b] + R.l[q][2] * verts[3 * cc] - ox);
                y.y = (float)(R.l[q][0] * verts[3 * a + 1] + R.l[q][1] * verts[3 * b + 1] + R.l[q][2] * verts[3 * cc + 1] -
                              oy);
                y.z = (float)(R.l[q][0] * verts[3 * a + 2] + R.l[q][1] * verts[3 * b + 2] + R.l[q][2] * verts[3 * cc + 2] -
                              oz);
                const float w = (float)(R.w[q] * area[j]);
                field_point32(r, y, n, w * sv, w * sk, F);
            }
        } else {
            for (int q = 0; q < K; ++q) {
                const float4 y = gp[j * K + q];
                field_point32(r, y, n, y.w * sv, y.w * sk, F);
            }
        }
    }
    double *o = part + (int64_t)blockIdx.y * 3 * nc;
    o[k] = F[0]; o[nc + k] = F[1]; o[2 * nc + k] = F[2];
}

__global__ void pack_colloc32_kernel(int64_t n, const double *__restrict__ cen, const double *__restrict__ w, double ox,
                                     double oy, double oz, float4 *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = make_float4((float)(cen[3 * i] - ox), (float)(cen[3 * i + 1] - oy), (float)(cen[3 * i + 2] - oz),
                         (float)w[i]);
}

__global__ void __launch_bounds__(128) colloc32_kernel(int64_t nc, const double *__restrict__ xyz, double ox,
                                                       double oy, double oz, int64_t m,
                                                       const float4 *__restrict__ src, float kappa, int64_t chunk,
                                                       double *__restrict__ part) {
    __shared__ float4 tile[128];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b0 = (int64_t)blockIdx.y * chunk, b1 = min(m, b0 + chunk);
    float rx = 0.f, ry = 0.f, rz = 0.f;
    if (k < nc) { rx = (float)(xyz[3 * k] - ox); ry = (float)(xyz[3 * k + 1] - oy); rz = (float)(xyz[3 * k + 2] - oz); }
    float P = 0.f, Fx = 0.f, Fy = 0.f, Fz = 0.f, D = 0.f;
    for (int64_t c0 = b0; c0 < b1; c0 += 128) {
        __syncthreads();
        if (c0 + threadIdx.x < b1) tile[threadIdx.x] = src[c0 + threadIdx.x];
        __syncthreads();
        const int cnt = (int)min((int64_t)128, b1 - c0);
        if (k < nc)
            for (int j = 0; j < cnt; ++j) {
                const float4 s = tile[j];
                const float dx = s.x - rx, dy = s.y - ry, dz = s.z - rz;
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float iv = rsqrtf(r2);
                const float e = kappa == 0.f ? 1.f : __expf(-kappa * r2 * iv);
                const float g = s.w * e * iv;
                P += g;
                const float f = g * (1.f + kappa * r2 * iv) * iv * iv;
                Fx += f * dx; Fy += f * dy; Fz += f * dz;
                D -= s.w * e;
            }
    }
    if (k < nc) {
        double *o = part + (int64_t)blockIdx.y * 5 * nc;
        o[k] = P; o[nc + k] = Fx; o[2 * nc + k] = Fy; o[3 * nc + k] = Fz; o[4 * nc + k] = D;
    }
}

// ---------------------------------------------------------------- host helpers
void upload_adjoint_tables() {
    int terms[3 * kMaxTerms1];
    int i = 0;
    for (int n = 0; n <= kMaxP + 1; ++n)
        for (int k1 = n; k1 >= 0; --k1)
            for (int k2 = n - k1; k2 >= 0; --k2) {
                const int k3 = n - k1 - k2;
                if (tindex(k1, k2, k3) != i) fail(PB_ECUDA, "term table layout");
                terms[3 * i] = k1; terms[3 * i + 1] = k2; terms[3 * i + 2] = k3;
                ++i;
            }
    PB_CUDA_TRY(cudaMemcpyToSymbol(c_aterms, terms, sizeof(terms)));
    TriRule r[4] = {make_rule(1), make_rule(3), make_rule(7), make_rule(19)};
    PB_CUDA_TRY(cudaMemcpyToSymbol(c_arules, r, sizeof(r)));
}

void rank_dot(AdjointState &A, int64_t n, const double *u, const int32_t *rank, const double *va, double ca,
              const double *vb, double cb, double scale, double *out, cudaStream_t s) {
    if (n <= 0) return;
    const int nb = std::min<int64_t>(kDotBlocks, div_up(n, 256));
    rdot_partial_kernel<<<nb, 256, 0, s>>>(n, u, rank, va, ca, vb, cb, A.part.p);
    PB_LAUNCH_CHECK();
    rdot_final_kernel<<<1, 256, 0, s>>>(A.part.p, nb, scale, out);
    PB_LAUNCH_CHECK();
}

// d c_{R,t} / d eps_p with c = 1 (R inner of t) or eps_inner(t) / eps_R.
double dcoef(const pb_problem *pb, int R, int t, int p) {
    const SurfDev &S = pb->S[t];
    if (S.inner == R) return 0.0;
    const double er = pb->regions[R].eps, ei = pb->regions[S.inner].eps;
    double d = 0.0;
    if (p == S.inner) d += 1.0 / er;
    if (p == R) d -= ei / (er * er);
    return d;
}

const Pair &forward_of(const pb_problem *pb, const TPair &tp) {
    return tp.charges ? pb->cpairs[tp.fwd] : pb->pairs[tp.fwd];
}

void init_tpair(pb_problem *pb, AdjointState &A, TPair &tp, const Tree &Tr) {
    cudaStream_t s = pb->stream;
    const Params &prm = pb->prm;
    const bool mixed = prm.precision == PB_MIXED;
    const Targets &G = A.GP[tp.tgt];
    const Pair &F = forward_of(pb, tp);
    const Targets &Gf = pb->G[tp.charges ? (int)pb->S.size() : tp.src];
    Pair &L = tp.L;
    L.tgt = tp.tgt;
    L.kappas = F.kappas;
    tp.nk = (int)F.kappas.size();
    const int nk = tp.nk;
    build_far_lists(L, G, Tr, prm, s);
    if (mixed) L.p2p_part32.alloc(2 * nk * std::max<int64_t>(1, L.n_p2p));
    else L.p2p_part.alloc(2 * nk * std::max<int64_t>(1, L.n_p2p));
    if (L.n_m2p > 0) {
        if (mixed) L.m2p_part32.alloc(2 * nk * L.n_m2p);
        else L.m2p_part64.alloc(2 * nk * L.n_m2p);
    }
    L.VK.resize(nk); L.dV.resize(nk); L.dK.resize(nk); L.selfV.resize(nk);
    for (int k = 0; k < nk; ++k) L.VK[k].alloc(2 * std::max<int64_t>(1, G.n));
    L.near_ptr.alloc(G.n + 1);
    L.near_ptr.zero(s);
    L.n_near = 0;
    if (mixed) targets_to_float(L, G, Tr, s);
    tp.fold.alloc(2 * nk * std::max<int64_t>(1, tp.nsrc));
    tp.src64.alloc(8 * std::max<int64_t>(1, Tr.npts));
    tp.srcA32.alloc(std::max<int64_t>(1, Tr.npts));
    tp.srcB32.alloc(std::max<int64_t>(1, Tr.npts));
    if (L.n_m2p > 0) {
        const size_t nm = (size_t)Tr.nnodes * 2 * nk * nterms(prm.P);
        if (mixed) tp.mom32.alloc(nm); else tp.mom64.alloc(nm);
        if (radial_pair(tp, prm)) tp.rmom32.alloc((size_t)Tr.nnodes * radialT_floats_per_node(prm.P));
    }
    // transposed near list: forward entries grouped by panel of the target surface
    const int64_t npan = pb->S[tp.tgt].n, nn = F.n_near;
    tp.nt_ptr.alloc(npan + 1);
    tp.nt_ent.alloc(std::max<int64_t>(1, nn));
    tp.nt_src.alloc(std::max<int64_t>(1, nn));
    TmpBuf<int32_t> cnt(std::max<int64_t>(1, npan), s);
    PB_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(int32_t) * std::max<int64_t>(1, npan), s));
    if (nn > 0) {
        TmpBuf<int32_t> owner(nn, s), idx(nn, s);
        TmpBuf<uint64_t> keys(nn, s);
        near_owner_kernel<<<div_up(Gf.n, 128), 128, 0, s>>>(Gf.n, F.near_ptr.p, owner.p);
        PB_LAUNCH_CHECK();
        near_keys_kernel<<<div_up(nn, 256), 256, 0, s>>>(nn, F.near_panel.p, keys.p, idx.p, cnt.p);
        PB_LAUNCH_CHECK();
        sort_key_index(keys.p, idx.p, nn, s);
        near_fill_kernel<<<div_up(nn, 256), 256, 0, s>>>(nn, idx.p, owner.p, Gf.order.p, tp.nt_ent.p, tp.nt_src.p);
        PB_LAUNCH_CHECK();
    }
    exclusive_scan_i32_to_i64(cnt.p, tp.nt_ptr.p, npan, s);
    PB_CUDA_TRY(cudaStreamSynchronize(s));
}

void prepare_adjoint(pb_problem *pb) {
    cudaStream_t s = pb->stream;
    const Params &prm = pb->prm;
    const int ns = (int)pb->S.size();
    const int64_t nc = pb->nc;
    auto A = std::make_shared<AdjointState>();
    upload_adjoint_tables();
    const int ncritT = prm.ncrit_adjoint > 0 ? prm.ncrit_adjoint : prm.ncrit;
    A->TC.resize(ns);
    A->GP.resize(ns);
    A->gn64.resize(ns);
    A->gn32.resize(ns);
    for (int t = 0; t < ns; ++t) {
        const SurfDev &S = pb->S[t];
        build_tree_points(A->TC[t], S.cen.p, nullptr, S.n, 1, ncritT, s);
        build_targets(A->GP[t], S.gy.p, S.n * prm.K, t, s, prm.K);
        const int64_t m = A->GP[t].n;
        A->gn64[t].alloc(3 * m);
        A->gn32[t].alloc(m);
        gnormals_kernel<<<div_up(m, 256), 256, 0, s>>>(m, prm.K, A->GP[t].order.p, S.nrm.p, A->gn64[t].p,
                                                       A->gn32[t].p);
        PB_LAUNCH_CHECK();
    }
    if (nc > 0) build_tree_points(A->TQ, pb->cxyz_d.p, nullptr, nc, 1, ncritT, s);
    if (prm.precision == PB_MIXED) {
        A->pc32.resize(ns);
        A->pn32.resize(ns);
        A->gp32.resize(ns);
        for (int t = 0; t < ns; ++t) {
            const SurfDev &S = pb->S[t];
            const double *o = pb->T[t].origin;
            A->pc32[t].alloc(S.n);
            A->pn32[t].alloc(S.n);
            A->gp32[t].alloc(S.n * prm.K);
            pack_panels32_kernel<<<div_up(S.n, 256), 256, 0, s>>>(S.n, prm.K, S.cen.p, S.L.p, S.nrm.p, S.gy.p, S.gwa.p,
                                                                  prm.thres, o[0], o[1], o[2], A->pc32[t].p,
                                                                  A->pn32[t].p, A->gp32[t].p);
            PB_LAUNCH_CHECK();
        }
    }
    for (size_t pi = 0; pi < pb->pairs.size(); ++pi) {
        const Pair &F = pb->pairs[pi];
        A->tp.emplace_back();
        TPair &tp = A->tp.back();
        tp.fwd = (int)pi;
        tp.src = F.tgt;
        tp.tgt = F.tree;
        tp.nsrc = pb->S[tp.src].n;
        for (int side = 0; side < 2; ++side)
            for (const Term &tm : pb->rows[2 * tp.src + side])
                if (tm.pair == (int)pi) {
                    tp.cV[tm.kidx][side] += tm.cV;
                    tp.cK[tm.kidx][side] += tm.cK;
                }
        init_tpair(pb, *A, tp, A->TC[tp.src]);
    }
    for (size_t ci = 0; ci < pb->cpairs.size(); ++ci) {
        const Pair &F = pb->cpairs[ci];
        A->tq.emplace_back();
        TPair &tp = A->tq.back();
        tp.charges = true;
        tp.fwd = (int)ci;
        tp.src = -1;
        tp.tgt = F.tree;
        tp.nsrc = nc;
        for (const Term &tm : pb->reac)
            if (tm.pair == (int)ci) {
                tp.cV[tm.kidx][0] += kC0 * tm.cV;
                tp.cK[tm.kidx][0] += kC0 * tm.cK;
            }
        init_tpair(pb, *A, tp, A->TQ);
    }
    A->minvT.alloc(4 * pb->N);
    transpose_minv_kernel<<<div_up(pb->N, 256), 256, 0, s>>>(pb->N, pb->minv.p, A->minvT.p);
    PB_LAUNCH_CHECK();
    A->lam.alloc(2 * pb->N);
    A->f.alloc(2 * pb->N);
    A->gacc.alloc(2 * pb->regions.size());
    A->part.alloc(kDotBlocks);
    // counters of the one-launch M2M (the transposed operator is captured into a graph: nothing allocates there)
    auto counters = [&](Tree &T) {
        if (T.nnodes > 0) {
            T.ucnt.alloc(T.nnodes);
            T.ucnt.zero(s);
        }
    };
    for (Tree &T : A->TC) counters(T);
    counters(A->TQ);
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    pb->adj = A;
}

void launch_p2pT(const TPair &tp, const Targets &G, const double *n64, const float4 *n32, const Tree &Tr, bool mixed,
                 cudaStream_t s) {
    const Pair &Pr = tp.L;
    const int64_t ni = Pr.n_p2p_items;
    if (!ni) return;
    const unsigned grid = (unsigned)((ni + 3) / 4);
    const int nk = tp.nk;
    const double k0 = Pr.kappas[0], k1 = nk > 1 ? Pr.kappas[1] : 0.0;
    const bool y0 = k0 != 0.0, y1 = k1 != 0.0;
    const int us = (!tp.charges && tp.src == tp.tgt) ? 1 : 0;
    if (mixed) {
        TKSet ks{{(float)k0, (float)k1}};
#define PB_P2PT32(NK, A_, B_)                                                                                   \
    p2pT32_kernel<NK, A_, B_><<<grid, 128, 0, s>>>(ni, Pr.p2p_items.p, Pr.p2p_inv.p, Pr.p2p_ent.p, Pr.x32.p, n32, \
                                                   G.self_panel.p, us, Tr.leaf_node.p, Tr.start.p, Tr.count.p, \
                                                   tp.srcA32.p, tp.srcB32.p, ks, Pr.p2p_part32.p)
        if (nk == 1) { if (y0) PB_P2PT32(1, true, false); else PB_P2PT32(1, false, false); }
        else if (!y0 && y1) PB_P2PT32(2, false, true);
        else if (y0 && !y1) PB_P2PT32(2, true, false);
        else if (y0 && y1) PB_P2PT32(2, true, true);
        else PB_P2PT32(2, false, false);
#undef PB_P2PT32
    } else {
#define PB_P2PT64(NK, A_, B_)                                                                                    \
    p2pT64_kernel<NK, A_, B_><<<grid, 128, 0, s>>>(ni, Pr.p2p_items.p, Pr.p2p_inv.p, Pr.p2p_ent.p, G.xs.p, n64,    \
                                                   G.self_panel.p,                                                \
                                                   us, Tr.leaf_node.p, Tr.start.p, Tr.count.p, tp.src64.p, k0,   \
                                                   k1, Pr.p2p_part.p)
        if (nk == 1) { if (y0) PB_P2PT64(1, true, false); else PB_P2PT64(1, false, false); }
        else if (!y0 && y1) PB_P2PT64(2, false, true);
        else if (y0 && !y1) PB_P2PT64(2, true, false);
        else if (y0 && y1) PB_P2PT64(2, true, true);
        else PB_P2PT64(2, false, false);
#undef PB_P2PT64
    }
    PB_LAUNCH_CHECK();
}

template <typename T>
void launch_m2pT_typed(int P, bool yuk, const TPair &tp, const Targets &G, const double *n64, const float4 *n32,
                       const Tree &Tr, const T *mom, int kslot, T *part, cudaStream_t s) {
    const Pair &Pr = tp.L;
    const int64_t ni = Pr.n_m2p_items;
    const unsigned grid = (unsigned)((ni + 3) / 4);
    const int64_t stride = (int64_t)2 * tp.nk * nterms(P);
    const double kap = Pr.kappas[kslot];
#define PB_M2PT_ARGS \
    ni, Pr.m2p_items.p, Pr.m2p_inv.p, Pr.m2p_ent.p, P, G.xs.p, Pr.x32.p, n64, n32, Tr.centre.p, Tr.cen32.p, mom,   \
        stride, kap, kslot, \
        tp.nk, part
#define PB_M2PT_CASE(PP)                                                      \
    case PP:                                                                  \
        if (yuk) m2pT_kernel<PP, true, T><<<grid, 128, 0, s>>>(PB_M2PT_ARGS);  \
        else m2pT_kernel<PP, false, T><<<grid, 128, 0, s>>>(PB_M2PT_ARGS);     \
        break;
    switch (P) {
        PB_M2PT_CASE(0)
        PB_M2PT_CASE(1)
        PB_M2PT_CASE(2)
        PB_M2PT_CASE(3)
        PB_M2PT_CASE(4)
        PB_M2PT_CASE(5)
        PB_M2PT_CASE(6)
        PB_M2PT_CASE(7)
        PB_M2PT_CASE(8)
        default:
            if (yuk) m2pT_kernel<-1, true, T><<<grid, 128, 0, s>>>(PB_M2PT_ARGS);
            else m2pT_kernel<-1, false, T><<<grid, 128, 0, s>>>(PB_M2PT_ARGS);
    }
#undef PB_M2PT_CASE
#undef PB_M2PT_ARGS
    PB_LAUNCH_CHECK();
}

// A mixed-precision pair of a Laplace (slot 0) and a Yukawa (slot 1) kernel takes the radial-form kernel.
bool radial_pair(const TPair &tp, const Params &prm) {
    return prm.precision == PB_MIXED && tp.nk == 2 && tp.L.kappas[0] == 0.0 && tp.L.kappas[1] != 0.0 &&
           prm.P >= 1 && prm.P <= kRadialMaxP;
}

size_t radialT_floats_per_node(int P) { return (size_t)radialT_stride(P); }

void launch_m2pT_radial(int P, TPair &tp, const Targets &G, const float4 *n32, const Tree &Tr, cudaStream_t s) {
    const Pair &Pr = tp.L;
    const int64_t ni = Pr.n_m2p_items;
    const unsigned grid = (unsigned)((ni + 3) / 4);
    const unsigned gt = (unsigned)div_up((int64_t)Tr.nnodes * radialT_stride(P), 128);
    float4 *part = reinterpret_cast<float4 *>(Pr.m2p_part32.p);
    const float kap = (float)Pr.kappas[1];
#define PB_RT(PP)                                                                                               \
    case PP:                                                                                                    \
        radialT_moments_kernel<PP><<<gt, 128, 0, s>>>(Tr.nnodes, tp.mom32.p, tp.rmom32.p);                      \
        PB_LAUNCH_CHECK();                                                                                      \
        m2pT_ly32_kernel<PP><<<grid, 128, 0, s>>>(ni, Pr.m2p_items.p, Pr.m2p_inv.p, Pr.m2p_ent.p, Pr.x32.p, n32, \
                                                  Tr.cen32.p,                                                    \
                                                  tp.rmom32.p, kap, part);                                      \
        break;
    switch (P) { PB_RT(1) PB_RT(2) PB_RT(3) PB_RT(4) PB_RT(5) PB_RT(6) PB_RT(7) PB_RT(8) default: break; }
#undef PB_RT
    PB_LAUNCH_CHECK();
}

// Transposed products of the listed pairs: sources folded from u (rows of each
// pair's source surface, or the charges), their sums at the Gauss points, and
// the per-panel combination into out (unknown order).  half: add the 1/2 phi
// terms of every row (the operator itself; not for the charge pairs).
void apply_tpairs(pb_problem *pb, std::vector<TPair> &list, const double *u, double *out, bool half) {
    AdjointState &A = *pb->adj;
    cudaStream_t s = pb->stream;
    const Params &prm = pb->prm;
    const bool mixed = prm.precision == PB_MIXED;
    const int ns = (int)pb->S.size();
    const int NT = nterms(prm.P);
    for (TPair &tp : list) {
        const Tree &Tr = tp.charges ? A.TQ : A.TC[tp.src];
        const Targets &G = A.GP[tp.tgt];
        const double *u0 = tp.charges ? u : u + 2 * pb->off[tp.src];
        const double *u1 = tp.charges ? nullptr : u0 + pb->S[tp.src].n;
        FoldCoef fc;
        std::memcpy(fc.cV, tp.cV, sizeof(fc.cV));
        std::memcpy(fc.cK, tp.cK, sizeof(fc.cK));
        if (tp.nsrc) {
            fold_kernel<<<div_up(tp.nsrc, 256), 256, 0, s>>>(tp.nsrc, tp.nk, fc, u0, u1, tp.fold.p);
            PB_LAUNCH_CHECK();
        }
        const int64_t np = Tr.npts;
        if (np) {
            if (mixed)
                tstrengths32_kernel<<<div_up(np, 256), 256, 0, s>>>(np, Tr.pos32.p, Tr.pids.p, tp.fold.p, tp.nsrc,
                                                                    tp.nk, tp.srcA32.p, tp.srcB32.p);
            else
                tstrengths64_kernel<<<div_up(np, 256), 256, 0, s>>>(np, Tr.ys.p, Tr.pids.p, tp.fold.p, tp.nsrc, tp.nk,
                                                                    tp.src64.p);
            PB_LAUNCH_CHECK();
        }
        // the direct sums need only the strengths: they run on the side stream beside the expansions
        const double *n64 = A.gn64[tp.tgt].p;
        const float4 *n32 = A.gn32[tp.tgt].p;
        const bool fork = pb->side != nullptr;
        if (fork) PB_CUDA_TRY(cudaEventRecord(pb->evf, s));
        if (tp.L.n_m2p > 0) {
            const int NS = 2 * tp.nk;
            if (mixed) {
                TSrc<float> sv{tp.srcA32.p, tp.srcB32.p};
                p2m_mono_kernel<float><<<Tr.nleaves, 128, 0, s>>>(Tr.nleaves, Tr.leaf_node.p, Tr.start.p, Tr.count.p,
                                                                  Tr.centre.p, Tr.origin[0], Tr.origin[1],
                                                                  Tr.origin[2], sv, prm.P, NT, NS, tp.mom32.p);
            } else {
                TSrc<double> sv{tp.src64.p};
                p2m_mono_kernel<double><<<Tr.nleaves, 128, 0, s>>>(Tr.nleaves, Tr.leaf_node.p, Tr.start.p,
                                                                   Tr.count.p, Tr.centre.p, Tr.origin[0], Tr.origin[1],
                                                                   Tr.origin[2], sv, prm.P, NT, NS, tp.mom64.p);
            }
            PB_LAUNCH_CHECK();
            void *mom = mixed ? (void *)tp.mom32.p : (void *)tp.mom64.p;
            if (climb_fits(NS * NT, mixed))
                m2m_climb(const_cast<Tree &>(Tr), prm.P, mixed, mom, NS * NT, s);
            else
                for (int k = 0; k < tp.nk; ++k) m2m_pass(Tr, prm.P, mixed, mom, NS * NT, 2 * k * NT, s);
        }
        if (fork) {
            PB_CUDA_TRY(cudaStreamWaitEvent(pb->side, pb->evf, 0));
            launch_p2pT(tp, G, n64, n32, Tr, mixed, pb->side);
            PB_CUDA_TRY(cudaEventRecord(pb->evj, pb->side));
        } else {
            launch_p2pT(tp, G, n64, n32, Tr, mixed, s);
        }
        if (tp.L.n_m2p_items > 0 && radial_pair(tp, prm)) {
            launch_m2pT_radial(prm.P, tp, G, n32, Tr, s);
        } else if (tp.L.n_m2p_items > 0) {
            for (int k = 0; k < tp.nk; ++k) {
                const bool yuk = tp.L.kappas[k] != 0.0;
                if (mixed) launch_m2pT_typed<float>(prm.P, yuk, tp, G, n64, n32, Tr, tp.mom32.p, k, tp.L.m2p_part32.p, s);
                else launch_m2pT_typed<double>(prm.P, yuk, tp, G, n64, n32, Tr, tp.mom64.p, k, tp.L.m2p_part64.p, s);
            }
        }
        if (fork) PB_CUDA_TRY(cudaStreamWaitEvent(s, pb->evj, 0));
        launch_gather(tp.L, G, mixed, false, u0, u0, nullptr, s);
    }
    for (int t = 0; t < ns; ++t) {
        TComb tc{};
        for (TPair &tp : list) {
            if (tp.tgt != t) continue;
            if (tc.np == 8) fail(PB_EINVAL, "a surface interacts with more than 8 others");
            const Pair &F = forward_of(pb, tp);
            TCombPair &c = tc.p[tc.np++];
            c.ntg = A.GP[t].n;
            c.nk = tp.nk;
            c.rank = A.GP[t].rank.p;
            c.nt_ptr = tp.nt_ptr.p;
            c.nt_ent = tp.nt_ent.p;
            c.nt_src = tp.nt_src.p;
            c.fold = tp.fold.p;
            c.nsrc = tp.nsrc;
            const bool self = !tp.charges && tp.src == tp.tgt;
            for (int k = 0; k < tp.nk; ++k) {
                c.VK[k] = tp.L.VK[k].p;
                if (mixed) {
                    c.dV32[k] = F.dV32.p + (int64_t)k * F.n_near;
                    c.dK32[k] = F.dK32.p + (int64_t)k * F.n_near;
                } else {
                    c.dV64[k] = F.dV[k].p;
                    c.dK64[k] = F.dK[k].p;
                }
                c.selfV[k] = self ? F.selfV[k].p : nullptr;
            }
        }
        const int64_t n = pb->S[t].n;
        double *o = out + 2 * pb->off[t];
        if (tc.np == 0) {
            PB_CUDA_TRY(cudaMemsetAsync(o, 0, 2 * n * sizeof(double), s));
            continue;
        }
        const double *h0 = half ? u + 2 * pb->off[t] : nullptr;
        const double *h1 = half ? h0 + n : nullptr;
        tcombine_kernel<<<div_up(n, 128), 128, 0, s>>>(n, prm.K, pb->S[t].gwa.p, tc, h0, h1, o, o + n);
        PB_LAUNCH_CHECK();
    }
}

void apply_precond_T(pb_problem *pb, const double *u, double *z) {
    cudaStream_t s = pb->stream;
    if (pb->use_cluster) {
        cluster_apply_T(pb->csurf, pb->cinv.p, u, z, s);
        return;
    }
    AdjointState &A = *pb->adj;
    for (size_t sf = 0; sf < pb->S.size(); ++sf) {
        const int64_t n = pb->S[sf].n, o = 2 * pb->off[sf];
        block_jacobi_apply(n, A.minvT.p + 4 * pb->off[sf], u + o, u + o + n, z + o, z + o + n, s);
    }
}

void launch_dkappa(pb_problem *pb, const Pair &P, const Targets &G, int kidx, bool use_self, const double *phi,
                   const double *dphi, const double *dself, double *outV, double *outK, cudaStream_t s) {
    const Params &prm = pb->prm;
    const Tree &Tr = pb->T[P.tree];
    const SurfDev &S = pb->S[P.tree];
    DkArgs g{};
    g.ntg = G.n;
    g.xs = G.xs.p;
    g.selfp = G.self_panel.p;
    g.use_self = use_self ? 1 : 0;
    g.p2p_ptr = P.p2p_ptr.p;
    g.p2p_node = P.p2p_node.p;
    g.start = Tr.start.p;
    g.count = Tr.count.p;
    g.src64 = Tr.src64.p;
    g.m2p_ptr = P.m2p_ptr.p;
    g.m2p_node = P.m2p_node.p;
    g.centre = Tr.centre.p;
    g.mom = P.n_m2p > 0 ? Tr.mom64.p : nullptr;
    g.NT = nterms(prm.P);
    g.Prt = prm.P;
    g.near_ptr = P.near_ptr.p;
    g.near_panel = P.near_panel.p;
    g.verts = S.verts.p;
    g.tris = S.tris.p;
    g.nrm = S.nrm.p;
    g.area = S.area.p;
    g.slotK = rule_slot(prm.K);
    g.slotF = rule_slot(prm.K_fine);
    g.kappa = P.kappas[kidx];
    g.phi = phi;
    g.dphi = dphi;
    g.dself = dself;
    if (!G.n) return;
    const unsigned grid = (unsigned)div_up(G.n, 4);
    switch (prm.P) {
        case 0: dkappa_kernel<0><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 1: dkappa_kernel<1><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 2: dkappa_kernel<2><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 3: dkappa_kernel<3><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 4: dkappa_kernel<4><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 5: dkappa_kernel<5><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 6: dkappa_kernel<6><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 7: dkappa_kernel<7><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 8: dkappa_kernel<8><<<grid, 128, 0, s>>>(g, outV, outK); break;
        default: dkappa_kernel<-1><<<grid, 128, 0, s>>>(g, outV, outK); break;
    }
    PB_LAUNCH_CHECK();
}

void launch_dkappa32(pb_problem *pb, const Pair &P, const Targets &G, int kidx, bool use_self, const double *phi,
                     const double *dphi, const double *dself, double *outV, double *outK, cudaStream_t s) {
    const Params &prm = pb->prm;
    const Tree &Tr = pb->T[P.tree];
    const SurfDev &S = pb->S[P.tree];
    Dk32Args g{};
    g.ntg = G.n;
    g.x32 = P.x32.p;
    g.selfp = G.self_panel.p;
    g.use_self = use_self ? 1 : 0;
    g.p2p_ptr = P.p2p_ptr.p;
    g.p2p_node = P.p2p_node.p;
    g.start = Tr.start.p;
    g.count = Tr.count.p;
    g.A = Tr.srcA32.p;
    g.B = Tr.srcB32.p;
    g.m2p_ptr = P.m2p_ptr.p;
    g.m2p_node = P.m2p_node.p;
    g.cen32 = Tr.cen32.p;
    g.mom = P.n_m2p > 0 ? Tr.mom32.p : nullptr;
    g.NT = nterms(prm.P);
    g.near_ptr = P.near_ptr.p;
    g.near_panel = P.near_panel.p;
    g.xs = G.xs.p;
    g.verts = S.verts.p;
    g.tris = S.tris.p;
    g.nrm = S.nrm.p;
    g.area = S.area.p;
    g.slotK = rule_slot(prm.K);
    g.slotF = rule_slot(prm.K_fine);
    g.kappa = (float)P.kappas[kidx];
    g.phi = phi;
    g.dphi = dphi;
    g.dself = dself;
    if (!G.n) return;
    const unsigned grid = (unsigned)div_up(G.n, 4);
    switch (prm.P) {
        case 0: dkappa32_kernel<0><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 1: dkappa32_kernel<1><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 2: dkappa32_kernel<2><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 3: dkappa32_kernel<3><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 4: dkappa32_kernel<4><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 5: dkappa32_kernel<5><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 6: dkappa32_kernel<6><<<grid, 128, 0, s>>>(g, outV, outK); break;
        case 7: dkappa32_kernel<7><<<grid, 128, 0, s>>>(g, outV, outK); break;
        default: dkappa32_kernel<8><<<grid, 128, 0, s>>>(g, outV, outK); break;
    }
    PB_LAUNCH_CHECK();
}

}  // namespace

void apply_transpose(pb_problem *pb, const double *lam, double *out) {
    if (!pb->adj) prepare_adjoint(pb);
    apply_tpairs(pb, pb->adj->tp, lam, out, true);
}

void energy_gradient(pb_problem *pb, pb_grad *out) {
    cudaStream_t s = pb->stream;
    const Params &prm = pb->prm;
    const int ns = (int)pb->S.size();
    const int64_t nc = pb->nc;
    const int nreg = (int)pb->regions.size();
    const int Rc = pb->cregion;
    if (!pb->have_solution) fail(PB_EINVAL, "pb_gradient needs a pb_solve since the last pb_setup");
    if (nc == 0) fail(PB_EINVAL, "pb_gradient needs charges");
    PB_CUDA_TRY(cudaEventRecord(pb->ev0, s));
    if (!pb->adj) prepare_adjoint(pb);
    AdjointState &A = *pb->adj;
    const double *x = pb->x.p;
    // adjoint right-hand side c0 Rm^T q and the adjoint solve
    apply_tpairs(pb, A.tq, pb->cq_d.p, A.f.p, false);
    DevOp op = [pb](const double *u, double *v) { apply_transpose(pb, u, v); };
    DevOp pc;
    if (prm.precond) pc = [pb](const double *u, double *z) { apply_precond_T(pb, u, z); };
    KrylovJob jb;
    jb.pb = pb;
    jb.op = op;
    jb.precond = pc;
    jb.b = A.f.p;
    jb.x = A.lam.p;
    jb.x_zero = true;
    // every Arnoldi step replays the transposed operator as one captured graph
    jb.graph = [pb](cudaStream_t gs) {
        launch_captured(pb, pb->adj_exec, pb->adj_kernels,
                        [pb] { apply_tpairs(pb, pb->adj->tp, pb->z1.p, pb->gm.w.p, true); }, gs);
    };
    // a whole cycle's Arnoldi steps as one graph, the loop ended on the device
    jb.cycle_op = [pb] { apply_tpairs(pb, pb->adj->tp, pb->z1.p, pb->gm.w.p, true); };
    jb.cycle_exec = &pb->adj_cyc_exec;
    jb.cycle_kernels = &pb->adj_cyc_kernels;
    std::vector<KrylovJob *> jobs{&jb};
    run_krylov(jobs);
    const KrylovStats st = jb.st;
    const double *lam = A.lam.p;
    // forward block sums at the solution
    reaction(pb, x);
    apply_operator(pb, x, pb->y.p);
    A.gacc.zero(s);
    double *geps = A.gacc.p, *gkap = A.gacc.p + nreg;
    const double eps_c = pb->regions[Rc].eps;
    // eps: coefficient derivatives of the row blocks and of the reaction map, and db/deps
    for (int sf = 0; sf < ns; ++sf)
        for (int side = 0; side < 2; ++side) {
            const double *lr = lam + 2 * pb->off[sf] + side * pb->S[sf].n;
            for (const Term &tm : pb->rows[2 * sf + side]) {
                const Pair &P = pb->pairs[tm.pair];
                for (int p = 0; p < nreg; ++p) {
                    const double dcV = -tm.cK * dcoef(pb, tm.region, P.tree, p);
                    if (dcV != 0.0)
                        rank_dot(A, pb->S[sf].n, lr, pb->G[sf].rank.p, P.VK[tm.kidx].p, -dcV, nullptr, 0.0, 1.0,
                                 geps + p, s);
                }
            }
        }
    for (const Term &tm : pb->reac) {
        const Pair &P = pb->cpairs[tm.pair];
        for (int p = 0; p < nreg; ++p) {
            const double dcV = -tm.cK * dcoef(pb, Rc, P.tree, p);
            if (dcV != 0.0)
                rank_dot(A, nc, pb->cq_d.p, pb->G[ns].rank.p, P.VK[tm.kidx].p, kC0 * dcV, nullptr, 0.0, 1.0,
                         geps + p, s);
        }
    }
    rank_dot(A, 2 * pb->N, lam, nullptr, pb->b.p, 1.0, nullptr, 0.0, -1.0 / eps_c, geps + Rc, s);
    // kappa: derivative kernels of every block; on the mixed path (P <= 8) in
    // FP32 on the sources and moments the forward product above left for x
    const bool dk32 = prm.precision == PB_MIXED && prm.P <= 8;
    if (!dk32)
        for (int t = 0; t < ns; ++t) {
            const double *phi = x + 2 * pb->off[t];
            compute_strengths(pb->T[t], pb->S[t], phi, phi + pb->S[t].n, false, s);
            if (pb->need_far[t]) upward_pass(pb->T[t], prm.P, false, s);
        }
    auto dk_pair = [&](const Pair &P, int pi, bool charges) {
        const Targets &G = pb->G[P.tgt];
        const bool use_self = !charges && P.tgt == P.tree;
        const double *phi = x + 2 * pb->off[P.tree];
        const double *dphi = phi + pb->S[P.tree].n;
        TmpBuf<double> dvk(2 * std::max<int64_t>(1, G.n), s), dself(std::max<int64_t>(1, pb->S[P.tree].n), s);
        for (size_t k = 0; k < P.kappas.size(); ++k) {
            if (use_self) self_integrals_dkappa(pb->S[P.tree], prm.N_k, P.kappas[k], dself.p, s);
            if (dk32) launch_dkappa32(pb, P, G, (int)k, use_self, phi, dphi, dself.p, dvk.p, dvk.p + G.n, s);
            else launch_dkappa(pb, P, G, (int)k, use_self, phi, dphi, dself.p, dvk.p, dvk.p + G.n, s);
            if (!charges) {
                const int sf = P.tgt;
                for (int side = 0; side < 2; ++side) {
                    const double *lr = lam + 2 * pb->off[sf] + side * pb->S[sf].n;
                    for (const Term &tm : pb->rows[2 * sf + side])
                        if (tm.pair == pi && tm.kidx == (int)k)
                            rank_dot(A, pb->S[sf].n, lr, G.rank.p, dvk.p, tm.cV, dvk.p + G.n, tm.cK, -1.0,
                                     gkap + tm.region, s);
                }
            } else {
                for (const Term &tm : pb->reac)
                    if (tm.pair == pi && tm.kidx == (int)k)
                        rank_dot(A, nc, pb->cq_d.p, G.rank.p, dvk.p, tm.cV, dvk.p + G.n, tm.cK, kC0, gkap + Rc, s);
            }
        }
    };
    for (size_t pi = 0; pi < pb->pairs.size(); ++pi) dk_pair(pb->pairs[pi], (int)pi, false);
    for (size_t ci = 0; ci < pb->cpairs.size(); ++ci) dk_pair(pb->cpairs[ci], (int)ci, true);
    // B^T lambda and its gradient at the charges (collocation points of the charged region's rows)
    int64_t m = 0;
    for (int sf = 0; sf < ns; ++sf)
        for (int side = 0; side < 2; ++side)
            if ((side == 0 ? pb->S[sf].inner : pb->S[sf].outer) == Rc) m += pb->S[sf].n;
    TmpBuf<dvec4> csrc(std::max<int64_t>(1, m), s);
    TmpBuf<float4> csrc32(std::max<int64_t>(1, m), s);
    const bool mixed = prm.precision == PB_MIXED;
    const double *co = pb->T[0].origin;
    {
        int64_t o = 0;
        for (int sf = 0; sf < ns; ++sf)
            for (int side = 0; side < 2; ++side)
                if ((side == 0 ? pb->S[sf].inner : pb->S[sf].outer) == Rc) {
                    const int64_t n = pb->S[sf].n;
                    if (mixed)
                        pack_colloc32_kernel<<<div_up(n, 256), 256, 0, s>>>(n, pb->S[sf].cen.p,
                                                                            lam + 2 * pb->off[sf] + side * n, co[0],
                                                                            co[1], co[2], csrc32.p + o);
                    else
                        pack_colloc_kernel<<<div_up(n, 256), 256, 0, s>>>(n, pb->S[sf].cen.p,
                                                                          lam + 2 * pb->off[sf] + side * n, csrc.p + o);
                    PB_LAUNCH_CHECK();
                    o += n;
                }
    }
    const int gx = div_up(nc, 128);
    const int nparts = std::max(1, std::min<int>(64, div_up(4 * 148, gx)));
    TmpBuf<double> part((size_t)nparts * 5 * nc, s), col(5 * nc, s), fld(3 * nc, s);
    {
        const int64_t chunk = std::max<int64_t>(1, (m + nparts - 1) / nparts);
        if (mixed)
            colloc32_kernel<<<dim3(gx, nparts), 128, 0, s>>>(nc, pb->cxyz_d.p, co[0], co[1], co[2], m, csrc32.p,
                                                             (float)pb->regions[Rc].kappa, chunk, part.p);
        else
            colloc_kernel<<<dim3(gx, nparts), 128, 0, s>>>(nc, pb->cxyz_d.p, m, csrc.p, pb->regions[Rc].kappa, chunk,
                                                           part.p);
        PB_LAUNCH_CHECK();
        sum_parts_kernel<<<div_up(5 * nc, 256), 256, 0, s>>>(nc, 5, nparts, part.p, kInv4Pi, 0, col.p);
        PB_LAUNCH_CHECK();
    }
    rank_dot(A, nc, pb->cq_d.p, nullptr, col.p + 4 * nc, 1.0, nullptr, 0.0, 1.0 / eps_c, gkap + Rc, s);
    PB_CUDA_TRY(cudaMemsetAsync(fld.p, 0, 3 * nc * sizeof(double), s));
    for (const Term &tm : pb->reac) {
        const int t = pb->cpairs[tm.pair].tree;
        const SurfDev &S = pb->S[t];
        const double *phi = x + 2 * pb->off[t];
        const int64_t chunk = std::max<int64_t>(1, (S.n + nparts - 1) / nparts);
        if (mixed) {
            const double *o = pb->T[t].origin;
            reac_field32_kernel<<<dim3(gx, nparts), 128, 0, s>>>(
                nc, pb->cxyz_d.p, o[0], o[1], o[2], S.n, prm.K, rule_slot(prm.K_fine), A.pc32[t].p, A.pn32[t].p,
                A.gp32[t].p, S.cen.p, S.L.p, S.area.p, S.verts.p, S.tris.p, prm.thres, (float)tm.cK, (float)tm.cV,
                pb->T[t].phf.p, chunk, part.p);
        } else {
            reac_field_kernel<<<dim3(gx, nparts), 128, 0, s>>>(nc, pb->cxyz_d.p, S.n, prm.K, rule_slot(prm.K_fine),
                                                               S.gy.p, S.gwa.p, S.cen.p, S.nrm.p, S.L.p, S.area.p,
                                                               S.verts.p, S.tris.p, prm.thres, tm.cK, tm.cV, phi,
                                                               phi + S.n, chunk, part.p);
        }
        PB_LAUNCH_CHECK();
        sum_parts_kernel<<<div_up(3 * nc, 256), 256, 0, s>>>(nc, 3, nparts, part.p, kInv4Pi, 1, fld.p);
        PB_LAUNCH_CHECK();
    }
    A.dq_d.alloc(nc);
    A.dxyz_d.alloc(3 * nc);
    assemble_charges_kernel<<<div_up(nc, 128), 128, 0, s>>>(nc, kC0, 1.0 / eps_c, pb->cq_d.p, pb->phi_reac.p, col.p,
                                                            fld.p, A.dq_d.p, A.dxyz_d.p);
    PB_LAUNCH_CHECK();
    std::vector<double> gh(2 * nreg);
    A.gacc.download(gh.data(), 2 * nreg, s);
    if (out->dq) A.dq_d.download(out->dq, nc, s);
    if (out->dxyz) A.dxyz_d.download(out->dxyz, 3 * nc, s);
    double energy = 0.0;
    PB_CUDA_TRY(cudaMemcpyAsync(&energy, pb->energy.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaEventRecord(pb->ev1, s));
    PB_CUDA_TRY(cudaEventSynchronize(pb->ev1));
    float ms = 0.f;
    PB_CUDA_TRY(cudaEventElapsedTime(&ms, pb->ev0, pb->ev1));
    if (out->deps) std::copy(gh.begin(), gh.begin() + nreg, out->deps);
    if (out->dkappa) std::copy(gh.begin() + nreg, gh.end(), out->dkappa);
    out->energy = energy;
    out->residual = st.rel;
    out->iterations = st.iters;
    out->matvecs = st.matvecs;
    out->grad_ms = ms;
    if (!(st.rel < prm.tol)) fail(PB_ENOCONV, "adjoint GMRES reached max_iter before the tolerance");
}

}  // namespace pb
