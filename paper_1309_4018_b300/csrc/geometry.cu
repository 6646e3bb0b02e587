// Panel geometry, Gauss points, singular and near-singular integrals, the
// right-hand side (Sec. 2.2 Eqs. nBEM_disc, matrix, matel; Sec. 2.3
// "Treecode-accelerated BEM").
#include <cmath>

#include "geometry.cuh"

namespace pb {

// Symmetric triangle rules (Dunavant 1985): barycentric nodes and weights
// (weights sum to 1).  Regular rules K = 1, 3, 7; near-singular rules 7, 19.
TriRule make_rule(int K) {
    TriRule r{};
    r.n = 0;
    auto add = [&](double a, double b, double c, double w) {
        r.l[r.n][0] = a; r.l[r.n][1] = b; r.l[r.n][2] = c; r.w[r.n] = w; ++r.n;
    };
    auto orbit3 = [&](double a, double b, double w) {  // (a, b, b) and its two rotations
        add(a, b, b, w); add(b, a, b, w); add(b, b, a, w);
    };
    auto orbit6 = [&](double a, double b, double c, double w) {
        add(a, b, c, w); add(a, c, b, w); add(b, a, c, w); add(b, c, a, w); add(c, a, b, w); add(c, b, a, w);
    };
    const double third = 1.0 / 3.0;
    if (K == 1) {
        add(third, third, third, 1.0);
    } else if (K == 3) {
        orbit3(2.0 / 3.0, 1.0 / 6.0, 1.0 / 3.0);
    } else if (K == 7) {
        add(third, third, third, 0.225);
        orbit3(0.059715871789770, 0.470142064105115, 0.132394152788506);
        orbit3(0.797426985353087, 0.101286507323456, 0.125939180544827);
    } else {  // 19 points, degree 9
        add(third, third, third, 0.097135796282799);
        orbit3(0.020634961602525, 0.489682519198738, 0.031334700227139);
        orbit3(0.125820817014127, 0.437089591492937, 0.077827541004774);
        orbit3(0.623592928761935, 0.188203535619033, 0.079647738927210);
        orbit3(0.910540973211095, 0.044729513394453, 0.025577675658698);
        orbit6(0.036838412054736, 0.221962989160766, 0.741198598784498, 0.043283539377289);
    }
    return r;
}

int rule_slot(int K) { return K == 1 ? 0 : K == 3 ? 1 : K == 7 ? 2 : 3; }

namespace {

__constant__ TriRule c_rules[4];  // 1, 3, 7, 19 points


__global__ void panel_geom_kernel(int64_t n, const double *__restrict__ v, const int32_t *__restrict__ t,
                                  double *__restrict__ cen, double *__restrict__ nrm, double *__restrict__ area,
                                  double *__restrict__ L, int32_t *__restrict__ bad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = t[3 * i], b = t[3 * i + 1], c = t[3 * i + 2];
    double p0[3], p1[3], p2[3];
    for (int k = 0; k < 3; ++k) { p0[k] = v[3 * a + k]; p1[k] = v[3 * b + k]; p2[k] = v[3 * c + k]; }
    for (int k = 0; k < 3; ++k) cen[3 * i + k] = __ddiv_rn(__dadd_rn(__dadd_rn(p0[k], p1[k]), p2[k]), 3.0);
    double e1[3], e2[3];
    for (int k = 0; k < 3; ++k) { e1[k] = __dsub_rn(p1[k], p0[k]); e2[k] = __dsub_rn(p2[k], p0[k]); }
    const double cx = __dsub_rn(__dmul_rn(e1[1], e2[2]), __dmul_rn(e1[2], e2[1]));
    const double cy = __dsub_rn(__dmul_rn(e1[2], e2[0]), __dmul_rn(e1[0], e2[2]));
    const double cz = __dsub_rn(__dmul_rn(e1[0], e2[1]), __dmul_rn(e1[1], e2[0]));
    const double n2 = __dadd_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)), __dmul_rn(cz, cz));
    const double nl = __dsqrt_rn(n2);
    if (!(nl > 0.0)) atomicExch(bad, 1);
    nrm[3 * i] = __ddiv_rn(cx, nl);
    nrm[3 * i + 1] = __ddiv_rn(cy, nl);
    nrm[3 * i + 2] = __ddiv_rn(cz, nl);
    const double ar = __dmul_rn(0.5, nl);
    area[i] = ar;
    L[i] = __dsqrt_rn(__dmul_rn(2.0, ar));
}

__global__ void gauss_points_kernel(int64_t n, int slot, const double *__restrict__ v, const int32_t *__restrict__ t,
                                    const double *__restrict__ area, double *__restrict__ gy, double *__restrict__ gwa) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const TriRule &R = c_rules[slot];
    const int a = t[3 * i], b = t[3 * i + 1], c = t[3 * i + 2];
    for (int k = 0; k < R.n; ++k) {
        for (int d = 0; d < 3; ++d) {
            const double y = __dadd_rn(__dadd_rn(__dmul_rn(R.l[k][0], v[3 * a + d]), __dmul_rn(R.l[k][1], v[3 * b + d])),
                                       __dmul_rn(R.l[k][2], v[3 * c + d]));
            gy[3 * (i * R.n + k) + d] = y;
        }
        gwa[i * R.n + k] = __dmul_rn(R.w[k], area[i]);
    }
}

// V = sum_k w_k A G(x, y_k), K = sum_k w_k A n . grad_y G(x, y_k) over one panel (FP64).
__device__ void panel_rule_sums(const double x[3], const double *__restrict__ v, const int32_t *__restrict__ t, int j,
                                const double nrm[3], double area, const TriRule &R, double kappa, double &V, double &K) {
    const int a = t[3 * j], b = t[3 * j + 1], c = t[3 * j + 2];
    double sv = 0.0, sk = 0.0;
    for (int k = 0; k < R.n; ++k) {
        double r[3];
        for (int d = 0; d < 3; ++d) {
            const double y = R.l[k][0] * v[3 * a + d] + R.l[k][1] * v[3 * b + d] + R.l[k][2] * v[3 * c + d];
            r[d] = x[d] - y;
        }
        const double r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        const double rho = sqrt(r2);
        const double rn = r[0] * nrm[0] + r[1] * nrm[1] + r[2] * nrm[2];
        const double e = kappa == 0.0 ? 1.0 : exp(-kappa * rho);
        const double wa = R.w[k] * area;
        sv += wa * e / rho;
        sk += wa * rn * (1.0 + kappa * rho) * e / (r2 * rho);
    }
    V = sv * kInv4Pi;
    K = sk * kInv4Pi;
}

// Near-singular corrections: for each near entry (target i, panel j) the
// K_fine-rule value minus the K-rule value that the direct sum evaluates.
// One thread per entry; its target is found by binary search in the CSR offsets.
__global__ void near_values_kernel(int64_t ntg, int64_t nnear, const double *__restrict__ xs,
                                   const int64_t *__restrict__ ptr, const int32_t *__restrict__ pan,
                                   const double *__restrict__ v, const int32_t *__restrict__ t,
                                   const double *__restrict__ nrm, const double *__restrict__ area, int slotK, int slotF,
                                   double kappa, double *__restrict__ dV, double *__restrict__ dK) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnear) return;
    int64_t lo = 0, hi = ntg;  // last i with ptr[i] <= e
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (ptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int64_t i = lo;
    const double x[3] = {xs[3 * i], xs[3 * i + 1], xs[3 * i + 2]};
    const int j = pan[e];
    const double nj[3] = {nrm[3 * j], nrm[3 * j + 1], nrm[3 * j + 2]};
    double vf, kf, vk, kk;
    panel_rule_sums(x, v, t, j, nj, area[j], c_rules[slotF], kappa, vf, kf);
    panel_rule_sums(x, v, t, j, nj, area[j], c_rules[slotK], kappa, vk, kk);
    dV[e] = vf - vk;
    dK[e] = kf - kk;
}

// Mixed path: the same corrections in FP32, with positions taken relative to
// the panel's first vertex (differences of nearby points stay exact enough).
// FP32 copies of the rules (the FP64 constants converted once, not per point).
struct TriRule32 {
    int n;
    float l1[19], l2[19], w[19];
};
__constant__ TriRule32 c_rules32[4];

// V and K of one panel at xr (relative to its first vertex) for NK kernels at once:
// the geometry of every rule point is shared by the kernels.
template <int NK>
__device__ void panel_rule_sums32(const float xr[3], const float e1[3], const float e2[3], const float nrm[3],
                                  float area, const TriRule32 &R, const float *kappa, float *V, float *K) {
    float sv[NK], sk[NK];
#pragma unroll
    for (int a = 0; a < NK; ++a) { sv[a] = 0.f; sk[a] = 0.f; }
    for (int k = 0; k < R.n; ++k) {
        const float l1 = R.l1[k], l2 = R.l2[k];
        const float rx = xr[0] - (l1 * e1[0] + l2 * e2[0]);
        const float ry = xr[1] - (l1 * e1[1] + l2 * e2[1]);
        const float rz = xr[2] - (l1 * e1[2] + l2 * e2[2]);
        const float r2 = rx * rx + ry * ry + rz * rz;
        const float inv = rsqrtf(r2);
        const float rho = r2 * inv;
        const float rn = rx * nrm[0] + ry * nrm[1] + rz * nrm[2];
        const float wa = R.w[k] * area;
        const float wi = wa * inv, wk = wa * rn * inv * inv * inv;
#pragma unroll
        for (int a = 0; a < NK; ++a) {
            const float e = kappa[a] == 0.f ? 1.f : __expf(-kappa[a] * rho);
            sv[a] += wi * e;
            sk[a] += wk * (1.f + kappa[a] * rho) * e;
        }
    }
#pragma unroll
    for (int a = 0; a < NK; ++a) {
        V[a] = sv[a] * (float)kInv4Pi;
        K[a] = sk[a] * (float)kInv4Pi;
    }
}

template <int NK>
__global__ void near_values32_kernel(int64_t ntg, int64_t nnear, const double *__restrict__ xs,
                                     const int64_t *__restrict__ ptr, const int32_t *__restrict__ pan,
                                     const double *__restrict__ v, const int32_t *__restrict__ t,
                                     const double *__restrict__ nrm, const double *__restrict__ area, int slotK,
                                     int slotF, float kap0, float kap1, float *__restrict__ dV,
                                     float *__restrict__ dK) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nnear) return;
    int64_t lo = 0, hi = ntg;  // last i with ptr[i] <= e
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (ptr[mid] <= e) lo = mid; else hi = mid;
    }
    const int64_t i = lo;
    const int j = pan[e];
    const int a = t[3 * j], b = t[3 * j + 1], c = t[3 * j + 2];
    float xr[3], e1[3], e2[3], nj[3];
    for (int d = 0; d < 3; ++d) {
        xr[d] = (float)(xs[3 * i + d] - v[3 * a + d]);
        e1[d] = (float)(v[3 * b + d] - v[3 * a + d]);
        e2[d] = (float)(v[3 * c + d] - v[3 * a + d]);
        nj[d] = (float)nrm[3 * j + d];
    }
    const float kap[2] = {kap0, kap1};
    float vf[NK], kf[NK], vk[NK], kk[NK];
    panel_rule_sums32<NK>(xr, e1, e2, nj, (float)area[j], c_rules32[slotF], kap, vf, kf);
    panel_rule_sums32<NK>(xr, e1, e2, nj, (float)area[j], c_rules32[slotK], kap, vk, kk);
#pragma unroll
    for (int a = 0; a < NK; ++a) {
        dV[a * nnear + e] = vf[a] - vk[a];
        dK[a * nnear + e] = kf[a] - kk[a];
    }
}

// Semi-analytical single-layer self integral at the centroid (Zhu et al.
// technique, N_k Gauss points per side).  Each edge at in-plane distance h
// from the centroid contributes int F(h cosh s) / cosh s ds over
// s = asinh(u / h), u the arclength from the foot of the perpendicular, with
// F(rho) = rho (Laplace) or (1 - exp(-kappa rho)) / kappa (Yukawa): the radial
// integral of G r dr in closed form, the angle (d angle = ds / cosh s) by
// Gauss-Legendre in s.
struct GL {
    int n;
    double x[32], w[32];
};

// NK kernels at once (kappa[a], out[a]): the edge geometry and the hyperbolic
// substitution are shared, only the radial function differs.
template <int NK>
__global__ void self_integral_kernel(int64_t n, const double *__restrict__ v, const int32_t *__restrict__ t,
                                     const double *__restrict__ cen, GL gl, double kappa0, double kappa1,
                                     double *__restrict__ out0, double *__restrict__ out1) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int idx[3] = {t[3 * i], t[3 * i + 1], t[3 * i + 2]};
    const double c[3] = {cen[3 * i], cen[3 * i + 1], cen[3 * i + 2]};
    const double kap[2] = {kappa0, kappa1};
    double tot[NK];
    for (int a = 0; a < NK; ++a) tot[a] = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *va = v + 3 * idx[e];
        const double *vb = v + 3 * idx[(e + 1) % 3];
        double d[3], len2 = 0.0;
        for (int k = 0; k < 3; ++k) { d[k] = vb[k] - va[k]; len2 += d[k] * d[k]; }
        const double len = sqrt(len2);
        double s0 = 0.0;
        for (int k = 0; k < 3; ++k) { d[k] /= len; s0 += (c[k] - va[k]) * d[k]; }
        double h2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double f = c[k] - (va[k] + s0 * d[k]);
            h2 += f * f;
        }
        const double h = sqrt(h2);
        const double s1 = asinh(-s0 / h), s2 = asinh((len - s0) / h);
        const double half = 0.5 * (s2 - s1), mid = 0.5 * (s2 + s1);
        for (int q = 0; q < gl.n; ++q) {
            const double ch = cosh(mid + half * gl.x[q]);
            const double rho = h * ch;
#pragma unroll
            for (int a = 0; a < NK; ++a) {
                const double F = kap[a] == 0.0 ? rho : -expm1(-kap[a] * rho) / kap[a];
                tot[a] += gl.w[q] * half * F / ch;
            }
        }
    }
    out0[i] = tot[0] * kInv4Pi;
    if (NK > 1) out1[i] = tot[NK - 1] * kInv4Pi;
}

// d V_ii / d kappa by the same rule: the radial integral of -exp(-kappa r) r dr
// is the kappa derivative of F(rho) = (1 - exp(-kappa rho)) / kappa,
// (kappa rho exp(-kappa rho) + expm1(-kappa rho)) / kappa^2, taken from its
// power series rho^2 sum_{n>=2} (-1)^(n-1) (n-1)/n! (kappa rho)^(n-2) when
// kappa rho < 0.1 (no cancellation; -rho^2/2 at kappa = 0).
__device__ double dF_dkappa(double rho, double kappa) {
    const double x = kappa * rho;
    if (x < 0.1) {
        double sum = 0.0, fact = 1.0, xp = 1.0;
        for (int n = 2; n < 16; ++n) {
            fact *= n;
            sum += ((n & 1) ? 1.0 : -1.0) * (n - 1) / fact * xp;
            xp *= x;
        }
        return rho * rho * sum;
    }
    return (x * exp(-x) + expm1(-x)) / (kappa * kappa);
}

__global__ void self_dkappa_kernel(int64_t n, const double *__restrict__ v, const int32_t *__restrict__ t,
                                   const double *__restrict__ cen, GL gl, double kappa, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int idx[3] = {t[3 * i], t[3 * i + 1], t[3 * i + 2]};
    const double c[3] = {cen[3 * i], cen[3 * i + 1], cen[3 * i + 2]};
    double total = 0.0;
    for (int e = 0; e < 3; ++e) {
        const double *va = v + 3 * idx[e];
        const double *vb = v + 3 * idx[(e + 1) % 3];
        double d[3], len2 = 0.0;
        for (int k = 0; k < 3; ++k) { d[k] = vb[k] - va[k]; len2 += d[k] * d[k]; }
        const double len = sqrt(len2);
        double s0 = 0.0;
        for (int k = 0; k < 3; ++k) { d[k] /= len; s0 += (c[k] - va[k]) * d[k]; }
        double h2 = 0.0;
        for (int k = 0; k < 3; ++k) {
            const double f = c[k] - (va[k] + s0 * d[k]);
            h2 += f * f;
        }
        const double h = sqrt(h2);
        const double s1 = asinh(-s0 / h), s2 = asinh((len - s0) / h);
        const double half = 0.5 * (s2 - s1), mid = 0.5 * (s2 + s1);
        for (int q = 0; q < gl.n; ++q) {
            const double ch = cosh(mid + half * gl.x[q]);
            total += gl.w[q] * half * dF_dkappa(h * ch, kappa) / ch;
        }
    }
    out[i] = total * kInv4Pi;
}

__global__ void rhs_kernel(int64_t n, const double *__restrict__ cen, int64_t nc, const double *__restrict__ q,
                           const double *__restrict__ xyz, double kappa, double eps, double *__restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = cen[3 * i], y = cen[3 * i + 1], z = cen[3 * i + 2];
    double s = 0.0;
    for (int64_t k = 0; k < nc; ++k) {
        const double dx = x - xyz[3 * k], dy = y - xyz[3 * k + 1], dz = z - xyz[3 * k + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        s += q[k] * (kappa == 0.0 ? 1.0 : exp(-kappa * r)) / r;
    }
    b[i] = s * kInv4Pi / eps;
}

// Mixed-precision right-hand side: charges staged in shared memory as FP32
// (relative to an origin near the molecule), FP32 terms, each 256-charge tile
// summed in FP32 and added into a compensated (hi, lo) FP32 pair.
__global__ void __launch_bounds__(256) rhs32_kernel(int64_t n, const double *__restrict__ cen, int64_t nc,
                                                    const double *__restrict__ q, const double *__restrict__ xyz,
                                                    double ox, double oy, double oz, float kappa, double eps,
                                                    double *__restrict__ b) {
    __shared__ float4 sc[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float x = 0.f, y = 0.f, z = 0.f;
    if (i < n) {
        x = (float)(cen[3 * i] - ox); y = (float)(cen[3 * i + 1] - oy); z = (float)(cen[3 * i + 2] - oz);
    }
    const float l2k = -kappa * 1.4426950408889634f;
    float hi = 0.f, lo = 0.f;
    for (int64_t c0 = 0; c0 < nc; c0 += 256) {
        const int64_t c = c0 + threadIdx.x;
        __syncthreads();
        if (c < nc)
            sc[threadIdx.x] = make_float4((float)(xyz[3 * c] - ox), (float)(xyz[3 * c + 1] - oy),
                                          (float)(xyz[3 * c + 2] - oz), (float)q[c]);
        __syncthreads();
        const int m = (int)(nc - c0 < 256 ? nc - c0 : 256);
        float p = 0.f;
        for (int k = 0; k < m; ++k) {
            const float4 ch = sc[k];
            const float dx = x - ch.x, dy = y - ch.y, dz = z - ch.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float inv = rsqrtf(r2);
            const float g = kappa == 0.f ? inv : inv * exp2f(l2k * r2 * inv);
            p = fmaf(ch.w, g, p);
        }
        const float t = hi + p;
        lo += (fabsf(hi) >= fabsf(p)) ? ((hi - t) + p) : ((p - t) + hi);
        hi = t;
    }
    if (i < n) b[i] = ((double)hi + (double)lo) * kInv4Pi / eps;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n.
GL gauss_legendre(int n) {
    GL g{};
    g.n = n;
    auto legendre = [n](double x, double &pn, double &pn1) {
        double p0 = 1.0, p1 = x;
        if (n == 0) { pn = 1.0; pn1 = 0.0; return; }
        for (int k = 2; k <= n; ++k) {
            const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        pn = p1;
        pn1 = p0;  // P_{n-1}
    };
    for (int i = 0; i < n; ++i) {
        double x = std::cos(kPi * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double pn, pm;
            legendre(x, pn, pm);
            const double dp = n * (x * pn - pm) / (x * x - 1.0);
            const double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        double pn, pm;
        legendre(x, pn, pm);
        const double dp = n * (x * pn - pm) / (x * x - 1.0);
        g.x[i] = x;
        g.w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    return g;
}

}  // namespace

void upload_rules() {
    TriRule r[4] = {make_rule(1), make_rule(3), make_rule(7), make_rule(19)};
    PB_CUDA_TRY(cudaMemcpyToSymbol(c_rules, r, sizeof(r)));
    TriRule32 r32[4] = {};
    for (int q = 0; q < 4; ++q) {
        r32[q].n = r[q].n;
        for (int k = 0; k < r[q].n; ++k) {
            r32[q].l1[k] = (float)r[q].l[k][1];
            r32[q].l2[k] = (float)r[q].l[k][2];
            r32[q].w[k] = (float)r[q].w[k];
        }
    }
    PB_CUDA_TRY(cudaMemcpyToSymbol(c_rules32, r32, sizeof(r32)));
}

bool valid_rule(int K) { return K == 1 || K == 3 || K == 7 || K == 19; }

void surface_geometry(SurfDev &S, int K, cudaStream_t s) {
    S.cen.alloc(3 * S.n); S.nrm.alloc(3 * S.n); S.area.alloc(S.n); S.L.alloc(S.n);
    TmpBuf<int32_t> bad(1, s);
    PB_CUDA_TRY(cudaMemsetAsync(bad.p, 0, 4, s));
    panel_geom_kernel<<<div_up(S.n, 128), 128, 0, s>>>(S.n, S.verts.p, S.tris.p, S.cen.p, S.nrm.p, S.area.p, S.L.p, bad.p);
    PB_LAUNCH_CHECK();
    S.gy.alloc(3 * S.n * K);
    S.gwa.alloc(S.n * K);
    gauss_points_kernel<<<div_up(S.n, 128), 128, 0, s>>>(S.n, rule_slot(K), S.verts.p, S.tris.p, S.area.p, S.gy.p, S.gwa.p);
    PB_LAUNCH_CHECK();
    int hb = 0;
    PB_CUDA_TRY(cudaMemcpyAsync(&hb, bad.p, 4, cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    if (hb) fail(PB_EINVAL, "surface has a zero-area triangle");
}

void near_values(const Pair &Pr, const Targets &G, const SurfDev &src, int K, int K_fine, double kappa, double *dV,
                 double *dK, cudaStream_t s) {
    if (G.n == 0 || Pr.n_near == 0) return;
    near_values_kernel<<<div_up(Pr.n_near, 128), 128, 0, s>>>(G.n, Pr.n_near, G.xs.p, Pr.near_ptr.p,
                                                               Pr.near_panel.p, src.verts.p, src.tris.p, src.nrm.p,
                                                               src.area.p, rule_slot(K), rule_slot(K_fine), kappa, dV,
                                                               dK);
    PB_LAUNCH_CHECK();
}

void near_values32(const Pair &Pr, const Targets &G, const SurfDev &src, int K, int K_fine, float *dV, float *dK,
                   cudaStream_t s) {
    if (G.n == 0 || Pr.n_near == 0) return;
    const int nk = (int)Pr.kappas.size();
    const float k0 = (float)Pr.kappas[0], k1 = nk > 1 ? (float)Pr.kappas[1] : 0.f;
    if (nk == 1)
        near_values32_kernel<1><<<div_up(Pr.n_near, 128), 128, 0, s>>>(
            G.n, Pr.n_near, G.xs.p, Pr.near_ptr.p, Pr.near_panel.p, src.verts.p, src.tris.p, src.nrm.p, src.area.p,
            rule_slot(K), rule_slot(K_fine), k0, k1, dV, dK);
    else
        near_values32_kernel<2><<<div_up(Pr.n_near, 128), 128, 0, s>>>(
            G.n, Pr.n_near, G.xs.p, Pr.near_ptr.p, Pr.near_panel.p, src.verts.p, src.tris.p, src.nrm.p, src.area.p,
            rule_slot(K), rule_slot(K_fine), k0, k1, dV, dK);
    PB_LAUNCH_CHECK();
}

namespace {
// out_i = selfv_i - (1/4pi) sum_k w_k A_i G(|c_i - y_ik|): the self value less the
// share of panel i's own K points in the direct sum at its centroid (FP64).
__global__ void self_minus_kpoint_kernel(int64_t n, int K, const double *__restrict__ cen,
                                         const double *__restrict__ gy, const double *__restrict__ gwa, double kappa,
                                         const double *__restrict__ selfv, double *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double sum = 0.0;
    for (int k = 0; k < K; ++k) {
        const int64_t q = i * K + k;
        const double dx = cen[3 * i] - gy[3 * q], dy = cen[3 * i + 1] - gy[3 * q + 1], dz = cen[3 * i + 2] - gy[3 * q + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        sum += gwa[q] * (kappa == 0.0 ? 1.0 / r : exp(-kappa * r) / r);
    }
    out[i] = selfv[i] - kInv4Pi * sum;
}
}  // namespace

void self_minus_kpoint(const SurfDev &S, int K, double kappa, const double *selfv, double *out, cudaStream_t s) {
    self_minus_kpoint_kernel<<<div_up(S.n, 128), 128, 0, s>>>(S.n, K, S.cen.p, S.gy.p, S.gwa.p, kappa, selfv, out);
    PB_LAUNCH_CHECK();
}

void self_integrals(const SurfDev &S, int N_k, double kappa, double *out, cudaStream_t s) {
    if (N_k < 1 || N_k > 32) fail(PB_EINVAL, "N_k must be in 1..32");
    GL gl = gauss_legendre(N_k);
    self_integral_kernel<1><<<div_up(S.n, 128), 128, 0, s>>>(S.n, S.verts.p, S.tris.p, S.cen.p, gl, kappa, 0.0, out,
                                                             nullptr);
    PB_LAUNCH_CHECK();
}

void self_integrals2(const SurfDev &S, int N_k, double kappa0, double kappa1, double *out0, double *out1,
                     cudaStream_t s) {
    if (N_k < 1 || N_k > 32) fail(PB_EINVAL, "N_k must be in 1..32");
    GL gl = gauss_legendre(N_k);
    self_integral_kernel<2><<<div_up(S.n, 128), 128, 0, s>>>(S.n, S.verts.p, S.tris.p, S.cen.p, gl, kappa0, kappa1,
                                                             out0, out1);
    PB_LAUNCH_CHECK();
}

void self_integrals_dkappa(const SurfDev &S, int N_k, double kappa, double *out, cudaStream_t s) {
    if (N_k < 1 || N_k > 32) fail(PB_EINVAL, "N_k must be in 1..32");
    GL gl = gauss_legendre(N_k);
    self_dkappa_kernel<<<div_up(S.n, 128), 128, 0, s>>>(S.n, S.verts.p, S.tris.p, S.cen.p, gl, kappa, out);
    PB_LAUNCH_CHECK();
}

void rhs_rows(const SurfDev &S, int64_t nc, const double *q, const double *xyz, double kappa, double eps, double *b,
              const double *origin, cudaStream_t s) {
    if (origin) {
        rhs32_kernel<<<div_up(S.n, 256), 256, 0, s>>>(S.n, S.cen.p, nc, q, xyz, origin[0], origin[1], origin[2],
                                                      (float)kappa, eps, b);
    } else {
        rhs_kernel<<<div_up(S.n, 128), 128, 0, s>>>(S.n, S.cen.p, nc, q, xyz, kappa, eps, b);
    }
    PB_LAUNCH_CHECK();
}

}  // namespace pb
