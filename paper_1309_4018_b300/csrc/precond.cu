// Cluster block preconditioner (see precond.cuh).
#include <cmath>

#include "gmres.cuh"
#include "precond.cuh"

namespace pb {

namespace {

constexpr int kMaxK = 19;                        // Gauss points per panel at most
constexpr float kInv4PiF = 0.0795774715459476678f;

struct BuildArgs {
    ClusterSurface sf;
    ClusterGeom g;
    ClusterRows r;
    float *binv;
    int *err;
};

// NB2: unknowns per block at most (twice the panels), a power of two; the
// kernels run 2 NB2 threads (build) and NB2 threads (apply).
template <int NB2>
size_t build_smem(int K) {
    constexpr int CB = NB2 / 2;
    return sizeof(float) * ((size_t)NB2 * (NB2 + 1) + CB * 6 + (size_t)CB * K * 4 + NB2 + 2 * CB) +
           sizeof(int) * 2 * NB2;
}

// One block per run: its couplings, then Gauss-Jordan elimination with
// partial pivoting in shared memory (in place; the row interchanges become a
// column relabelling of the result), the inverse written transposed.
// Local unknown u = 2 b + (0: phi, 1: dphi) of panel b; local row w = 2 a + side.
template <int NB2>
__global__ void __launch_bounds__(2 * NB2) cluster_build_kernel(BuildArgs a) {
    constexpr int kBlockDim = NB2, kPad = NB2 + 1, kBuildThreads = 2 * NB2, CB = NB2 / 2;
    extern __shared__ __align__(16) unsigned char smem[];
    const int K = a.g.K;
    float *A = reinterpret_cast<float *>(smem);                  // [NB2][NB2 + 1]
    float *cx = A + kBlockDim * kPad;                            // centroids, relative to the first panel's
    float *nx = cx + 3 * CB;                                     // normals
    float *gp = nx + 3 * CB;                                     // Gauss points (x, y, z, w A) relative
    float *fcol = gp + 4 * CB * K;                               // the pivot column of a step
    float *sv = fcol + kBlockDim;                                // self values, per side
    int *perm = reinterpret_cast<int *>(sv + 2 * CB);            // pivot row of every step
    int *col = perm + kBlockDim;                                 // result column -> working column
    __shared__ int s_piv;
    __shared__ float s_pval;
    const ClusterSurface &sf = a.sf;
    const int tid = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * sf.cb;
    const int nb = (int)min((int64_t)sf.cb, sf.n - c0);
    const int n2 = 2 * nb;
    const int ref = sf.order[c0];
    const double rx = a.g.cen[3 * ref], ry = a.g.cen[3 * ref + 1], rz = a.g.cen[3 * ref + 2];
    for (int b = tid; b < nb; b += kBuildThreads) {
        const int p = sf.order[c0 + b];
        cx[3 * b] = (float)(a.g.cen[3 * p] - rx);
        cx[3 * b + 1] = (float)(a.g.cen[3 * p + 1] - ry);
        cx[3 * b + 2] = (float)(a.g.cen[3 * p + 2] - rz);
        for (int d = 0; d < 3; ++d) nx[3 * b + d] = (float)a.g.nrm[3 * p + d];
        for (int s = 0; s < 2; ++s) sv[s * CB + b] = a.r.selfV[s] ? (float)a.r.selfV[s][p] : 0.f;
    }
    for (int e = tid; e < nb * K; e += kBuildThreads) {
        const int b = e / K, k = e - b * K;
        const int64_t q = (int64_t)sf.order[c0 + b] * K + k;
        gp[4 * e] = (float)(a.g.gy[3 * q] - rx);
        gp[4 * e + 1] = (float)(a.g.gy[3 * q + 1] - ry);
        gp[4 * e + 2] = (float)(a.g.gy[3 * q + 2] - rz);
        gp[4 * e + 3] = (float)a.g.gwa[q];
    }
    __syncthreads();
    const float k0 = (float)a.r.kappa[0], k1 = (float)a.r.kappa[1];
    const float cK0 = (float)a.r.cK[0], cK1 = (float)a.r.cK[1], cV0 = (float)a.r.cV[0], cV1 = (float)a.r.cV[1];
    for (int e = tid; e < nb * nb; e += kBuildThreads) {
        const int ta = e / nb, sb = e - ta * nb;
        float K0 = 0.f, K1 = 0.f, V0 = 0.f, V1 = 0.f;
        if (ta != sb) {
            const float x = cx[3 * ta], y = cx[3 * ta + 1], z = cx[3 * ta + 2];
            const float n0 = nx[3 * sb], n1 = nx[3 * sb + 1], n2v = nx[3 * sb + 2];
            for (int k = 0; k < K; ++k) {
                const float *q = gp + 4 * (sb * K + k);
                const float dx = x - q[0], dy = y - q[1], dz = z - q[2];
                const float r2 = dx * dx + dy * dy + dz * dz;
                const float ri = rsqrtf(r2), r = r2 * ri;
                const float rn = (dx * n0 + dy * n1 + dz * n2v) * ri * ri * ri;
                const float e0 = __expf(-k0 * r), e1 = __expf(-k1 * r);
                V0 += q[3] * e0 * ri;
                V1 += q[3] * e1 * ri;
                K0 += q[3] * rn * (1.f + k0 * r) * e0;
                K1 += q[3] * rn * (1.f + k1 * r) * e1;
            }
            K0 *= kInv4PiF; K1 *= kInv4PiF; V0 *= kInv4PiF; V1 *= kInv4PiF;
        } else {
            V0 = sv[ta];
            V1 = sv[CB + ta];
        }
        const float h = ta == sb ? 0.5f : 0.f;
        A[(2 * ta) * kPad + 2 * sb] = h + cK0 * K0;
        A[(2 * ta) * kPad + 2 * sb + 1] = cV0 * V0;
        A[(2 * ta + 1) * kPad + 2 * sb] = h + cK1 * K1;
        A[(2 * ta + 1) * kPad + 2 * sb + 1] = cV1 * V1;
    }
    __syncthreads();
    // Gauss-Jordan elimination.  Thread (rg, c) = (tid / NB2, tid % NB2) owns
    // column c of the rows rg, rg + 2, ...: no index division in the loops.
    const int cc = tid & (kBlockDim - 1), rg = tid / kBlockDim;
    constexpr int kRowStep = kBuildThreads / kBlockDim;
    for (int k = 0; k < n2; ++k) {
        if (tid < 32) {
            float best = -1.f, bval = 0.f;
            int bi = k;
            for (int r = k + tid; r < n2; r += 32) {
                const float v = A[r * kPad + k];
                if (fabsf(v) > best) { best = fabsf(v); bval = v; bi = r; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ob = __shfl_xor_sync(0xffffffffu, best, o);
                const float ov = __shfl_xor_sync(0xffffffffu, bval, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bval = ov; bi = oi; }
            }
            if (tid == 0) {
                s_piv = bi;
                s_pval = bval;
                perm[k] = bi;
                if (!(best > 0.f)) atomicExch(a.err, 1);
            }
        }
        __syncthreads();
        const int p = s_piv;
        if (p != k && rg == 0 && cc < n2) {
            const float t = A[k * kPad + cc];
            A[k * kPad + cc] = A[p * kPad + cc];
            A[p * kPad + cc] = t;
        }
        __syncthreads();
        const float ip = s_pval != 0.f ? 1.f / s_pval : 0.f;
        if (tid < n2 && tid != k) fcol[tid] = A[tid * kPad + k];
        if (rg == 1 && cc < n2) A[k * kPad + cc] = (cc == k ? 1.f : A[k * kPad + cc]) * ip;
        __syncthreads();
        if (cc < n2) {
            const float akc = A[k * kPad + cc];
            const bool diag = cc == k;
#pragma unroll
            for (int i = 0; i < kBlockDim / kRowStep; ++i) {
                const int r = rg + kRowStep * i;
                if (r < n2 && r != k) {
                    const float base = diag ? 0.f : A[r * kPad + cc];
                    A[r * kPad + cc] = base - fcol[r] * akc;
                }
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        for (int c = 0; c < n2; ++c) col[c] = c;
        for (int k = n2 - 1; k >= 0; --k) {
            const int p = perm[k];
            const int t = col[k];
            col[k] = col[p];
            col[p] = t;
        }
    }
    __syncthreads();
    float *out = a.binv + (sf.first + blockIdx.x) * (int64_t)kBlockDim * kBlockDim;
#pragma unroll 4
    for (int e = tid; e < kBlockDim * kBlockDim; e += kBuildThreads) {
        const int w = e / kBlockDim, u = e & (kBlockDim - 1);
        out[e] = (u < n2 && w < n2) ? A[u * kPad + col[w]] : 0.f;
    }
}

// z = M^-1 v for the runs of one surface, one block per run, thread u for
// local unknown u (FP64 sums of the FP32 inverse times the FP64 entries).
// PREP: v is v_j of the device Arnoldi loop, formed and stored here.
template <bool PREP, int NB2, bool TRANS = false>
__global__ void __launch_bounds__(NB2) cluster_apply_kernel(ClusterSurface sf, const float *__restrict__ binv,
                                                                  const double *__restrict__ u,
                                                                  double *__restrict__ z, const GmresState *st,
                                                                  double *__restrict__ V, int64_t ld,
                                                                  const double *__restrict__ w,
                                                                  const double *__restrict__ num_sq) {
    constexpr int kBlockDim = NB2;
    __shared__ float2 vl2[NB2];
    __shared__ int pan[NB2 / 2];
    __shared__ double s_inv;
    const int t = threadIdx.x;
    const int64_t c0 = (int64_t)blockIdx.x * sf.cb;
    const int nb = (int)min((int64_t)sf.cb, sf.n - c0);
    const int n2 = 2 * nb;
    if (t < nb) pan[t] = sf.order[c0 + t];
    int pend = 0;
    if (PREP) {
        pend = st->pend;
        if (t == 0 && pend) {
            const double d = sqrt(*num_sq);
            s_inv = d > 0.0 ? 1.0 / d : 0.0;
        }
    }
    __syncthreads();
    if (t < n2) {
        const int64_t gi = 2 * sf.off + (int64_t)(t & 1) * sf.n + pan[t >> 1];
        double v;
        if (PREP) {
            double *colj = V + (int64_t)st->j * ld;
            if (pend) {
                v = w[gi] * s_inv;
                colj[gi] = v;
            } else {
                v = colj[gi];
            }
        } else {
            v = u[gi];
        }
        const float vh = (float)v;
        vl2[t] = make_float2(vh, (float)(v - (double)vh));
    }
    __syncthreads();
    if (t >= n2) return;
    // FP32 pairs (hi + lo, ~48 significant bits) on the FP32 pipe: the products
    // m v_hi exactly by fma, m v_lo rounded, the sum compensated (TwoSum), so
    // the map is linear to ~1e-14 relative without FP64 arithmetic per term
    // TRANS: the transpose (z_w = sum_u Binv[u][w] v_u), row w of the stored block
    const float *bt = binv + (sf.first + blockIdx.x) * (int64_t)kBlockDim * kBlockDim + (TRANS ? t * kBlockDim : t);
    float sh = 0.f, sl = 0.f;
    for (int c = 0; c < n2; ++c) {
        const float m = bt[TRANS ? c : (int64_t)c * kBlockDim];
        const float2 v = vl2[c];
        const float ph = m * v.x;
        const float pe = fmaf(m, v.y, fmaf(m, v.x, -ph));
        const float s1 = sh + ph;
        const float bb = s1 - sh;
        sl += ((sh - (s1 - bb)) + (ph - bb)) + pe;
        sh = s1;
    }
    z[2 * sf.off + (int64_t)(t & 1) * sf.n + pan[t >> 1]] = (double)sh + (double)sl;
}

}  // namespace

int cluster_block_dim(int cb) { return cb <= 8 ? 16 : cb <= 16 ? 32 : cb <= 32 ? 64 : 128; }

namespace {

template <int NB2>
void build_launch(const BuildArgs &a, cudaStream_t s) {
    static bool attr = false;
    const size_t smem = build_smem<NB2>(kMaxK);
    if (!attr) {
        PB_CUDA_TRY(cudaFuncSetAttribute(cluster_build_kernel<NB2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
        attr = true;
    }
    cluster_build_kernel<NB2><<<(unsigned)a.sf.nblocks(), 2 * NB2, build_smem<NB2>(a.g.K), s>>>(a);
    PB_LAUNCH_CHECK();
}

template <bool PREP, int NB2, bool TRANS>
void apply_launch(const ClusterSurface &sf, const float *binv, const double *u, double *z, const GmresState *st,
                  double *V, int64_t ld, const double *w, const double *num_sq, cudaStream_t s) {
    cluster_apply_kernel<PREP, NB2, TRANS><<<(unsigned)sf.nblocks(), NB2, 0, s>>>(sf, binv, u, z, st, V, ld, w,
                                                                                    num_sq);
    PB_LAUNCH_CHECK();
}

template <bool PREP, bool TRANS = false>
void apply_any(const ClusterSurface &sf, const float *binv, const double *u, double *z, const GmresState *st,
               double *V, int64_t ld, const double *w, const double *num_sq, cudaStream_t s) {
    switch (cluster_block_dim(sf.cb)) {
        case 16: apply_launch<PREP, 16, TRANS>(sf, binv, u, z, st, V, ld, w, num_sq, s); break;
        case 32: apply_launch<PREP, 32, TRANS>(sf, binv, u, z, st, V, ld, w, num_sq, s); break;
        case 64: apply_launch<PREP, 64, TRANS>(sf, binv, u, z, st, V, ld, w, num_sq, s); break;
        default: apply_launch<PREP, 128, TRANS>(sf, binv, u, z, st, V, ld, w, num_sq, s);
    }
}

}  // namespace

void cluster_blocks(const ClusterSurface &sf, const ClusterGeom &g, const ClusterRows &r, float *binv, int *err,
                    cudaStream_t s) {
    if (sf.n == 0) return;
    if (g.K > kMaxK || sf.cb < 1 || sf.cb > kClusterMax) fail(PB_EINVAL, "internal: preconditioner block shape");
    const BuildArgs a{sf, g, r, binv, err};
    switch (cluster_block_dim(sf.cb)) {
        case 16: build_launch<16>(a, s); break;
        case 32: build_launch<32>(a, s); break;
        case 64: build_launch<64>(a, s); break;
        default: build_launch<128>(a, s);
    }
}

void cluster_apply(const std::vector<ClusterSurface> &sfs, const float *binv, const double *u, double *z,
                   cudaStream_t s) {
    for (const ClusterSurface &sf : sfs)
        if (sf.n) apply_any<false>(sf, binv, u, z, nullptr, nullptr, 0, nullptr, nullptr, s);
}

void cluster_apply_T(const std::vector<ClusterSurface> &sfs, const float *binv, const double *u, double *z,
                     cudaStream_t s) {
    for (const ClusterSurface &sf : sfs)
        if (sf.n) apply_any<false, true>(sf, binv, u, z, nullptr, nullptr, 0, nullptr, nullptr, s);
}

void cluster_prep(const std::vector<ClusterSurface> &sfs, const float *binv, const GmresState *st, double *V,
                  int64_t ld, const double *w, const double *num_sq, double *z, cudaStream_t s) {
    for (const ClusterSurface &sf : sfs)
        if (sf.n) apply_any<true>(sf, binv, nullptr, z, st, V, ld, w, num_sq, s);
}

}  // namespace pb
