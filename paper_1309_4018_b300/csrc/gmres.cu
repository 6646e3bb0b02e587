// Device-resident restarted GMRES in FP64 (Sec. 2.3, last paragraph: a Krylov
// solver with one treecode evaluation per iteration; stopping tolerance
// gmres_tol of Tables 1 and 3) and the energy reductions (Eqs. solv, total_energy).
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2): two block
// projections per step instead of j sequential ones, with the orthogonality
// of modified Gram-Schmidt.  The Hessenberg least-squares problem is reduced by
// Givens rotations on the device; the host only reads the residual estimate.
// All reductions use a fixed block count and a fixed combination order, so
// results do not depend on scheduling.
#include "gmres.cuh"

namespace pb {

namespace {

constexpr int kRedBlocks = 148;   // one per SM: two elements per thread halve the FP64 block reductions
constexpr int kRedThreads = 256;

// partial[v * kRedBlocks + block] = sum over the block's slice of V[v] . w.
// Vectors are taken 8 at a time: each thread keeps 8 running sums, so w is
// read once per group and the block synchronises once per group.
constexpr int kDotGroup = 8;
constexpr int kSliceGroup = 16;     // basis vectors per pass of the fused Arnoldi dots
constexpr int kMaxRestart = 200;    // the largest restart length (checked when the parameters are set)

__global__ void __launch_bounds__(kRedThreads) mdot_kernel(const double *__restrict__ V, int64_t ld, int nv,
                                                           const double *__restrict__ w, int64_t n,
                                                           double *__restrict__ partial) {
    __shared__ double sm[kDotGroup][kRedThreads / 32];
    const int64_t per = (n + kRedBlocks - 1) / kRedBlocks;
    const int64_t lo = blockIdx.x * per, hi = min(n, lo + per);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int v0 = 0; v0 < nv; v0 += kDotGroup) {
        const int nb = min(kDotGroup, nv - v0);
        double s[kDotGroup];
#pragma unroll
        for (int b = 0; b < kDotGroup; ++b) s[b] = 0.0;
        for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) {
            const double wi = w[i];
#pragma unroll
            for (int b = 0; b < kDotGroup; ++b)
                if (b < nb) s[b] += V[(int64_t)(v0 + b) * ld + i] * wi;
        }
#pragma unroll
        for (int b = 0; b < kDotGroup; ++b) {
            double t = s[b];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) sm[b][wid] = t;
        }
        __syncthreads();
        if (threadIdx.x < nb) {
            double t = 0.0;
            for (int k = 0; k < kRedThreads / 32; ++k) t += sm[threadIdx.x][k];
            partial[(v0 + threadIdx.x) * kRedBlocks + blockIdx.x] = t;
        }
        __syncthreads();
    }
}

// out[v] (+)= sum_b partial[v][b]; one warp per vector, fixed order.
__global__ void mdot_finish_kernel(const double *__restrict__ partial, int nv, double *__restrict__ out, int accumulate) {
    const int v = blockIdx.x;
    if (v >= nv) return;
    double s = 0.0;
    for (int b = threadIdx.x; b < kRedBlocks; b += 32) s += partial[v * kRedBlocks + b];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[v] = accumulate ? out[v] + s : s;
}

// dst = src / sqrt(*num_sq): the reciprocal is formed once per block (FP64
// division and square root are long sequences on the narrow FP64 pipe).
__global__ void scale_copy_kernel(const double *__restrict__ src, const double *__restrict__ num_sq,
                                  double *__restrict__ dst, int64_t n) {
    __shared__ double inv;
    if (threadIdx.x == 0) {
        const double d = sqrt(*num_sq);
        inv = d > 0.0 ? 1.0 / d : 0.0;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i] * inv;
}

__global__ void axpby_kernel(double a, const double *__restrict__ x, double b, const double *__restrict__ y,
                             double *__restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a * x[i] + b * y[i];
}

// y = H[0..k)^-1 g (back substitution) into st->y.
// y = R^-1 g for the k x k upper triangle of H (columns of stride m + 1).  Up
// to kBackStage columns the block stages the triangle in shared memory first
// and one thread runs the substitution there; longer cycles read it from
// global memory.  Either way the same sums in the same order.
constexpr int kBackThreads = 256;
constexpr int kBackStage = 64;

__global__ void __launch_bounds__(kBackThreads) back_solve_kernel(GmresState *st, int k) {
    __shared__ double sH[kBackStage * kBackStage];
    __shared__ double sy[kBackStage];
    const int m = st->m;
    const double *H = st->H, *g = st->g;
    if (k > kBackStage) {
        if (threadIdx.x != 0) return;
        for (int i = k - 1; i >= 0; --i) {
            double s = g[i];
            for (int c = i + 1; c < k; ++c) s -= H[(int64_t)c * (m + 1) + i] * st->y[c];
            st->y[i] = s / H[(int64_t)i * (m + 1) + i];
        }
        return;
    }
    for (int e = threadIdx.x; e < k * k; e += kBackThreads) {
        const int c = e / k, i = e - c * k;
        sH[e] = H[(int64_t)c * (m + 1) + i];
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = k - 1; i >= 0; --i) {
        double s = g[i];
        for (int c = i + 1; c < k; ++c) s -= sH[c * k + i] * sy[c];
        sy[i] = s / sH[i * k + i];
    }
    for (int i = 0; i < k; ++i) st->y[i] = sy[i];
}

// x += sum_c V[c] y[c]
__global__ void update_x_kernel(const double *__restrict__ V, int64_t ld, int k, const GmresState *st,
                                double *__restrict__ x, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = x[i];
    for (int c = 0; c < k; ++c) s += V[c * ld + i] * st->y[c];
    x[i] = s;
}

__global__ void set_bnorm_kernel(GmresState *st, double bn) {
    if (threadIdx.x == 0) st->bnorm = bn;
}

__global__ void set_cycle_kernel(GmresState *st, int maxit) {
    if (threadIdx.x != 0) return;
    st->j = 0;
    st->pend = 0;
    st->maxit = maxit;
    st->steps = 0.0;
}

// Fused first kernel of a device-loop step for the panels [off, off + n) of
// one surface: v = w / ||w|| (pend: the previous step's new vector, stored as
// column j) or column j; z = M^-1 v with the panels' 2x2 blocks (minv), or
// z = v without a preconditioner.  Elements off + i and off + n + i form a
// panel's pair.
__global__ void prep_step_kernel(int64_t n, int64_t off, const double *__restrict__ minv,
                                 const GmresState *__restrict__ st, double *__restrict__ V, int64_t ld,
                                 const double *__restrict__ w, const double *__restrict__ num_sq,
                                 double *__restrict__ z) {
    __shared__ double inv;
    const int pend = st->pend;
    if (threadIdx.x == 0 && pend) {
        const double d = sqrt(*num_sq);
        inv = d > 0.0 ? 1.0 / d : 0.0;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double *col = V + (int64_t)st->j * ld;
    const int64_t i1 = off + i, i2 = off + n + i;
    double a, b;
    if (pend) {
        a = w[i1] * inv;
        b = w[i2] * inv;
        col[i1] = a;
        col[i2] = b;
    } else {
        a = col[i1];
        b = col[i2];
    }
    if (minv) {
        z[i1] = minv[4 * i] * a + minv[4 * i + 1] * b;
        z[i2] = minv[4 * i + 2] * a + minv[4 * i + 3] * b;
    } else {
        z[i1] = a;
        z[i2] = b;
    }
}

__global__ void copy_basis_kernel(const double *__restrict__ V, int64_t ld, const GmresState *st,
                                  double *__restrict__ dst, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = V[(int64_t)st->j * ld + i];
}

// v_{j+1} = w / ||w|| for the device column j (one reciprocal per block).
__global__ void scale_copy_next_kernel(const double *__restrict__ src, const double *__restrict__ num_sq,
                                       double *__restrict__ V, int64_t ld, const GmresState *st, int64_t n) {
    __shared__ double inv;
    if (threadIdx.x == 0) {
        const double d = sqrt(*num_sq);
        inv = d > 0.0 ? 1.0 / d : 0.0;
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) V[(int64_t)(st->j + 1) * ld + i] = src[i] * inv;
}

// After step j: record the steps and either advance to column j + 1 or end the loop.
__global__ void arnoldi_control_kernel(GmresState *st, cudaGraphConditionalHandle h, double tol) {
    if (threadIdx.x != 0) return;
    const int steps = st->j + 1;
    st->steps = (double)steps;
    const bool stop = !(st->res_est >= tol) || steps >= st->maxit || steps >= st->m;
    if (!stop) st->j = steps;
    cudaGraphSetConditional(h, stop ? 0u : 1u);
}

__global__ void init_cycle_kernel(GmresState *st, const double *__restrict__ beta2) {
    if (threadIdx.x != 0) return;
    const double beta = sqrt(*beta2);
    for (int i = 0; i <= st->m; ++i) st->g[i] = 0.0;
    st->g[0] = beta;
    st->beta = beta;
}

// ---------------------------------------------------------------- energies
// out = scale * sum_k q_k phi[k] (fixed-order reduction in one block).
__global__ void weighted_sum_kernel(const double *__restrict__ q, const double *__restrict__ phi, int64_t n,
                                    double scale, double *__restrict__ out) {
    __shared__ double sm[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += q[i] * phi[i];
    sm[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = scale * sm[0];
}

// rowv[i] = sum_{j != i} q_j / r_ij
__global__ void coulomb_rows_kernel(const double *__restrict__ xyz, const double *__restrict__ q, int64_t n,
                                    double *__restrict__ rowv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    double s = 0.0;
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        const double dx = x - xyz[3 * j], dy = y - xyz[3 * j + 1], dz = z - xyz[3 * j + 2];
        s += q[j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    rowv[i] = s;
}

__global__ void bj_inverse_kernel(int64_t n, double cin, const double *__restrict__ sa_in, double cout,
                                  const double *__restrict__ sa_out, double *__restrict__ minv) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a11 = 0.5, a12 = cin * sa_in[i], a21 = 0.5, a22 = cout * sa_out[i];
    const double det = a11 * a22 - a12 * a21;
    minv[4 * i] = a22 / det;
    minv[4 * i + 1] = -a12 / det;
    minv[4 * i + 2] = -a21 / det;
    minv[4 * i + 3] = a11 / det;
}

__global__ void bj_apply_kernel(int64_t n, const double *__restrict__ minv, const double *__restrict__ u1,
                                const double *__restrict__ u2, double *__restrict__ z1, double *__restrict__ z2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = u1[i], b = u2[i];
    z1[i] = minv[4 * i] * a + minv[4 * i + 1] * b;
    z2[i] = minv[4 * i + 2] * a + minv[4 * i + 3] * b;
}

__global__ void combination_kernel(const double *__restrict__ V, int64_t ld, int k, const GmresState *st,
                                   double *__restrict__ out, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int c = 0; c < k; ++c) s += V[c * ld + i] * st->y[c];
    out[i] = s;
}

void dot_device(const double *V, int64_t ld, int nv, const double *w, int64_t n, double *partial, double *out,
                cudaStream_t s) {
    mdot_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(V, ld, nv, w, n, partial);
    PB_LAUNCH_CHECK();
    mdot_finish_kernel<<<nv, 32, 0, s>>>(partial, nv, out, 0);
    PB_LAUNCH_CHECK();
}

// ---------------------------------------------------------------- fused Arnoldi step
// One CGS2 step in four launches.  Every block owns a fixed slice of the
// vector; its partial dot products go to `partial`, and the block that
// arrives last (an atomic count, each block announcing itself after a fence)
// adds the partials in block order, so the sums are deterministic.
struct ArnoldiArgs {
    const double *V;
    int64_t ld, n;
    int nv;                 // j + 1 basis vectors
    double *w;
    double *h1, *h2, *nrm2; // device scalars
    double *partial;        // kDotGroup-blocked partials
    unsigned *count;        // zero between launches
    GmresState *st;
    int j;
    // fused device loop: the last block of the norm kernel also ends or advances the loop
    int control;
    double tol;
    cudaGraphConditionalHandle h;
};

__device__ __forceinline__ bool arrive_last(unsigned *count) {
    __shared__ bool last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last) __threadfence();
    return last;
}

// a.j < 0: the column is the device state's (device-driven loop).
__device__ __forceinline__ ArnoldiArgs device_column(ArnoldiArgs a) {
    if (a.j < 0) {
        a.j = a.st->j;
        a.nv = a.j + 1;
    }
    return a;
}

// Block partials of V[v] . w over the block's slice, for v < nv, up to 16
// vectors per pass (all of a pass's loads per element in flight at once).
// The FP64 pipe is narrow on this part, so a pass computes its vectors
// rounded up to a multiple of four (not always 16) and the block reduction is arranged to issue few FP64
// instructions: every thread's partials go to shared memory, each (vector,
// 8-thread chunk) is summed by one thread, and one warp per vector adds the
// 32 chunk sums by a butterfly (each warp takes two vectors of the pass).
template <int NB>
__device__ __forceinline__ void slice_pass(const ArnoldiArgs &a, int64_t lo, int64_t hi, int v0, int nb,
                                           double (*red)[kRedThreads + 1]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double acc[NB];
#pragma unroll
    for (int b = 0; b < NB; ++b) acc[b] = 0.0;
#pragma unroll 1
    for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) {
        const double wi = a.w[i];
        // unconditional loads (the index clamped to the pass's last vector;
        // the extra sums are never stored), so the NB are issued together
        double x[NB];
#pragma unroll
        for (int b = 0; b < NB; ++b) x[b] = a.V[(int64_t)(v0 + min(b, nb - 1)) * a.ld + i];
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] += x[b] * wi;
    }
#pragma unroll
    for (int b = 0; b < NB; ++b) red[b][threadIdx.x] = acc[b];
    __syncthreads();
    // warp wid sums vectors wid and wid + 8: lane adds the partials of threads 8 lane .. 8 lane + 7
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int vb = wid + 8 * h;
        if (vb < nb) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < 8; ++k) t += red[vb][8 * lane + k];
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
            if (lane == 0) a.partial[(v0 + vb) * kRedBlocks + blockIdx.x] = t;
        }
    }
    __syncthreads();
}

// A pass takes its nb vectors in a form for 4, 8, 12 or 16.
__device__ void slice_dots(const ArnoldiArgs &a, int64_t lo, int64_t hi) {
    constexpr int G = kSliceGroup;
    static_assert(kRedThreads == 256 && G == 16, "the reduction layout assumes 256 threads, 16 vectors");
    __shared__ double red[G][kRedThreads + 1];
    for (int v0 = 0; v0 < a.nv; v0 += G) {
        const int nb = min(G, a.nv - v0);
        if (nb <= 4) slice_pass<4>(a, lo, hi, v0, nb, red);
        else if (nb <= 8) slice_pass<8>(a, lo, hi, v0, nb, red);
        else if (nb <= 12) slice_pass<12>(a, lo, hi, v0, nb, red);
        else slice_pass<16>(a, lo, hi, v0, nb, red);
    }
}

// w[i] - sum_v V[v][i] h[v], subtracted in v order: eight basis loads in
// flight per step, then four, then one at a time for the last few.
__device__ __forceinline__ double project_elem(const ArnoldiArgs &a, const double *__restrict__ sh, int64_t i,
                                               double t) {
    int v = 0;
    for (; v + 8 <= a.nv; v += 8) {
        double x[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = a.V[(int64_t)(v + u) * a.ld + i];
#pragma unroll
        for (int u = 0; u < 8; ++u) t -= x[u] * sh[v + u];
    }
    if (v + 4 <= a.nv) {
        double x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = a.V[(int64_t)(v + u) * a.ld + i];
#pragma unroll
        for (int u = 0; u < 4; ++u) t -= x[u] * sh[v + u];
        v += 4;
    }
    for (; v < a.nv; ++v) t -= a.V[(int64_t)v * a.ld + i] * sh[v];
    return t;
}

// h[0 .. nv) into shared memory, zero up to the next multiple of eight.
__device__ __forceinline__ void stage_h(double *sh, const double *__restrict__ h, int nv) {
    const int nv8 = (nv + 7) & ~7;
    for (int v = threadIdx.x; v < nv8; v += kRedThreads) sh[v] = v < nv ? h[v] : 0.0;
    __syncthreads();
}

// One warp per vector: lanes take the block partials in a fixed stride, then a butterfly.
__device__ void finish_dots(const ArnoldiArgs &a, int nv, double *out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int v = wid; v < nv; v += kRedThreads / 32) {
        double t = 0.0;
#pragma unroll
        for (int b = lane; b < kRedBlocks; b += 32) t += __ldcg(a.partial + v * kRedBlocks + b);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) out[v] = t;
    }
}

// h1 = V^T w
__global__ void __launch_bounds__(kRedThreads) arnoldi_dots_kernel(ArnoldiArgs a0) {
    const ArnoldiArgs a = device_column(a0);
    const int64_t per = (a.n + kRedBlocks - 1) / kRedBlocks;
    const int64_t lo = blockIdx.x * per, hi = min(a.n, lo + per);
    slice_dots(a, lo, hi);
    if (arrive_last(a.count)) {
        finish_dots(a, a.nv, a.h1);
        if (threadIdx.x == 0) *a.count = 0;
    }
}

// w -= V h1, then h2 = V^T w (the block projects its own slice first)
__global__ void __launch_bounds__(kRedThreads) arnoldi_project_dots_kernel(ArnoldiArgs a0) {
    const ArnoldiArgs a = device_column(a0);
    const int64_t per = (a.n + kRedBlocks - 1) / kRedBlocks;
    const int64_t lo = blockIdx.x * per, hi = min(a.n, lo + per);
    __shared__ double sh[kMaxRestart + 8];
    stage_h(sh, a.h1, a.nv);
    for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) a.w[i] = project_elem(a, sh, i, a.w[i]);
    __syncthreads();
    slice_dots(a, lo, hi);
    if (arrive_last(a.count)) {
        finish_dots(a, a.nv, a.h2);
        if (threadIdx.x == 0) *a.count = 0;
    }
}

// w -= V h2; nrm2 = w . w; the last block also forms the Hessenberg column
// h1 + h2 and applies the Givens rotations (residual estimate in st).
__global__ void __launch_bounds__(kRedThreads) arnoldi_project_norm_kernel(ArnoldiArgs a0) {
    const ArnoldiArgs a = device_column(a0);
    __shared__ double sm[kRedThreads / 32];
    const int64_t per = (a.n + kRedBlocks - 1) / kRedBlocks;
    const int64_t lo = blockIdx.x * per, hi = min(a.n, lo + per);
    __shared__ double sh[kMaxRestart + 8];
    // the Hessenberg column h1 + h2 and the earlier rotations, for the last
    // block's Givens update: fixed since the previous launches, so every block
    // stages them now and the last block does not wait for them after its arrival
    __shared__ double scol[kMaxRestart + 2], scs[kMaxRestart], ssn[kMaxRestart];
    {
        const GmresState *st = a.st;
        for (int i = threadIdx.x; i <= a.j; i += kRedThreads) scol[i] = a.h1[i] + a.h2[i];
        for (int i = threadIdx.x; i < a.j; i += kRedThreads) {
            scs[i] = st->cs[i];
            ssn[i] = st->sn[i];
        }
    }
    stage_h(sh, a.h2, a.nv);
    double s2 = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) {
        const double t = project_elem(a, sh, i, a.w[i]);
        a.w[i] = t;
        s2 += t * t;
    }
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kRedThreads / 32; ++k) t += sm[k];
        a.partial[blockIdx.x] = t;
    }
    if (arrive_last(a.count)) {
        // ||w||^2 from the block partials: a fixed tree over the whole block
        double p = 0.0;
        for (int b = threadIdx.x; b < kRedBlocks; b += kRedThreads) p += __ldcg(a.partial + b);
        for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
        if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = p;
        __syncthreads();
        // thread 0 applies the rotations to the staged column (no global
        // round trip per step), then the block writes it back
        GmresState *st = a.st;
        const int m = st->m, j = a.j;
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kRedThreads / 32; ++k) t += sm[k];
            *a.nrm2 = t;
            *a.count = 0;
            double *col = scol;
            const double hn = sqrt(t);
            col[j + 1] = hn;
            st->hnext = hn;
            for (int i = 0; i < j; ++i) {
                const double u = scs[i] * col[i] + ssn[i] * col[i + 1];
                col[i + 1] = -ssn[i] * col[i] + scs[i] * col[i + 1];
                col[i] = u;
            }
            const double den = hypot(col[j], col[j + 1]);
            const double c = den > 0.0 ? col[j] / den : 1.0, sn = den > 0.0 ? col[j + 1] / den : 0.0;
            st->cs[j] = c;
            st->sn[j] = sn;
            col[j] = den;
            col[j + 1] = 0.0;
            const double gj = st->g[j];
            st->g[j + 1] = -sn * gj;
            st->g[j] = c * gj;
            st->res_est = fabs(-sn * gj) / st->bnorm;
            if (a.control) {
                // every block has read the column index: the loop may advance it now
                const int steps = j + 1;
                st->steps = (double)steps;
                const bool stop = !(st->res_est >= a.tol) || steps >= st->maxit || steps >= m;
                if (!stop) {
                    st->j = steps;
                    st->pend = 1;
                }
                cudaGraphSetConditional(a.h, stop ? 0u : 1u);
            }
        }
        __syncthreads();
        double *col = st->H + (int64_t)j * (m + 1);
        for (int i = threadIdx.x; i <= j + 1; i += kRedThreads) col[i] = scol[i];
    }
}

}  // namespace

void Gmres::init(int64_t n_, int m_, cudaStream_t s) {
    n = n_;
    m = m_;
    ld = (n + 31) / 32 * 32;
    V.alloc((size_t)(m + 1) * ld);
    w.alloc(n);
    partial.alloc((size_t)kRedBlocks * (m + 2));
    hcol.alloc(m + 2);
    h2.alloc(m + 2);
    scal.alloc(4);
    H.alloc((size_t)(m + 1) * m);
    cs.alloc(m); sn.alloc(m); g.alloc(m + 1); y.alloc(m);
    st.alloc(1);
    count.alloc(1);
    count.zero(s);
    GmresState h{};
    h.m = m;
    h.H = H.p; h.cs = cs.p; h.sn = sn.p; h.g = g.p; h.y = y.p;
    h.bnorm = 1.0;
    hs.alloc(4);
    // page-locked source that outlives the copy: no host wait here (a later
    // init runs after the setup's final synchronisation)
    hst.alloc(1);
    *hst.p = h;
    PB_CUDA_TRY(cudaMemcpyAsync(st.p, hst.p, sizeof(h), cudaMemcpyHostToDevice, s));
}

void Gmres::norm2_async(const double *x, cudaStream_t s) {
    dot_device(x, 0, 1, x, n, partial.p, scal.p + 2, s);
    PB_CUDA_TRY(cudaMemcpyAsync(hs.p, scal.p + 2, sizeof(double), cudaMemcpyDeviceToHost, s));
}

void Gmres::set_bnorm(double bn, cudaStream_t s) {
    set_bnorm_kernel<<<1, 1, 0, s>>>(st.p, bn);
    PB_LAUNCH_CHECK();
}

void Gmres::start_cycle(const double *r, cudaStream_t s) {
    dot_device(r, ld, 1, r, n, partial.p, scal.p, s);
    scale_copy_kernel<<<div_up(n, 256), 256, 0, s>>>(r, scal.p, V.p, n);
    PB_LAUNCH_CHECK();
    init_cycle_kernel<<<1, 1, 0, s>>>(st.p, scal.p);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaMemcpyAsync(hs.p + 1, scal.p, sizeof(double), cudaMemcpyDeviceToHost, s));
}

void Gmres::arnoldi_step(int j, cudaStream_t s) {
    ArnoldiArgs a{};
    a.V = V.p;
    a.ld = ld;
    a.n = n;
    a.nv = j + 1;
    a.w = w.p;
    a.h1 = hcol.p;
    a.h2 = h2.p;
    a.nrm2 = scal.p + 1;
    a.partial = partial.p;
    a.count = count.p;
    a.st = st.p;
    a.j = j;
    arnoldi_dots_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(a);
    PB_LAUNCH_CHECK();
    arnoldi_project_dots_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(a);
    PB_LAUNCH_CHECK();
    arnoldi_project_norm_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(a);
    PB_LAUNCH_CHECK();
    scale_copy_kernel<<<div_up(n, 256), 256, 0, s>>>(w.p, scal.p + 1, V.p + (int64_t)(j + 1) * ld, n);
    PB_LAUNCH_CHECK();
    PB_CUDA_TRY(cudaMemcpyAsync(hs.p + 2, &st.p->res_est, sizeof(double), cudaMemcpyDeviceToHost, s));
}

void Gmres::set_cycle(int maxit, cudaStream_t s) {
    set_cycle_kernel<<<1, 1, 0, s>>>(st.p, maxit);
    PB_LAUNCH_CHECK();
}

void Gmres::copy_basis(double *dst, cudaStream_t s) {
    copy_basis_kernel<<<div_up(n, 256), 256, 0, s>>>(V.p, ld, st.p, dst, n);
    PB_LAUNCH_CHECK();
}

void Gmres::prep_step(const double *minv, const std::vector<std::pair<int64_t, int64_t>> &surfaces, double *z,
                      cudaStream_t s) {
    for (const auto &sf : surfaces) {
        if (sf.second == 0) continue;
        prep_step_kernel<<<div_up(sf.second, 256), 256, 0, s>>>(sf.second, 2 * sf.first, minv ? minv + 4 * sf.first : nullptr,
                                                                 st.p, V.p, ld, w.p, scal.p + 1, z);
        PB_LAUNCH_CHECK();
    }
}

void Gmres::arnoldi_step_dev(cudaGraphConditionalHandle h, double tol, cudaStream_t s, bool fused) {
    ArnoldiArgs a{};
    a.V = V.p;
    a.ld = ld;
    a.n = n;
    a.nv = 0;
    a.w = w.p;
    a.h1 = hcol.p;
    a.h2 = h2.p;
    a.nrm2 = scal.p + 1;
    a.partial = partial.p;
    a.count = count.p;
    a.st = st.p;
    a.j = -1;
    a.control = fused ? 1 : 0;
    a.tol = tol;
    a.h = h;
    arnoldi_dots_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(a);
    PB_LAUNCH_CHECK();
    arnoldi_project_dots_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(a);
    PB_LAUNCH_CHECK();
    arnoldi_project_norm_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(a);
    PB_LAUNCH_CHECK();
    if (fused) return;   // v_{j+1} is formed by the next step's prep_step, the loop control ran above
    scale_copy_next_kernel<<<div_up(n, 256), 256, 0, s>>>(w.p, scal.p + 1, V.p, ld, st.p, n);
    PB_LAUNCH_CHECK();
    arnoldi_control_kernel<<<1, 1, 0, s>>>(st.p, h, tol);
    PB_LAUNCH_CHECK();
}

void Gmres::read_cycle_async(cudaStream_t s) {
    PB_CUDA_TRY(cudaMemcpyAsync(hs.p + 2, &st.p->res_est, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
}

void Gmres::update_solution(int k, double *x, cudaStream_t s) {
    if (k <= 0) return;
    back_solve_kernel<<<1, kBackThreads, 0, s>>>(st.p, k);
    PB_LAUNCH_CHECK();
    update_x_kernel<<<div_up(n, 256), 256, 0, s>>>(V.p, ld, k, st.p, x, n);
    PB_LAUNCH_CHECK();
}

void block_jacobi_inverse(int64_t n, double cV_in, const double *sa_in, double cV_out, const double *sa_out,
                          double *minv, cudaStream_t s) {
    if (!n) return;
    bj_inverse_kernel<<<div_up(n, 256), 256, 0, s>>>(n, cV_in, sa_in, cV_out, sa_out, minv);
    PB_LAUNCH_CHECK();
}

void block_jacobi_apply(int64_t n, const double *minv, const double *u_in, const double *u_out, double *z_phi,
                        double *z_dphi, cudaStream_t s) {
    if (!n) return;
    bj_apply_kernel<<<div_up(n, 256), 256, 0, s>>>(n, minv, u_in, u_out, z_phi, z_dphi);
    PB_LAUNCH_CHECK();
}

void basis_combination(const Gmres &G, int k, double *out, cudaStream_t s) {
    back_solve_kernel<<<1, kBackThreads, 0, s>>>(G.st.p, k);
    PB_LAUNCH_CHECK();
    combination_kernel<<<div_up(G.n, 256), 256, 0, s>>>(G.V.p, G.ld, k, G.st.p, out, G.n);
    PB_LAUNCH_CHECK();
}

void axpby(double a, const double *x, double b, const double *y, double *out, int64_t n, cudaStream_t s) {
    if (!n) return;
    axpby_kernel<<<div_up(n, 256), 256, 0, s>>>(a, x, b, y, out, n);
    PB_LAUNCH_CHECK();
}

void weighted_sum(const double *q, const double *phi, int64_t n, double scale, double *out, cudaStream_t s) {
    weighted_sum_kernel<<<1, 1024, 0, s>>>(q, phi, n, scale, out);
    PB_LAUNCH_CHECK();
}

void coulomb_rows(const double *xyz, const double *q, int64_t n, double *rowv, cudaStream_t s) {
    if (!n) return;
    coulomb_rows_kernel<<<div_up(n, 128), 128, 0, s>>>(xyz, q, n, rowv);
    PB_LAUNCH_CHECK();
}

}  // namespace pb
