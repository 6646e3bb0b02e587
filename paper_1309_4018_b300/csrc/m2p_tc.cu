// M2P in radial form with the contraction on the tensor pipe (an evaluated
// variant of the FP32 M2P; pb_params.m2p_variant = 1).
//
// The radial-form far field of a (target, box) pair (Sec. 2.3, Eq. multexp,
// regrouped as in radial.cuh) is
//   V = sum_n F_n(|u|) S_n,   S_n = sum_alpha u^alpha N_{alpha,n},
// for the monopole (M) and dipole (D) moment sets.  Over the 32 targets of a
// work item that all use the same box, S is a dense product
//   S[32 x 2(P+1)] = U[32 x NA] . B[NA x 2(P+1)],
// U the targets' monomials u^alpha and B the box's N values (zero where
// n lies outside [|alpha|, (|alpha| + P)/2]).  Here the product runs as
// mma.sync m16n8k8 TF32 tensor instructions with every operand split in two
// TF32 parts (a = a_hi + a_lo, three products a_hi b_hi + a_hi b_lo + a_lo b_hi,
// FP32 accumulation), which keeps the FP32 path's accuracy; the monomials,
// the radial functions F_n and the two final dot products stay on the FP32
// pipe.  The dense form carries 4.5 times the multiply-adds of the sparse
// contraction (588 against 130 per moment set at P = 6) and the split
// another factor three.  Only for pairs of one Laplace and one Yukawa kernel
// and P <= 7; results differ from the FP32 path by rounding only.
#include "radial.cuh"
#include "treecode.cuh"

namespace pb {

namespace {

template <int P>
struct TcDims {
    static constexpr int NA = (P + 1) * (P + 2) * (P + 3) / 6;   // monomials
    static constexpr int KP = (NA + 7) / 8 * 8;                    // K padded to the instruction's 8
    static constexpr int KT = KP / 8;
    static constexpr int NC = 2 * (P + 1);                         // S_M[0..P], S_D[0..P]
    static constexpr int AS = KP + 4;                              // U row stride: conflict-free fragment loads
    static constexpr int BS = 24;                                  // B row stride: conflict-free fragment loads
    static constexpr int DS = 17;                                  // S row stride
    static constexpr int WARP_FLOATS = 32 * AS + 2 * KP * BS + 32 * DS;
};

// (alpha index k, order n) of every radial entry r, in the radial moment order
template <int P>
struct RadialKN {
    int16_t k[radial_terms(P)];
    int8_t n[radial_terms(P)];
};

template <int P>
constexpr RadialKN<P> make_radial_kn() {
    RadialKN<P> t{};
    int r = 0, k = 0;
    for (int a1 = 0; a1 <= P; ++a1)
        for (int a2 = 0; a2 <= P - a1; ++a2)
            for (int a3 = 0; a3 <= P - a1 - a2; ++a3, ++k) {
                const int a = a1 + a2 + a3;
                for (int n = a; 2 * n <= a + P; ++n, ++r) {
                    t.k[r] = (int16_t)k;
                    t.n[r] = (int8_t)n;
                }
            }
    return t;
}

template <int P>
__device__ const RadialKN<P> g_radial_kn = make_radial_kn<P>();

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t y;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = to_tf32(x);
    lo = to_tf32(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One warp per (box, up to 32 targets) item, two warps per block.
template <int P>
__global__ void __launch_bounds__(64) m2p_tc_kernel(int64_t nitems, M2PArgs32 g) {
    using D = TcDims<P>;
    extern __shared__ __align__(16) float tc_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = (int64_t)blockIdx.x * 2 + warp;
    if (item >= nitems) return;
    float *U = tc_smem + warp * D::WARP_FLOATS;              // [32][AS]
    uint32_t *Bh = reinterpret_cast<uint32_t *>(U + 32 * D::AS);   // [KP][BS]
    uint32_t *Bl = Bh + D::KP * D::BS;                             // [KP][BS]
    float *S = reinterpret_cast<float *>(Bl + D::KP * D::BS);      // [32][DS]
    const int4 it = g.items[item];
    const int b = it.x;
    // the box's B, split in TF32 parts
    for (int q = lane; q < D::KP * D::BS; q += 32) {
        Bh[q] = 0u;
        Bl[q] = 0u;
    }
    __syncwarp();
    const float2 *R = reinterpret_cast<const float2 *>(g.rmom + (int64_t)b * radial_stride(P));
    for (int r = lane; r < radial_terms(P); r += 32) {
        const float2 v = R[r];
        const int k = g_radial_kn<P>.k[r], n = g_radial_kn<P>.n[r];
        split_tf32(v.x, Bh[k * D::BS + n], Bl[k * D::BS + n]);
        split_tf32(v.y, Bh[k * D::BS + P + 1 + n], Bl[k * D::BS + P + 1 + n]);
    }
    // this lane's target and its monomials u^alpha, one row of U
    const int64_t slot = (int64_t)it.y + (lane < it.z ? lane : 0);
    const float4 c = g.cen32[b];
    const float4 x = g.x32[g.inv[slot]];
    const float ux = c.x - x.x, uy = c.y - x.y, uz = c.z - x.z;
    {
        float px[P + 1], py[P + 1], pz[P + 1];
        px[0] = py[0] = pz[0] = 1.f;
#pragma unroll
        for (int i = 1; i <= P; ++i) {
            px[i] = px[i - 1] * ux;
            py[i] = py[i - 1] * uy;
            pz[i] = pz[i - 1] * uz;
        }
        float *row = U + lane * D::AS;
        int k = 0;
#pragma unroll
        for (int a1 = 0; a1 <= P; ++a1)
#pragma unroll
            for (int a2 = 0; a2 <= P - a1; ++a2) {
                const float base = px[a1] * py[a2];
#pragma unroll
                for (int a3 = 0; a3 <= P - a1 - a2; ++a3) row[k++] = base * pz[a3];
            }
#pragma unroll
        for (int q = D::NA; q < D::KP; ++q) row[q] = 0.f;
    }
    __syncwarp();
    // S = U . B on the tensor pipe: two 16-row tiles x two 8-column tiles
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[mt][nt][e] = 0.f;
#pragma unroll 2
    for (int kt = 0; kt < D::KT; ++kt) {
        uint32_t bh[2][2], bl[2][2];
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            const int col = nt * 8 + gq;
            bh[nt][0] = Bh[(kt * 8 + tq) * D::BS + col];
            bh[nt][1] = Bh[(kt * 8 + tq + 4) * D::BS + col];
            bl[nt][0] = Bl[(kt * 8 + tq) * D::BS + col];
            bl[nt][1] = Bl[(kt * 8 + tq + 4) * D::BS + col];
        }
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const float *r0 = U + (mt * 16 + gq) * D::AS + kt * 8 + tq;
            const float *r1 = r0 + 8 * D::AS;
            uint32_t ah[4], al[4];
            split_tf32(r0[0], ah[0], al[0]);
            split_tf32(r1[0], ah[1], al[1]);
            split_tf32(r0[4], ah[2], al[2]);
            split_tf32(r1[4], ah[3], al[3]);
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                mma_tf32(acc[mt][nt], ah, bh[nt][0], bh[nt][1]);
                mma_tf32(acc[mt][nt], ah, bl[nt][0], bl[nt][1]);
                mma_tf32(acc[mt][nt], al, bh[nt][0], bh[nt][1]);
            }
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
            float *s0 = S + (mt * 16 + gq) * D::DS + nt * 8 + 2 * tq;
            float *s1 = s0 + 8 * D::DS;
            s0[0] = acc[mt][nt][0];
            s0[1] = acc[mt][nt][1];
            s1[0] = acc[mt][nt][2];
            s1[1] = acc[mt][nt][3];
        }
    __syncwarp();
    // radial functions and the two dot products, as in the FP32 path
    const float *srow = S + lane * D::DS;
    const float r2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    const float rinv = rsqrtf(r2), ir2 = rinv * rinv;
    float FL[P + 1], FY[P + 1];
    FL[0] = rinv;
#pragma unroll
    for (int n = 0; n < P; ++n) FL[n + 1] = (-(float)(2 * n + 1) * ir2) * FL[n];
    const float rho = r2 * rinv;
    const float e = __expf(-g.kappa * rho);
    FY[0] = e * rinv;
    if (P >= 1) FY[1] = -fmaf(g.kappa, rho, 1.f) * FY[0] * ir2;
    const float k2 = g.kappa * g.kappa;
#pragma unroll
    for (int n = 1; n < P; ++n) FY[n + 1] = fmaf(k2, FY[n - 1], -(float)(2 * n + 1) * FY[n]) * ir2;
    float VL = 0.f, KL = 0.f, VY = 0.f, KY = 0.f;
#pragma unroll
    for (int n = 0; n <= P; ++n) {
        const float sm = srow[n], sd = srow[P + 1 + n];
        VL = fmaf(FL[n], sm, VL);
        KL = fmaf(FL[n], sd, KL);
        VY = fmaf(FY[n], sm, VY);
        KY = fmaf(FY[n], sd, KY);
    }
    if (lane < it.z) g.part[g.ent[slot]] = make_float4(VL, KL, VY, KY);
}

template <int P>
size_t tc_smem_bytes() {
    return (size_t)2 * TcDims<P>::WARP_FLOATS * sizeof(float);
}

}  // namespace

void m2p_tc_prepare() {
#define PB_TCA(PP)                                                                                     \
    PB_CUDA_TRY(cudaFuncSetAttribute(m2p_tc_kernel<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)tc_smem_bytes<PP>()));
    PB_TCA(1) PB_TCA(2) PB_TCA(3) PB_TCA(4) PB_TCA(5) PB_TCA(6) PB_TCA(7)
#undef PB_TCA
}

bool m2p_tc_eligible(const Pair &Pr, int P, bool mixed) {
    return mixed && Pr.kappas.size() == 2 && Pr.kappas[0] == 0.0 && Pr.kappas[1] != 0.0 && P >= 1 && P <= 7;
}

void launch_m2p_tc(const M2PArgs32 &a, int64_t nitems, int P, cudaStream_t s) {
    if (!nitems) return;
    const unsigned grid = (unsigned)((nitems + 1) / 2);
    switch (P) {
#define PB_TCL(PP) \
    case PP: m2p_tc_kernel<PP><<<grid, 64, tc_smem_bytes<PP>(), s>>>(nitems, a); break;
        PB_TCL(1) PB_TCL(2) PB_TCL(3) PB_TCL(4) PB_TCL(5) PB_TCL(6) PB_TCL(7)
#undef PB_TCL
        default: fail(PB_EINVAL, "internal: tensor-pipe M2P needs 1 <= P <= 7");
    }
    PB_LAUNCH_CHECK();
}

}  // namespace pb
