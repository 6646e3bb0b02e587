// Taylor expansions of radial kernels in radial form (FP32 M2P, forward and
// transposed treecode).  Included by treecode.cu and adjoint.cu; everything
// here has internal linkage.
#pragma once

#include "common.cuh"

namespace pb {
namespace {

// The kernels are radial, G = F(|u|), u = y_c - x, and the Taylor coefficient
// of order k is (1/k!) d^k F(u), with (one axis at a time, since d_i F_m = u_i F_{m+1})
//   d^k F(u) = sum_j prod_i k_i! / (2^j_i j_i! (k_i - 2 j_i)!) u^(k - 2j) F_{|k| - |j|}(|u|),
//   F_m = ((1/r) d/dr)^m F.
// Grouping the expansion sum_{|k| <= P} (1/k!) d^k F(u) M^k by (alpha = k - 2j, n = |k| - |j|):
//   sum_{alpha, n} u^alpha F_n(|u|) N_{alpha,n},
//   N_{alpha,n} = sum_{|j| = n - |alpha|, |alpha| + 2|j| <= P} prod_i 1 / (2^j_i j_i! alpha_i!) M^(alpha + 2j).
// N depends only on the box's moments, so it is formed once per box for M and
// for D and serves the Laplace and the Yukawa kernel alike; per (target, box)
// there remain the monomials u^alpha, the radial functions
//   Laplace F = 1/r:        F_{n+1} = -(2n + 1) F_n / r^2,
//   Yukawa  F = e^{-kr}/r:  F_1 = -(kr + 1) e^{-kr} / r^3,  F_{n+1} = (k^2 F_{n-1} - (2n + 1) F_n) / r^2
// (the second from r^2 F_{n+1} + (2n + 1) F_n - k^2 F_{n-1} = 0, which
// (1/r d/dr)^n of the Yukawa equation gives), and two dot products.
// The sum equals the Taylor sum exactly; only the rounding differs.
// graded term index (n = |k|, then k1 descending, then k2 descending), the moment layout
__host__ __device__ constexpr int graded_index(int k1, int k2, int k3) {
    return (k1 + k2 + k3) * (k1 + k2 + k3 + 1) * (k1 + k2 + k3 + 2) / 6 + (k2 + k3) * (k2 + k3 + 1) / 2 + k3;
}

__host__ __device__ constexpr int radial_terms(int P) {
    int n = 0;
    for (int a = 0; a <= P; ++a) n += ((P - a) / 2 + 1) * (a + 1) * (a + 2) / 2;
    return n;
}
// floats per node in the radial moment array (N^M, N^D interleaved), padded to 16 bytes
__host__ __device__ constexpr int radial_stride(int P) { return (2 * radial_terms(P) + 3) / 4 * 4; }

__host__ __device__ constexpr int radial_table_terms(int P) {
    int q = 0;
    for (int a = 0; a <= P; ++a)
        for (int m = 0; a + 2 * m <= P; ++m) q += (a + 1) * (a + 2) / 2 * (m + 1) * (m + 2) / 2;
    return q;
}

// The transform N = T M as a sparse table, built at compile time: for output
// r = (alpha, n) in the order alpha_1, alpha_2, alpha_3 ascending (nested),
// then n ascending, the terms start[r] .. start[r + 1] - 1 are
// (moment index of alpha + 2j, weight prod_i 1 / (2^j_i j_i! alpha_i!)).
template <int P>
struct RadialTable {
    int16_t start[radial_terms(P) + 1];
    int16_t k[radial_table_terms(P)];
    float w[radial_table_terms(P)];
};

__host__ __device__ constexpr double fact_d(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

template <int P>
constexpr RadialTable<P> make_radial_table() {
    RadialTable<P> t{};
    int r = 0, q = 0;
    for (int a1 = 0; a1 <= P; ++a1)
        for (int a2 = 0; a2 <= P - a1; ++a2)
            for (int a3 = 0; a3 <= P - a1 - a2; ++a3) {
                const int a = a1 + a2 + a3;
                for (int n = a; 2 * n <= a + P; ++n) {
                    const int m = n - a;
                    t.start[r++] = (int16_t)q;
                    for (int j1 = 0; j1 <= m; ++j1)
                        for (int j2 = 0; j2 <= m - j1; ++j2) {
                            const int j3 = m - j1 - j2;
                            t.k[q] = (int16_t)graded_index(a1 + 2 * j1, a2 + 2 * j2, a3 + 2 * j3);
                            t.w[q] = (float)(1.0 / ((double)(1 << m) * fact_d(j1) * fact_d(j2) * fact_d(j3) *
                                                    fact_d(a1) * fact_d(a2) * fact_d(a3)));
                            ++q;
                        }
                }
            }
    t.start[r] = (int16_t)q;
    return t;
}

template <int P>
__device__ const RadialTable<P> g_radial = make_radial_table<P>();

}  // namespace
}  // namespace pb
