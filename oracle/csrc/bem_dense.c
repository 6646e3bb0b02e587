/* Matrix-free dense FP64 collocation BEM block sums (oracle, test infrastructure only).
 *
 * For targets x_i and the panels j of one source surface, with kernel
 * G = exp(-kappa r) / (4 pi r) (kappa = 0: 1 / (4 pi r)) it accumulates
 *
 *   V_i = sum_j V_ij dphi_j,   K_i = sum_j K_ij phi_j,
 *   V_ij = A_j sum_k w_k G(x_i, y_jk),   K_ij = A_j sum_k w_k n_j . grad_y G(x_i, y_jk)
 *
 * (Sec. 2.2, Eqs. nBEM_disc and matel with the 1/4pi kept), using the K-point
 * rule, the K_fine-point rule when |x_i - c_j|^2 < (thres L_j)^2 (near-singular
 * region), and the precomputed semi-analytical V_ii with K_ii = 0 on the
 * target's own panel (self_idx[i] = j).  One OpenMP thread per target row.
 * Built with -ffp-contract=off; no blocking or reordering beyond the sums.
 */
#include <math.h>
#include <stdint.h>

static void pair_sums(const double *xi, const double *y, const double *wa, int nq,
                      const double *nrm, double kappa, double *v, double *k)
{
    const double inv4pi = 1.0 / (4.0 * M_PI);
    double sv = 0.0, sk = 0.0;
    for (int q = 0; q < nq; ++q) {
        double rx = xi[0] - y[3 * q + 0];
        double ry = xi[1] - y[3 * q + 1];
        double rz = xi[2] - y[3 * q + 2];
        double r2 = rx * rx + ry * ry + rz * rz;
        double r = sqrt(r2);
        double rn = rx * nrm[0] + ry * nrm[1] + rz * nrm[2];
        double e = kappa == 0.0 ? 1.0 : exp(-kappa * r);
        sv += wa[q] * e / r;
        sk += wa[q] * rn * (1.0 + kappa * r) * e / (r2 * r);
    }
    *v = sv * inv4pi;
    *k = sk * inv4pi;
}

void bem_dense_block_sums(int64_t m, const double *x, const int64_t *self_idx,
                          int64_t n, const double *cen, const double *nrm, const double *L,
                          int K, const double *y, const double *wa,
                          int Kf, const double *yf, const double *waf,
                          const double *selfV, double thres, double kappa,
                          const double *phi, const double *dphi,
                          double *Vout, double *Kout)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        const double *xi = x + 3 * i;
        double sv = 0.0, sk = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double v, k;
            if (self_idx && self_idx[i] == j) {
                v = selfV[j];
                k = 0.0;
            } else {
                double dx = xi[0] - cen[3 * j + 0];
                double dy = xi[1] - cen[3 * j + 1];
                double dz = xi[2] - cen[3 * j + 2];
                double d2 = (dx * dx + dy * dy) + dz * dz;
                double tl = thres * L[j];
                if (d2 < tl * tl)
                    pair_sums(xi, yf + 3 * Kf * j, waf + Kf * j, Kf, nrm + 3 * j, kappa, &v, &k);
                else
                    pair_sums(xi, y + 3 * K * j, wa + K * j, K, nrm + 3 * j, kappa, &v, &k);
            }
            sv += v * dphi[j];
            sk += k * phi[j];
        }
        Vout[i] = sv;
        Kout[i] = sk;
    }
}
