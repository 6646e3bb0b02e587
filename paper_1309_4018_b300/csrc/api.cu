// C-ABI of the pbbem library (include/pbbem.h): problem assembly, setup,
// treecode operator application, device GMRES solve and energies.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "adjoint.cuh"
#include "geometry.cuh"
#include "gmres.cuh"
#include "model.cuh"
#include "validate.cuh"
#include "problem.cuh"
#include "surface.cuh"
#include "tree.cuh"
#include "treecode.cuh"

using namespace pb;

namespace pb {
std::atomic<long long> g_launches{0};
}

pb_problem::~pb_problem() {
    if (mv_exec) cudaGraphExecDestroy(mv_exec);
    if (adj_exec) cudaGraphExecDestroy(adj_exec);
    if (cyc_exec) cudaGraphExecDestroy(cyc_exec);
    if (adj_cyc_exec) cudaGraphExecDestroy(adj_cyc_exec);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (evf) cudaEventDestroy(evf);
    if (evj) cudaEventDestroy(evj);
    if (ev2a) cudaEventDestroy(ev2a);
    if (ev2b) cudaEventDestroy(ev2b);
    if (ev2c) cudaEventDestroy(ev2c);
    if (side) cudaStreamDestroy(side);
    if (lists2) cudaStreamDestroy(lists2);
}

namespace {

int fail_ctx(pb_ctx *c, const Error &e) {
    if (c) c->err = e.msg;
    return e.code;
}

template <typename F>
int guard(pb_ctx *c, F &&f) {
    try {
        f();
        if (c) c->err.clear();
        return PB_OK;
    } catch (const Error &e) {
        return fail_ctx(c, e);
    } catch (const std::bad_alloc &) {
        return fail_ctx(c, Error{PB_ENOMEM, "host allocation failed"});
    } catch (const std::exception &e) {
        return fail_ctx(c, Error{PB_EINVAL, e.what()});
    }
}

void set_device(pb_ctx *c) { PB_CUDA_TRY(cudaSetDevice(c->device)); }

Params resolve(const pb_params *p) {
    Params r;
    if (p) {
        if (p->K) r.K = p->K;
        if (p->K_fine) r.K_fine = p->K_fine;
        if (p->N_k) r.N_k = p->N_k;
        if (p->thres != 0.0) r.thres = p->thres;
        if (p->P) r.P = p->P;
        if (p->theta != 0.0) r.theta = p->theta;
        if (p->ncrit) r.ncrit = p->ncrit;
        if (p->gmres_tol != 0.0) r.tol = p->gmres_tol;
        if (p->restart) r.restart = p->restart;
        if (p->max_iter) r.max_iter = p->max_iter;
        r.precision = p->precision;
        r.precond = p->no_precond == 0;
        r.ncrit_adjoint = p->ncrit_adjoint;
        if (p->p2p_tile) r.p2p_tile = p->p2p_tile;
        r.m2p_variant = p->m2p_variant;
        if (p->precond_block) r.precond_block = p->precond_block;
    }
    if (!valid_rule(r.K)) fail(PB_EINVAL, "K must be 1, 3, 7 or 19");
    if (!valid_rule(r.K_fine)) fail(PB_EINVAL, "K_fine must be 1, 3, 7 or 19");
    if (r.N_k < 1 || r.N_k > 32) fail(PB_EINVAL, "N_k must be in 1..32");
    if (r.P < 0 || r.P > kMaxP) fail(PB_EINVAL, "P must be in 0..12");
    if (r.ncrit < 1) fail(PB_EINVAL, "ncrit must be >= 1");
    if (r.ncrit_adjoint < 0) fail(PB_EINVAL, "ncrit_adjoint must be >= 0");
    if (r.p2p_tile < 1 || r.p2p_tile > 64) fail(PB_EINVAL, "p2p_tile must be in 1..64");
    if (r.m2p_variant != 0 && r.m2p_variant != 1) fail(PB_EINVAL, "m2p_variant must be 0 or 1");
    if (r.precond_block < 1 || r.precond_block > 64) fail(PB_EINVAL, "precond_block must be in 1..64");
    if (r.restart < 1 || r.restart > 200) fail(PB_EINVAL, "restart must be in 1..200");
    if (r.max_iter < 1) fail(PB_EINVAL, "max_iter must be >= 1");
    if (!(r.tol > 0.0)) fail(PB_EINVAL, "gmres_tol must be > 0");
    if (!(r.thres >= 0.0)) fail(PB_EINVAL, "thres must be >= 0");
    if (!std::isfinite(r.theta)) fail(PB_EINVAL, "theta must be finite");
    if (r.precision != PB_FP64 && r.precision != PB_MIXED) fail(PB_EINVAL, "unknown precision");
    return r;
}

// Index of the (tgt, tree) pair in v, appending it if new; a pair of the
// previous setup with the same surfaces (in `old`) is reused with its buffers.
int find_pair(std::vector<Pair> &v, std::vector<Pair> &old, int tgt, int tree) {
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i].tgt == tgt && v[i].tree == tree) return (int)i;
    bool reused = false;
    for (auto &o : old)
        if (o.tgt == tgt && o.tree == tree) {
            v.push_back(std::move(o));
            o.tgt = -1;
            v.back().kappas.clear();
            reused = true;
            break;
        }
    if (!reused) v.emplace_back();
    v.back().tgt = tgt;
    v.back().tree = tree;
    return (int)v.size() - 1;
}

int kernel_slot(Pair &p, double kappa) {
    for (size_t i = 0; i < p.kappas.size(); ++i)
        if (p.kappas[i] == kappa) return (int)i;
    p.kappas.push_back(kappa);
    return (int)p.kappas.size() - 1;
}

void setup_problem(pb_problem *pb) {
    cudaStream_t s = pb->stream;
    const Params &prm = pb->prm;
    const int ns = (int)pb->sin.size();
    if (ns == 0) fail(PB_EINVAL, "no surface");
    for (const auto &si : pb->sin)
        if (si.inner < 0 || si.inner >= (int)pb->regions.size() || si.outer < 0 ||
            si.outer >= (int)pb->regions.size() || si.inner == si.outer)
            fail(PB_EINVAL, "surface references an unknown region");
    PB_CUDA_TRY(cudaEventRecord(pb->ev0, s));
    pb->adj.reset();
    if (pb->mv_exec) {
        cudaGraphExecDestroy(pb->mv_exec);
        pb->mv_exec = nullptr;
    }
    if (pb->adj_exec) {
        cudaGraphExecDestroy(pb->adj_exec);
        pb->adj_exec = nullptr;
    }
    for (cudaGraphExec_t *e : {&pb->cyc_exec, &pb->adj_cyc_exec})
        if (*e) {
            cudaGraphExecDestroy(*e);
            *e = nullptr;
        }
    // geometry, trees and pairs of a previous setup keep their device buffers
    if (pb->S.size() != (size_t)ns) {
        pb->S.clear(); pb->T.clear(); pb->G.clear();
        pb->S.resize(ns);
        pb->T.resize(ns);
    }
    std::vector<Pair> old_pairs = std::move(pb->pairs), old_cpairs = std::move(pb->cpairs);
    pb->pairs.clear();
    pb->cpairs.clear();
    pb->off.assign(ns + 1, 0);
    for (int t = 0; t < ns; ++t) {
        SurfDev &S = pb->S[t];
        const SurfIn &si = pb->sin[t];
        S.n = si.nt;
        S.nv = si.nv;
        S.inner = si.inner;
        S.outer = si.outer;
        S.off = pb->off[t];
        pb->off[t + 1] = pb->off[t] + S.n;
        S.verts.alloc(3 * S.nv);
        S.tris.alloc(3 * S.n);
        PB_CUDA_TRY(cudaMemcpyAsync(S.verts.p, si.v.p, 3 * S.nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
        PB_CUDA_TRY(cudaMemcpyAsync(S.tris.p, si.t.p, 3 * S.n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        surface_geometry(S, prm.K, s);
    }
    pb->N = pb->off[ns];
    pb->G.resize(ns + 1);
    // the target sorts run on the second list stream beside the trees
    cudaStream_t s2 = pb->lists2 ? pb->lists2 : s;
    if (s2 != s) {
        PB_CUDA_TRY(cudaEventRecord(pb->ev2a, s));
        PB_CUDA_TRY(cudaStreamWaitEvent(s2, pb->ev2a, 0));
    }
    for (int t = 0; t < ns; ++t) build_targets(pb->G[t], pb->S[t].cen.p, pb->S[t].n, t, s2);
    const int64_t nc = pb->nc;
    build_targets(pb->G[ns], pb->cxyz_d.p, nc, -1, s2);
    if (s2 != s) PB_CUDA_TRY(cudaEventRecord(pb->ev2c, s2));
    for (int t = 0; t < ns; ++t) build_tree(pb->T[t], pb->S[t], prm.K, prm.ncrit, s);
    // the charges must lie in their region: inside every surface that has it as
    // inner region, outside every surface that has it as outer region
    int n_wind = 0;
    // the near-field values, self integrals and right-hand side go to the side
    // stream as soon as their inputs exist, beside the next pair's list build
    // (latency-bound: small kernels and host reads); joined before the
    // preconditioner
    cudaStream_t fs = pb->side ? pb->side : s;
    if (nc > 0) {
        std::vector<int32_t> expect;
        std::vector<int> wsurf;
        for (int t = 0; t < ns; ++t)
            if (pb->S[t].inner == pb->cregion || pb->S[t].outer == pb->cregion) {
                wsurf.push_back(t);
                expect.push_back(pb->S[t].inner == pb->cregion ? 1 : 0);
            }
        n_wind = (int)wsurf.size();
        if (n_wind > 8) fail(PB_EINVAL, "the charged region is bounded by more than 8 surfaces");
        if (n_wind > 0) {
            // on the side stream, beside the latency-bound list construction below
            cudaStream_t ws = pb->side ? pb->side : s;
            if (ws != s) {
                PB_CUDA_TRY(cudaEventRecord(pb->evf, s));
                PB_CUDA_TRY(cudaStreamWaitEvent(ws, pb->evf, 0));
            }
            pb->wind.alloc(n_wind * nc);
            pb->wind.zero(ws);
            for (int k = 0; k < n_wind; ++k)
                winding_numbers(pb->S[wsurf[k]].verts.p, pb->S[wsurf[k]].tris.p, pb->S[wsurf[k]].n, pb->cxyz_d.p,
                                nc, pb->wind.p + k * nc, ws);
            pb->wind_bad.alloc(3);
            pb->wind_bad_h.alloc(3);
            winding_mismatch(pb->wind.p, nc, n_wind, expect.data(), pb->wind_bad.p, ws);
            PB_CUDA_TRY(cudaMemcpyAsync(pb->wind_bad_h.p, pb->wind_bad.p, 3 * sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, ws));
        }
    }
    // block structure (multi-surface rule): row (s, R) gets sigma (K - c V) of every t in dR
    pb->rows.assign(2 * ns, {});
    auto eps = [&](int R) { return pb->regions[R].eps; };
    for (int sf = 0; sf < ns; ++sf) {
        const int Rs[2] = {pb->S[sf].inner, pb->S[sf].outer};
        for (int side = 0; side < 2; ++side) {
            const int R = Rs[side];
            for (int t = 0; t < ns; ++t) {
                const bool in = pb->S[t].inner == R, out = pb->S[t].outer == R;
                if (!in && !out) continue;
                const double sigma = in ? 1.0 : -1.0;
                const double cc = in ? 1.0 : eps(pb->S[t].inner) / eps(R);
                const int pi = find_pair(pb->pairs, old_pairs, sf, t);
                const int ki = kernel_slot(pb->pairs[pi], pb->regions[R].kappa);
                pb->rows[2 * sf + side].push_back(Term{pi, ki, sigma, -sigma * cc, R});
            }
            if (pb->rows[2 * sf + side].size() > 8) fail(PB_EINVAL, "a region is bounded by more than 8 surfaces");
        }
    }
    pb->reac.clear();
    if (nc > 0) {
        const int Rc = pb->cregion;
        for (int t = 0; t < ns; ++t) {
            const bool in = pb->S[t].inner == Rc, out = pb->S[t].outer == Rc;
            if (!in && !out) continue;
            const double sigma = in ? 1.0 : -1.0;
            const double cc = in ? 1.0 : eps(pb->S[t].inner) / eps(Rc);
            const int pi = find_pair(pb->cpairs, old_cpairs, ns, t);
            const int ki = kernel_slot(pb->cpairs[pi], pb->regions[Rc].kappa);
            pb->reac.push_back(Term{pi, ki, -sigma, sigma * cc, Rc});
        }
        if (pb->reac.size() > 8) fail(PB_EINVAL, "the charged region is bounded by more than 8 surfaces");
    }
    pb->need_far.assign(ns, false);
    const bool mixed = prm.precision == PB_MIXED;
    // the side stream starts on what needs only the geometry and trees: the
    // self integrals and the right-hand side, beside the list builds
    if (fs != s) {
        PB_CUDA_TRY(cudaEventRecord(pb->evf, s));
        PB_CUDA_TRY(cudaStreamWaitEvent(fs, pb->evf, 0));
    }
    auto self_terms = [&](Pair &P) {
        const SurfDev &src = pb->S[P.tree];
        const size_t nk = P.kappas.size();
        P.VK.resize(nk); P.dV.resize(nk); P.dK.resize(nk); P.selfV.resize(nk); P.selfV32.resize(nk);
        // the FP32 direct sum keeps a panel's own points when none sits at its centroid (K = 3);
        // the self value then carries the correction
        P.p2p_self_in = mixed && P.tgt == P.tree && prm.K == 3;
        if (P.tgt != P.tree) return;
        for (size_t k = 0; k < nk; ++k) {
            P.selfV[k].alloc(src.n);
            if (nk == 2 && k == 1) {
                self_integrals2(src, prm.N_k, P.kappas[0], P.kappas[1], P.selfV[0].p, P.selfV[1].p, fs);
            } else if (nk == 1) {
                self_integrals(src, prm.N_k, P.kappas[k], P.selfV[k].p, fs);
            }
        }
        if (P.p2p_self_in)
            for (size_t k = 0; k < nk; ++k) {
                P.selfV32[k].alloc(src.n);
                self_minus_kpoint(src, prm.K, P.kappas[k], P.selfV[k].p, P.selfV32[k].p, fs);
            }
    };
    for (auto &P : pb->pairs) self_terms(P);
    for (auto &P : pb->cpairs) {
        const size_t nk = P.kappas.size();
        P.VK.resize(nk); P.dV.resize(nk); P.dK.resize(nk); P.selfV.resize(nk); P.selfV32.resize(nk);
        P.p2p_self_in = false;
    }
    // right-hand side
    pb->b.alloc(2 * pb->N);
    pb->b.zero(fs);
    if (nc > 0) {
        const Region &Rg = pb->regions[pb->cregion];
        for (int sf = 0; sf < ns; ++sf) {
            const int Rs[2] = {pb->S[sf].inner, pb->S[sf].outer};
            for (int side = 0; side < 2; ++side)
                if (Rs[side] == pb->cregion)
                    rhs_rows(pb->S[sf], nc, pb->cq_d.p, pb->cxyz_d.p, Rg.kappa, Rg.eps,
                             pb->b.p + 2 * pb->off[sf] + side * pb->S[sf].n, mixed ? pb->T[sf].origin : nullptr, fs);
        }
    }
    // cluster block preconditioner, on the side stream after the self values and the target sorts
    pb->use_cluster = prm.precond && prm.precond_block > 1;
    if (pb->use_cluster) {
        pb->csurf.assign(ns, ClusterSurface{});
        int64_t nblk = 0;
        for (int sf = 0; sf < ns; ++sf) {
            ClusterSurface &cs = pb->csurf[sf];
            cs.n = pb->S[sf].n;
            cs.off = pb->off[sf];
            cs.order = pb->G[sf].order.p;
            cs.cb = prm.precond_block;
            cs.first = nblk;
            nblk += cs.nblocks();
        }
        const int nb2 = cluster_block_dim(prm.precond_block);
        pb->cinv.alloc((size_t)std::max<int64_t>(1, nblk) * nb2 * nb2);
        pb->cerr.alloc(1);
        pb->cerr.zero(fs);
        pb->cerr_h.alloc(1);
        if (s2 != fs) PB_CUDA_TRY(cudaStreamWaitEvent(fs, pb->ev2c, 0));
        for (int sf = 0; sf < ns; ++sf) {
            ClusterRows cr{};
            for (int side = 0; side < 2; ++side)
                for (const Term &tm : pb->rows[2 * sf + side]) {
                    const Pair &P = pb->pairs[tm.pair];
                    if (P.tree != sf || P.tgt != sf) continue;
                    cr.cK[side] = tm.cK;
                    cr.cV[side] = tm.cV;
                    cr.kappa[side] = P.kappas[tm.kidx];
                    cr.selfV[side] = P.selfV[tm.kidx].p;
                }
            const SurfDev &S = pb->S[sf];
            cluster_blocks(pb->csurf[sf], ClusterGeom{S.cen.p, S.nrm.p, S.gy.p, S.gwa.p, prm.K}, cr, pb->cinv.p,
                           pb->cerr.p, fs);
        }
        PB_CUDA_TRY(cudaMemcpyAsync(pb->cerr_h.p, pb->cerr.p, sizeof(int32_t), cudaMemcpyDeviceToHost, fs));
    }
    // the list builds, pairs alternating between the two list streams (both see the trees and the targets)
    if (s2 != s) {
        PB_CUDA_TRY(cudaEventRecord(pb->ev2a, s));
        PB_CUDA_TRY(cudaStreamWaitEvent(s2, pb->ev2a, 0));
        PB_CUDA_TRY(cudaEventRecord(pb->ev2b, s2));
        PB_CUDA_TRY(cudaStreamWaitEvent(s, pb->ev2b, 0));
    }
    {
        std::vector<ListJob> jobs;
        int k = 0;
        for (auto &P : pb->pairs) {
            const bool odd = k++ % 2;
            jobs.push_back(ListJob{&P, &pb->G[P.tgt], &pb->T[P.tree], &pb->S[P.tree], P.tgt == P.tree, odd ? s2 : s,
                                   odd ? s : s2});
        }
        for (auto &P : pb->cpairs) {
            const bool odd = k++ % 2;
            jobs.push_back(ListJob{&P, &pb->G[P.tgt], &pb->T[P.tree], &pb->S[P.tree], false, odd ? s2 : s,
                                   odd ? s : s2});
        }
        build_lists_multi(jobs, prm);
    }
    if (s2 != s) {
        PB_CUDA_TRY(cudaEventRecord(pb->ev2b, s2));
        PB_CUDA_TRY(cudaStreamWaitEvent(s, pb->ev2b, 0));
    }
    // near-field values on the side stream once the lists exist
    if (fs != s) {
        PB_CUDA_TRY(cudaEventRecord(pb->evf, s));
        PB_CUDA_TRY(cudaStreamWaitEvent(fs, pb->evf, 0));
    }
    auto near_field = [&](Pair &P) {
        const Targets &G = pb->G[P.tgt];
        const SurfDev &src = pb->S[P.tree];
        if (P.n_m2p > 0) pb->need_far[P.tree] = true;
        const size_t nk = P.kappas.size();
        if (mixed) P.p2p_part32.alloc(2 * nk * std::max<int64_t>(1, P.n_p2p));
        else P.p2p_part.alloc(2 * nk * std::max<int64_t>(1, P.n_p2p));
        if (P.n_m2p > 0) {
            if (mixed) P.m2p_part32.alloc(2 * nk * P.n_m2p);
            else P.m2p_part64.alloc(2 * nk * P.n_m2p);
        }
        if (mixed) {
            P.dV32.alloc(std::max<int64_t>(1, (int64_t)nk * P.n_near));
            P.dK32.alloc(std::max<int64_t>(1, (int64_t)nk * P.n_near));
            near_values32(P, G, src, prm.K, prm.K_fine, P.dV32.p, P.dK32.p, fs);
        }
        for (size_t k = 0; k < nk; ++k) {
            P.VK[k].alloc(2 * std::max<int64_t>(1, G.n));
            if (!mixed) {
                P.dV[k].alloc(std::max<int64_t>(1, P.n_near));
                P.dK[k].alloc(std::max<int64_t>(1, P.n_near));
                near_values(P, G, src, prm.K, prm.K_fine, P.kappas[k], P.dV[k].p, P.dK[k].p, fs);
            }
        }
    };
    for (auto &P : pb->pairs) near_field(P);
    for (auto &P : pb->cpairs) near_field(P);
    if (mixed) {
        for (auto &P : pb->pairs) targets_to_float(P, pb->G[P.tgt], pb->T[P.tree], s);
        for (auto &P : pb->cpairs) targets_to_float(P, pb->G[P.tgt], pb->T[P.tree], s);
    }
    if (fs != s) {
        PB_CUDA_TRY(cudaEventRecord(pb->evj, fs));
        PB_CUDA_TRY(cudaStreamWaitEvent(s, pb->evj, 0));
    }
    pb->x.alloc(2 * pb->N);
    pb->x.zero(s);
    pb->y.alloc(2 * pb->N);
    pb->r.alloc(2 * pb->N);
    pb->phi_reac.alloc(std::max<int64_t>(1, nc));
    pb->energy.alloc(1);
    pb->gm.init(2 * pb->N, prm.restart, s);
    // block-Jacobi right preconditioner from every panel's 2x2 self block
    pb->z1.alloc(2 * pb->N);
    pb->z2.alloc(2 * pb->N);
    pb->minv.alloc(4 * pb->N);
    for (int sf = 0; sf < ns; ++sf) {
        const double *sa[2] = {nullptr, nullptr};
        double cv[2] = {0.0, 0.0};
        for (int side = 0; side < 2; ++side)
            for (const Term &tm : pb->rows[2 * sf + side]) {
                const Pair &P = pb->pairs[tm.pair];
                if (P.tree == sf) { sa[side] = P.selfV[tm.kidx].p; cv[side] = tm.cV; }
            }
        if (!sa[0] || !sa[1]) fail(PB_EINVAL, "internal: missing self block");
        block_jacobi_inverse(pb->S[sf].n, cv[0], sa[0], cv[1], sa[1], pb->minv.p + 4 * pb->off[sf], s);
    }
    // moments for every tree with a far field, and the FP32 densities, so that no
    // operator application allocates (it may be captured into a CUDA graph)
    for (int t = 0; t < ns; ++t) {
        if (prm.precision == PB_MIXED) pb->T[t].phf.alloc(pb->S[t].n);
        pb->T[t].ucnt.alloc(pb->T[t].nnodes);
        pb->T[t].ucnt.zero(s);
    }
    for (int t = 0; t < ns; ++t)
        if (pb->need_far[t]) {
            const size_t nm = (size_t)pb->T[t].nnodes * 2 * nterms(prm.P);
            if (prm.precision == PB_MIXED) pb->T[t].mom32.alloc(nm); else pb->T[t].mom64.alloc(nm);
            if (prm.precision == PB_MIXED && prm.P <= kRadialMaxP)
                pb->T[t].rmom32.alloc((size_t)pb->T[t].nnodes * radial_floats(prm.P));
        }
    PB_CUDA_TRY(cudaEventRecord(pb->ev1, s));
    PB_CUDA_TRY(cudaEventSynchronize(pb->ev1));
    // a run whose block had a vanishing pivot: the 2 x 2 self blocks instead
    if (pb->use_cluster && *pb->cerr_h.p) pb->use_cluster = false;
    if (n_wind > 0 && pb->wind_bad_h.p[0] > 0) {
        const int32_t *bad = pb->wind_bad_h.p;
        fail(PB_EINVAL, std::to_string(bad[0]) + " charge(s) lie outside their region (first: charge " +
                            std::to_string(bad[1]) + ", against surface " +
                            std::to_string(bad[2] < n_wind ? bad[2] : -1) + " of the region's boundary)");
    }
    float ms = 0.f;
    PB_CUDA_TRY(cudaEventElapsedTime(&ms, pb->ev0, pb->ev1));
    pb->setup_ms = ms;
    pb->is_setup = true;
    pb->have_solution = false;
}

}  // namespace

namespace pb {

namespace {

void strengths_all(pb_problem *pb, const double *xd, cudaStream_t s) {
    const bool mixed = pb->prm.precision == PB_MIXED;
    for (size_t t = 0; t < pb->S.size(); ++t) {
        const double *phi = xd + 2 * pb->off[t];
        const double *dphi = phi + pb->S[t].n;
        compute_strengths(pb->T[t], pb->S[t], phi, dphi, mixed, s);
    }
}

void upward_all(pb_problem *pb, cudaStream_t s) {
    const bool mixed = pb->prm.precision == PB_MIXED;
    for (size_t t = 0; t < pb->S.size(); ++t)
        if (pb->need_far[t]) upward_pass(pb->T[t], pb->prm.P, mixed, s);
}

}  // namespace

// y = A x, both device pointers of 2N doubles; optional event marks between the phases.
void apply_operator(pb_problem *pb, const double *xd, double *yd, PhaseEvents *ph) {
    cudaStream_t s = pb->stream;
    const Params &prm = pb->prm;
    const bool mixed = prm.precision == PB_MIXED;
    const int ns = (int)pb->S.size();
    auto mark = [&](int k) {
        if (ph) PB_CUDA_TRY(cudaEventRecord(ph->ev[k], s));
    };
    mark(0);
    // Without phase marks the direct sums (which need only the source
    // strengths) run on the side stream while the upward pass and the
    // expansions run here; the gather waits for both.
    const bool fork = !ph && pb->side;
    strengths_all(pb, xd, s);
    if (fork) PB_CUDA_TRY(cudaEventRecord(pb->evf, s));
    // the upward pass is enqueued first: its blocks (one per leaf) start before the direct sums fill the GPU
    upward_all(pb, s);
    if (fork) {
        PB_CUDA_TRY(cudaStreamWaitEvent(pb->side, pb->evf, 0));
        for (auto &P : pb->pairs) launch_p2p(P, pb->G[P.tgt], pb->T[P.tree], P.tgt == P.tree, mixed, pb->side);
        PB_CUDA_TRY(cudaEventRecord(pb->evj, pb->side));
    }
    mark(1);
    if (!fork)
        for (auto &P : pb->pairs) launch_p2p(P, pb->G[P.tgt], pb->T[P.tree], P.tgt == P.tree, mixed, s);
    mark(2);
    for (auto &P : pb->pairs) launch_m2p(P, pb->G[P.tgt], pb->T[P.tree], prm.P, mixed, s, prm.m2p_variant);
    if (fork) PB_CUDA_TRY(cudaStreamWaitEvent(s, pb->evj, 0));
    mark(3);
    for (auto &P : pb->pairs) {
        const double *phi = xd + 2 * pb->off[P.tree];
        launch_gather(P, pb->G[P.tgt], mixed, P.tgt == P.tree, phi, phi + pb->S[P.tree].n, pb->T[P.tree].phf.p, s);
    }
    mark(4);
    operator_post(pb, xd, yd, s);
    mark(5);
}

void operator_pre(pb_problem *pb, const double *xd, cudaStream_t s) {
    strengths_all(pb, xd, s);
    upward_all(pb, s);
}

void operator_post(pb_problem *pb, const double *xd, double *yd, cudaStream_t s) {
    const int ns = (int)pb->S.size();
    for (int sf = 0; sf < ns; ++sf) {
        CombineRow row[2]{};
        for (int side = 0; side < 2; ++side) {
            const auto &terms = pb->rows[2 * sf + side];
            row[side].nterm = (int)terms.size();
            for (int k = 0; k < row[side].nterm; ++k) {
                const Pair &P = pb->pairs[terms[k].pair];
                row[side].term[k] = CombineTerm{P.VK[terms[k].kidx].p, pb->G[P.tgt].n, terms[k].cK, terms[k].cV};
            }
        }
        // both rows of the surface (the two sides of its panels) in one launch
        launch_combine_pair(pb->S[sf].n, pb->G[sf].rank.p, xd + 2 * pb->off[sf], 0.5, row[0], row[1],
                            yd + 2 * pb->off[sf], s);
    }
}

// phi_reac at the charges (input order) for the unknowns x (device); then
// energy = 1/2 C sum_k q_k 4 pi phi_reac (device scalar).
void reaction(pb_problem *pb, const double *xd) {
    cudaStream_t s = pb->stream;
    const Params &prm = pb->prm;
    const bool mixed = prm.precision == PB_MIXED;
    const int ns = (int)pb->S.size();
    const int64_t nc = pb->nc;
    if (nc == 0) {
        pb->energy.zero(s);
        return;
    }
    for (int t = 0; t < ns; ++t) {
        bool used = false;
        for (auto &P : pb->cpairs) used = used || P.tree == t;
        if (!used) continue;
        const double *phi = xd + 2 * pb->off[t];
        compute_strengths(pb->T[t], pb->S[t], phi, phi + pb->S[t].n, mixed, s);
        if (pb->need_far[t]) upward_pass(pb->T[t], prm.P, mixed, s);
    }
    for (auto &P : pb->cpairs) {
        const Targets &G = pb->G[P.tgt];
        const Tree &Tr = pb->T[P.tree];
        const double *phi = xd + 2 * pb->off[P.tree];
        launch_p2p(P, G, Tr, false, mixed, s);
        launch_m2p(P, G, Tr, prm.P, mixed, s, prm.m2p_variant);
        launch_gather(P, G, mixed, false, phi, phi + pb->S[P.tree].n, pb->T[P.tree].phf.p, s);
    }
    CombineRow row{};
    row.nterm = (int)pb->reac.size();
    for (int k = 0; k < row.nterm; ++k) {
        const Pair &P = pb->cpairs[pb->reac[k].pair];
        row.term[k] = CombineTerm{P.VK[pb->reac[k].kidx].p, nc, pb->reac[k].cK, pb->reac[k].cV};
    }
    launch_combine(nc, pb->G[ns].rank.p, nullptr, 0.0, row, pb->phi_reac.p, s);
    weighted_sum(pb->cq_d.p, pb->phi_reac.p, nc, 0.5 * kKjPerMol * 4.0 * kPi, pb->energy.p, s);
}

// z = M^-1 u (block-Jacobi), both 2N device vectors.
void apply_precond(pb_problem *pb, const double *u, double *z) {
    cudaStream_t s = pb->stream;
    if (pb->use_cluster) {
        cluster_apply(pb->csurf, pb->cinv.p, u, z, s);
        return;
    }
    for (size_t sf = 0; sf < pb->S.size(); ++sf) {
        const int64_t n = pb->S[sf].n, o = 2 * pb->off[sf];
        block_jacobi_apply(n, pb->minv.p + 4 * pb->off[sf], u + o, u + o + n, z + o, z + o + n, s);
    }
}

void launch_captured(pb_problem *pb, cudaGraphExec_t &exec, long long &nk, const std::function<void()> &body,
                     cudaStream_t s) {
    if (!exec) {
        cudaStream_t cs = pb->stream;
        const long long k0 = g_launches.load();
        PB_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t graph = nullptr;
        try {
            body();
        } catch (...) {
            cudaStreamEndCapture(cs, &graph);
            if (graph) cudaGraphDestroy(graph);
            throw;
        }
        PB_CUDA_TRY(cudaStreamEndCapture(cs, &graph));
        const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        PB_CUDA_TRY(e);
        nk = g_launches.load() - k0;
        g_launches.fetch_sub(nk);   // captured, not executed
    }
    PB_CUDA_TRY(cudaGraphLaunch(exec, s));
    g_launches.fetch_add(nk);
}

void launch_operator_graph(pb_problem *pb, cudaStream_t s) {
    launch_captured(pb, pb->mv_exec, pb->mv_kernels, [pb] { apply_operator(pb, pb->z1.p, pb->gm.w.p); }, s);
}

namespace {

void sync_streams(const std::vector<KrylovJob *> &jobs, bool only_active) {
    std::vector<cudaStream_t> done;
    for (const KrylovJob *jb : jobs) {
        if (only_active && jb->act == 0) continue;
        cudaStream_t s = jb->pb->stream;
        if (std::find(done.begin(), done.end(), s) != done.end()) continue;
        done.push_back(s);
        PB_CUDA_TRY(cudaStreamSynchronize(s));
    }
}

}  // namespace

// One GMRES cycle's Arnoldi loop as a graph: a WHILE node whose body takes
// v_j (column j in the device state), applies the preconditioner and the
// operator, runs the Arnoldi step and lets the control kernel end the loop.
void build_cycle_graph(KrylovJob *jb) {
    pb_problem *pb = jb->pb;
    cudaStream_t cs = pb->stream;
    Gmres &gm = pb->gm;
    cudaGraph_t g = nullptr;
    PB_CUDA_TRY(cudaGraphCreate(&g, 0));
    struct GraphGuard {
        cudaGraph_t &g;
        ~GraphGuard() { if (g) cudaGraphDestroy(g); }
    } guard{g};
    cudaGraphConditionalHandle h;
    PB_CUDA_TRY(cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    PB_CUDA_TRY(cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    const long long k0 = g_launches.load();
    PB_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    try {
        if (jb->prep) {
            jb->prep(cs);
        } else if (jb->precond) {
            gm.copy_basis(pb->z2.p, cs);
            jb->precond(pb->z2.p, pb->z1.p);
        } else {
            gm.copy_basis(pb->z1.p, cs);
        }
        jb->cycle_op();
        gm.arnoldi_step_dev(h, pb->prm.tol, cs, (bool)jb->prep);
    } catch (...) {
        cudaStreamEndCapture(cs, &body);
        throw;
    }
    PB_CUDA_TRY(cudaStreamEndCapture(cs, &body));
    *jb->cycle_kernels = g_launches.load() - k0;
    g_launches.fetch_sub(*jb->cycle_kernels);   // captured, counted per executed step
    PB_CUDA_TRY(cudaGraphInstantiate(jb->cycle_exec, g, 0));
}

void run_krylov(std::vector<KrylovJob *> &jobs, BatchPlan *plan) {
    for (KrylovJob *jb : jobs) {
        pb_problem *pb = jb->pb;
        jb->st = KrylovStats{};
        jb->act = 0;
        if (jb->x_zero) PB_CUDA_TRY(cudaMemsetAsync(jb->x, 0, 2 * pb->N * sizeof(double), pb->stream));
        pb->gm.norm2_async(jb->b, pb->stream);
    }
    sync_streams(jobs, false);
    for (KrylovJob *jb : jobs) {
        pb_problem *pb = jb->pb;
        jb->bnorm = std::sqrt(pb->gm.host(0));
        if (jb->bnorm == 0.0) {
            PB_CUDA_TRY(cudaMemsetAsync(jb->x, 0, 2 * pb->N * sizeof(double), pb->stream));
            jb->phase = 3;
        } else {
            pb->gm.set_bnorm(jb->bnorm, pb->stream);
            jb->phase = 1;
        }
    }
    while (true) {
        bool any = false;
        for (KrylovJob *jb : jobs) {
            pb_problem *pb = jb->pb;
            cudaStream_t s = pb->stream;
            Gmres &gm = pb->gm;
            const int64_t n2 = 2 * pb->N;
            jb->act = 0;
            if (jb->phase == 1) {
                if (jb->x_zero) {
                    PB_CUDA_TRY(cudaMemcpyAsync(pb->r.p, jb->b, n2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
                } else {
                    jb->op(jb->x, pb->y.p);
                    ++jb->st.matvecs;
                    axpby(1.0, jb->b, -1.0, pb->y.p, pb->r.p, n2, s);
                }
                jb->x_zero = false;
                gm.start_cycle(pb->r.p, s);
                jb->act = 1;
            } else if (jb->phase == 2 && plan) {
                // the step's operator input, then the ends of the operator that stay per problem
                if (jb->precond) jb->precond(gm.basis(jb->j), pb->z1.p);
                else PB_CUDA_TRY(cudaMemcpyAsync(pb->z1.p, gm.basis(jb->j), n2 * sizeof(double),
                                                 cudaMemcpyDeviceToDevice, s));
                operator_pre(pb, pb->z1.p, s);
                PB_CUDA_TRY(cudaEventRecord(pb->evf, s));
                jb->act = 2;
            } else if (jb->phase == 2 && jb->cycle_exec) {
                gm.set_cycle(pb->prm.max_iter - jb->st.iters, s);
                if (!*jb->cycle_exec) build_cycle_graph(jb);
                PB_CUDA_TRY(cudaGraphLaunch(*jb->cycle_exec, s));
                gm.read_cycle_async(s);
                jb->act = 3;
            } else if (jb->phase == 2) {
                if (jb->graph) {
                    if (jb->precond) jb->precond(gm.basis(jb->j), pb->z1.p);
                    else PB_CUDA_TRY(cudaMemcpyAsync(pb->z1.p, gm.basis(jb->j), n2 * sizeof(double),
                                                     cudaMemcpyDeviceToDevice, s));
                    jb->graph(s);
                } else if (jb->precond) {
                    jb->precond(gm.basis(jb->j), pb->z1.p);
                    jb->op(pb->z1.p, gm.w.p);
                } else {
                    jb->op(gm.basis(jb->j), gm.w.p);
                }
                ++jb->st.matvecs;
                gm.arnoldi_step(jb->j, s);
                jb->act = 2;
            }
            any = any || jb->act != 0;
        }
        if (plan && any) {
            // one persistent launch for the direct sums, far field and gathers of every
            // problem taking an Arnoldi step, then each problem's combine and step
            cudaStream_t bs = jobs[0]->pb->ctx->stream;
            bool stepping = false;
            for (size_t i = 0; i < jobs.size(); ++i) {
                const bool on = jobs[i]->act == 2;
                plan->active_h.p[i] = on ? 1 : 0;
                if (on) {
                    PB_CUDA_TRY(cudaStreamWaitEvent(bs, jobs[i]->pb->evf, 0));
                    stepping = true;
                }
            }
            if (stepping) {
                batch_operator_launch(*plan, bs);
                PB_CUDA_TRY(cudaEventRecord(plan->ev, bs));
                for (KrylovJob *jb : jobs) {
                    if (jb->act != 2) continue;
                    pb_problem *pb = jb->pb;
                    PB_CUDA_TRY(cudaStreamWaitEvent(pb->stream, plan->ev, 0));
                    operator_post(pb, pb->z1.p, pb->gm.w.p, pb->stream);
                    ++jb->st.matvecs;
                    pb->gm.arnoldi_step(jb->j, pb->stream);
                }
            }
        }
        if (!any) break;
        sync_streams(jobs, true);
        if (plan && plan->status_h.p[0] != PB_OK) {
            PB_CUDA_TRY(cudaStreamSynchronize(jobs[0]->pb->ctx->stream));
            fail(PB_ETIMEOUT, "batched operator: a gather's bounded wait for its pair's direct and far-field "
                              "sums ran out");
        }
        for (KrylovJob *jb : jobs) {
            pb_problem *pb = jb->pb;
            const Params &prm = pb->prm;
            cudaStream_t s = pb->stream;
            Gmres &gm = pb->gm;
            if (jb->act == 1) {
                jb->st.rel = std::sqrt(gm.host(1)) / jb->bnorm;
                if (!(jb->st.rel >= prm.tol) || jb->st.iters >= prm.max_iter) {
                    jb->phase = 3;
                } else {
                    jb->phase = 2;
                    jb->j = 0;
                }
            } else if (jb->act == 3) {
                // the device ran the cycle's steps; the solution update follows
                const int steps = (int)gm.host(3);
                jb->st.iters += steps;
                jb->st.matvecs += steps;
                g_launches.fetch_add(*jb->cycle_kernels * steps);
                if (steps > 0) {
                    if (jb->precond) {
                        basis_combination(gm, steps, pb->z1.p, s);
                        jb->precond(pb->z1.p, pb->z2.p);
                        axpby(1.0, jb->x, 1.0, pb->z2.p, jb->x, 2 * pb->N, s);
                    } else {
                        gm.update_solution(steps, jb->x, s);
                    }
                }
                jb->phase = 1;
            } else if (jb->act == 2) {
                ++jb->st.iters;
                const int k = jb->j + 1;
                const double est = gm.host(2);
                if (!(est >= prm.tol) || jb->st.iters >= prm.max_iter || k == gm.m) {
                    if (jb->precond) {
                        basis_combination(gm, k, pb->z1.p, s);
                        jb->precond(pb->z1.p, pb->z2.p);
                        axpby(1.0, jb->x, 1.0, pb->z2.p, jb->x, 2 * pb->N, s);
                    } else {
                        gm.update_solution(k, jb->x, s);
                    }
                    jb->phase = 1;
                } else {
                    ++jb->j;
                }
            }
        }
    }
}

KrylovStats run_gmres(pb_problem *pb, const DevOp &op, const DevOp &precond, const double *b, double *x,
                      bool x_zero) {
    KrylovJob jb;
    jb.pb = pb;
    jb.op = op;
    jb.precond = precond;
    jb.b = b;
    jb.x = x;
    jb.x_zero = x_zero;
    std::vector<KrylovJob *> jobs{&jb};
    run_krylov(jobs);
    return jb.st;
}

}  // namespace pb

namespace {

void require_setup(pb_problem *pb) {
    if (!pb->is_setup) fail(PB_ENOTSETUP, "pb_setup has not been called since the last input change");
}

void fill_result(pb_problem *pb, const KrylovStats &st, float ms, pb_result *out) {
    std::memset(out, 0, sizeof(*out));
    out->dG_solv = pb->dG;
    out->residual = st.rel;
    out->iterations = st.iters;
    out->converged = st.rel < pb->prm.tol;
    out->matvecs = st.matvecs;
    out->setup_ms = pb->setup_ms;
    out->solve_ms = ms;
    for (auto &P : pb->pairs) {
        out->p2p_pairs += P.p2p_pairs;
        out->m2p_pairs += P.n_m2p * (int64_t)P.kappas.size();
        out->near_pairs += P.n_near;
        out->near_excluded += P.near_excl;
    }
}

// Whether a batch takes the persistent batched operator: two or more
// problems, all FP32-mixed with the same expansion order in the radial form,
// and every pair of each one a Laplace-inside / Yukawa-outside pair
// (single-surface molecules: binding triplets, ligand fleets).
bool batch_persistent_eligible(const std::vector<pb_problem *> &probs) {
    if (probs.size() < 2 || !probs[0]->ctx->batch_persistent) return false;
    for (pb_problem *pb : probs) {
        if (pb->prm.precision != PB_MIXED || pb->prm.P != probs[0]->prm.P) return false;
        for (const Pair &P : pb->pairs)
            if (!batch_pair_eligible(P, pb->prm, P.tgt == P.tree)) return false;
    }
    return true;
}

// Solve every problem of `probs` (set up, distinct) by lock-step GMRES, each on
// its current stream, then its reaction potential and energy.
void solve_many(const std::vector<pb_problem *> &probs, const std::vector<const double *> &x0s,
                std::vector<KrylovStats> &stats, std::vector<float> &ms) {
    const size_t n = probs.size();
    std::vector<KrylovJob> jobs(n);
    std::vector<KrylovJob *> jp(n);
    for (size_t i = 0; i < n; ++i) {
        pb_problem *pb = probs[i];
        require_setup(pb);
        cudaStream_t s = pb->stream;
        PB_CUDA_TRY(cudaEventRecord(pb->ev0, s));
        const int64_t n2 = 2 * pb->N;
        if (x0s[i]) PB_CUDA_TRY(cudaMemcpyAsync(pb->x.p, x0s[i], n2 * sizeof(double), cudaMemcpyHostToDevice, s));
        KrylovJob &jb = jobs[i];
        jb.pb = pb;
        jb.op = [pb](const double *u, double *v) { apply_operator(pb, u, v); };
        if (pb->prm.precond) jb.precond = [pb](const double *u, double *z) { apply_precond(pb, u, z); };
        jb.b = pb->b.p;
        jb.x = pb->x.p;
        jb.x_zero = x0s[i] == nullptr;
        jb.graph = [pb](cudaStream_t gs) { launch_operator_graph(pb, gs); };
        jb.cycle_op = [pb] { apply_operator(pb, pb->z1.p, pb->gm.w.p); };
        jb.prep = [pb](cudaStream_t ps) {
            if (pb->use_cluster) {
                Gmres &gm = pb->gm;
                cluster_prep(pb->csurf, pb->cinv.p, gm.st.p, gm.V.p, gm.ld, gm.w.p, gm.scal.p + 1, pb->z1.p, ps);
                return;
            }
            std::vector<std::pair<int64_t, int64_t>> sf;
            for (size_t t = 0; t < pb->S.size(); ++t) sf.emplace_back(pb->off[t], pb->S[t].n);
            pb->gm.prep_step(pb->prm.precond ? pb->minv.p : nullptr, sf, pb->z1.p, ps);
        };
        jb.cycle_exec = &pb->cyc_exec;
        jb.cycle_kernels = &pb->cyc_kernels;
        jp[i] = &jb;
    }
    std::unique_ptr<BatchPlan> plan;
    if (batch_persistent_eligible(probs)) {
        plan = std::make_unique<BatchPlan>();
        std::vector<BatchPairRef> refs;
        for (size_t i = 0; i < n; ++i) {
            pb_problem *pb = probs[i];
            for (const Pair &P : pb->pairs)
                refs.push_back(BatchPairRef{&P, &pb->G[P.tgt], &pb->T[P.tree], P.tgt == P.tree,
                                            pb->z1.p + 2 * pb->off[P.tree] + pb->S[P.tree].n, (int)i});
        }
        batch_plan_build(*plan, refs, (int)n, probs[0]->prm.P, probs[0]->ctx->stream);
    }
    run_krylov(jp, plan.get());
    for (size_t i = 0; i < n; ++i) {
        pb_problem *pb = probs[i];
        reaction(pb, pb->x.p);
        PB_CUDA_TRY(cudaMemcpyAsync(pb->gm.hs.p + 3, pb->energy.p, sizeof(double), cudaMemcpyDeviceToHost,
                                    pb->stream));
        PB_CUDA_TRY(cudaEventRecord(pb->ev1, pb->stream));
    }
    stats.resize(n);
    ms.resize(n);
    for (size_t i = 0; i < n; ++i) {
        pb_problem *pb = probs[i];
        PB_CUDA_TRY(cudaEventSynchronize(pb->ev1));
        PB_CUDA_TRY(cudaEventElapsedTime(&ms[i], pb->ev0, pb->ev1));
        pb->dG = pb->gm.host(3);
        pb->have_solution = true;
        stats[i] = jobs[i].st;
    }
}

void solve(pb_problem *pb, const double *x0, pb_result *out) {
    std::vector<KrylovStats> st;
    std::vector<float> ms;
    solve_many({pb}, {x0}, st, ms);
    if (out) fill_result(pb, st[0], ms[0], out);
    if (!(st[0].rel < pb->prm.tol)) fail(PB_ENOCONV, "GMRES reached max_iter before the tolerance");
}

// Runs `f` with problem i on pool stream i mod (pool size), forked from and
// joined back to the context stream, so the call stays ordered on it.
template <typename F>
void on_pool_streams(pb_ctx *c, const std::vector<pb_problem *> &probs, F &&f) {
    const size_t np = std::min<size_t>(std::max<size_t>(1, probs.size()), 8);
    while (c->pool.size() < np) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        PB_CUDA_TRY(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        PB_CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        c->pool.push_back(st);
        c->pool_ev.push_back(ev);
    }
    PB_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    for (size_t k = 0; k < np; ++k) PB_CUDA_TRY(cudaStreamWaitEvent(c->pool[k], c->ev0, 0));
    for (size_t i = 0; i < probs.size(); ++i) probs[i]->stream = c->pool[i % np];
    auto restore = [&] {
        for (size_t k = 0; k < np; ++k) {
            cudaEventRecord(c->pool_ev[k], c->pool[k]);
            cudaStreamWaitEvent(c->stream, c->pool_ev[k], 0);
        }
        for (pb_problem *pb : probs) pb->stream = c->stream;
    };
    try {
        f();
    } catch (...) {
        restore();
        throw;
    }
    restore();
}

double coulomb(pb_problem *pb) {
    cudaStream_t s = pb->stream;
    const int64_t nc = pb->nc;
    if (nc == 0) return 0.0;
    TmpBuf<double> rowv(nc, s);
    coulomb_rows(pb->cxyz_d.p, pb->cq_d.p, nc, rowv.p, s);
    weighted_sum(pb->cq_d.p, rowv.p, nc, 0.5 * kKjPerMol / pb->regions[pb->cregion].eps, pb->energy.p, s);
    double out = 0.0;
    PB_CUDA_TRY(cudaMemcpyAsync(&out, pb->energy.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    PB_CUDA_TRY(cudaStreamSynchronize(s));
    return out;
}

void check_batch(pb_ctx *c, pb_problem *const *probs, int n, std::vector<pb_problem *> &v) {
    if (n < 0 || (n > 0 && !probs)) fail(PB_EINVAL, "bad problem array");
    for (int i = 0; i < n; ++i) {
        if (!probs[i]) fail(PB_EINVAL, "null problem in batch");
        if (probs[i]->ctx != c) fail(PB_EINVAL, "problem belongs to another context");
        if (std::find(v.begin(), v.end(), probs[i]) != v.end()) fail(PB_EINVAL, "problem repeated in batch");
        require_setup(probs[i]);
        v.push_back(probs[i]);
    }
}

}  // namespace

extern "C" {

int pb_ctx_create(int device, pb_ctx **out) {
    if (!out) return PB_EINVAL;
    *out = nullptr;
    auto c = std::make_unique<pb_ctx>();
    c->device = device;
    int rc = guard(nullptr, [&] {
        int nd = 0;
        PB_CUDA_TRY(cudaGetDeviceCount(&nd));
        if (device < 0 || device >= nd) fail(PB_EINVAL, "no such CUDA device");
        set_device(c.get());
        PB_CUDA_TRY(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
        // stream-ordered temporaries come back from the device's pool without
        // returning memory to the driver at every synchronisation
        cudaMemPool_t mp = nullptr;
        PB_CUDA_TRY(cudaDeviceGetDefaultMemPool(&mp, device));
        uint64_t keep = UINT64_MAX;
        PB_CUDA_TRY(cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep));
        PB_CUDA_TRY(cudaEventCreate(&c->ev0));
        PB_CUDA_TRY(cudaEventCreate(&c->ev1));
        // constant tables (quadrature rules, Taylor term indices, binomials) and
        // kernel attributes, once per context instead of at every setup
        upload_rules();
        upload_term_tables();
    });
    if (rc != PB_OK) return rc;
    *out = c.release();
    return PB_OK;
}

void pb_ctx_destroy(pb_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (size_t k = 0; k < c->pool.size(); ++k) {
        cudaStreamSynchronize(c->pool[k]);
        cudaStreamDestroy(c->pool[k]);
        cudaEventDestroy(c->pool_ev[k]);
    }
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char *pb_last_error(pb_ctx *c) { return c ? c->err.c_str() : "null context"; }

int pb_ctx_set_option(pb_ctx *c, int option, long long value) {
    if (!c) return PB_EINVAL;
    return guard(c, [&] {
        if (option == PB_OPT_BATCH_PERSISTENT) {
            if (value != 0 && value != 1) fail(PB_EINVAL, "PB_OPT_BATCH_PERSISTENT takes 0 or 1");
            c->batch_persistent = (int)value;
        } else {
            fail(PB_EINVAL, "unknown option");
        }
    });
}

void *pb_ctx_stream(pb_ctx *c) { return c ? (void *)c->stream : nullptr; }

int pb_problem_create(pb_ctx *c, pb_problem **out) {
    if (!c || !out) return PB_EINVAL;
    *out = nullptr;
    auto pb = std::make_unique<pb_problem>();
    pb->ctx = c;
    pb->stream = c->stream;
    const int rc = guard(c, [&] {
        set_device(c);
        PB_CUDA_TRY(cudaEventCreate(&pb->ev0));
        PB_CUDA_TRY(cudaEventCreate(&pb->ev1));
        PB_CUDA_TRY(cudaStreamCreateWithFlags(&pb->side, cudaStreamNonBlocking));
        PB_CUDA_TRY(cudaEventCreateWithFlags(&pb->evf, cudaEventDisableTiming));
        PB_CUDA_TRY(cudaEventCreateWithFlags(&pb->evj, cudaEventDisableTiming));
        PB_CUDA_TRY(cudaStreamCreateWithFlags(&pb->lists2, cudaStreamNonBlocking));
        PB_CUDA_TRY(cudaEventCreateWithFlags(&pb->ev2a, cudaEventDisableTiming));
        PB_CUDA_TRY(cudaEventCreateWithFlags(&pb->ev2b, cudaEventDisableTiming));
        PB_CUDA_TRY(cudaEventCreateWithFlags(&pb->ev2c, cudaEventDisableTiming));
    });
    if (rc != PB_OK) return rc;
    *out = pb.release();
    return PB_OK;
}

void pb_problem_destroy(pb_problem *pb) {
    if (!pb) return;
    cudaSetDevice(pb->ctx->device);
    cudaStreamSynchronize(pb->stream);
    delete pb;
}

int pb_add_region(pb_problem *pb, double eps, double kappa, int *region_id) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        if (!(eps > 0.0) || !(kappa >= 0.0) || !std::isfinite(eps) || !std::isfinite(kappa))
            fail(PB_EINVAL, "region needs eps > 0 and kappa >= 0");
        pb->regions.push_back(Region{eps, kappa});
        pb->is_setup = false;
        if (region_id) *region_id = (int)pb->regions.size() - 1;
    });
}

namespace {

void check_surface_args(pb_problem *pb, const void *verts, int64_t nv, const void *tris, int64_t nt, int inner,
                        int outer) {
    if (!verts || !tris || nv < 3 || nt < 1) fail(PB_EINVAL, "empty surface");
    if (inner < 0 || outer < 0 || inner >= (int)pb->regions.size() || outer >= (int)pb->regions.size() ||
        inner == outer)
        fail(PB_EINVAL, "surface references an unknown region");
    if (nt > ((int64_t)1 << 29) / 19) fail(PB_EINVAL, "too many triangles");
}

// The mesh check, then the surface joins the problem (si holds the device copy).
void add_checked_surface(pb_problem *pb, SurfIn &&si, int inner, int outer, int *surface_id) {
    pb->mesh_chk_h.alloc(1);
    check_mesh_async(si.v.p, si.nv, si.t.p, si.nt, pb->mesh_chk_h.p, pb->stream);
    PB_CUDA_TRY(cudaStreamSynchronize(pb->stream));
    mesh_check_result(*pb->mesh_chk_h.p);
    si.inner = inner;
    si.outer = outer;
    pb->sin.push_back(std::move(si));
    pb->is_setup = false;
    if (surface_id) *surface_id = (int)pb->sin.size() - 1;
}

// p must be device (or managed) memory of the context's device.
void require_device_ptr(pb_ctx *ctx, const void *p, const char *what) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        fail(PB_EINVAL, std::string(what) + " is not a CUDA pointer");
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        fail(PB_EINVAL, std::string(what) + " is not device memory");
    if (at.device != ctx->device)
        fail(PB_EINVAL, std::string(what) + " is memory of device " + std::to_string(at.device) +
                            ", not of the context's device " + std::to_string(ctx->device));
}

// Fails with PB_EINVAL naming the first bad element found by check_values_async.
void value_check_result(const ValueCheck &r, const char *value_what, const char *index_what) {
    if (r.bad_value != ~0ull)
        fail(PB_EINVAL, std::string("non-finite ") + value_what + " (element " + std::to_string(r.bad_value) + ")");
    if (r.bad_index != ~0ull)
        fail(PB_EINVAL, std::string(index_what) + " out of range (element " + std::to_string(r.bad_index) + ")");
}

}  // namespace

int pb_add_surface(pb_problem *pb, const double *verts, int64_t nv, const int32_t *tris, int64_t nt, int inner,
                   int outer, int *surface_id) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        check_surface_args(pb, verts, nv, tris, nt, inner, outer);
        for (int64_t i = 0; i < 3 * nv; ++i)
            if (!std::isfinite(verts[i])) fail(PB_EINVAL, "non-finite vertex coordinate");
        for (int64_t i = 0; i < 3 * nt; ++i)
            if (tris[i] < 0 || tris[i] >= nv) fail(PB_EINVAL, "triangle vertex index out of range");
        set_device(pb->ctx);
        SurfIn si;
        si.nv = nv;
        si.nt = nt;
        si.v.upload(verts, 3 * nv, pb->stream);
        si.t.upload(tris, 3 * nt, pb->stream);
        add_checked_surface(pb, std::move(si), inner, outer, surface_id);
    });
}

int pb_add_surface_dev(pb_problem *pb, const double *verts, int64_t nv, const int32_t *tris, int64_t nt, int inner,
                       int outer, int *surface_id) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        check_surface_args(pb, verts, nv, tris, nt, inner, outer);
        set_device(pb->ctx);
        require_device_ptr(pb->ctx, verts, "verts");
        require_device_ptr(pb->ctx, tris, "tris");
        cudaStream_t s = pb->stream;
        SurfIn si;
        si.nv = nv;
        si.nt = nt;
        si.v.alloc(3 * nv);
        si.t.alloc(3 * nt);
        PB_CUDA_TRY(cudaMemcpyAsync(si.v.p, verts, 3 * nv * sizeof(double), cudaMemcpyDeviceToDevice, s));
        PB_CUDA_TRY(cudaMemcpyAsync(si.t.p, tris, 3 * nt * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        pb->val_chk_h.alloc(1);
        check_values_async(si.v.p, 3 * nv, si.t.p, 3 * nt, nv, pb->val_chk_h.p, s);
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        value_check_result(*pb->val_chk_h.p, "vertex coordinate", "triangle vertex index");
        add_checked_surface(pb, std::move(si), inner, outer, surface_id);
    });
}

int pb_add_gaussian_surface(pb_problem *pb, const double *xyz, const double *radius, int64_t na,
                            const pb_surf_params *sp, int inner, int outer, int *surface_id) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        if (!sp) fail(PB_EINVAL, "surface parameters missing");
        if (inner < 0 || outer < 0 || inner >= (int)pb->regions.size() || outer >= (int)pb->regions.size() ||
            inner == outer)
            fail(PB_EINVAL, "surface references an unknown region");
        SurfGenParams gp;
        gp.spacing = sp->spacing;
        if (sp->beta != 0.0) gp.beta = sp->beta;
        if (sp->cutoff != 0.0) gp.cutoff = sp->cutoff;
        gp.radius_offset = sp->radius_offset;
        if (sp->margin != 0.0) gp.margin = sp->margin;
        if (sp->level != 0.0) gp.level = sp->level;
        if (sp->tclamp != 0.0) gp.tclamp = sp->tclamp < 0.0 ? 0.0 : sp->tclamp;
        if (sp->relax != 0.0) gp.relax = sp->relax;
        if (sp->max_step != 0.0) gp.max_step = sp->max_step;
        if (sp->smooth_iters != 0) gp.smooth_iters = sp->smooth_iters < 0 ? 0 : sp->smooth_iters;
        if (sp->newton_steps != 0) gp.newton_steps = sp->newton_steps < 0 ? 0 : sp->newton_steps;
        set_device(pb->ctx);
        SurfIn si;
        gaussian_surface(xyz, radius, na, gp, pb->stream, si);
        if (si.nt > ((int64_t)1 << 29) / 19) fail(PB_EINVAL, "too many triangles");
        si.inner = inner;
        si.outer = outer;
        pb->sin.push_back(std::move(si));
        pb->is_setup = false;
        if (surface_id) *surface_id = (int)pb->sin.size() - 1;
    });
}

int pb_surface_info_get(pb_problem *pb, int surface, pb_surface_info *out) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        if (!out || surface < 0 || surface >= (int)pb->sin.size()) fail(PB_EINVAL, "unknown surface");
        const SurfIn &si = pb->sin[surface];
        std::memset(out, 0, sizeof(*out));
        out->nv = si.nv;
        out->nt = si.nt;
        out->generated = si.generated ? 1 : 0;
        for (int d = 0; d < 3; ++d) out->grid[d] = si.gen.shape[d];
        out->rounds = si.gen.rounds;
        out->components = si.gen.components;
        out->raw_nv = si.gen.raw_nv;
        out->raw_nt = si.gen.raw_nt;
        out->gen_ms = si.gen.ms;
    });
}

int pb_surface_export(pb_problem *pb, int surface, double *verts, int32_t *tris) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        if (surface < 0 || surface >= (int)pb->sin.size()) fail(PB_EINVAL, "unknown surface");
        set_device(pb->ctx);
        const SurfIn &si = pb->sin[surface];
        if (verts) si.v.download(verts, 3 * si.nv, pb->stream);
        if (tris) si.t.download(tris, 3 * si.nt, pb->stream);
        PB_CUDA_TRY(cudaStreamSynchronize(pb->stream));
    });
}

int pb_set_charges(pb_problem *pb, const double *xyz, const double *q, int64_t nc, int region) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        if (nc < 0 || (nc > 0 && (!xyz || !q))) fail(PB_EINVAL, "bad charge arrays");
        if (region < 0 || region >= (int)pb->regions.size()) fail(PB_EINVAL, "unknown charge region");
        if (pb->regions[region].kappa != 0.0) fail(PB_EINVAL, "charges must sit in a kappa = 0 region");
        for (int64_t i = 0; i < 3 * nc; ++i)
            if (!std::isfinite(xyz[i])) fail(PB_EINVAL, "non-finite charge position");
        set_device(pb->ctx);
        pb->cq_d.upload(q, nc, pb->stream);
        pb->cxyz_d.upload(xyz, 3 * nc, pb->stream);
        PB_CUDA_TRY(cudaStreamSynchronize(pb->stream));
        pb->nc = nc;
        pb->cregion = region;
        pb->is_setup = false;
    });
}

int pb_set_charges_dev(pb_problem *pb, const double *xyz, const double *q, int64_t nc, int region) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        if (nc < 0 || (nc > 0 && (!xyz || !q))) fail(PB_EINVAL, "bad charge arrays");
        if (region < 0 || region >= (int)pb->regions.size()) fail(PB_EINVAL, "unknown charge region");
        if (pb->regions[region].kappa != 0.0) fail(PB_EINVAL, "charges must sit in a kappa = 0 region");
        set_device(pb->ctx);
        cudaStream_t s = pb->stream;
        if (nc > 0) {
            require_device_ptr(pb->ctx, xyz, "xyz");
            require_device_ptr(pb->ctx, q, "q");
        }
        pb->cq_d.alloc(nc);
        pb->cxyz_d.alloc(3 * nc);
        if (nc > 0) {
            PB_CUDA_TRY(cudaMemcpyAsync(pb->cq_d.p, q, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
            PB_CUDA_TRY(cudaMemcpyAsync(pb->cxyz_d.p, xyz, 3 * nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        pb->val_chk_h.alloc(1);
        check_values_async(pb->cxyz_d.p, 3 * nc, nullptr, 0, 0, pb->val_chk_h.p, s);
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        pb->nc = 0;
        pb->is_setup = false;
        value_check_result(*pb->val_chk_h.p, "charge position", "index");
        pb->nc = nc;
        pb->cregion = region;
    });
}

int pb_setup(pb_problem *pb, const pb_params *params) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        set_device(pb->ctx);
        pb->is_setup = false;
        pb->prm = resolve(params);
        setup_problem(pb);
    });
}

int64_t pb_num_unknowns(pb_problem *pb) { return (pb && pb->is_setup) ? 2 * pb->N : -1; }

int pb_apply_operator(pb_problem *pb, const double *x, double *y, int device_ptrs) {
    if (!pb || !x || !y) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        set_device(pb->ctx);
        cudaStream_t s = pb->stream;
        const int64_t n2 = 2 * pb->N;
        if (device_ptrs) {
            require_device_ptr(pb->ctx, x, "x");
            require_device_ptr(pb->ctx, y, "y");
            apply_operator(pb, x, y);
        } else {
            pb->xin.upload(x, n2, s);
            pb->yout.alloc(n2);
            apply_operator(pb, pb->xin.p, pb->yout.p);
            pb->yout.download(y, n2, s);
        }
        PB_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int pb_rhs(pb_problem *pb, double *bh) {
    if (!pb || !bh) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        pb->b.download(bh, 2 * pb->N, pb->stream);
        PB_CUDA_TRY(cudaStreamSynchronize(pb->stream));
    });
}

int pb_solve(pb_problem *pb, const double *x0, pb_result *out) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        set_device(pb->ctx);
        solve(pb, x0, out);
    });
}

int pb_gradient(pb_problem *pb, pb_grad *g) {
    if (!pb || !g) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        set_device(pb->ctx);
        energy_gradient(pb, g);
    });
}

int pb_apply_transpose(pb_problem *pb, const double *x, double *y, int device_ptrs) {
    if (!pb || !x || !y) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        set_device(pb->ctx);
        cudaStream_t s = pb->stream;
        const int64_t n2 = 2 * pb->N;
        if (device_ptrs) {
            require_device_ptr(pb->ctx, x, "x");
            require_device_ptr(pb->ctx, y, "y");
            apply_transpose(pb, x, y);
        } else {
            pb->xin.upload(x, n2, s);
            pb->yout.alloc(n2);
            apply_transpose(pb, pb->xin.p, pb->yout.p);
            pb->yout.download(y, n2, s);
        }
        PB_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int pb_get_solution(pb_problem *pb, double *xh) {
    if (!pb || !xh) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        if (!pb->have_solution) fail(PB_EINVAL, "no solution yet");
        pb->x.download(xh, 2 * pb->N, pb->stream);
        PB_CUDA_TRY(cudaStreamSynchronize(pb->stream));
    });
}

int pb_reaction_potential(pb_problem *pb, const double *xh, double *phi) {
    if (!pb || !xh || !phi) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        set_device(pb->ctx);
        cudaStream_t s = pb->stream;
        pb->xin.upload(xh, 2 * pb->N, s);
        reaction(pb, pb->xin.p);
        pb->phi_reac.download(phi, pb->nc, s);
        PB_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int pb_coulomb_energy(pb_problem *pb, double *out) {
    if (!pb || !out) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        set_device(pb->ctx);
        *out = coulomb(pb);
    });
}

int pb_solve_batch(pb_ctx *c, pb_problem *const *probs, int n, pb_result *out) {
    if (!c) return PB_EINVAL;
    return guard(c, [&] {
        set_device(c);
        std::vector<pb_problem *> v;
        check_batch(c, probs, n, v);
        if (v.empty()) return;
        std::vector<KrylovStats> st;
        std::vector<float> ms;
        on_pool_streams(c, v, [&] { solve_many(v, std::vector<const double *>(v.size(), nullptr), st, ms); });
        bool conv = true;
        for (size_t i = 0; i < v.size(); ++i) {
            if (out) fill_result(v[i], st[i], ms[i], out + i);
            conv = conv && st[i].rel < v[i]->prm.tol;
        }
        PB_CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (!conv) fail(PB_ENOCONV, "GMRES reached max_iter before the tolerance in a batched problem");
    });
}

int pb_binding_energy(pb_ctx *c, pb_problem *cx, pb_problem *rec, pb_problem *lig, double *ddG) {
    if (!c || !ddG) return PB_EINVAL;
    return guard(c, [&] {
        set_device(c);
        pb_problem *arr[3] = {cx, rec, lig};
        std::vector<pb_problem *> v;
        check_batch(c, arr, 3, v);
        std::vector<KrylovStats> st;
        std::vector<float> ms;
        double e[3] = {0.0, 0.0, 0.0};
        on_pool_streams(c, v, [&] {
            solve_many(v, std::vector<const double *>(3, nullptr), st, ms);
            for (int i = 0; i < 3; ++i) e[i] = v[i]->dG + coulomb(v[i]);
        });
        PB_CUDA_TRY(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < 3; ++i)
            if (!(st[i].rel < v[i]->prm.tol)) fail(PB_ENOCONV, "GMRES reached max_iter before the tolerance");
        *ddG = e[0] - e[1] - e[2];
    });
}

int pb_profile_operator(pb_problem *pb, const double *xh, int reps, double *phase_ms) {
    if (!pb || !xh || !phase_ms || reps < 1) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        set_device(pb->ctx);
        cudaStream_t s = pb->stream;
        const int64_t n2 = 2 * pb->N;
        pb->xin.upload(xh, n2, s);
        pb->yout.alloc(n2);
        PhaseEvents ph;
        for (auto &e : ph.ev) PB_CUDA_TRY(cudaEventCreate(&e));
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int r = 0; r < reps; ++r) {
            apply_operator(pb, pb->xin.p, pb->yout.p, &ph);
            PB_CUDA_TRY(cudaEventSynchronize(ph.ev[5]));
            for (int k = 0; k < 5; ++k) {
                float ms = 0.f;
                PB_CUDA_TRY(cudaEventElapsedTime(&ms, ph.ev[k], ph.ev[k + 1]));
                acc[k] += ms;
            }
            float tot = 0.f;
            PB_CUDA_TRY(cudaEventElapsedTime(&tot, ph.ev[0], ph.ev[5]));
            acc[5] += tot;
        }
        for (auto &e : ph.ev) cudaEventDestroy(e);
        for (int k = 0; k < 6; ++k) phase_ms[k] = acc[k] / reps;
    });
}

long long pb_launch_count(void) { return pb::g_launches.load(); }

int pb_tree_info_get(pb_problem *pb, int surface, pb_tree_info *out) {
    if (!pb || !out) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        if (surface < 0 || surface >= (int)pb->T.size()) fail(PB_EINVAL, "no such surface");
        const Tree &T = pb->T[surface];
        out->n_points = T.npts;
        out->n_nodes = T.nnodes;
        out->n_leaves = T.nleaves;
        for (int a = 0; a < 3; ++a) out->corner[a] = T.corner[a];
        out->side = T.side;
    });
}

int pb_tree_export(pb_problem *pb, int surface, uint64_t *keys, int32_t *perm, int32_t *node_level,
                   int64_t *node_start, int64_t *node_count, int32_t *node_first_child, int32_t *node_nchild) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        if (surface < 0 || surface >= (int)pb->T.size()) fail(PB_EINVAL, "no such surface");
        const Tree &T = pb->T[surface];
        cudaStream_t s = pb->stream;
        if (keys) T.keys.download(keys, T.npts, s);
        if (perm) T.perm.download(perm, T.npts, s);
        if (node_level) T.level.download(node_level, T.nnodes, s);
        if (node_start) T.start.download(node_start, T.nnodes, s);
        if (node_count) T.count.download(node_count, T.nnodes, s);
        if (node_first_child) T.first_child.download(node_first_child, T.nnodes, s);
        if (node_nchild) T.nchild.download(node_nchild, T.nnodes, s);
        PB_CUDA_TRY(cudaStreamSynchronize(s));
    });
}

int pb_lists_export(pb_problem *pb, int target_surface, int source_surface, int64_t *counts, int64_t *m2p_ptr,
                    int32_t *m2p_nodes, int64_t *p2p_ptr, int32_t *p2p_nodes, int64_t *near_ptr,
                    int32_t *near_panels) {
    if (!pb) return PB_EINVAL;
    return guard(pb->ctx, [&] {
        require_setup(pb);
        const int ns = (int)pb->S.size();
        if (target_surface < -1 || target_surface >= ns || source_surface < 0 || source_surface >= ns)
            fail(PB_EINVAL, "no such surface");
        const int tg = target_surface < 0 ? ns : target_surface;
        std::vector<Pair> &v = target_surface < 0 ? pb->cpairs : pb->pairs;
        const Pair *P = nullptr;
        for (auto &q : v)
            if (q.tgt == tg && q.tree == source_surface) P = &q;
        if (!P) fail(PB_EINVAL, "these surfaces do not interact");
        const Targets &G = pb->G[tg];
        cudaStream_t s = pb->stream;
        const int64_t m = G.n;
        if (counts) {
            counts[0] = P->n_m2p; counts[1] = P->n_p2p; counts[2] = P->n_near;
            counts[3] = P->near_excl; counts[4] = P->self_excl; counts[5] = m;
        }
        std::vector<int32_t> order(m);
        G.order.download(order.data(), m, s);
        PB_CUDA_TRY(cudaStreamSynchronize(s));
        auto reorder = [&](const DevBuf<int64_t> &dptr, const DevBuf<int32_t> &dent, int64_t total, int64_t *hptr,
                           int32_t *hent) {
            if (!hptr && !hent) return;
            std::vector<int64_t> ptr(m + 1);
            std::vector<int32_t> ent(std::max<int64_t>(1, total));
            dptr.download(ptr.data(), m + 1, s);
            if (total) dent.download(ent.data(), total, s);
            PB_CUDA_TRY(cudaStreamSynchronize(s));
            std::vector<int64_t> len(m);
            for (int64_t q = 0; q < m; ++q) len[order[q]] = ptr[q + 1] - ptr[q];
            std::vector<int64_t> optr(m + 1, 0);
            for (int64_t i = 0; i < m; ++i) optr[i + 1] = optr[i] + len[i];
            if (hptr) std::copy(optr.begin(), optr.end(), hptr);
            if (hent)
                for (int64_t q = 0; q < m; ++q)
                    std::copy(ent.begin() + ptr[q], ent.begin() + ptr[q + 1], hent + optr[order[q]]);
        };
        reorder(P->m2p_ptr, P->m2p_node, P->n_m2p, m2p_ptr, m2p_nodes);
        reorder(P->p2p_ptr, P->p2p_node, P->n_p2p, p2p_ptr, p2p_nodes);
        reorder(P->near_ptr, P->near_panel, P->n_near, near_ptr, near_panels);
    });
}

}  // extern "C"
