/* pbbem: treecode-accelerated boundary-element Poisson-Boltzmann solver for B300 (sm_103a).
 *
 * The library computes the electrostatic solvation energy of molecules in
 * implicit solvent with the boundary-integral formulation of Cooper, Bardhan &
 * Barba (arXiv:1309.4018): flat triangular panels with constant phi and
 * dphi/dn, centroid collocation (Sec. 2.2, Eqs. nBEM_disc, matrix, matel),
 * several interacting surfaces (molecular surface, Stern layer,
 * solvent-filled cavities; Sec. 2.2 "Multi-surface problems"), a
 * Cartesian-Taylor treecode for every matrix-vector product (Sec. 2.3, Eqs.
 * nbody, taylor, multexp, MAC) and a Krylov solver (Sec. 2.3, last
 * paragraph); the reaction potential and energies follow Eqs. reac_integral,
 * solv, bind_energy and total_energy.
 *
 * Units: Angstrom, elementary charge, relative permittivity, kappa in 1/A,
 * energies in kJ/mol.
 *
 * Conventions shared by every entry point:
 *   - All functions return PB_OK (0) or one of the PB_E* codes below; the
 *     message of the last failure is pb_last_error(ctx).
 *   - Host input arrays are copied during the call (surfaces and charges go
 *     straight to device memory, so pb_setup reads only device-resident
 *     inputs); the library never keeps a caller pointer.  Output arrays are
 *     caller-allocated and written in full.
 *   - All device memory is owned by the library and released by the matching
 *     *_destroy call.
 *   - A context serves one host thread at a time; its work runs on one CUDA
 *     stream (pb_ctx_stream).
 *   - Triangles are wound counter-clockwise seen from the surface's outer
 *     region, so the normal (v1 - v0) x (v2 - v0) points from the inner
 *     region to the outer region.
 *   - The unknown vector of a problem has 2 N entries, N the total panel
 *     count: surface by surface, phi on the panels of that surface followed
 *     by dphi/dn taken on its inner side.  The two row blocks of a surface
 *     are the equation of its inner region, then that of its outer region.
 */
#ifndef PBBEM_H
#define PBBEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PB_OK 0
#define PB_EINVAL 1      /* bad argument or malformed input (message says which) */
#define PB_ENOMEM 2      /* device or host allocation failed */
#define PB_ECUDA 3       /* a CUDA call failed */
#define PB_ENOCONV 4     /* GMRES reached max_iter; the partial result is still written */
#define PB_ETIMEOUT 5    /* a bounded device-side wait gave up */
#define PB_ENOTSETUP 6   /* pb_setup has not been called since the last input change */

#define PB_FP64 0        /* every treecode step in FP64 */
#define PB_MIXED 1       /* P2P, P2M, M2M, M2P in FP32 (compensated sums); Krylov, near field, energy FP64 */

typedef struct pb_ctx pb_ctx;
typedef struct pb_problem pb_problem;

/* Parameters (Tables 1, 3, 4 and 6).  A zero field takes the default in brackets. */
typedef struct {
    int K;             /* Gauss points per panel in the regular case: 1, 3, 7 or 19 [3] */
    int K_fine;        /* Gauss points per panel in the near-singular region: 1, 3, 7 or 19 [19] */
    int N_k;           /* Gauss points per triangle side, semi-analytical self integral, 1..32 [5] */
    double thres;      /* near-singular region |x - c_j| < thres * L_j, L_j = sqrt(2 A_j) [2.0] */
    int P;             /* Taylor expansion order, 0..12 [6] */
    double theta;      /* MAC parameter (Eq. MAC); negative selects direct summation [0.5] */
    int ncrit;         /* a box with >= ncrit sources is split [300] */
    double gmres_tol;  /* relative residual tolerance [1e-4] */
    int restart;       /* GMRES restart length, 1..200 [50] */
    int max_iter;      /* total GMRES iteration cap [1000] */
    int precision;     /* PB_FP64 or PB_MIXED [PB_FP64] */
    int no_precond;    /* 1: plain GMRES; 0: right-preconditioned by the inverse of every
                          panel's 2x2 self block (not in the paper; same solution) [0] */
    int ncrit_adjoint; /* a box of the transposed treecode (pb_gradient, pb_apply_transpose)
                          with >= ncrit_adjoint collocation points is split [ncrit] */
    int p2p_tile;      /* targets per direct-sum (P2P) work item, 1..64: a warp sums one leaf's
                          sources, staged 32 at a time, for this many targets that list the
                          leaf, two per lane above 32 (PB_MIXED; PB_FP64 takes at most 32)
                          (not in the paper; the results do not depend on it) [64] */
    int m2p_variant;   /* 1: the PB_MIXED far field of a Laplace/Yukawa pair (P <= 7) forms its
                          radial-form contraction on the tensor pipe (TF32 instructions, every
                          operand split in two TF32 parts, FP32 accumulation; rounding differs
                          from 0, accuracy the same); 0: on the FP32 pipe (not in the paper) [0] */
    int precond_block; /* panels per block of the right preconditioner, 1..64: runs of this many
                          Morton-consecutive panels of a surface, whose 2 x 2 panel couplings
                          (self terms exact, the rest by the K-point rule) form a dense block
                          inverted at setup (FP32, applied with ~48-bit sums); 1: every panel's
                          2 x 2 self block (not in the paper; the same solution to the GMRES
                          tolerance) [32] */
} pb_params;

typedef struct {
    double dG_solv;        /* solvation energy, kJ/mol (Eq. solv) */
    double residual;       /* final true relative residual ||b - A x|| / ||b|| */
    int iterations;        /* GMRES iterations */
    int converged;         /* 1 if residual < gmres_tol */
    int matvecs;           /* treecode evaluations during the solve */
    int pad_;
    double setup_ms;       /* time of the last pb_setup (device, CUDA events) */
    double solve_ms;       /* time of this solve (device, CUDA events) */
    int64_t p2p_pairs;     /* direct (target, source point) pairs per treecode evaluation */
    int64_t m2p_pairs;     /* (target, box, kernel) expansion evaluations per treecode evaluation */
    int64_t near_pairs;    /* near-singular (target, panel) corrections */
    int64_t near_excluded; /* near-singular panels left uncorrected (a point fell in an accepted box) */
} pb_result;

/* Context: one CUDA device, one stream. */
int pb_ctx_create(int device, pb_ctx **out);
void pb_ctx_destroy(pb_ctx *ctx);
const char *pb_last_error(pb_ctx *ctx);
/* The cudaStream_t all work of this context is issued on (for event timing). */
void *pb_ctx_stream(pb_ctx *ctx);
/* Context options (not in the paper).  PB_OPT_BATCH_PERSISTENT (0, the
 * default, or 1): whether pb_solve_batch runs the operator applications of
 * an eligible batch as one persistent launch per GMRES step (see
 * pb_solve_batch).  PB_EINVAL for an unknown option or value. */
#define PB_OPT_BATCH_PERSISTENT 1
int pb_ctx_set_option(pb_ctx *ctx, int option, long long value);

/* Problem: regions, surfaces and charges (Sec. 2.1, Eq. pde; Sec. 2.2). */
int pb_problem_create(pb_ctx *ctx, pb_problem **out);
void pb_problem_destroy(pb_problem *pb);
/* A region with permittivity eps > 0 and inverse Debye length kappa >= 0
 * (kappa = 0: Poisson/Laplace kernel; > 0: linearised PB/Yukawa kernel).
 * Regions are numbered 0, 1, ... in call order. */
int pb_add_region(pb_problem *pb, double eps, double kappa, int *region_id);
/* A closed triangle mesh separating region `inner` from region `outer`.
 * verts: nv x 3 doubles; tris: nt x 3 vertex indices.  PB_EINVAL on an
 * index out of range or an unknown region; pb_setup fails with PB_EINVAL on
 * a zero-area triangle. */
int pb_add_surface(pb_problem *pb, const double *verts, int64_t nv, const int32_t *tris,
                   int64_t nt, int inner, int outer, int *surface_id);
/* pb_add_surface with verts and tris in device (or managed) memory of the
 * context's device, as a torch CUDA tensor holds them: nv x 3 doubles and
 * nt x 3 ints, row-major, contiguous; the caller keeps ownership (they are
 * copied on the context stream, and the call returns once the copy and the
 * checks are done).  Writes to them on another stream must be complete
 * before the call.  The checks are those of pb_add_surface (finite
 * coordinates and indices in range, here run on the device, then the mesh
 * check); PB_EINVAL also for a pointer that is not device memory of the
 * context's device. */
int pb_add_surface_dev(pb_problem *pb, const double *verts, int64_t nv, const int32_t *tris,
                       int64_t nt, int inner, int outer, int *surface_id);
/* Molecular surface generated on the device from atoms.  The paper meshes the
 * solvent-excluded surface with MSMS (Sec. 2.2, Sec. 3); this builds instead
 * the level set rho = level of the Gaussian density
 *   rho(x) = sum_a [|x - x_a| <= cutoff R_a] exp(-beta (|x - x_a|^2 / R_a^2 - 1)),
 * R_a = radius[a] + radius_offset, on the nodes lo + spacing (i, j, k) of a grid
 * reaching margin + max R_a beyond the atoms; the triangles are those of
 * marching tetrahedra on the six-tetrahedron (Kuhn) split of every grid cube,
 * with a vertex at the linear zero of rho - level on every crossing edge (edge
 * parameter clamped to [tclamp, 1 - tclamp]); only the connected component of
 * the crossing of largest grid x index (the outer surface) is kept, oriented
 * towards rho < level; then up to smooth_iters rounds move every vertex a
 * fraction relax towards the mean of its neighbours and project it
 * newton_steps times onto the level set along grad rho (steps capped at
 * max_step), using the largest round count that leaves no triangle facing up
 * grad rho.  A zero field takes the default in brackets. */
typedef struct {
    double spacing;        /* grid spacing in A; required, > 0 */
    double beta;           /* density decay [0.5] */
    double cutoff;         /* an atom contributes within cutoff * R_a [2.7] */
    double radius_offset;  /* added to every radius (a Stern layer: 2) [0] */
    double margin;         /* grid padding in A beyond the largest radius [4] */
    double level;          /* iso level [1] */
    double tclamp;         /* edge parameter clamp, < 0.5 [0.02]; negative: no clamp */
    double relax;          /* umbrella step fraction, (0, 1] [0.5] */
    double max_step;       /* length cap of a projection step in A [0.3] */
    int smooth_iters;      /* smoothing rounds, <= 64 [5]; negative: none */
    int newton_steps;      /* projections per round, <= 64 [3]; negative: none */
} pb_surf_params;
/* Adds the generated surface between regions inner and outer, exactly as
 * pb_add_surface would add its mesh.  xyz: na x 3 doubles, radius: na doubles
 * (host; copied).  PB_EINVAL on bad parameters or atoms, a grid of more than
 * 4096 nodes per axis or 2^31 nodes, or a density with no crossing on the
 * grid; PB_ETIMEOUT if the device component labelling ran out of its bounded
 * step budget.  Synchronises the context stream. */
int pb_add_gaussian_surface(pb_problem *pb, const double *xyz, const double *radius, int64_t na,
                            const pb_surf_params *sp, int inner, int outer, int *surface_id);
/* Sizes of a surface and, for a generated one, how it was made. */
typedef struct {
    int64_t nv, nt;          /* vertices, triangles */
    int generated;           /* 1: made by pb_add_gaussian_surface */
    int grid[3];             /* density grid nodes per axis */
    int rounds;              /* smoothing rounds used */
    int pad_;
    int64_t components;      /* connected components of the level set on the grid */
    int64_t raw_nv, raw_nt;  /* vertices, triangles before the outer component was taken */
    double gen_ms;           /* device time of the generation (CUDA events) */
} pb_surface_info;
int pb_surface_info_get(pb_problem *pb, int surface, pb_surface_info *out);
/* Copies a surface's mesh to host arrays of nv x 3 doubles and nt x 3 ints (either may be NULL). */
int pb_surface_export(pb_problem *pb, int surface, double *verts, int32_t *tris);
/* Point charges (Eq. pde) inside region `region` (which must have kappa = 0). */
int pb_set_charges(pb_problem *pb, const double *xyz, const double *q, int64_t nc, int region);
/* pb_set_charges with xyz (nc x 3 doubles) and q (nc doubles) in device (or
 * managed) memory of the context's device; copied on the context stream,
 * caller keeps ownership, writes on another stream must be complete before
 * the call.  PB_EINVAL for a pointer that is not device memory of the
 * context's device, or a non-finite position (found on the device after the
 * copy; the problem then holds no charges). */
int pb_set_charges_dev(pb_problem *pb, const double *xyz, const double *q, int64_t nc, int region);

/* Geometry, octrees, interaction lists, near-singular corrections and the
 * right-hand side (Sec. 2.3: built once, reused by every iteration). */
int pb_setup(pb_problem *pb, const pb_params *params);
int64_t pb_num_unknowns(pb_problem *pb);  /* 2 N, or -1 before pb_setup */

/* y = A x for the assembled operator (one treecode evaluation, Sec. 2.3
 * "Treecode-accelerated BEM").  x, y: 2 N doubles; on the host if
 * device_ptrs == 0, else device pointers of this context's device (the call
 * is ordered on the context stream and returns when y is complete; PB_EINVAL
 * for a pointer that is not device memory of that device). */
int pb_apply_operator(pb_problem *pb, const double *x, double *y, int device_ptrs);
/* b of Eq. matrix (2 N host doubles). */
int pb_rhs(pb_problem *pb, double *b);
/* Solve A x = b by restarted GMRES on the device, then dG (Eqs. reac_integral, solv).
 * x0: optional initial guess (2 N host doubles) or NULL for zero. */
int pb_solve(pb_problem *pb, const double *x0, pb_result *out);
/* Solve n set-up problems of this context together (the binding triplet, a
 * fleet of ligands; the batching pattern of the production workload, applied
 * to Eq. bind_energy's three solves).  By default every problem runs its
 * GMRES cycles as device-driven graphs on one of up to 8 pool streams, one
 * host synchronisation per cycle round for the whole batch.  With
 * PB_OPT_BATCH_PERSISTENT = 1 an eligible batch (two or more problems, all
 * PB_MIXED with the same P <= 8, every surface between a kappa = 0 region
 * and a kappa > 0 region with K = 3: single-surface molecules) instead
 * advances its Arnoldi steps in lock step, one host synchronisation per step,
 * and each step's direct sums, far-field sums and per-target gathers of all
 * problems run as ONE persistent launch over a device queue of (problem,
 * phase, tile) entries; a problem's gathers wait, with a bounded number of
 * polls, for its direct and far-field entries, and a wait that runs out ends
 * the call with PB_ETIMEOUT (the context stays usable).  Either way the
 * energies equal those of single pb_solve calls bit for bit.  The call is
 * ordered on the context stream.  out: n results (may be NULL).  PB_ENOCONV
 * if any problem reached max_iter (every result is still written). */
int pb_solve_batch(pb_ctx *ctx, pb_problem *const *probs, int n, pb_result *out);
/* Binding energy (Eq. bind_energy): solves complex, receptor and ligand as one
 * batch and returns ddG = E_cx - E_rec - E_lig with E = dG_solv + the Coulomb
 * energy of the molecule's charges (Eq. total_energy), kJ/mol. */
int pb_binding_energy(pb_ctx *ctx, pb_problem *cx, pb_problem *rec, pb_problem *lig, double *ddG);
/* The solution of the last pb_solve (2 N host doubles). */
int pb_get_solution(pb_problem *pb, double *x);
/* Reaction potential at the charges (Eq. reac_integral) for a given unknown
 * vector x (host, 2 N); phi_reac: nc doubles in the 1/(4 pi) units of the kernels. */
int pb_reaction_potential(pb_problem *pb, const double *x, double *phi_reac);
/* Coulomb energy 1/2 C sum_{i != j} q_i q_j / (eps_R r_ij) of the charges, kJ/mol
 * (the Coulomb term of Eq. total_energy). */
int pb_coulomb_energy(pb_problem *pb, double *out);

/* Adjoint gradient of the solvation energy (Eq. solv) of the last pb_solve.
 * With E = c0 q^T Rm x (Rm: the reaction-potential map of Eq.
 * reac_integral, c0 = C/2 * 4 pi), A x = b = B q, and the adjoint
 * A^T lambda = c0 Rm^T q solved by GMRES on the transposed treecode operator
 * (same parameters, tolerance and preconditioner as the forward solve):
 *   dE/dq_k   = c0 (Rm x)_k + (B^T lambda)_k
 *   dE/dr_k   = c0 q_k grad(Rm x)_k + q_k lambda^T grad_k B
 *   dE/dp     = c0 q^T (dRm/dp) x + lambda^T (db/dp - (dA/dp) x),  p = eps_R or kappa_R
 * for every region R (the paper computes no gradients: this is the adjoint of
 * its discrete operator).  The kappa derivatives use the kernel derivatives
 * dG/dkappa and the derivative of the near-singular and semi-analytical
 * rules; the near/far rule choice is held fixed.  The charged region's
 * kappa derivative is the one-sided derivative at kappa = 0.
 * Arrays are caller-owned host buffers (NULL: not wanted): dq [nc], dxyz
 * [3 nc], deps [n_regions], dkappa [n_regions].  Units: kJ/mol per e, per A,
 * per unit eps, and kJ/mol * A.  Needs a converged pb_solve since the last
 * pb_setup (else PB_EINVAL); PB_ENOCONV if the adjoint GMRES reaches
 * max_iter (the arrays are still written).  dkappa with P > 8 needs
 * ~14 KB of local memory per device thread. */
typedef struct {
    double *dq;
    double *dxyz;
    double *deps;
    double *dkappa;
    double energy;      /* out: dG_solv of the solution differentiated */
    double residual;    /* out: relative residual of the adjoint solve */
    int iterations;     /* out: adjoint GMRES iterations */
    int matvecs;        /* out: transposed treecode evaluations */
    double grad_ms;     /* out: device time of the whole gradient (CUDA events) */
} pb_grad;
int pb_gradient(pb_problem *pb, pb_grad *g);
/* y = A^T x for the assembled operator by the transposed treecode (sources at
 * the collocation points, targets at the Gauss points).  x in row order, y in
 * unknown order, 2 N doubles each; host or device pointers as in
 * pb_apply_operator. */
int pb_apply_transpose(pb_problem *pb, const double *x, double *y, int device_ptrs);

/* Per-phase device time of one operator application (CUDA events on the
 * context stream), averaged over `reps` applications to the given unknown
 * vector x (host, 2 N).  phase_ms[0..5]: source strengths + P2M/M2M, P2P,
 * M2P, per-target gather of the partials with the near-singular and self
 * corrections, block combine, total.  Not in the paper:
 * instrumentation for the per-phase timings of the measurement. */
int pb_profile_operator(pb_problem *pb, const double *x, int reps, double *phase_ms);
/* Number of kernels this library has launched since it was loaded. */
long long pb_launch_count(void);

/* Coulomb energy 1/2 C sum_{i != j} q_i q_j / (eps r_ij) of nc charges, in
 * kJ/mol, computed without allocating device memory.  The paper has no
 * counterpart: this serves callers that cannot let a library allocate, such as
 * applications that own all device memory through their own pool or budget,
 * or loops that must not pay the synchronisation cudaMalloc/cudaFree imply.
 * xyz (3 nc doubles), q (nc doubles) and energy (1 double) are device
 * pointers on `device`; the work is queued on `stream` (a cudaStream_t, NULL
 * for the default stream) and the call returns before it completes.  Scratch
 * lives in a static device array of 262,144 doubles (2 MiB per GPU, held while
 * the library is loaded): nc > 262144 returns PB_EINVAL.  Every call shares
 * that array, so calls whose work overlaps on the GPU (other streams, other
 * threads) race; each call rewrites all the entries it reads.  The first call
 * on a device resolves the array's device address, so make it before any
 * stream capture.  That address is cached for the life of the process: after
 * cudaDeviceReset (or any other reset of the device's primary context) it no
 * longer belongs to the array, so do not call this function on that device
 * again in the same process.  *err (optional) receives a static message on
 * failure. */
int pb_coulomb_energy_noalloc(int device, const double *xyz, const double *q, int64_t nc, double eps,
                              double *energy, void *stream, const char **err);

/* Introspection of the integer work (Sec. 2.3, Eq. MAC), for bit-exact checks.
 * Octree over the Gauss points of surface `surface` (point j*K + k is Gauss
 * point k of panel j).  Nodes are numbered breadth first, children in octant
 * order.  Sizes first, then arrays of those sizes. */
typedef struct {
    int64_t n_points;
    int32_t n_nodes;
    int32_t n_leaves;
    double corner[3];
    double side;
} pb_tree_info;
int pb_tree_info_get(pb_problem *pb, int surface, pb_tree_info *out);
/* keys: n_points sorted Morton keys; perm: sorted position -> point index;
 * node_level, node_start, node_count, node_first_child (-1 for a leaf),
 * node_nchild: n_nodes each.  Any pointer may be NULL. */
int pb_tree_export(pb_problem *pb, int surface, uint64_t *keys, int32_t *perm,
                   int32_t *node_level, int64_t *node_start, int64_t *node_count,
                   int32_t *node_first_child, int32_t *node_nchild);
/* Interaction lists of the targets of `target_surface` (-1: the charges) against
 * the octree of `source_surface`, indexed by the targets' input order.
 * counts[0..5]: total M2P entries, P2P entries, near entries, excluded near
 * panels, targets whose own panel had a point in an accepted box, targets.
 * Arrays (any may be NULL): m2p_ptr/p2p_ptr/near_ptr (targets + 1 each),
 * m2p_nodes, p2p_nodes (node ids, depth-first pre-order per target),
 * near_panels (ascending per target).  PB_EINVAL if the pair never interacts. */
int pb_lists_export(pb_problem *pb, int target_surface, int source_surface, int64_t *counts,
                    int64_t *m2p_ptr, int32_t *m2p_nodes, int64_t *p2p_ptr,
                    int32_t *p2p_nodes, int64_t *near_ptr, int32_t *near_panels);

#ifdef __cplusplus
}
#endif
#endif /* PBBEM_H */
