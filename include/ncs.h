/*
 * ncs.h - C ABI of the GB300 narrow capture / narrow escape solver.
 *
 * The library solves the block-preconditioned second-kind multiple-scattering
 * system of Kaye & Greengard, "A fast solver for the narrow capture and narrow
 * escape problems in the sphere" (arXiv 1906.04209), Section 6, eq. (opinteqnsdisc):
 *
 *     f_i + P sum_{j != i} S_ij B f_j = P 1,     i = 1..N,
 *
 * for N disk patches of geodesic radius eps on the unit sphere, with K Zernike
 * coefficients per patch. The matrix-vector product runs on the GPU
 * (Section 7, Step 3): the outgoing map rho_j = T f_j, the far-field sums of the
 * Neumann Green's function over skeleton points, and the Zernike transform P.
 *
 * Conventions (all entry points):
 *   - Return 0 (NCS_OK) on success or a negative NCS_E_* code; no exceptions
 *     cross the ABI. ncs_last_error() describes the most recent failure on a
 *     context. Inputs are validated before any device work is issued.
 *   - Host arrays are owned by the caller, read (or written) only during the
 *     call, and copied where the library keeps the data.
 *   - Device pointers are owned by the caller, must be resident on the device
 *     bound to the context (the one current at its first GPU call), are used only
 *     on the given CUDA stream and only until the call's work on that stream
 *     completes.
 *   - Vectors over all patches are patch-major: x[i*K + k] is coefficient k of
 *     patch i; k follows the Zernike ordering (n ascending, then m ascending,
 *     cos before sin) of Section 4.
 *   - Patch frames: for a centre c, e3 = c, e1 = (z x c)/|z x c| (e1 = x when c
 *     is a pole), e2 = e3 x e1; the local point (t, theta) is
 *     cos t c + sin t (cos theta e1 + sin theta e2), t the arclength from c.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef NCS_H
#define NCS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NCS_OK 0
#define NCS_E_INPUT (-1)   /* invalid argument or infeasible patch layout */
#define NCS_E_NOCONV (-2)  /* iteration cap reached before the tolerance */
#define NCS_E_NUMERIC (-3) /* breakdown, NaN or Inf in the iteration */
#define NCS_E_CUDA (-4)    /* CUDA runtime error (message in ncs_last_error) */
#define NCS_E_TIMEOUT (-5) /* a bounded device wait gave up */
#define NCS_E_OOM (-6)     /* device or host allocation failed */
#define NCS_E_STATE (-7)   /* call out of order (e.g. matvec before set_patches) */

#define NCS_EXTERIOR 0 /* narrow capture: G_E, Section 2.2 */
#define NCS_INTERIOR 1 /* narrow escape:  G_I, Section 2.3 */

#define NCS_FP64 0  /* all pair sums and transforms in FP64 */
#define NCS_FP32 1  /* FP32 pair sums / transforms in patch- or group-local frames */
#define NCS_MIXED 2 /* solve only: FP32 inner GMRES + FP64-accurate iterative refinement */
#define NCS_DF64 3  /* pair sums and interpolation in float-float (two FP32 words, ~48-bit
                       significand, ~1e-14 relative) on the FP32 pipes; GEMMs, grid
                       transforms and offsets in FP64: FP64-accurate products at a
                       fraction of the FP64-pipe cost */
#define NCS_PRECISION_DEFAULT (-1) /* the context's precision (ncs_set_precision); for a
                                      product, NCS_MIXED means NCS_FP32 */

#define NCS_METHOD_AUTO 0   /* tree when N >= tree_min_patches, else direct */
#define NCS_METHOD_DIRECT 1 /* compressed sums over all other patches, O(N^2) (Section 7.1) */
#define NCS_METHOD_TREE 2   /* cube-sphere quadtree, O(N log N) (Sections 7.2-7.3, Step 3) */

typedef struct ncs_ctx ncs_ctx;

typedef struct ncs_params {
  int npan;            /* radial panels of the one-patch solver (Section 8.2), default 13 */
  int nord;            /* nodes per panel, default 20 */
  int ntheta_fine;     /* fine-grid azimuths; 0 = M + 40 rounded up to even */
  double id_tol;       /* interpolative-decomposition tolerance (Section 7.1), default 1e-11 */
  int threads;         /* host threads for the precompute and the tree set-up; 0 = all */
  double grid_tol;     /* incoming-grid tolerance (Section 7.3), default 1e-8 */
  int method;          /* NCS_METHOD_*, default AUTO */
  int tree_min_patches;/* AUTO switches to the tree at this N, default 128 (on GB300 the tree
                          product is faster from N ~ 200: 0.36 vs 0.49 ms at N = 200, 1.6 vs
                          17.9 ms at N = 2000, K = 128) */
  int gmres_maxit;     /* GMRES iteration cap, default 200 */
  int verbose;         /* 0 silent .. 3 chatty (stderr) */
  int mixed_residual;  /* precision of the refinement residual of NCS_MIXED:
                          NCS_DF64 (default) or NCS_FP64 */
  int tensor_cores;    /* 1 (default): the FP32 product runs its dense contractions
                          (rho = T x, y = x + P z) on the tcgen05 tensor cores (3xTF32
                          splits, ~2^-22 per operand: product error a few 1e-6 relative);
                          0: FP32 SIMT kernels (~1e-6) */
  int residual_update; /* NCS_MIXED: 1 (default) forms the refinement residual as
                          r - A corr with an FP32 product once |r| <= 1e-4 |b| (its error,
                          ~1e-6 |r|, is then below 1e-10 |b|); 0 always recomputes
                          b - A x at mixed_residual precision */
  double id_ladder_max;/* largest far-field radius (radians) for which an extra, smaller ID
                          representation is built (far fields beyond 2, 2.52, 3.17, 4, ... eps;
                          Section 7.1 recompression), default 1.0; 0: only the 2 eps one.
                          Fewer representations shorten the precompute (one CPQR of the
                          sketch per representation) and lengthen the products */
  int device_precompute;/* 1 (default): the precompute forms the one-patch modal
                          collocation matrices (Section 8.2; the modal kernels at every
                          quadrature node, ~1e5 nodes x ~500 theta nodes) and runs its
                          interpolative decompositions (the Gaussian sketch of the
                          far-field kernel matrix, ~1e10 FP64 FMAs, the column-pivoted QRs
                          and the T assembly) on the CUDA device current at ncs_create
                          when there is one, else on the host; 0: always on the host. The
                          per-mode LUs and solves stay on the host */
  int cuda_graphs;     /* 1 (default): ncs_solve captures one GMRES step (the product, the
                          orthogonalisation and the Givens update, all reading the step
                          index from device memory) as a CUDA graph on its first use and
                          replays it; 0: the same kernels launched one by one. While a
                          capture runs, no other host thread may synchronise the whole
                          device (cudaDeviceSynchronize, or calls that imply it): with
                          contexts driven from several threads set 0 (ncs_batch_solve does) */
  int batch_ladder_by_n; /* ncs_batch_solve only. 1 (default): each sphere's ID ladder extent is
                          min(id_ladder_max, 0 below 1000 patches, 0.1 rad below 3000, else
                          1.0 rad), the measured balance between the precompute (one more
                          representation per rung) and its products; 0: id_ladder_max for all */
  int batch_grouped;     /* ncs_batch_solve with NCS_MIXED only. 1 (default): spheres with fewer
                          than tree_min_patches patches (and method not NCS_METHOD_TREE) are
                          solved together, one concatenated system per mode with one launch per
                          product stage and Krylov step for all of them (each keeps its own
                          eps, operator and GMRES state); 0: each on its own context */
  double inner_grid_tol; /* NCS_MIXED with the tree on >= 10000 patches: incoming-grid tolerance of
                          the tree that the inner FP32 solves (and the FP32 residual update) use,
                          default 1e-5:
                          their products need only the accuracy of FP32 pair sums, so coarser
                          grids (fewer grid points and pair evaluations) serve them, while the
                          refinement residuals keep grid_tol. Built with the product's tree when
                          the context's precision is NCS_MIXED (else at the first mixed solve).
                          Values <= grid_tol (e.g. 0) use the product's tree throughout */
} ncs_params;

/* Fills *p with the defaults listed above. */
void ncs_default_params(ncs_params* p);

/*
 * Launch configuration of the tree product's FP32 path, chosen per workload by ncs_tune
 * (no counterpart in the paper, whose Section 7 "Optimizations and parallelization"
 * leaves such choices to the implementation). Every setting gives the same product up to
 * the FP32 rounding of its pair sums; none changes the accuracy of the FP64 or
 * float-float products.
 */
typedef struct ncs_tuning {
  int p2l_tile;       /* interaction-list patches per shared-memory tile of a P2L block: 8, 16 */
  int p2l_poly;       /* of every 16 packed pair chains in the P2L kernel, how many take
                         their logarithm on the FMA pipe instead of the MUFU unit: 0, 2, 4, 6 */
  int direct_poly;    /* the same for the direct lists at the Zernike nodes: 0, 2, 4, 6 */
  int item_patches;   /* interaction-list patches per P2L work item (one block): 8..64, a
                         multiple of p2l_tile; changing it rebuilds the host tree */
  double l2p_weight;  /* cost of one L2P node-grid product in pair evaluations, weighed when
                         a group chooses its incoming grid or direct evaluation (Step 3):
                         0.01..1; changing it rebuilds the host tree */
  int p2l_rsq;        /* of every 16 packed pair chains in the P2L kernel, how many take the
                         reciprocal square root by Newton steps on the FMA pipe (Lomont's
                         seed) instead of the MUFU unit: 0, 4, 8 (with p2l_poly <= 16) */
  int direct_rsq;     /* the same for the direct lists: 0, 4, 8 */
} ncs_tuning;

/*
 * Creates a context for patch radius eps (0 < eps < 1), problem mode
 * (NCS_EXTERIOR / NCS_INTERIOR) and K Zernike functions per patch (1 <= K <= 2000),
 * and runs the one-patch precompute (Section 7, Step 1): modal solves giving B
 * (Sections 5 and 8), I = w^T B (eq. getI), the interpolative decompositions and
 * T = Pi W B (Section 7.1, eq. Tmap), and the Zernike transform P (Section 4). With
 * params->device_precompute (the default) its collocation matrices and interpolative
 * decompositions run on the CUDA device current at this call, synchronously, with
 * temporary device buffers freed before it returns (on the host if there is no device
 * or no room). params may be NULL (defaults). The CUDA device current at the first
 * call that needs the GPU for the context (a product, solve or evaluation) is bound to
 * the context for its lifetime and receives the uploads. On success *out owns host and
 * device memory that ncs_destroy releases.
 * Errors: NCS_E_INPUT, NCS_E_NUMERIC (precompute failure, including a CUDA error in its
 * device kernels), NCS_E_OOM; *out is NULL.
 */
int ncs_create(double eps, int mode, int K, const ncs_params* params, ncs_ctx** out);

/*
 * Like ncs_create, but takes the outgoing operator from the caller instead of
 * computing it: T (p x K row-major), the skeleton points' local polar coordinates
 * skel_t, skel_theta (p each, t in [0, eps]) and I (K). P and the Zernike
 * sampling nodes are still formed by the library (Section 4). The arrays are
 * copied. Used to reuse a stored precompute.
 * Errors: NCS_E_INPUT (sizes, NULL arrays, skeleton t outside [0, eps], non-finite T),
 * NCS_E_OOM; *out is NULL.
 */
int ncs_create_from_operator(double eps, int mode, int K, int p, const double* T,
                             const double* skel_t, const double* skel_theta, const double* I,
                             const ncs_params* params, ncs_ctx** out);

/*
 * Like ncs_create_from_operator with several outgoing representations: nrep far-field
 * radii rho_min (geodesic, increasing, the first >= 2 eps), their ranks p, and T,
 * skel_t, skel_theta concatenated in that order (sum(p) rows / entries). A source is
 * represented by the coarsest representation whose far field contains every target
 * it is summed onto (per-level recompression, Section 7 "Optimizations").
 * Errors: as ncs_create_from_operator, and NCS_E_INPUT for radii that do not start at
 * 2 eps or more and increase.
 */
int ncs_create_from_operators(double eps, int mode, int K, int nrep, const double* rho_min, const int* p,
                              const double* T, const double* skel_t, const double* skel_theta,
                              const double* I, const ncs_params* params, ncs_ctx** out);

/* Number of outgoing representations in *nrep; with rho_min and p non-NULL (and
 * *nrep at least that number on entry) also their far-field radii and ranks, into caller
 * arrays. Errors: NCS_E_INPUT (NULL ctx or nrep, *nrep too small). */
int ncs_get_reps(const ncs_ctx* ctx, int* nrep, double* rho_min, int* p);

/*
 * Representation r (0 <= r < nrep) of the outgoing operator (Section 7.1, eq. Tmap with
 * the far field beyond rho_min[r]): T (p_r x K row-major) and the skeleton points' local
 * polar coordinates skel_t, skel_theta (p_r each), copied into caller arrays; any
 * pointer may be NULL. Errors: NCS_E_INPUT (bad r or context).
 */
int ncs_get_rep(const ncs_ctx* ctx, int r, double* T, double* skel_t, double* skel_theta);

/*
 * Writes context sizes into out[0..n): K, Kstar, p, M, nf (fine-grid points),
 * N (patches set, 0 if none), nrad (radial nodes), tree levels (0 if no tree),
 * grid points over all tree groups, pair evaluations per tree matvec (FP counts
 * of far-field kernel evaluations), direct pairs per matvec, and the grid points and
 * pair evaluations of the mixed solve's inner tree (0 if not built; see inner_grid_tol);
 * at most 13 values. out: n caller int64s. Errors: NCS_E_INPUT (NULL).
 */
int ncs_info(const ncs_ctx* ctx, int64_t* out, int n);

/* Precompute timings in seconds: out[0] one-patch solve, out[1] ID; out[2] = 1 if the ID
 * ran on a CUDA device, else 0; parts of out[1]: out[3] sketch, out[4] CPQRs, out[5]
 * assembly of the T operators; out[6] = 1 if the modal collocation matrices were formed
 * on a CUDA device, else 0; parts of out[0]: out[7] collocation matrices, out[8] LUs and
 * modal solves. n < 9 fills the first n. */
int ncs_timings(const ncs_ctx* ctx, double* out, int n);

/*
 * Copies the finest outgoing representation (far field beyond 2 eps) and the
 * rest of the precompute out (any pointer may be NULL to skip it): T (p x K),
 * skeleton (t, theta) (p each), I (K), P (K x Kstar), Zernike nodes on the unit
 * disk (r, theta) (Kstar each), into caller arrays of those sizes.
 * Errors: NCS_E_INPUT (NULL ctx).
 */
int ncs_get_operator(const ncs_ctx* ctx, double* T, double* skel_t, double* skel_theta,
                     double* I, double* P, double* znode_r, double* znode_theta);

/*
 * Copies the one-patch solution (Section 8): radial collocation nodes trad (nrad)
 * and radial profiles beta (nrad x K, row-major), so that b_j(t, theta) =
 * beta_j(t) trig(m_j theta). NCS_E_STATE for contexts made from an operator.
 */
int ncs_get_onepatch(const ncs_ctx* ctx, double* trad, double* beta);

/*
 * Sets the patch layout: N >= 1 unit centres (N x 3 row-major, host, copied).
 * Validates |c| = 1 (to 1e-10) and the geodesic separation >= 3 eps (Section 3)
 * and, for the tree method, builds the cube-sphere quadtree, interaction lists and
 * incoming grids on the host (Section 7, Step 2). Device copies are made at the
 * next call that uses the GPU. Errors: NCS_E_INPUT (bad centre, separation), NCS_E_OOM.
 */
int ncs_set_patches(ncs_ctx* ctx, int64_t N, const double* centres);

/*
 * Diagnostics of the cube-sphere quadtree (Section 7.2): every ordered (target,
 * source) patch pair the tree product accounts for, with its level and kind (0 =
 * interaction list, 2 = leaf-level neighbour; Step 3 note: each ordered pair of
 * distinct patches must appear exactly once). Call with target == NULL to get the
 * count in *count; then with buffers of at least *count ints each.
 * Errors: NCS_E_INPUT (NULL, buffers smaller than the count), NCS_E_STATE (no patches).
 */
int ncs_tree_pairs(ncs_ctx* ctx, int64_t* count, int* target, int* source, int* level, int* kind);

/*
 * Tree statistics into out[0..n): levels, grid groups, grid points, P2L work items,
 * P2L kernel evaluations, direct kernel evaluations, L2P node-grid products,
 * direct (target, source) patch pairs, distinct grid shapes, grid-to-grid links of
 * the downward pass, their point-grid products. Builds the host tree if needed
 * (host-only). Errors: NCS_E_INPUT (NULL), NCS_E_STATE (no patches).
 */
int ncs_tree_stats(ncs_ctx* ctx, int64_t* out, int n);

/* Selects NCS_METHOD_AUTO / DIRECT / TREE for later products and solves (a tree is
 * built on the host if needed). Errors: NCS_E_INPUT (NULL ctx, bad method). */
int ncs_set_method(ncs_ctx* ctx, int method);

/*
 * Sets the context's precision (NCS_FP64, NCS_FP32, NCS_MIXED or NCS_DF64; default
 * NCS_MIXED), used by every call whose precision argument is NCS_PRECISION_DEFAULT: solves
 * run at it, products at it with NCS_MIXED read as NCS_FP32 (the inner products of the mixed
 * solve). Errors: NCS_E_INPUT.
 */
int ncs_set_precision(ncs_ctx* ctx, int precision);

/*
 * y = A x for the system of eq. (opinteqnsdisc): y_i = x_i + P sum_{j != i} S_ij B x_j,
 * evaluated by the compressed representation (Section 7, Step 3). x, y: host,
 * N*K doubles. precision: NCS_FP64, NCS_DF64 or NCS_FP32 (FP32 kernels, FP64 in/out).
 * x and y belong to the caller and are used only during the call (synchronous).
 * Errors: NCS_E_INPUT (NULL, bad precision), NCS_E_STATE (no patches), NCS_E_OOM,
 * NCS_E_CUDA, NCS_E_TIMEOUT (a bounded device wait of the tensor-core GEMM gave up).
 */
int ncs_matvec(ncs_ctx* ctx, const double* x, double* y, int precision);

/* As ncs_matvec with device pointers x, y (N*K doubles, caller-owned, not overlapping)
 * on the given stream (cudaStream_t, NULL = legacy default stream). Asynchronous: errors
 * of the enqueued work surface at a later synchronising call. Errors: as ncs_matvec. */
int ncs_matvec_dev(ncs_ctx* ctx, const double* x, double* y, int precision, void* stream);

/*
 * As ncs_matvec_dev, synchronous, with CUDA-event times (milliseconds) of each stage
 * of Step 3 written to ms[0..n): outgoing map (3.1), P2L onto incoming grids (3.2),
 * grid coefficients (first half of 3.4), direct sums at the Zernike nodes (3.3 and
 * small groups; the whole sum for the direct method), L2P interpolation (second half
 * of 3.4), apply P (3.5), total. Stages that do not run report 0. ms: n caller doubles.
 * Errors: as ncs_matvec.
 */
int ncs_profile_matvec(ncs_ctx* ctx, const double* x, double* y, int precision, void* stream, double* ms, int n);

/*
 * The multiple-scattering field before the transform P (Section 7, end of Step 4):
 * z_i(k) = sum_{j != i} [S_ij B x_j](k) at the Zernike sampling nodes, z: device,
 * N*Kstar doubles, patch-major, caller-owned. Asynchronous on `stream`.
 * Errors: as ncs_matvec_dev.
 */
int ncs_field_dev(ncs_ctx* ctx, const double* x, double* z, int precision, void* stream);

/*
 * Solves the system by GMRES (Section 7, Step 3; x0 = 0, relative residual tol).
 * precision: NCS_FP64 (all FP64), NCS_DF64 (float-float products, FP64 Arnoldi),
 * NCS_FP32 (FP32 products, FP64 Arnoldi) or NCS_MIXED (FP32 inner GMRES wrapped in
 * iterative refinement whose residuals use NCS_DF64 products, or, once the residual
 * is below 1e-4 |b|, the FP32 residual update of ncs_params.residual_update).
 * Outputs (each may be NULL): fhat (N*K host doubles, the densities in the b_n
 * basis, Remark sigrep), scalar = mean first passage time mu = 1/(3 I_sigma) - 3/5
 * (interior, eq. mufromsigma2) or capacitance C = 4 pi I_sigma (exterior, |J|
 * of Section 2.2), I_sigma (eq. getI), iterations (total products by A), and the
 * final relative residual (recomputed as b - A x, or updated as above). Errors: NCS_E_NOCONV (cap reached; outputs hold
 * the last iterate), NCS_E_NUMERIC, NCS_E_STATE, NCS_E_CUDA.
 */
int ncs_solve(ncs_ctx* ctx, double tol, int precision, double* fhat, double* scalar,
              double* Isigma, int* iterations, double* relres);

/*
 * Autotuner of the tree product. Times FP32 tree products of the context's layout under
 * candidate launch configurations (flags & 1: the pair-kernel variants (tile, polynomial
 * logarithm and Newton reciprocal-square-root shares), each stage timed with CUDA events; flags & 2: the work-item size and the grid-or-direct weight, each
 * candidate on a rebuilt tree), keeps a candidate only if its product matches the
 * float-float product of the same input to 2e-5 of the largest entry, and applies the
 * fastest to ctx (products and solves that follow use it). With cache_path non-NULL the
 * choice is looked up first in, and then appended to, that text file, keyed by mode, K,
 * eps, N and the default tree's shape (levels, share of direct pairs); a hit costs no
 * trial products. out (may be NULL) receives the chosen configuration; report (may be
 * NULL, n entries) receives [0] default product ms, [1] tuned product ms, [2] trial
 * products, [3] the chosen product's error against float-float (relative to max |z|),
 * [4] seconds spent, [5] 1 if the choice came from the cache. Uses the device, the
 * context's stream and one temporary device buffer (2 N K* doubles).
 * Errors: NCS_E_INPUT (flags), NCS_E_STATE (no patches, or not the tree method),
 * NCS_E_OOM, NCS_E_CUDA.
 */
int ncs_tune(ncs_ctx* ctx, int flags, const char* cache_path, ncs_tuning* out, double* report, int n);

/* Applies a launch configuration (as from ncs_tune) to ctx. Errors: NCS_E_INPUT (a value
 * outside the ranges of ncs_tuning). */
int ncs_set_tuning(ncs_ctx* ctx, const ncs_tuning* t);

/* The context's current launch configuration. Errors: NCS_E_INPUT (NULL). */
int ncs_get_tuning(const ncs_ctx* ctx, ncs_tuning* t);

/*
 * Counters of the last ncs_solve on ctx, into out[0..n): [0] GMRES steps (products at the
 * inner precision), [1] residuals recomputed as b - A x (products at the residual
 * precision: NCS_MIXED's mixed_residual, else the solve's), [2] FP32 residual updates
 * r - A corr, [3] refinement steps (NCS_MIXED), [4] the final relative residual, [5] steps
 * run as a replay of the captured CUDA graph, [6] wall seconds of the solve, [7] 1 if the
 * final residual was recomputed as b - A x (always, unless the solve stopped early on an
 * error). Errors: NCS_E_INPUT (NULL).
 */
int ncs_solve_stats(const ncs_ctx* ctx, double* out, int n);

/*
 * Single-layer potential at M targets off the patches (Section 2, eqs. urep and
 * intBVPansatz, off-surface Green's functions eqs. Gextoffsurface / Gintoffsurface):
 * u(x) = sum_j S sigma_j(x). A patch whose centre lies farther than 2.5 eps (geodesic, from
 * the target's radial projection) is summed from its skeletons, rho_j = T fhat_j; a nearer
 * patch is integrated directly against its density sigma_j = sum_k fhat_jk b_k (the
 * one-patch solution, Section 8) with radial and angular rules graded toward the target
 * (FP64 on the device), which serves targets close to the sphere such as the paper's maps
 * at |x| = 1 - eps/5 (Section 9.2). targets: M x 3 host (|x| >= 1 exterior, |x| <= 1
 * interior); fhat: N*K host. out (M): exterior ubar = 1 - u; interior
 * vbar = (v - 1)/(3D) + (1 - |x|^2)/6 with D = -I_sigma (eq. vtilde).
 * Errors: NCS_E_INPUT (a target on the sphere inside a patch, where u is the boundary data;
 * targets within 2.5 eps of a patch on a context made from an operator, which has no
 * one-patch data; a near target with Zernike degree M > 31; a target so close that its
 * radial rule would exceed 2048 nodes), NCS_E_STATE, NCS_E_CUDA.
 */
int ncs_eval(ncs_ctx* ctx, int64_t M, const double* targets, const double* fhat, double* out);

/*
 * Relative L2 residual of the multiple-scattering system on patch i (Section 9, eq.
 * l2res, the error measure of the paper's large runs): the root mean square over Gamma_i
 * of r = S sigma_i + sum_{j != i} S_ij sigma_j - 1. S sigma_i = sum_k fhat_ik q_k (each
 * basis density solves the one-patch equation S b_k = q_k, Section 8); the other
 * patches' potential comes from their finest skeleton representation (FP64 on the
 * device; every point of Gamma_i is at least 2 eps from the other centres). The printed
 * normalisation (the norm over |Gamma_i|) is read as the relative residual
 * ||r|| / ||1|| = ||r|| / sqrt(|Gamma_i|). Quadrature: nt Gauss-Legendre nodes in the
 * arclength t on [0, eps] (measure sin t dt) times nth equispaced angles; 0 selects
 * M + 8 and 2M + 10. fhat: N*K host doubles (as from ncs_solve); rms: one double.
 * Errors: NCS_E_INPUT (index out of range, grid above 4096 x 8192, NULL), NCS_E_STATE,
 * NCS_E_OOM, NCS_E_CUDA.
 */
int ncs_patch_residual(ncs_ctx* ctx, int64_t i, const double* fhat, int nt, int nth, double* rms);

/*
 * The projections of one GMRES Arnoldi step (Section 7, Step 3; classical Gram-Schmidt
 * on the device): out[j] = V_j . w for j < k, V_j = V + j*ld, all device FP64 arrays
 * (n entries each; out holds k), reduced deterministically in two stages (fixed
 * chunks, then a per-vector sum). Allocates its k x 64 partial sums with cudaMalloc
 * for the duration of the call; synchronous on `stream`.
 * Errors: NCS_E_INPUT, NCS_E_OOM, NCS_E_CUDA.
 */
int ncs_block_dots(int64_t n, int k, const double* V, int64_t ld, const double* w, double* out, void* stream);

/*
 * ncs_block_dots without any allocation, for callers that cannot call cudaMalloc (a
 * host application that manages the device memory itself, a loop that must not block
 * on the allocator, work recorded into a stream capture). The paper has no
 * counterpart: this is a property of the library, not of the method. The partial sums
 * live in a fixed device array inside the library (room for k <= 1024 vectors, 512 KiB,
 * held by every GPU that loads the library until the process exits); the first call on
 * a device looks its address up with that device current (which may load the library's
 * device code on that device), so make that first call before any stream capture.
 * Asynchronous on `stream`; calls that overlap on the GPU share the array and race, so
 * serialise them. Nothing is allocated or freed.
 * Errors: NCS_E_INPUT (k > 1024, bad sizes or NULL), NCS_E_CUDA (also when an earlier,
 * unrelated CUDA error is pending on the calling thread: it is reported, and cleared,
 * before anything is launched).
 */
int ncs_block_dots_noalloc(int64_t n, int k, const double* V, int64_t ld, const double* w, double* out,
                           void* stream);

/*
 * The library's tensor-core GEMM on its own: D = A B^T with A (rows x kdim), B
 * (cols x kdim) and D (rows x cols), all row-major FP32 device arrays, computed with
 * tcgen05 kind::tf32 MMAs on hi/lo TF32 splits (3 products, ~FP32 accuracy) - the
 * kernel behind the per-patch operator contractions (eq. Tmap, Step 3.5). Synchronous
 * on `stream`. Errors: NCS_E_INPUT, NCS_E_CUDA, NCS_E_TIMEOUT (bounded wait gave up).
 */
int ncs_tc_gemm_f32(int64_t rows, int cols, int kdim, const float* A, const float* B, float* D, void* stream);

/*
 * Solves B independent spheres (each its own eps, mode, patch layout; common K) to
 * relative residual tol at `precision`, as ncs_solve does for one (Section 7, Step 3):
 * `workers` host threads (0 = all cores) each take instances from a shared queue,
 * run the precompute and tree set-up for it on one host core, solve it on the GPU on
 * its own stream, and release it, so set-up, transfers and GPU work of different
 * instances overlap and at most `workers` instances hold device memory at once.
 * With params->batch_ladder_by_n each sphere's ID ladder extent follows its patch count;
 * with params->batch_grouped (NCS_MIXED only) the spheres below tree_min_patches are set
 * up by the workers and then solved together on the calling thread, one grouped system per
 * mode (direct products, the mixed refinement of ncs_solve per instance in lock step, the
 * Krylov step of all of them captured once as a CUDA graph and replayed when
 * params->cuda_graphs is set).
 * centres[b] points to N[b] x 3 host doubles. Per-instance outputs (each may be NULL):
 * scalar (mu or C), I_sigma, iterations, relres, status (NCS_OK or the instance's error
 * code). seconds (may be NULL): [set-up summed over instances, solve summed over
 * instances, wall clock of the batch]. Returns NCS_OK if every instance converged,
 * else the first failing instance's code.
 */
int ncs_batch_solve(int B, const double* eps, const int* mode, const int64_t* N, const double* const* centres,
                    int K, double tol, int precision, const ncs_params* params, int workers, double* scalar,
                    double* Isigma, int* iterations, double* relres, int* status, double* seconds);

/*
 * Peak FMA throughput of the current device at precision NCS_FP64 or NCS_FP32, measured by
 * the library's own microkernel (independent FMA chains on every SM, CUDA-event timed, best
 * of three launches after a warm-up), in TFLOP/s (2 flops per FMA) into *tflops: the
 * denominator of the pair kernels' pipe fractions. No counterpart in the paper.
 * Synchronous; about 0.1 s. Errors: NCS_E_INPUT, NCS_E_CUDA.
 */
int ncs_fma_peak(int precision, double* tflops);

/* Message of the last failure on ctx (static string if ctx is NULL). */
const char* ncs_last_error(const ncs_ctx* ctx);

/*
 * Number of CUDA kernels this library has launched in this process so far, over all
 * contexts and threads (diagnostic; not part of the method). The difference across a
 * call is the number of kernels that call launched, when no other thread uses the
 * library meanwhile. Never fails.
 */
int64_t ncs_launch_count(void);

/* Releases all host and device memory of ctx (NULL is ignored). */
void ncs_destroy(ncs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* NCS_H */
