/*
 * fdmpc.h -- C-ABI of the GB300 (sm_103a) vertex-star FDM/sparse relaxation
 * library (Brubeck & Farrell, arXiv 2107.14758).
 *
 * The library solves the Q_p continuous Galerkin discretisation of
 * -div(kappa grad u) = f with homogeneous Dirichlet data on a structured
 * nx x ny x nz hexahedral mesh (Section 2.1), by PCG preconditioned with the
 * hybrid p-multigrid/Schwarz V(1,1) cycle of Section 2.5: additive
 * vertex-star relaxation in the FDM basis (Section 2.4) with sparse patch
 * Cholesky factors (Section 2.6), and a Q1 coarse space on the same mesh.
 *
 * General conventions
 *   - All vectors are full-grid GLL nodal arrays of length
 *     (nx p + 1)(ny p + 1)(nz p + 1) doubles, x fastest, DEVICE resident and
 *     owned by the caller.  Entries on the Dirichlet boundary are ignored on
 *     input and written as 0 on output.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are stream-ordered and asynchronous unless stated.
 *   - Every call returns 0 on success or a negative FDM_E* code; the text of
 *     the last error of a context is returned by fdm_last_error().  No C++
 *     exception crosses this interface.
 *   - A context owns all of its device memory (factors, coefficients,
 *     work vectors).  Concurrent calls on one context must be serialised by
 *     the caller (one stream at a time).
 */
#ifndef FDMPC_H
#define FDMPC_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ---- */
#define FDM_OK 0
#define FDM_EINVAL (-1)   /* bad argument */
#define FDM_ENOMEM (-2)   /* device or host allocation failed, or a context's device allocations would
                           * exceed the byte limit in the environment variable FDM_ALLOC_LIMIT_BYTES
                           * (unset, empty or not a number: no limit) */
#define FDM_ENOTSPD (-3)  /* a patch or coarse Cholesky pivot was <= 0 */
#define FDM_ENOCONV (-4)  /* PCG reached maxit before rtol */
#define FDM_ENAN (-5)     /* a non-finite scalar appeared in PCG */
#define FDM_ETIMEOUT (-6) /* a bounded device-side wait gave up */
#define FDM_ECUDA (-7)    /* a CUDA runtime call failed */

/* ---- precision of the preconditioner (Section 2.8; FP64 outer PCG) ---- */
#define FDM_PREC_FP64 0  /* everything FP64 */
#define FDM_PREC_FP32 1  /* basis changes, patch solves, V-cycle in FP32 */

/* ---- preconditioner structure ---- */
#define FDM_PC_NONE 0    /* identity */
#define FDM_PC_ASM 1     /* omega * P_ASM^{-1} alone */
#define FDM_PC_VCYCLE 2  /* hybrid multiplicative V(1,1) with the Q1 coarse space */

/* ---- separable surrogate on curved cells (Section 2.7) ---- */
#define FDM_SURR_AVERAGED 0 /* mu_j = cell average of kappa * Ghat_jj */
#define FDM_SURR_EXTERNAL 1 /* mu supplied by fdm_surrogate_load */

typedef struct fdm_ctx fdm_ctx;

/* Mesh: nx, ny, nz cells per axis on a tensor grid with HOST vertex
 * coordinates xv[nx+1], yv[ny+1], zv[nz+1] (strictly increasing).
 * jac (HOST, optional): for curved cells, the Jacobian dx/dxhat (row-major
 * 3x3) at the (p+1)^3 Gauss-Legendre points of every cell, points x fastest,
 * cells x fastest (9 (p+1)^3 nx ny nz doubles); NULL = box cells, for which
 * the exact Kronecker form of eq. (kron) is used.  The arrays are copied. */
typedef struct {
  int nx, ny, nz;
  const double *xv, *yv, *zv;
  const double *jac;
} fdm_mesh;

/* Coefficients (HOST, optional, copied): kappa at the same Gauss points as
 * jac ((p+1)^3 nx ny nz doubles); NULL = kappa == 1.  Curved cells only.
 * samples27 (HOST, optional, copied): inputs of the learned surrogate,
 * kappa and J (row-major) at the 3x3x3 Gauss-Legendre points of every cell
 * (points x fastest, cells x fastest): 270 nx ny nz doubles, kappa > 0;
 * curved cells only.
 * mu (HOST, optional, copied): the per-cell separable coefficients of the
 * relaxation (3 per cell: x, y, z scalings, cells x fastest, > 0), used
 * instead of the box-cell values or the averaged surrogate; the same as a
 * later fdm_surrogate_load without refactoring. */
typedef struct {
  const double *kappa_q;
  const double *samples27;
  const double *mu;
} fdm_coeff;

typedef struct {
  int precision;      /* FDM_PREC_* (default FP32 preconditioner) */
  int pc;             /* FDM_PC_* (default V-cycle) */
  int surrogate;      /* FDM_SURR_* (default averaged) */
  int lanczos_steps;  /* CG-Lanczos steps for omega (default 20) */
  double omega;       /* > 0: use this damping instead of Lanczos */
  uint64_t lanczos_seed; /* seed of the N(0,1) Lanczos start vector (default 12345) */
  int flexible_beta;  /* 1: Polak-Ribiere beta in PCG (default 1 for FP32 PC) */
  double wait_timeout_s; /* bound on any device-side spin wait (default 1.0) */
  const double *lanczos_start; /* HOST, optional: Lanczos start vector (ndof doubles);
                                  NULL = N(0,1) from lanczos_seed (splitmix64 + Box-Muller) */
  int kernel_timing;  /* 1: record CUDA events around every kernel group (FDM_Q_KERNEL_TIMES) */
  int patch_ctas_per_sm; /* resident patch-solve CTAs per SM (0 = automatic); bounds the
                            patch factors in flight so that both solves find them in L2 */
  int patch_threads;  /* threads per patch-solve CTA: 256, 512 or 1024 (0 = 256, or 1024 when
                         an interface exceeds 1000 dofs) */
  int patch_kernel;   /* 0 = automatic (= 1), 1 = one CTA per patch reading the factor
                         directly, 2 = streamed: bulk copies into a shared-memory ring,
                         3 = resident: persistent CTAs that bulk-copy each patch's whole factor
                         into shared memory (falls back to 1 where it does not fit), 4 = cluster:
                         the interior stars on thread-block clusters that hold L21 in shared
                         memory across both solves, the other stars as 1; 5 = persistent CTAs in
                         the Schur-coupling form that stage the next patch's lower-block values in
                         shared memory and its S_TB and W in L2 while solving the current one;
                         6 = persistent CTAs in the Schur-coupling form that bulk-copy each patch's
                         whole operator (pivots, L10, line blocks, S_TB, W) into one of two
                         shared-memory buffers while solving the previous patch from the other
                         (FDM_EINVAL at set-up where two operators do not fit in 227 KB) */
  int stream_buffers; /* ring buffers of the streamed solve (0 = 4) */
  int stream_buffer_kb; /* size of each ring buffer in KiB (0 = 16) */
  int inject_stall;   /* test hook: the streamed, resident, cluster and (where it stages values in
                         shared memory) Schur-coupling solves wait on a barrier that is never
                         completed, give up after wait_timeout_s and report FDM_ETIMEOUT */
  int patch_prefetch; /* one-CTA-per-patch solve: L2 bulk prefetch of the factor, 1 = all at
                         the start, 2 = one section ahead of use, 3 = none (0 = 3) */
  int pcg_graph;      /* 1 (default): pcg_solve runs its loop on the device in a captured CUDA
                         graph (as pcg_solve_batched, a batch of one; the graph is rebuilt when
                         b, x, rtol or maxit change); 0, or kernel_timing = 1: a host loop with one
                         synchronisation per iteration */
  int patch_l2_hints; /* one-CTA-per-patch solve: 0 (default) or 1 = L2 eviction priorities
                         (forward solve reads the large factor sections evict-last, backward
                         solve evict-first), 2 = none */
  int autotune;       /* 1: at set-up, time one relaxation sweep with each patch-solve variant
                         (256 threads with four or eight rows per warp in the forward products,
                         512, 1024 threads, the resident kernel where it fits; in the
                         Schur-coupling form its one-CTA-per-patch shapes and the persistent
                         kernels 5 and 6, the latter where it fits) and keep the
                         fastest (FDM_Q_TUNING); 0 (default): the fixed rule (patch_threads,
                         patch_kernel).  Variants sum in different orders: results of contexts
                         tuned differently agree to rounding, not bit for bit */
  int patch_rows_per_warp; /* rows a warp keeps in flight in the forward products of the
                              one-CTA-per-patch solve: 4 or 8 (0 = 8 for 256 threads and L21
                              rows of 200 or more, else 4); L form only */
  int patch_form;     /* layout of the patch factors: 1 = L form (the Cholesky factor L_G:
                         diagonal level 0, sparse L10/L20, line blocks, dense L21, Z = L_TT^{-1});
                         2 = Schur-coupling form (y_B = S_BB^{-1} g_B, x_T = W (g_T - S_TB y_B),
                         x_B = y_B - S_BB^{-1} S_BT x_T with B = levels 0 and 1, T = the top
                         level, S_TB in S_G's own sparsity and W = (L_TT L_TT^T)^{-1}: no dense
                         L21, W read once), patch_kernel 0, 1, 5 or 6 only; 0 (default) = 2 for
                         patch_kernel 0, 1, 5 or 6, else 1 */
  int coarse_levels;  /* solve of the Q1 coarse problem (Section 3): 0 = exact (dense inverse
                         from a banded Cholesky factor); k > 0 = one geometric multigrid V-cycle
                         with at most k coarsenings (every other vertex per axis while all cell
                         counts are even and >= 4; linear interpolation in the vertex coordinates;
                         Galerkin operators P^T A P; gmg_nu damped point-Jacobi sweeps before and
                         after each coarse-grid correction; the exact solve on the coarsest level);
                         -1 (default) = exact up to 4096 Q1 unknowns, else multigrid on every level
                         the mesh allows */
  int gmg_nu;         /* Jacobi sweeps before and after the coarse-grid correction (<= 0: 2) */
  double gmg_omega;   /* Jacobi damping (<= 0: 2/3) */
  int sc_variant;     /* Schur-coupling one-CTA-per-patch solve with 256 threads: 1 (0 = default) =
                         two rows of W per warp, lower-block values and S_TB staged in shared
                         memory (five CTAs per SM); 2 = four rows of W per warp (four CTAs per SM);
                         3 = two rows, only the lower-block values staged (six CTAs per SM);
                         4 = two rows, nothing staged, the patch's whole value block prefetched
                         into L2 when its CTA starts (six CTAs per SM) */
  int tensor_core;    /* 1: the SIPG star solves of the FP32 preconditioner (and sipg_patch_solve in
                         FP32) run their six 1D contractions on the tensor cores (tcgen05.mma,
                         TF32 inputs rounded to nearest, FP32 accumulation in tensor memory); DQ_7
                         only (FDM_EINVAL at set-up otherwise); a completion wait that runs out
                         gives FDM_ETIMEOUT.  0 (default): FP32 CUDA-core contractions */
} fdm_options;

/* Fills the defaults listed above. */
int fdm_default_options(fdm_options *opt);

/* Set-up (Sections 2.3-2.6): 1D GLL basis and interior eigenbasis,
 * per-cell surrogate coefficients, vertex-star patch assembly in the FDM
 * basis, symbolic factorisation once per patch class (interface ordered by
 * nested dissection on the star's three vertex planes), FP64 numeric
 * factorisation of every patch on the device (plus an FP32 copy for the
 * FP32 preconditioner), the Galerkin Q1 coarse operator, and the damping
 * omega by CG-Lanczos on P_ASM^{-1} A (Section 2.5).  p in [1, 15].
 * Synchronises `stream`.  On success *out owns the context. */
int fdm_setup(const fdm_mesh *mesh, int p, const fdm_coeff *coeff, const fdm_options *opt,
              fdm_ctx **out, void *stream);

/* y = A u: matrix-free sum-factorised stiffness apply in FP64 (eq. (kron)
 * on box cells; Gauss quadrature with Ghat = kappa |det J| J^{-1} J^{-T} on
 * curved cells, Section 2.7).  u, y: device, ndof doubles. */
int stiffness_apply(fdm_ctx *ctx, const double *u_dev, double *y_dev, void *stream);

/* y = A u exactly as stiffness_apply, for callers that must not allocate
 * device memory when they call (for example code that runs inside a
 * memory-pool-free or allocation-forbidden section, or a runtime that owns
 * all device memory and forbids cudaMalloc after start-up).  No counterpart
 * in the paper: the method does not depend on where scratch memory lives.
 * The cell-local partial results go to a fixed 16 MiB device array of the
 * library (2^21 doubles, reserved on every GPU that loads the library until
 * the process exits) instead of the context's buffer; calls with
 * nx*ny*nz*(p+1)^3 > 2^21 are rejected with FDM_EINVAL.  This call performs
 * no cudaMalloc/cudaFree and no allocating library call.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture.  All calls share the array and
 * it keeps the last call's contents (every entry is written before it is
 * read, nothing needs clearing); calls that overlap on the GPU race on it. */
int stiffness_apply_noalloc(fdm_ctx *ctx, const double *u_dev, double *y_dev, void *stream);

/* b = M f: the mass matrix (load vector of nodal data f).  Device arrays. */
int mass_apply(fdm_ctx *ctx, const double *f_dev, double *b_dev, void *stream);

/* z = omega * P_ASM^{-1} r (Section 2.5): one additive vertex-star sweep:
 * basis change to the FDM basis, patch gather, Schur condensation, sparse
 * Cholesky forward and backward solves, interior back-substitution,
 * deterministic additive scatter, basis change back.  In the context's
 * preconditioner precision.  Device arrays. */
int asm_apply(fdm_ctx *ctx, const double *r_dev, double *z_dev, void *stream);

/* z = P^{-1} r: the context's preconditioner (V(1,1) by default). */
int pc_apply(fdm_ctx *ctx, const double *r_dev, double *z_dev, void *stream);

/* Solve information filled by pcg_solve. */
typedef struct {
  int iterations;        /* number of PCG iterations performed */
  int converged;         /* 1 if ||r||_2 <= rtol ||b||_2 was reached */
  double rnorm0;         /* ||b||_2 */
  double rnorm;          /* final recursive residual ||r_k||_2 */
  double true_rnorm;     /* ||b - A x||_2 recomputed in FP64 */
  double seconds;        /* device time of the solve (CUDA events) */
} fdm_solve_info;

/* PCG from x0 = 0 until ||r||_2 <= rtol ||b||_2 (Euclidean norm of the
 * unpreconditioned residual, Section 2.8) or maxit iterations.  FP64 dot
 * products (fixed-order reductions), FP64 vector updates and FP64 stiffness
 * apply.  b, x: device.  info (HOST, may be NULL) is filled; the call
 * synchronises `stream`.  Returns FDM_ENOCONV if maxit was reached,
 * FDM_ENAN on a non-finite scalar. */
int pcg_solve(fdm_ctx *ctx, const double *b_dev, double *x_dev, double rtol, int maxit,
              fdm_solve_info *info, void *stream);

/* ---- batched solves of independent problems ---- */
typedef struct fdm_batch fdm_batch;
/* Groups k set-up contexts (of any sizes and degrees) for one batched PCG
 * call.  The contexts stay owned by the caller and must outlive the batch. */
int fdm_batch_setup(int k, fdm_ctx *const *ctxs, fdm_batch **out);
/* The same with a schedule:
 *   FDM_BATCH_BRANCHES (fdm_batch_setup): one CUDA graph, every problem's PCG
 *     loop a branch of its own (a conditional WHILE node), its kernels at a
 *     priority ranked by problem size (smaller first);
 *   FDM_BATCH_LOCKSTEP: one device-driven loop in which every problem still
 *     iterating takes one PCG iteration per pass (its cell kernels, coarse
 *     solve and vector work in a conditional IF node of its own), and the star
 *     solves of all those problems run in one launch per relaxation sweep over
 *     a global list of (problem, patch) sorted by patch size, largest first,
 *     with one CTA per patch (the Schur-coupling form, 256 threads); a problem
 *     that has converged (true residual) or reached maxit drops out of every
 *     later launch.  Needs FP32 preconditioners with the V(1,1) cycle and the
 *     Schur-coupling form (patch_form 2, the default) in every context, else
 *     FDM_EINVAL.
 * Results of the two agree to the rounding of the star solves' kernel
 * variant, not bit for bit. */
#define FDM_BATCH_BRANCHES 0
#define FDM_BATCH_LOCKSTEP 1
int fdm_batch_setup_mode(int k, fdm_ctx *const *ctxs, int mode, fdm_batch **out);
/* Solves all k problems: b[i], x[i] device vectors of problem i; infos
 * (HOST, k entries, may be NULL).  Synchronises `stream`. */
int pcg_solve_batched(fdm_batch *batch, const double *const *b_dev, double *const *x_dev,
                      double rtol, int maxit, fdm_solve_info *infos, void *stream);
void fdm_batch_destroy(fdm_batch *batch);

/* ---- surrogate coefficients (Section 2.7) ---- */
/* Replaces the per-cell surrogate coefficients mu (HOST, 3 per cell, x,y,z
 * scalings, cells x fastest) and refactors every patch. */
int fdm_surrogate_load(fdm_ctx *ctx, const double *mu_host, void *stream);

/* ---- learned separable surrogate (Section 2.7, Theorem 1) ----
 * Not in the paper: the paper's surrogate on curved cells is the cell
 * average mu_avg of kappa Ghat_jj.  Here a network predicts a per-direction
 * correction c per cell, mu = mu_avg exp(c), from the 27 samples of
 * fdm_coeff.samples27.  Inputs (189 per cell, per sample point): log kappa
 * minus its cell average; log(M_aa / nu_a), with M = kappa Ghat and nu the
 * 27-point average of M_aa; and the correlations M_ab / sqrt(M_aa M_bb) for
 * ab = 01, 02, 12.  Network: 189 -> 64 (tanh) -> 64 (tanh) -> 3 (linear),
 * FP32 weights packed as W1[64][189], b1[64], W2[64][64], b2[64], W3[3][64],
 * b3[3] (FDM_MLP_NPARAM floats; W[out][in]).  Training label per cell (the
 * default, FDM_LABEL_THEOREM1; see fdm_surrogate_labels for the other kind):
 * c* = log(mu_opt / mu_avg) with mu_opt the scalings that minimise the ratio hi/lo
 * of Theorem 1's bound lo a~ <= a <= hi a~ (the extreme eigenvalues of
 * diag(mu)^{-1/2} M_q diag(mu)^{-1/2} over the cell's (p+1)^3 Gauss points),
 * found by the central-cut ellipsoid method on the ratio, which is convex in
 * log mu (start mu_avg, disc radius 6 in log mu, at most 600 steps, optimality
 * gap bound 1e-10), and scaled so that lo hi = 1.  Loss:
 * (1/(2 N)) sum over the N cells of |c - c*|^2.  All calls need a context set
 * up with curved cells and samples27 (else FDM_EINVAL). */
#define FDM_MLP_NPARAM 16515

/* Loss and gradient (HOST, FDM_MLP_NPARAM floats) at the weights w (HOST)
 * over the cells of ctx, computed by the library's FP32 training kernels.
 * loss (HOST, may be NULL).  Synchronises `stream`. */
int fdm_surrogate_grad(fdm_ctx *ctx, const float *w, float *grad, double *loss, void *stream);

/* Training labels.  FDM_LABEL_THEOREM1 (the default): the per-cell optimum of
 * Theorem 1's bound ratio above.  FDM_LABEL_PATCH_KAPPA: each candidate mu is
 * scored by the Lanczos estimate of kappa(A~_P(mu)^{-1} A_P) on the cell's
 * interior patch P (the functions of the cell's interior, homogeneous
 * Dirichlet on its boundary): A_P the true cell stiffness (Gauss quadrature
 * with kappa Ghat), A~_P(mu) the separable surrogate's interior block, which
 * the interior FDM basis S = S_1 (x) S_1 (x) S_1 diagonalises:
 * A~_P = S^{-T} D S^{-1}, D = mu_x lam_i + mu_y lam_j + mu_z lam_k.  The
 * estimate: min(48, (p-1)^3) steps of Lanczos with full reorthogonalisation
 * (two Gram-Schmidt passes) on D^{-1/2} S^T A_P S D^{-1/2} from
 * r0[i] = frac(i 2654435769 / 2^32) - 1/2, ended early when the next vector's
 * norm is below 1e-10 times the largest diagonal entry; the extreme
 * eigenvalues of the Lanczos matrix (bisection) estimate lambda_min,
 * lambda_max.  With mu = mu_avg exp((0, t1, t2) + gamma), (t1, t2) minimises
 * log(lambda_max / lambda_min) by compass search from 0 (step 1/2, the best
 * of the four moves +-step that lowers it by more than 1e-9 is taken, else the
 * step halves, until it is below 1/256 or after 48 rounds) and gamma =
 * log(lambda_min lambda_max) / 2 centres the labelled spectrum.  Degrees 2..8
 * (FDM_EINVAL otherwise).
 * fdm_surrogate_labels computes the labels of `kind` (once per context) and
 * selects them for this context's fdm_surrogate_grad and fdm_surrogate_train.
 * labels (HOST, 3 ncell: c per cell, may be NULL); score (HOST, 2 ncell, may
 * be NULL): per cell the label's criterion at mu_avg, then at the label
 * (THEOREM1: log(hi/lo) of the bound; PATCH_KAPPA: log(lambda_max/lambda_min)).
 * Synchronises `stream`. */
#define FDM_LABEL_THEOREM1 0
#define FDM_LABEL_PATCH_KAPPA 1
int fdm_surrogate_labels(fdm_ctx *ctx, int kind, double *labels, double *score, void *stream);

/* Trains the network on every cell of the k contexts (all on the current
 * device): `steps` full-batch Adam steps (beta1 0.9, beta2 0.999, eps 1e-8,
 * bias-corrected, step size lr, decoupled weight decay weight_decay >= 0)
 * from w_init (HOST), against each context's selected labels.  w_out (HOST) receives the weights, loss_hist (HOST,
 * steps + 1 doubles, may be NULL) the loss before each step and after the
 * last.  Device scratch is allocated and freed inside the call.
 * Synchronises `stream`. */
int fdm_surrogate_train(int k, fdm_ctx *const *ctxs, const float *w_init, int steps, double lr,
                        double weight_decay, float *w_out, double *loss_hist, void *stream);

/* Inference: mu = mu_avg exp(c) per cell with the network w (HOST); a cell
 * whose outputs are not finite or exceed 2 in magnitude keeps mu_avg.  Then
 * every patch is refactored and omega re-estimated (unless fixed).  With
 * judge = 1 the averaged surrogate judges the result: if the Lanczos
 * estimate lmax/lmin of P_ASM^{-1} A grew, mu_avg is restored (needs omega
 * not fixed).  nfallback (HOST, may be NULL): number of fallback cells;
 * kept (HOST, may be NULL): 1 if the network's scalings were kept.
 * Synchronises `stream`. */
int fdm_surrogate_apply(fdm_ctx *ctx, const float *w, int judge, int *nfallback, int *kept,
                        void *stream);

/* ---- primal linear elasticity (Section 4.1) ----
 * a(v, u) = int 2 mu eps(v):eps(u) + lambda div v div u on box cells
 * (mesh->jac must be NULL), Q_p per displacement component on the GLL grid of
 * the scalar problem, clamped (homogeneous Dirichlet) on the whole boundary.
 * Vectors are DEVICE FP64 arrays of 3 ndof doubles, component-major
 * ([component][node], nodes x fastest); Dirichlet entries are ignored on input
 * and 0 on output.
 * The preconditioner (opt->pc): FDM_PC_ASM = omega times the separate
 * displacement components (SDC) relaxation, i.e. block-Jacobi over the
 * components, each block A_jj (per-axis coefficients mu + (mu + lambda)
 * delta_aj: separable on box cells) relaxed by the vertex-star FDM/sparse
 * additive Schwarz of the scalar problem; FDM_PC_VCYCLE (default) = the hybrid
 * V(1,1) with that relaxation, the elasticity residual and the vector Q1
 * Galerkin coarse problem solved exactly.  omega from opt->lanczos_steps
 * CG-Lanczos steps on A_SDC^{-1} A (opt->lanczos_start: 3 ndof HOST doubles,
 * or N(0,1) from opt->lanczos_seed), unless opt->omega > 0.  opt->precision
 * selects the FP32 or FP64 preconditioner; PCG is FP64 (flexible beta with
 * FP32).  The patch-solve options apply to the three scalar relaxations.
 * Degrees 1..15.  Errors as for the scalar problem; fdm_elast_last_error. */
typedef struct fdm_elast fdm_elast;
int fdm_elast_setup(const fdm_mesh *mesh, int p, double mu, double lambda, const fdm_options *opt,
                    fdm_elast **out, void *stream);
/* The same, clamped only on the faces in dirichlet_faces and traction-free
 * (the natural condition) on the others, as in Sec. 4.1's tests (x_1 = 0
 * clamped: dirichlet_faces = 1): bit 2a is the face at the lower end of axis a
 * (a = 0, 1, 2 for x, y, z), bit 2a+1 the upper end; 63 = every face
 * (fdm_elast_setup).  At least one face is clamped (1..63), so that A is
 * positive definite.  The nodes on traction-free faces are unknowns; the star
 * of a vertex holds the free nodes within p - 1 of it along each axis (on a
 * traction-free face its boundary nodes), and the Q1 coarse space has every
 * vertex off the clamped faces.  sdc_form selects how the SDC blocks' star systems are
 * solved (both exact, so both give the same relaxation up to rounding):
 *   FDM_SDC_FDM_SPARSE  the scalar problem's vertex-star FDM/sparse relaxation
 *                       (every face clamped only);
 *   FDM_SDC_STAR_FDM    the star-local fast diagonalisation: block j's star
 *                       matrix is the Kronecker sum sum_a c_a A_a (x) M_b (x) M_c
 *                       of the star's 1D stiffness and mass (c_a = mu + (mu +
 *                       lambda) delta_aj), inverted as (S (x) S (x) S) D^{-1}
 *                       (S (x) S (x) S)^T with the 1D generalised eigenvectors;
 *                       stars up to 29 nodes per axis in shared memory;
 *   FDM_SDC_AUTO        FDM/sparse with every face clamped, else star FDM.
 * FDM_EINVAL for a mask or form outside these. */
#define FDM_SDC_AUTO 0
#define FDM_SDC_FDM_SPARSE 1
#define FDM_SDC_STAR_FDM 2
int fdm_elast_setup_bc(const fdm_mesh *mesh, int p, double mu, double lambda, int dirichlet_faces, int sdc_form,
                       const fdm_options *opt, fdm_elast **out, void *stream);
/* y = A u */
int elast_apply(fdm_elast *e, const double *u_dev, double *y_dev, void *stream);
/* z = P^{-1} r (the preconditioner selected by opt->pc) */
int elast_pc_apply(fdm_elast *e, const double *r_dev, double *z_dev, void *stream);
/* PCG from x = 0 to ||r||_2 <= rtol ||b||_2 (as pcg_solve, host-driven loop) */
int elast_pcg_solve(fdm_elast *e, const double *b_dev, double *x_dev, double rtol, int maxit,
                    fdm_solve_info *info, void *stream);
/* FDM_Q_NDOF (int64, nodes per component), FDM_Q_OMEGA, FDM_Q_LAMBDA, FDM_Q_LAUNCHES,
 * FDM_Q_RECURSIVE_ITS */
int fdm_elast_query(fdm_elast *e, int what, void *out, size_t *len);
const char *fdm_elast_last_error(const fdm_elast *e);
void fdm_elast_destroy(fdm_elast *e);

/* ---- symmetric interior penalty DG, DQ_p (Section 5) ----
 * The Poisson equation -div grad u = f discretised by SIPG on the DQ_p space
 * of GLL Lagrange nodal functions: box cells only (mesh->jac NULL), at least
 * 2 cells per axis, 1 <= p <= 10, homogeneous Dirichlet condition imposed
 * weakly on the whole boundary.  Vectors are cell-major: value (i, j, k) of
 * cell (cx, cy, cz) at ((cx + nx (cy + ny cz)) (p+1) + k) (p+1)^2 + j (p+1) + i,
 * ndof = nx ny nz (p+1)^3 doubles (DEVICE).  The operator is
 *   a(v, u) = sum_K int_K grad v.grad u + sum_e int_e eta h_e^{-1} [v].[u]
 *             - [v].{grad u} - {grad v}.[u]   (interior facets and boundary),
 * h_e^{-1} = |e| {|K|^{-1}}, eta > 0 (eta <= 0 selects the default p (p+1)).
 * Relaxation: additive Schwarz over the vertex stars of the interior vertices
 * ((2p+2)^3 values each, exact solves: on a Cartesian star the star matrix is
 * a Kronecker sum of 1D two-cell pencils and is inverted by their
 * eigendecompositions); coarse space: the conforming Q1 functions vanishing
 * on the boundary (Galerkin operator: the Q1 stiffness, solved as for the
 * conforming problem: opt->coarse_levels); preconditioner selected by
 * opt->pc (FDM_PC_ASM: omega ASM; FDM_PC_VCYCLE: the hybrid V(1,1)) in
 * opt->precision; omega from opt->lanczos_steps CG-Lanczos steps on
 * ASM^{-1} A unless opt->omega > 0.  A relaxation sweep solves every star in
 * one launch into a per-star buffer ((2p+2)^3 values per star, allocated on
 * first use) and sums each value over the stars holding it in a fixed corner
 * order (default), or with opt->patch_kernel = 1 in eight launches, one per
 * vertex parity class, that add into z; opt->tensor_core = 1 moves the star
 * solves' contractions to the tensor cores (DQ_7, FP32 preconditioner).
 * Errors as for the scalar problem (FDM_ENOTSPD if a star pencil is not
 * positive definite: eta too small; FDM_ETIMEOUT from sipg_pcg_solve when a
 * bounded wait of the tensor-core star solve ran out, FDM_Q_STATUS reads and
 * clears that flag); fdm_sipg_last_error. */
typedef struct fdm_sipg fdm_sipg;
int fdm_sipg_setup(const fdm_mesh *mesh, int p, double eta, const fdm_options *opt, fdm_sipg **out, void *stream);
/* y = A u */
int sipg_apply(fdm_sipg *s, const double *u_dev, double *y_dev, void *stream);
/* z = omega sum_v R_v^T A_v^{-1} R_v r (the 8 vertex parity classes, each one launch, in a fixed order) */
int sipg_asm_apply(fdm_sipg *s, const double *r_dev, double *z_dev, void *stream);
/* z = P^{-1} r (the preconditioner selected by opt->pc) */
int sipg_pc_apply(fdm_sipg *s, const double *r_dev, double *z_dev, void *stream);
/* for nv interior vertices (HOST list, index vx + (nx+1) (vy + (ny+1) vz)),
 * out[k][(2p+2)^3] = A_v^{-1} R_v r in star order [Z][Y][X], X = a (p+1) + i
 * for the cell at x offset a (0, 1) around the vertex (the same for Y, Z);
 * FDM_EINVAL for a vertex that is not interior; synchronises the stream */
int sipg_patch_solve(fdm_sipg *s, const double *r_dev, int nv, const int *vertices, double *out_dev, void *stream);
/* PCG from x = 0 to ||r||_2 <= rtol ||b||_2 (host-driven loop) */
int sipg_pcg_solve(fdm_sipg *s, const double *b_dev, double *x_dev, double rtol, int maxit, fdm_solve_info *info,
                   void *stream);
/* FDM_Q_NDOF (int64), FDM_Q_OMEGA, FDM_Q_LAMBDA, FDM_Q_LAUNCHES, FDM_Q_NPATCH (int32: stars) */
int fdm_sipg_query(fdm_sipg *s, int what, void *out, size_t *len);
const char *fdm_sipg_last_error(const fdm_sipg *s);
void fdm_sipg_destroy(fdm_sipg *s);

/* ---- general hexahedral meshes: host topology (no CUDA call) ----
 * The vertex-star relaxation on an unstructured conforming hexahedral mesh
 * (Sections 2.4 and 2.6 on the general meshes of the Section 3 experiments)
 * needs, besides the cell kernels, a node numbering that neighbouring cells of
 * any orientation share, the vertex stars in FDM order, the signed map from
 * each cell's tensor-product FDM functions to the global ones, and each star's
 * sparsity pattern.  fdm_hexmesh_create builds them on the host from
 * cells[nc][8] (HOST; vertex ids in [0, nv) at the corners (a, b, c) of the
 * reference cube, index a + 2 b + 4 c) for degree 1 <= p <= 15.  Numbering:
 * one node per used vertex (by vertex id), then (p-1) per edge (from its
 * lower-id vertex), (p-1)^2 per face (frame at its lowest-id corner, first
 * axis towards the lower-id neighbouring corner), (p-1)^3 per cell (cell-local
 * lexicographic); the FDM functions use the same slots (eigen-index m - 1 on
 * an edge or face axis), with a sign -1 where a cell sees an odd interior
 * function reversed.  Dirichlet nodes: the closure of the faces of one cell.
 * Stars: every used vertex with at least one free node; its FDM functions
 * in canonical order (the star's cells walked from the start cell and edge
 * labelling with the smallest encoding of their shared faces and edges, so
 * that equal configurations get equal orders in any cell orientation): cell
 * interiors first, then the interface (faces, edges, the vertex) entity by
 * entity in minimum-degree order of the interface Schur complement's
 * pattern; the pattern of
 * its separable surrogate matrix in the FDM basis as CSR over star positions
 * (its interior block is diagonal, Section 2.6).  Stars with equal patterns
 * form a class, which shares the symbolic Cholesky factorisation (elimination
 * tree and fill) of the interface Schur complement (Section 2.6, eq. LDLT).
 * FDM_EINVAL for a vertex id out of range, a degenerate cell, a face of more
 * than two cells or more than 2^31 - 1 nodes; fdm_hexmesh_last_error. */
typedef struct fdm_hexmesh fdm_hexmesh;
int fdm_hexmesh_create(int nv, int nc, const int *cells, int p, fdm_hexmesh **out);
/* The same with a natural (homogeneous Neumann, traction-free) condition on
 * part of the boundary (Sec. 4.1's clamped face with the others free):
 * dirichlet_vertex[nv] (HOST) marks vertices; a boundary face is Dirichlet when
 * its 4 corner vertices are marked (the closure of the Dirichlet faces holds
 * the Dirichlet nodes), the other boundary faces are natural, so the stars of
 * vertices on them keep their boundary nodes, and the Q1 coarse space keeps
 * their vertices.  NULL: every boundary face is Dirichlet (fdm_hexmesh_create). */
int fdm_hexmesh_create_bc(int nv, int nc, const int *cells, int p, const unsigned char *dirichlet_vertex,
                          fdm_hexmesh **out);
#define FDM_HQ_NNODE 1          /* int64: number of nodes */
#define FDM_HQ_CELL_NODES 2     /* int32[nc][(p+1)^3]: node of each cell-local GLL node (i + n (j + n k)) */
#define FDM_HQ_CELL_FDM 3       /* int32[nc][(p+1)^3]: global FDM function of each cell-local FDM function */
#define FDM_HQ_CELL_SIGN 4      /* int8[nc][(p+1)^3]: its sign (+1 or -1) */
#define FDM_HQ_DIRICHLET 5      /* uint8[nnode]: 1 on Dirichlet nodes */
#define FDM_HQ_NSTAR 6          /* int32: number of stars */
#define FDM_HQ_STAR_VERTEX 7    /* int32[nstar]: the vertex of each star */
#define FDM_HQ_STAR_PTR 8       /* int64[nstar + 1]: offsets into FDM_HQ_STAR_NODES */
#define FDM_HQ_STAR_NODES 9     /* int32[...]: each star's nodes in star order */
#define FDM_HQ_PATTERN_PTR 10   /* int64[nstar + 1]: offsets into FDM_HQ_PATTERN_ROWPTR (star size + 1 each) */
#define FDM_HQ_PATTERN_ROWPTR 11 /* int64[...]: per star, CSR row pointers starting at 0 */
#define FDM_HQ_PATTERN_COLPTR 12 /* int64[nstar + 1]: offsets into FDM_HQ_PATTERN_COLS */
#define FDM_HQ_PATTERN_COLS 13  /* int32[...]: per star, CSR column positions (sorted per row) */
#define FDM_HQ_STAR_NINT 14     /* int32[nstar]: cell-interior functions of each star (its first positions) */
#define FDM_HQ_STAR_CLASS 15    /* int32[nstar]: sparsity class (equal pattern and interior count) */
#define FDM_HQ_NCLASS 16        /* int32: number of classes */
#define FDM_HQ_CLASS_STAR 17    /* int32[nclass]: the first star of each class */
#define FDM_HQ_CLASS_NNZL 18    /* int64[nclass]: nonzeros of the Cholesky factor L of the class's
                                 * interface Schur complement S_G = A_GG - A_GI D^{-1} A_IG
                                 * (interface positions in star order, diagonal included) */
#define FDM_HQ_FILL_PTR 19      /* int64[nclass + 1]: offsets into FDM_HQ_FILL_ROWPTR (interface size + 1 each) */
#define FDM_HQ_FILL_ROWPTR 20   /* int64[...]: per class, CSR row pointers of L starting at 0 */
#define FDM_HQ_FILL_COLPTR 21   /* int64[nclass + 1]: offsets into FDM_HQ_FILL_COLS */
#define FDM_HQ_FILL_COLS 22     /* int32[...]: per class, the columns of each row of L (sorted) */
#define FDM_HQ_ETREE_PTR 23     /* int64[nclass + 1]: offsets into FDM_HQ_ETREE */
#define FDM_HQ_ETREE 24         /* int32[...]: per class, the elimination-tree parent of each
                                 * interface column (-1 for a root) */
#define FDM_HQ_MU 25            /* double[nc][3]: averaged surrogate coefficients (after fdm_hexmesh_factor) */
#define FDM_HQ_DIAG_PTR 26      /* int64[nstar + 1]: offsets into FDM_HQ_DIAG */
#define FDM_HQ_DIAG 27          /* double[...]: per star, the diagonal interior block D of its surrogate matrix */
#define FDM_HQ_FACTOR_PTR 28    /* int64[nstar + 1]: offsets into FDM_HQ_FACTOR */
#define FDM_HQ_FACTOR 29        /* double[...]: per star, L of S_G (S_G = L L^T) in its class's fill
                                 * pattern, row by row (FDM_HQ_FILL_*) */
#define FDM_HQ_SLOT_CELLS_PTR 30 /* int64[nnode + 1]: offsets into FDM_HQ_SLOT_CELLS */
#define FDM_HQ_SLOT_CELLS 31    /* int32[nc (p+1)^3]: per FDM slot, e (p+1)^3 + c of every cell-local
                                 * FDM function mapped to it (by cell): the assembly of the global FDM
                                 * residual from the cells' ones */
#define FDM_HQ_SLOT_STARS_PTR 32 /* int64[nnode + 1]: offsets (in pairs) into FDM_HQ_SLOT_STARS */
#define FDM_HQ_SLOT_STARS 33    /* int32[2 ...]: per FDM slot, the (star, position) pairs holding it (by star):
                                 * the sum of the star solutions */
#define FDM_HQ_NODE_OWNER 34    /* int32[nnode]: e (p+1)^3 + l of the lowest cell holding each node */
#define FDM_HQ_NODE_CELLS_PTR 35 /* int64[nnode + 1]: offsets into FDM_HQ_NODE_CELLS */
#define FDM_HQ_NODE_CELLS 36    /* int32[nc (p+1)^3]: per node, e (p+1)^3 + l of every cell-local copy (by cell):
                                 * the deterministic sum of the cells' operator results */
#define FDM_HQ_GEOM 37          /* double[nc][(p+1)^3][6] (after fdm_hexmesh_factor): w_q kappa |det J| J^{-1} J^{-T}
                                 * at the Gauss points (x fastest), entries xx, yy, zz, xy, xz, yz: the
                                 * stiffness a(v, u) = sum_K sum_q grad_xi v^T G grad_xi u */
#define FDM_HQ_COARSE_OF 38     /* int32[nv]: coarse unknown of each vertex, -1 on boundary faces or unused */
#define FDM_HQ_COARSE 39        /* double[nco][nco] (after fdm_hexmesh_factor): the Q1 Galerkin operator
                                 * P^T A P, P the Q1 functions of the coarse vertices in Q_p */
#define FDM_HQ_SC_SPLIT 40      /* int32[nclass]: size t of the top block T of the Schur-coupling form (the
                                 * last t interface positions, whole entities, chosen to minimise the stored
                                 * values nnz(L_BB) + nnz(S_TB) + t (t + 1) / 2) */
#define FDM_HQ_SC_PTR 41        /* int64[nclass + 1]: offsets into FDM_HQ_SC_ROWPTR */
#define FDM_HQ_SC_ROWPTR 42     /* int64[...]: per class, the row pointers of L_BB (nB + 1, from 0) and of
                                 * S_TB (t + 1, from 0); nB = interface size - t */
#define FDM_HQ_SC_COLPTR 43     /* int64[nclass + 1]: offsets into FDM_HQ_SC_COLS */
#define FDM_HQ_SC_COLS 44       /* int32[...]: per class, L_BB's columns then S_TB's (B positions) */
#define FDM_HQ_SC_VALUES_PTR 45 /* int64[nstar + 1]: offsets into FDM_HQ_SC_VALUES */
#define FDM_HQ_SC_VALUES 46     /* double[...] (after fdm_hexmesh_factor): per star, the values of L_BB
                                 * (S_BB = L_BB L_BB^T), of S_TB, and the lower triangle of
                                 * W = (S_TT - S_TB S_BB^{-1} S_BT)^{-1} row by row: the star's interface
                                 * solve is y_B = S_BB^{-1} g_B, x_T = W (g_T - S_TB y_B),
                                 * x_B = y_B - S_BB^{-1} S_BT x_T */
/* Numeric set-up on the host, FP64 (Sections 2.6-2.7): X[nv][3] (HOST) the
 * vertex coordinates, kappa_q NULL or the coefficient at the (p+1)^3 Gauss
 * points of every cell (x fastest).  Per cell the averaged surrogate mu_d =
 * (1/8) sum_q w_q G_dd, G = kappa |det J| J^{-1} J^{-T} of the trilinear map;
 * the geometry factors of the stiffness at the Gauss points (FDM_HQ_GEOM);
 * the Q1 coarse operator (FDM_HQ_COARSE, the Q1 stiffness of the same
 * quadrature, which is P^T A P since the trilinear functions lie in Q_p);
 * per star its surrogate matrix in the FDM basis (sum over its cells of
 * sum_d mu_d (A_f along axis d, B_f along the others), with the map's
 * signs), the interior pivots D and the Cholesky factor of the interface
 * Schur complement in the class's fill.  FDM_ENOTSPD for a pivot <= 0,
 * FDM_EINVAL for degenerate geometry or nv other than at creation. */
int fdm_hexmesh_factor(fdm_hexmesh *h, int nv, const double *X, const double *kappa_q);
/* The same for the coefficient kappa_q diag(kaxes) (HOST, 3 positive values:
 * a constant diagonal tensor in physical axes, e.g. the SDC blocks of
 * Sec. 4.1, mu + (mu + lam) delta_aj): G = kappa |det J| J^{-1} diag(kaxes) J^{-T}.
 * kaxes NULL: fdm_hexmesh_factor.  FDM_EINVAL for a value <= 0. */
int fdm_hexmesh_factor_axes(fdm_hexmesh *h, int nv, const double *X, const double *kappa_q, const double *kaxes);
/* Copies `what` into out (HOST); *len is the capacity in bytes on input and
 * the size written on output (out NULL: the size only). */
int fdm_hexmesh_query(fdm_hexmesh *h, int what, void *out, size_t *len);
const char *fdm_hexmesh_last_error(const fdm_hexmesh *h);
void fdm_hexmesh_destroy(fdm_hexmesh *h);

/* ---------------------------------------------------------------------------
 * General hexahedral meshes on the GPU (Sections 2.4-2.8 on the meshes of the
 * unstructured experiments, Sec. 3 and Table 1): a device context built from
 * an fdm_hexmesh after fdm_hexmesh_factor.  Vectors are FP64 DEVICE arrays of
 * nnode values in the hexmesh's node numbering (FDM_HQ_NNODE), caller-owned;
 * Dirichlet entries are ignored on input and written as 0 on output.
 *   hex_stiffness_apply: y = A u, the Gauss-quadrature stiffness with the
 *     geometry factors FDM_HQ_GEOM, summed per node over its cells in cell order;
 *   hex_asm_apply: one damped sweep z = omega sum_v R_v^T A~_v^{-1} R_v r of the
 *     vertex-star relaxation with the averaged surrogate (Sec. 2.7) in the glued
 *     FDM basis: per-cell basis change and Schur condensation, exact interface
 *     solves, per-cell back-substitution and basis change back; in opt.precision.
 *     The interface solve uses the dense inverse of each star's interface Schur
 *     complement (lower triangle, formed at set-up from its Cholesky factor;
 *     default) or, with opt.patch_form = 2, the Schur-coupling form (FDM_HQ_SC_*)
 *     with level-scheduled sparse solves with L_BB;
 *   hex_pc_apply: the hybrid V(1,1) with the Q1 coarse space (dense inverse of
 *     FDM_HQ_COARSE), or opt.pc = FDM_PC_ASM / FDM_PC_NONE;
 *   hex_pcg_solve: PCG from x = 0 to ||b - A x|| <= rtol ||b|| (FP64), as pcg_solve.
 * omega: opt.omega if > 0, else 2 / (1.25 lmax + 0.75 lmin) from
 * opt.lanczos_steps CG-Lanczos steps on ASM^{-1} A from opt.lanczos_start (HOST,
 * nnode values) or a seeded normal vector.  fdm_hex_setup copies what it needs
 * (the hexmesh may be destroyed afterwards); it returns FDM_EINVAL for a mesh
 * without its numeric set-up, FDM_ENOTSPD for a coarse operator that is not
 * positive definite, FDM_ENOMEM when device memory runs out.  The calls are
 * stream-ordered; hex_pcg_solve synchronises to read its scalars. */
typedef struct fdm_hexgpu fdm_hexgpu;
int fdm_hex_setup(const fdm_hexmesh *h, const fdm_options *opt, fdm_hexgpu **out, void *stream);
int hex_stiffness_apply(fdm_hexgpu *ctx, const double *u_dev, double *y_dev, void *stream);
int hex_asm_apply(fdm_hexgpu *ctx, const double *r_dev, double *z_dev, void *stream);
int hex_pc_apply(fdm_hexgpu *ctx, const double *r_dev, double *z_dev, void *stream);
int hex_pcg_solve(fdm_hexgpu *ctx, const double *b_dev, double *x_dev, double rtol, int maxit,
                  fdm_solve_info *info, void *stream);
#define FDM_XQ_NNODE 1       /* int64: nodes */
#define FDM_XQ_OMEGA 2       /* double: damping */
#define FDM_XQ_LAMBDA 3      /* double[2]: Lanczos lambda_min, lambda_max (0 with opt.omega given) */
#define FDM_XQ_LAUNCHES 4    /* int64: kernels launched since the last query */
#define FDM_XQ_SIZES 5       /* int64[6]: cells, stars, star interface values, stored factor values,
                                coarse unknowns, largest star interface */
#define FDM_XQ_ALGO_BYTES 6  /* double[2]: bytes of one relaxation sweep moved once (FP64, FP32 factors):
                                the stored factor values, twice the cell-local residual, the slot values
                                and star solutions, the surrogate, the per-cell maps, r in and z out */
/* Copies `what` into out (HOST); *len is the capacity in bytes on input and
 * the size written on output. */
int fdm_hex_query(fdm_hexgpu *ctx, int what, void *out, size_t *len);
const char *fdm_hex_last_error(const fdm_hexgpu *ctx);
void fdm_hex_destroy(fdm_hexgpu *ctx);

/* ---- introspection ---- */
#define FDM_Q_NDOF 1         /* int64: number of grid nodes */
#define FDM_Q_OMEGA 2        /* double: damping */
#define FDM_Q_LAMBDA 3       /* double[2]: Lanczos lambda_min, lambda_max */
#define FDM_Q_MU 4           /* double[3*ncell]: surrogate coefficients */
#define FDM_Q_NPATCH 5       /* int32: number of vertex-star patches */
#define FDM_Q_PATCH_CLASS 6  /* int32[npatch]: class (0..7) of each patch */
#define FDM_Q_CLASS_INFO 7   /* int32[8*8]: per class nd, nI, nG, n0, n1, n2, nlines, nnzL */
#define FDM_Q_GAMMA_ORDER 8  /* int32[...]: per class, star-local index of each interface dof in factor order */
#define FDM_Q_FACTOR_NNZ 9   /* int64: total structurally nonzero entries of all L_Gamma */
#define FDM_Q_PATTERN 10     /* uint8[nG*nG] of class `arg` (in: *(int*)out): pattern of L_Gamma */
#define FDM_Q_FACTOR 11      /* double[nG*nG] of patch `arg` (in: *(int*)out): dense L_Gamma (FP64) */
#define FDM_Q_BASIS 12       /* double[5 (p+1)^2]: A_hat, B_hat, T, Af, Bf */
#define FDM_Q_FACTOR_BYTES 13 /* int64[2]: bytes of the FP64 and FP32 factor value arrays */
#define FDM_Q_SETUP_SECONDS 14 /* double[4]: symbolic, numeric factor, coarse, Lanczos seconds */
#define FDM_Q_KERNEL_TIMES 15  /* double[2*FDM_NTIMER]: per timer (launch count, total ms) since the
                                  last query; needs opt.kernel_timing; synchronises the device */
#define FDM_Q_LAUNCHES 16      /* int64: kernels launched by this context since the last query */
#define FDM_Q_ALGO_BYTES 17    /* double[4]: algorithmic bytes of one patch-solve launch (FP64, FP32),
                                  and of one asm_apply (FP64, FP32) */
#define FDM_Q_STATUS 18        /* int32: device status word (1 = a bounded wait ran out); reading
                                  it clears it; synchronises the device */
#define FDM_Q_SURR_FEATURES 19 /* float[189*ncell]: network inputs */
#define FDM_Q_SURR_LABELS 20   /* double[3*ncell]: labels c* (computed on first use) */
#define FDM_Q_SURR_BOUNDS 21   /* double[3*ncell]: per cell log(hi/lo) of Theorem 1's bound at mu_avg,
                                  at mu* (NaN without samples27) and at the current mu */
#define FDM_Q_MUBAR 22         /* double[3*ncell]: averaged surrogate mu_avg (curved cells) */
#define FDM_Q_SURR_OUTPUT 23   /* float[3*ncell]: network outputs c of the last fdm_surrogate_apply */
#define FDM_Q_TUNING 24        /* double[8]: autotuner choice: patch kernel (L form: 1 one CTA per
                                  patch, 3 resident; Schur-coupling form: 5 one CTA per patch,
                                  6 persistent, 7 fully staged persistent, 8 one warp per patch),
                                  threads, rows-per-warp variant, sweep time (us), candidates
                                  timed; zeros without autotune */
#define FDM_Q_GMG_LEVELS 25    /* int32[1 + 4 (L+1)]: coarsenings L of the Q1 multigrid (0 = exact
                                  coarse solve), then per level cells nx, ny, nz and unknowns nf */
#define FDM_Q_GMG_STENCIL 26   /* double[sum of 27 nf]: each level's 27-point operator, level by
                                  level, coefficient-major [27][nf] with offset
                                  k = (dx+1) + 3 (dy+1) + 9 (dz+1) (unknowns lexicographic in
                                  the free vertices, x fastest) */
#define FDM_Q_ALGO_BYTES_LFORM 27 /* double[2]: FDM_Q_ALGO_BYTES' patch-solve bytes (FP64, FP32) of the L
                                     form, whichever form the context uses */
#define FDM_Q_RECURSIVE_ITS 28  /* int32[2] (fdm_elast_query): for the last elast_pcg_solve, the iteration
                                   at which the recursive residual first met the test (-1: never) and
                                   the number of true-residual checks that did not */
/* timers of FDM_Q_KERNEL_TIMES */
#define FDM_T_RESTRICT 0  /* basis change to the FDM basis */
#define FDM_T_PATCH 1     /* patch gather + condense + triangular solves + back-substitution */
#define FDM_T_INTERP 2    /* scatter + basis change back */
#define FDM_T_OP64 3      /* FP64 stiffness apply (2 kernels) */
#define FDM_T_OP32 4      /* FP32 stiffness apply inside the preconditioner */
#define FDM_T_COARSE 5    /* coarse restriction + dense solve + prolongation */
#define FDM_T_VEC 6       /* PCG dot products and vector updates */
#define FDM_NTIMER 7
/* Copies the quantity `what` into out (HOST); *len is the capacity in bytes
 * on input and the size written on output. */
int fdm_query(fdm_ctx *ctx, int what, void *out, size_t *len);

const char *fdm_last_error(const fdm_ctx *ctx);
void fdm_destroy(fdm_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Box partition of the structured mesh over ranks (host only, no GPU): the
 * layout of a sharded solve.  The path's sums over cells are the direct
 * stiffness summation of the cell operators (Section 2.2) and the additive
 * Schwarz sum of the star solutions (Section 2.5); split over ranks, each node
 * on a box face, edge or corner takes contributions from cells of several
 * ranks.  Ranks form a px x py x pz grid (rank = rx + px (ry + py rz)); rank r
 * owns the cells [c0, c1) per axis of a balanced split, c0 = floor(r n / P),
 * and holds the nodes [c0 p, c1 p] of its cells (its node box, x fastest).
 * Per-cell contributions of the owned cells are laid out E[local cell][(p+1)^3]
 * (local cells x fastest within the box, nodes x fastest within a cell).
 *   send lists: per neighbour (a rank whose node box meets this one, ascending
 *     rank), the local E indices of this rank's contributions at the shared
 *     nodes (nodes in ascending global index, then cells in ascending global
 *     index); the neighbour receives them in that order;
 *   receive buffer: the neighbours' messages concatenated in neighbour order
 *     (FDM_PQ_RECV_PTR gives the offsets);
 *   sum plan: per node of the node box, its contributions in ascending global
 *     cell index, each >= 0 (local E index) or < 0 (-1 - receive-buffer slot).
 * Summing the plan in order from 0 gives the single-domain node gather's sum
 * (ascending global cell index) bit for bit.  Node ownership (FDM_PQ_OWNED):
 * the box whose half-open cell range holds the node's lower cell along every
 * axis (the last box for the upper boundary): each node has one owner, which
 * takes it in dot products.  A vertex star belongs to its vertex's owner
 * (FDM_PQ_STARS, global vertex indices x fastest); its cells lie in the owner's
 * cells plus a one-cell halo (FDM_PQ_HALO_BOX).
 * fdm_partition_create: FDM_EINVAL unless 1 <= p <= 15, 1 <= px <= nx (same for
 * y, z) and 0 <= rank < px py pz.  The handle owns host memory only. */
typedef struct fdm_partition fdm_partition;
int fdm_partition_create(int nx, int ny, int nz, int p, int px, int py, int pz, int rank, fdm_partition **out);
#define FDM_PQ_CELL_BOX 1   /* int32[6]: owned cells [c0, c1) along x, y, z */
#define FDM_PQ_NODE_BOX 2   /* int32[6]: node box [g0, g1] (inclusive) along x, y, z */
#define FDM_PQ_HALO_BOX 3   /* int32[6]: owned cells plus a one-cell halo, [c0, c1) clamped to the mesh */
#define FDM_PQ_NNEIGH 4     /* int32: number of neighbours */
#define FDM_PQ_NEIGHBORS 5  /* int32[nneigh]: neighbour ranks, ascending */
#define FDM_PQ_SEND_PTR 6   /* int64[nneigh + 1]: offsets of the send lists */
#define FDM_PQ_SEND 7       /* int64[]: local E indices to send, concatenated over neighbours */
#define FDM_PQ_RECV_PTR 8   /* int64[nneigh + 1]: offsets of each neighbour's message in the receive buffer */
#define FDM_PQ_SUM_PTR 9    /* int64[nodes + 1]: offsets of each node's sum plan */
#define FDM_PQ_SUM 10       /* int64[]: sum plans (>= 0 local E index, < 0: -1 - receive slot) */
#define FDM_PQ_OWNED 11     /* uint8[nodes]: 1 where this rank owns the node */
#define FDM_PQ_STARS 12     /* int64[]: global indices of the vertices whose stars this rank owns */
/* Copies the quantity into out (HOST); *len is the capacity in bytes on input
 * and the size written (or, on FDM_EINVAL for a small buffer, needed) on output. */
int fdm_partition_query(const fdm_partition *part, int what, void *out, size_t *len);
const char *fdm_partition_last_error(void);
void fdm_partition_destroy(fdm_partition *part);

#ifdef __cplusplus
}
#endif
#endif
