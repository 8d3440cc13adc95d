/*
 * oracle.h -- plain FP64 CPU reference of the sparse vertex-star relaxation
 * (Brubeck & Farrell, "A scalable and robust vertex-star relaxation for
 * high-order FEM", arXiv 2107.14758).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link or call
 * this library: only the test suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or table with the CUDA
 * library; it is written to be slow and obviously correct.
 *
 * Conventions (all functions):
 *   - p >= 1 is the polynomial degree, n = p + 1 GLL points per direction.
 *   - The mesh is a structured nx x ny x nz hexahedral mesh.  Vertex
 *     coordinates per axis are given (tensor-product "box" cells), and
 *     optionally a Jacobian per Gauss point for curved cells.
 *   - Vectors are full-grid GLL nodal arrays of length
 *     (nx p + 1)(ny p + 1)(nz p + 1), x fastest.  Entries on the Dirichlet
 *     boundary are ignored on input and written as 0 on output (Section 2.1,
 *     homogeneous Dirichlet data).
 *   - Vertex-star patches are numbered by mesh vertex, x fastest.
 *   - Every function returning int returns 0 on success, a negative value on
 *     error (message in or_last_error()).
 *
 * Parity unpinned: none (every function is pinned by a test against closed
 * forms, brute-force dense solves or invariants; see tests/test_oracle_*.py).
 */
#ifndef FDM_ORACLE_H
#define FDM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

#define OR_PMAX 31

/* ---- 1D building blocks (Section 2.1, eq. for l_j; Section 2.3 eq:eig;
 *      Section 2.4 FDM basis) ------------------------------------------- */

/* Gauss-Legendre rule with q points on [-1,1] (ascending). */
int or_gauss(int q, double *x, double *w);
/* Gauss-Lobatto-Legendre nodes (roots of (1-x^2) P'_p) and weights. */
int or_gll(int p, double *xi, double *w);
/* Lagrange basis on the nodes xi[0..p] evaluated at m points:
 * V[t*(p+1)+j] = l_j(x_t), D[t*(p+1)+j] = l_j'(x_t). */
void or_lagrange(int p, const double *xi, int m, const double *x, double *V, double *D);
/* Reference 1D stiffness A and mass B in the GLL Lagrange basis ((p+1)^2,
 * row-major), interior generalised eigenpairs (S: (p-1)^2 row-major,
 * S[i*(p-1)+j] = value of eigenvector j at interior node i+1; lam ascending),
 * the basis change T ((p+1)^2, u_gll = T u_fdm) and the FDM-basis matrices
 * Af = T^T A T, Bf = T^T B T with their structural zeros set to 0 after
 * checking that they are below 1e-12 relative.  Any output may be NULL. */
int or_basis1d(int p, double *xi, double *A, double *B, double *S, double *lam,
               double *T, double *Af, double *Bf);

/* ---- problem context ------------------------------------------------ */
typedef struct or_ctx or_ctx;

/* Create a problem.  xv/yv/zv: nx+1, ny+1, nz+1 vertex coordinates.
 * jac: NULL for box cells; else J = dx/dxhat (row-major 3x3) at the
 *   (p+1)^3 Gauss-Legendre points of every cell (points x fastest), cells x
 *   fastest: 9*(p+1)^3*nx*ny*nz doubles.
 * kappa: NULL for kappa = 1; else kappa at the same points.
 * The stiffness uses a(v,u) = int kappa grad v . grad u with Gauss-Legendre
 * quadrature of p+1 points per direction (exact on box cells, where the
 * Kronecker form of eq. (kron) is used instead). */
or_ctx *or_create(int p, int nx, int ny, int nz, const double *xv, const double *yv,
                  const double *zv, const double *jac, const double *kappa);
void or_free(or_ctx *c);
const char *or_last_error(void);
long or_ndof(const or_ctx *c);
int or_npatch(const or_ctx *c);

/* Per-cell separable surrogate coefficients mu (3 per cell, x,y,z).  Box
 * cells: mu_j = prod_i L_i / L_j^2 (Section 2.2); curved cells: cell average
 * of kappa*Ghat_jj (Section 2.7).  get copies out, set overrides (e.g. with
 * learned values). */
void or_get_mu(const or_ctx *c, double *mu);
void or_set_mu(or_ctx *c, const double *mu);

/* y = A u (FP64), matrix-free, Dirichlet rows/cols removed. */
void or_stiffness_apply(const or_ctx *c, const double *u, double *y);
/* b = M f (mass matrix, same quadrature), Dirichlet rows removed. */
void or_mass_apply(const or_ctx *c, const double *f, double *b);

/* Patch set-up: assemble every vertex-star patch matrix in the FDM basis
 * from mu, form the interface Schur complement and its dense Cholesky
 * factor (Section 2.6, eq:LDLT).  vertices = NULL: all vertices; else the
 * listed vertex ids only (patch solves are then available for those only).
 * nthreads <= 0: OpenMP default. */
int or_setup_patches(or_ctx *c, const int *vertices, int nvert, int nthreads);
/* Star of a vertex: number of dofs and their global grid indices in the
 * oracle's order (lexicographic over the star box, x fastest), plus the
 * number of cell-interior dofs.  gidx may be NULL. */
int or_patch_dofs(const or_ctx *c, int vertex, int *nd, int *nI, long *gidx);
/* Dense patch matrix A_j in the FDM basis (nd x nd, oracle order). */
int or_patch_matrix(const or_ctx *c, int vertex, double *Aj);
/* Interface Schur complement S_G (nG x nG, oracle Gamma order = the
 * interface dofs in star order) -- requires or_setup_patches. */
int or_patch_schur(const or_ctx *c, int vertex, double *S);
/* x = A_j^{-1} r on the star (FDM basis, oracle order). */
int or_patch_solve(const or_ctx *c, int vertex, const double *r, double *x);
/* Dense Cholesky S = L L^T of a given SPD matrix in place (lower triangle
 * of S holds L on return, upper set to 0).  Returns -1 on a pivot <= 0. */
int or_cholesky(int m, double *S);
/* Structural fill of the Cholesky factor of a pattern (dense char matrix,
 * symmetric, m x m): on return pat holds the pattern of L (lower). */
void or_symbolic_fill(int m, unsigned char *pat);

/* Global basis changes (Section 2.4 "interpolation and restriction"):
 * r_fdm = T_g^T r and u = T_g u_fdm on the full grid. */
void or_restrict_fdm(const or_ctx *c, const double *r, double *r_fdm);
void or_interp_fdm(const or_ctx *c, const double *u_fdm, double *u);

/* z = omega * P_ASM^{-1} r  (Section 2.5, additive over all set-up patches). */
int or_asm_apply(const or_ctx *c, const double *r, double *z);
void or_set_omega(or_ctx *c, double omega);
double or_get_omega(const or_ctx *c);

/* Q1 coarse space on the same mesh (Section 2.5): Galerkin A_c = P^T A P,
 * dense Cholesky.  z = P A_c^{-1} P^T r. */
int or_setup_coarse(or_ctx *c);
int or_coarse_apply(const or_ctx *c, const double *r, double *z);
int or_coarse_matrix(const or_ctx *c, int *nc, double *Ac);

/* Geometric multigrid for the Q1 problem (the paper's solver for the
 * p-coarse problem, Section 3 solver diagram): `levels` nested coarsenings
 * (every other vertex per axis, while all cell counts are even and >= 4), P
 * linear interpolation in the level's vertex coordinates, A_{l+1} = P^T A_l P,
 * `nu` damped point-Jacobi sweeps (damping omega) before and after the
 * coarse-grid correction, Cholesky on the coarsest level.  After this call the
 * coarse correction of or_coarse_apply / or_pc_apply is one V-cycle instead of
 * the exact solve.  Returns the number of levels built (0: exact solve kept),
 * negative on error.  Requires or_setup_coarse. */
int or_setup_coarse_gmg(or_ctx *c, int levels, int nu, double omega);
/* level l's dense operator (nf x nf; A may be NULL to query nf) */
int or_gmg_level(const or_ctx *c, int l, int *nf, double *A);
/* x = one V-cycle on the Q1 problem applied to b (free coarse dofs) */
int or_gmg_vcycle(const or_ctx *c, const double *b, double *x);

/* Hybrid multiplicative V(1,1): z = P^{-1} r (Section 2.5). */
int or_pc_apply(const or_ctx *c, const double *r, double *z);

/* Damping from k CG-Lanczos steps on P_ASM^{-1} A started from b0
 * (Section 2.5, omega = 2/[(1+a) lmax + (1-a) lmin], a = 1/4).  Sets the
 * context's omega.  lmin/lmax/omega may be NULL. */
int or_lanczos_omega(or_ctx *c, const double *b0, int k, double *lmin, double *lmax,
                     double *omega);

/* PCG from x0 = 0 until ||r||_2 <= rtol ||b||_2 (Section 2.8).
 * pc: 0 none, 1 omega*ASM, 2 V(1,1).  hist (maxit+1 doubles, may be NULL)
 * receives ||r_k||_2.  Returns 0 on convergence, 1 if maxit was reached. */
int or_pcg(const or_ctx *c, const double *b, double *x, double rtol, int maxit, int pc,
           int *iters, double *hist);

/* ---- learned separable surrogate (surrogate.c) -----------------------
 * Section 2.7 / Theorem 1: for a cell with points q, M_q = kappa Ghat_q and a
 * separable surrogate D = diag(mu), the true and surrogate cell stiffnesses
 * satisfy lo * a~ <= a <= hi * a~ with lo (hi) the smallest (largest)
 * eigenvalue of D^{-1/2} M_q D^{-1/2} over q.  A network maps 27 samples per
 * cell to c, mu = mu_avg exp(c); its label is the mu minimising hi / lo. */
#define OR_MLP_NIN 189  /* 27 points x (log kappa, 6 scaled Ghat entries) */
#define OR_MLP_NH 64
#define OR_MLP_NOUT 3
#define OR_MLP_NPARAM (OR_MLP_NH * OR_MLP_NIN + OR_MLP_NH + OR_MLP_NH * OR_MLP_NH + OR_MLP_NH + \
                       OR_MLP_NOUT * OR_MLP_NH + OR_MLP_NOUT)
#define OR_SURR_MAXIT 600     /* ellipsoid steps of the label search */
#define OR_SURR_RADIUS 6.0    /* initial disc of the label search (in log mu) */
#define OR_SURR_TOL 1e-10     /* optimality-gap bound that ends the search */
#define OR_SURR_CMAX 2.0
#define OR_ADAM_BETA1 0.9
#define OR_ADAM_BETA2 0.999
#define OR_ADAM_EPS 1e-8

/* log(hi / lo) of the Theorem 1 bound over nq points G[q][6] = kappa Ghat
 * (00, 11, 22, 01, 02, 12) for the scalings mu[3]; lo/hi may be NULL. */
double or_surr_bound(int nq, const double *G, const double *mu, double *lo, double *hi);
/* kappa Ghat at the (p+1)^3 Gauss points of every cell (unweighted,
 * G[cell][q][6]) and the averaged surrogate mubar[cell][3]. */
int or_surr_cell_ghat(int p, int ncell, const double *jac, const double *kappa, double *G,
                      double *mubar);
/* Labels from the cells' full quadrature data (jac/kappa as or_create):
 * mubar (averaged surrogate), cstar = log(mu_opt / mubar) with mu_opt the
 * minimiser of the bound ratio (ellipsoid method on the convex ratio in
 * log mu, surrogate.c) scaled so that lo * hi = 1, and the
 * ratios F0 = log(hi/lo) at mubar and F1 at mu*.  Arrays of 3, 3, 1, 1
 * doubles per cell. */
int or_surr_label(int p, int ncell, const double *jac, const double *kappa, double *mubar,
                  double *cstar, double *F0, double *F1);
/* Network inputs from s27[cell][27][10] = (kappa, J row-major) at the
 * 3x3x3 Gauss points (x fastest): per point, log kappa minus its cell
 * average, log(Ghat_aa / nu_a) with nu the 27-point averaged surrogate,
 * and the correlations Ghat_ab / sqrt(Ghat_aa Ghat_bb) for ab = 01, 02, 12
 * (Ghat here includes kappa).  feat[cell][189]. */
int or_surr_features(int ncell, const double *s27, double *feat);
/* Network 189 -> 64 (tanh) -> 64 (tanh) -> 3 (linear); parameters packed
 * W1[64][189], b1[64], W2[64][64], b2[64], W3[3][64], b3[3]. */
void or_mlp_forward(int ncell, const double *params, const double *feat, double *c);
/* mean-squared loss (1 / (2 ncell)) sum (c - label)^2 and its gradient
 * (grad may be NULL). */
double or_mlp_loss_grad(int ncell, const double *params, const double *feat, const double *label,
                        double *grad);
/* one Adam step t >= 1 (beta1, beta2, eps above). */
void or_mlp_adam(int nparam, double *params, const double *grad, double *m, double *v, int t,
                 double lr);
/* mu = mubar exp(c) per cell, or mubar where any c is non-finite or
 * |c| > OR_SURR_CMAX; returns the number of such fallback cells. */
int or_surr_apply(int ncell, const double *mubar, const double *c, double *mu);

#ifdef __cplusplus
}
#endif
#endif
