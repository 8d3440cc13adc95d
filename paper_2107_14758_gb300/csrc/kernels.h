// Host-side declarations of the kernel launchers.
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "device.cuh"

namespace fdm {

constexpr int PATCH_THREADS_MAX = 1024;  // largest patch-solve block (tmp sizing)

template <typename T>
struct PatchSolveArgs {
  Grid g;
  const ClassDev *cls;
  const PatchDev *patches;
  const int *order;
  const T *E;
  const double *mu;
  const T *tab;
  const T *L;
  T *X;
  int tmpcap;    // elements of the tmp shared-memory area
  int prefetch;  // L2 bulk prefetch of the factor: 0 none, 1 all at start, 2 section ahead of use
  // resident (persistent) variant: bound of the mbarrier waits, status word, test hook
  uint64_t timeout_ns;
  int *status;
  int inject_stall;
  int l2hint;  // L2 eviction priorities: forward reads evict-last, backward reads evict-first
  int rows8;   // eight rows per warp in the forward products (else four)
  int headcap = 0;  // Schur-coupling form: elements of shared memory for the patch's values
                    // before S_TB (stage_st = 0) or before W (stage_st = 1), staged by one
                    // bulk copy where they fit; 0 = none
  int stage_st = 1;
};
int patch_tmp_elems(int maxN1, int maxN2);
// Schur-coupling form of the patch solve (one CTA per patch, 256 or 512 threads)
int patch_sc_tmp(int maxN1, int maxN2, int threads);
template <typename T>
size_t patch_sc_smem(int maxG, int maxN1, int maxN2, int threads, int headcap);
template <typename T>
void launch_patch_sc(const PatchSolveArgs<T> &a, int npatch, size_t smem, int threads, cudaStream_t st);
// the Schur-coupling solves of many problems in one launch (256 threads, four rows
// of W per warp, the values before W staged): args[problem] in device memory,
// work[b] = (problem, position in its patch order), problems with active == 0 skipped
template <typename T>
void launch_patch_sc_multi(const PatchSolveArgs<T> *args, const int2 *work, int nwork, const int *active, size_t smem,
                           cudaStream_t st);
// persistent variant (256 threads): headcap = elements of each of its two staging buffers
template <typename T>
void launch_patch_scp(const PatchSolveArgs<T> &a, int npatch, size_t smem, cudaStream_t st);
// persistent, each patch's whole operator staged in one of two shared-memory
// buffers of a.headcap elements (>= the largest class's value count)
template <typename T>
void launch_patch_scf(const PatchSolveArgs<T> &a, int npatch, size_t smem, int threads, cudaStream_t st);
// one warp per patch: ws = per-warp shared-memory elements (patch_scw_ws),
// warps = patches per CTA (4 or 8), maxN2 <= patch_scw_max_n2(4)
int patch_scw_ws(int maxG, int maxN0, int maxN1);
int patch_scw_max_n2(int nq);
template <typename T>
void launch_patch_scw(const PatchSolveArgs<T> &a, int npatch, int ws, int warps, int maxN2, cudaStream_t st);
// the resident variant: fcap factor elements per CTA in shared memory (one
// patch's values), tmp sized for `threads`
int patch_resident_tmp(int maxN1, int maxN2, int threads);
template <typename T>
size_t patch_resident_smem(int fcap, int maxG, int tmpcap);
template <typename T>
void launch_patch_resident(const PatchSolveArgs<T> &a, int npatch, int fcap, size_t smem, int threads,
                           cudaStream_t st);

template <typename T>
struct InterpArgs {
  Grid g;
  const PatchDev *patches;
  const ClassDev *cls;
  const T *X;       // interface solutions of all stars
  const T *E;       // condensed cell-local FDM residual (interior entries unchanged)
  const double *mu; // surrogate coefficients
  const T *tab;
  // [8 classes][8 corners][n^3]: star-interface index of each cell node in the
  // star of the cell's corner (bit 0: +x, bit 1: +y, bit 2: +z), -1 if none
  const int *cmap;
  const T *addv;  // optional: z = addv + omega * relaxation (grid vector)
};

// streamed patch solve: per-class chunk schedules over the factor values
template <typename T>
struct StreamArgs {
  Grid g;
  const ClassDev *cls;
  const PatchDev *patches;
  const int *order;   // patches with an interface, heaviest first
  int npatch;
  const T *E;
  const T *L;
  T *X;
  int maxG, maxN0, maxN1, tmpcap;
  int nbuf, buf_bytes;  // ring of shared-memory chunk buffers
  int ctas_per_sm;      // 0 = as many as fit
  uint64_t timeout_ns;  // bound of every mbarrier wait
  int inject_stall;     // test hook: wait on a barrier that nothing completes
  int *status;          // set to 1 when a bounded wait ran out
};
template <typename T>
size_t stream_smem_bytes(const StreamArgs<T> &a);
template <typename T>
int launch_patch_stream(const StreamArgs<T> &a, int threads, cudaStream_t st);

// patch solve on a thread-block cluster (classes with a dense top level), k_cluster.cu
template <typename T>
struct ClusterArgs {
  Grid g;
  const ClassDev *cls;
  const PatchDev *patches;
  const int *order;  // the patches solved by clusters
  int npatch;
  const T *E;
  const T *L;
  T *X;
  int cs;        // CTAs per cluster (one patch per cluster)
  int rows_cap;  // L21 rows held per CTA (>= ceil(n2 / cs))
  int ld_cap;    // >= ld21
  int n2_cap;    // >= n2, a multiple of 4
  int maxG;
  int tmpcap;    // >= max(n2_cap, ld_cap), >= 4 * threads
  uint64_t timeout_ns;
  int *status;
  int inject_stall;
};
template <typename T>
size_t patch_cluster_smem(const ClusterArgs<T> &a);
// clusters that can be resident at once (0: the configuration cannot run)
template <typename T>
int patch_cluster_fits(const ClusterArgs<T> &a, int threads);
template <typename T>
void launch_patch_cluster(const ClusterArgs<T> &a, int threads, cudaStream_t st);

// basis change and relaxation
template <typename T, typename Tin>
void launch_restrict_fdm(const Grid &g, const Tin *r, const T *tab, const double *mu, T *E, cudaStream_t st);
template <typename T, typename Tout>
void launch_interp_fdm(const InterpArgs<T> &a, double omega, Tout *z, cudaStream_t st);
template <typename T>
size_t patch_smem_bytes(int n, int maxG, int maxN1, int maxN2);
template <typename T>
void launch_patch_solve(const PatchSolveArgs<T> &a, int npatch, size_t smem, int threads, cudaStream_t st);
template <typename T>
size_t patch_smem_for_occupancy(size_t need, int ctas_per_sm);

// operators
struct OpArgs {
  Grid g;
  int general;          // 0: box cells (Kronecker), 1: quadrature
  const double *mu_box; // [ncell][3] (box)
  const void *Gw;       // [ncell][nq][6] in the op precision (general)
  const void *detw;     // [ncell][nq] (general mass)
  const void *tab;      // 1D tables in the op precision
};
// y = A u (stiffness) or M u (mass); E is a work buffer of ncell*n^3 elements.
template <typename T, typename Tin, typename Tout>
void launch_operator(const OpArgs &a, bool mass, const Tin *u, Tout *y, T *E, cudaStream_t st);
// cell kernels specialised on n (k_cell.cu); false when no specialisation applies
template <typename T, typename Tin, typename Tout>
bool launch_box_op_fast(const OpArgs &a, const Tin *u, Tout *y, T *E, cudaStream_t st, const double *rsub = nullptr);
template <typename T, typename Tin>
bool launch_restrict_fast(const Grid &g, const Tin *r, const T *tab, const double *mu, T *E, cudaStream_t st);
template <typename T, typename Tout>
bool launch_interp_fast(const InterpArgs<T> &a, double omega, Tout *z, cudaStream_t st);

template <typename T, typename Tin>
bool launch_coarse_restrict_fast(const Grid &g, const Tin *r, const T *tab, T *cellbuf, cudaStream_t st);
template <typename T, typename Tout>
bool launch_coarse_prolong_fast(const Grid &g, const T *xc, const T *tab, const int *cfree, Tout *z, bool accumulate,
                                cudaStream_t st);

// per-cell Galerkin coarse matrices P_K^T A^K P_K (FP64), [ncell][8][8]
void launch_coarse_cell_matrices(const OpArgs &a, double *Ac, cudaStream_t st);

// context accessors (defined with the C-ABI)
OpArgs ctx_op_args64(const fdm_ctx *c);
void ctx_count_launches(fdm_ctx *c, int k);
int ctx_device(const fdm_ctx *c);  // the device that holds the context's data
int ctx_fail(fdm_ctx *c, int code, const std::string &msg);

// coarse space
template <typename T, typename Tin>
void launch_coarse_restrict(const Grid &g, const Tin *r, const T *tab, const int *cfree, T *rc, T *cellbuf,
                            cudaStream_t st);
// one level of the geometric multigrid on the Q1 problem: m free vertices per
// axis (lexicographic, x fastest), 27-point stencil A[k][nf] with offset
// k = (dx+1) + 3 (dy+1) + 9 (dz+1), dw = omega / A[13], and per axis the
// interpolation parameter t[v] = (x_v - x_{v-1}) / (x_{v+1} - x_{v-1}) at the odd
// vertices v of this level (used when this level is the fine side of a transfer)
// sums cell-local values E [cell][n^3] over the cells of each grid node: y = sum
// (or rsub - sum), Dirichlet nodes 0
template <typename T, typename Tout>
void launch_gather_cells(const Grid &g, const T *E, const double *rsub, Tout *y, cudaStream_t st);
// linear elasticity on box cells: cell-local y^K = K^K u^K for the three
// components (u [3][ndof], G scratch [9][ncell][n^3], E [3][ncell][n^3]);
// Lc = half-widths [cell][3]; tab = the 1D tables (Gauss V, D), wq = Gauss weights
template <typename T>
size_t elast_smem(int n);
template <typename T, typename Tin>
void launch_elast_cells(const Grid &g, const Tin *u, const T *tab, const T *wq, const double *Lc, double mu, double lam,
                        T *G, T *E, cudaStream_t st);
// Star-local fast diagonalisation on box cells for a scalar block with a
// constant coefficient diag(c) (the SDC blocks of Section 4.1, c_a = mu +
// (mu + lam) delta_aj): the star matrix of vertex v is the Kronecker sum
// sum_a c_a A_a (x) M_b (x) M_c of its 1D star matrices, so
// A_v^{-1} = (S_x (x) S_y (x) S_z) D^{-1} (S_x (x) S_y (x) S_z)^T with the 1D
// generalised eigenpairs A_a S_a = M_a S_a Lam_a, S_a^T M_a S_a = I, and
// D = sum_a c_a Lam_a.  A 1D star spans the free nodes within p - 1 of its
// vertex: a vertex on a natural (traction-free) end keeps its boundary node, one
// on a Dirichlet end loses it (its star is empty for p = 1).
constexpr int STAR_FDM_MAX_LEN = 29;  // 2 p - 1 for p <= 15
struct StarFdmAxis {
  const int *lo = nullptr;    // [n_a + 1] first node of the 1D star of vertex coordinate v
  const int *len = nullptr;   // [n_a + 1] its nodes (0: empty)
  const int *soff = nullptr;  // [n_a + 1] offset in tab of S (len x len, row-major, column i =
                              // eigenvector i), the eigenvalues following at soff + len^2
};
template <typename T>
struct StarFdmDev {
  Grid g;                        // the grid with its Dirichlet face mask
  StarFdmAxis ax[3];
  const T *tab = nullptr;        // the 1D stars' S and eigenvalues
  const int *vstar = nullptr;    // [(nx+1)(ny+1)(nz+1)] star of each vertex or -1 (empty)
  const int *svert = nullptr;    // [nstar] vertex of each star
  const int64_t *off = nullptr;  // [nstar] first value of each star's block in X
  int64_t xstride = 0;           // values of one component's star blocks
  int nstar = 0, maxlen = 0;
  double c[3][3] = {};           // c[j][a]: coefficient of axis a in block j
};
// X[j xstride + off[s] + local] = A_s^{-1} R_s r_j for every star s and block
// j < ncomp (r: component-major [ncomp][ndof])
template <typename T, typename Tin>
void launch_star_fdm_solve(const StarFdmDev<T> &d, const Tin *r, T *X, int ncomp, cudaStream_t st);
// z_j = omega sum_s R_s^T X_s (+ addv_j), summed per node over its stars in
// lexicographic order of their vertices; Dirichlet nodes 0
template <typename T, typename Tout>
void launch_star_fdm_gather(const StarFdmDev<T> &d, const T *X, double omega, const T *addv, Tout *z, int ncomp,
                            cudaStream_t st);
size_t star_fdm_smem(int maxlen, size_t elem);

// SIPG on DQ_p box cells (Section 5): cell-major vectors, (p+1)^3 values per cell
constexpr int SIPG_MAX_N = 11;  // p <= 10
template <typename T>
struct SipgDev {
  int p = 0, n = 0, nx = 0, ny = 0, nz = 0, ncell = 0;
  double eta = 0.0;
  const double *hx = nullptr, *hy = nullptr, *hz = nullptr;  // half-widths per axis
  const T *tab = nullptr;  // A_hat, B_hat (n x n), l_i'(-1), l_i'(+1), GLL nodes (n each)
  // per axis a and interior vertex v (1..nc_a - 1): the 1D star pencil's
  // eigenvectors S[soff[a] + (v - 1) (2n)^2] (row-major, column i = vector i)
  // and eigenvalues lam[loff[a] + (v - 1) 2n]
  const T *S = nullptr, *lam = nullptr;
  int64_t soff[3] = {0, 0, 0}, loff[3] = {0, 0, 0};
};
template <typename T>
size_t sipg_cell_smem(int n);
template <typename T>
size_t sipg_patch_smem(int n);
// y = A u, or y = rsub - A u (rsub != nullptr); F: face data [ncell][12][n^2]
template <typename T, typename Tin>
void launch_sipg_op(const SipgDev<T> &d, const Tin *u, T *F, const double *rsub, T *y, cudaStream_t st);
// the stars of one vertex parity class (color = px | py << 1 | pz << 2, nblocks
// of them), or of the listed vertices (vlist): z += omega A_v^{-1} R_v r on
// their cells, or (zpatch != nullptr) A_v^{-1} R_v r into zpatch[block][(2n)^3]
template <typename T, typename Tin, typename Tout>
void launch_sipg_patch(const SipgDev<T> &d, int color, int nblocks, const int *vlist, const Tin *r, Tout *z,
                       T *zpatch, double omega, cudaStream_t st);
// z = (addv or 0) + omega * sum of the star solutions zp[star][(2n)^3] of all
// interior vertices (lexicographic) holding each value, in a fixed order
template <typename T, typename Tout>
void launch_sipg_star_gather(const SipgDev<T> &d, const T *zp, double omega, const T *addv, Tout *z,
                             cudaStream_t st);
// the same stars' solves with the six 1D contractions on the tensor cores
// (tcgen05, TF32 in, FP32 accumulation); DQ_7 only; status: 1 when a bounded
// completion wait ran out
template <typename Tin, typename Tout>
void launch_sipg_patch_tc(const SipgDev<float> &d, int color, int nblocks, const int *vlist, const Tin *r, Tout *z,
                          float *zpatch, double omega, uint64_t timeout_ns, int *status, cudaStream_t st);
template <typename T, typename Tin>
void launch_sipg_restrict(const SipgDev<T> &d, const Tin *r, const int *cfree, T *cellbuf, T *rc, cudaStream_t st);
template <typename T>
void launch_sipg_prolong(const SipgDev<T> &d, const int *cfree, const T *xc, T *x, cudaStream_t st);  // x += P xc

template <typename T>
struct GmgDev {
  int m[3] = {0, 0, 0};
  int nf = 0;
  const T *A = nullptr;
  const T *dw = nullptr;
  const T *t[3] = {nullptr, nullptr, nullptr};
};
template <typename T>
void launch_gmg_pre(const GmgDev<T> &L, int nu, const T *b, T *x, cudaStream_t st);  // min(nu, 2) sweeps from 0
template <typename T>
void launch_gmg_sweep(const GmgDev<T> &L, const T *b, const T *x, T *out, cudaStream_t st);
template <typename T>
void launch_gmg_resid(const GmgDev<T> &L, const T *b, const T *x, T *r, cudaStream_t st);
template <typename T>
void launch_gmg_restrict(const GmgDev<T> &F, const GmgDev<T> &C, const T *r, T *bc, cudaStream_t st);
template <typename T>
void launch_gmg_prolong(const GmgDev<T> &F, const GmgDev<T> &C, const T *xc, T *x, cudaStream_t st);  // x += P xc
template <typename T>
void launch_dense_symv(int m, const T *Ainv, const T *x, T *y, cudaStream_t st);
template <typename T, typename Tout>
void launch_coarse_prolong(const Grid &g, const T *xc, const T *tab, const int *cfree, Tout *z, bool accumulate,
                           cudaStream_t st);

// vectors
constexpr int DOT_BLOCKS = 608;  // 4 x 152 SMs; fixed so reductions are deterministic
void launch_dot(int64_t n, const double *a, const double *b, double *partial, double *out, cudaStream_t st);
void launch_dot2(int64_t n, const double *a, const double *b, const double *c, double *partial, double *out,
                 cudaStream_t st);  // out[0] = a.b, out[1] = a.c
template <typename Ta, typename Tb>
void launch_convert(int64_t n, const Ta *a, Tb *b, cudaStream_t st);
template <typename T>
void launch_axpby(int64_t n, T alpha, const T *x, T beta, const T *y, T *z, cudaStream_t st);  // z = a x + b y
template <typename T>
void launch_sub(int64_t n, const T *x, const T *y, T *z, cudaStream_t st);  // z = x - y
template <typename T>
void launch_add(int64_t n, const T *x, T *y, cudaStream_t st);  // y += x
// PCG scalar/vector steps (scalars on the device)
void launch_pcg_update_xr(int64_t n, const double *sc, const double *d, const double *q, double *x, double *r,
                          cudaStream_t st);
void launch_pcg_update_d(int64_t n, const double *sc, const double *z, double *d, cudaStream_t st);
void launch_pcg_scalars(int which, double *sc, const double *dots, cudaStream_t st);

// learned separable surrogate: network 189 -> 64 -> 64 -> 3 (FP32 weights)
constexpr int MLP_NIN = 189, MLP_NH = 64, MLP_NOUT = 3;
constexpr int MLP_NPARAM = MLP_NH * MLP_NIN + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NOUT * MLP_NH + MLP_NOUT;
constexpr int SURR_MAXIT = 600;       // ellipsoid steps of the label search
constexpr double SURR_RADIUS = 6.0;   // initial disc of the label search (log mu)
constexpr double SURR_TOL = 1e-10;    // optimality-gap bound that ends the search
constexpr float SURR_CMAX = 2.0f;   // |c| above this falls back to the averaged surrogate
constexpr float ADAM_BETA1 = 0.9f, ADAM_BETA2 = 0.999f, ADAM_EPS = 1e-8f;
void launch_surr_features(int ncell, const double *s27, const double w3[3], float *feat, cudaStream_t st);
void launch_surr_label(int ncell, int n, const double *Gw, const double *wq, const double *mubar, double *cstar,
                       double *F0, double *F1, cudaStream_t st);
void launch_surr_bound(int ncell, int n, const double *Gw, const double *wq, const double *mu, double *F,
                       cudaStream_t st);
// labels scored by the Lanczos estimate of kappa(A~_P^{-1} A_P) on each cell's
// interior patch: compass search over the scaling ratios, centred spectrum.
// cstar [cell][3]; F [cell][2] log kappa at mubar and at the label; evals
// [cell] (may be null) the estimates taken.  Degrees 2..PATCH_KAPPA_PMAX.
constexpr int PATCH_KAPPA_STEPS = 48;          // Lanczos steps per estimate (at most)
constexpr double PATCH_KAPPA_BREAKDOWN = 1e-10;  // relative norm of the next vector that ends a run
constexpr double PATCH_KAPPA_S0 = 0.5;         // first compass step (log mu)
constexpr double PATCH_KAPPA_SMIN = 1.0 / 256.0;
constexpr int PATCH_KAPPA_ROUNDS = 48;
constexpr double PATCH_KAPPA_IMPROVE = 1e-9;   // a move must lower log kappa by more than this
constexpr int PATCH_KAPPA_PMAX = 8;            // the Lanczos vectors stay in shared memory
void launch_surr_patch_label(int ncell, int p, const double *Gw, const double *tab, const double *S,
                             const double *lam, const double *mubar, double *cstar, double *F, int *evals,
                             cudaStream_t st);
int mlp_blocks(int ncell);
// forward (label == nullptr) or forward + loss + per-CTA partial gradient
void launch_mlp(int ncell, const float *P, const float *feat, const float *label, float *out, float *partial,
                float *lossp, cudaStream_t st);
void launch_mlp_reduce(int nblk, const float *partial, const float *lossp, float *grad, double *loss,
                       cudaStream_t st);
void launch_adam(float *P, const float *g, float *m, float *v, int t, double lr, double wd, cudaStream_t st);
void launch_surr_apply(int ncell, const float *c, const double *mubar, double *mu, int *nfall, cudaStream_t st);

}  // namespace fdm
