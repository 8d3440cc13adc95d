// C-ABI entry points of the fdmpc library (declared in include/fdmpc.h).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "factor.h"
#include "internal.h"
#include "kernels.h"
#include "ctx.h"

namespace fdm {
[[noreturn]] void fail(int code, const std::string &msg) { throw Error{code, msg}; }

void *device_alloc(size_t bytes, size_t &used) {
  bytes = std::max<size_t>(bytes, 1);
  size_t limit = SIZE_MAX;
  if (const char *s = std::getenv("FDM_ALLOC_LIMIT_BYTES")) {
    char *end = nullptr;
    const unsigned long long v = std::strtoull(s, &end, 10);
    if (end != s && *end == '\0' && s[0] != '-') limit = (size_t)v;
  }
  if (bytes > limit || used > limit - bytes)
    fail(FDM_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes would exceed FDM_ALLOC_LIMIT_BYTES = " +
                         std::to_string(limit) + " (" + std::to_string(used) + " bytes allocated)");
  void *ptr = nullptr;
  if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    fail(FDM_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  used += bytes;
  return ptr;
}
static_assert(MLP_NPARAM == FDM_MLP_NPARAM, "network size of the public header");
}  // namespace fdm

using namespace fdm;

namespace {
thread_local std::string g_last_error;
double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}
}  // namespace

struct fdm_batch {
  std::vector<fdm_ctx *> ctxs;
  // the captured solve: one graph with a device-driven PCG loop per problem
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;
  unsigned long long *d_times = nullptr;  // [1 + k] global timer: start, end of each solve
  std::vector<const double *> key_b;
  std::vector<double *> key_x;
  std::vector<size_t> init_kernels, body_kernels, verify_kernels;  // kernel nodes per problem: set-up, one
                                                                   // iteration, one true-residual check
  double key_rtol = -1.0;
  int key_maxit = -1;
  // lockstep mode: every problem steps one PCG iteration at a time inside one
  // device-driven loop, the star solves of all problems in one launch over a
  // global (problem, patch) list sorted largest first; converged problems drop out
  int mode = FDM_BATCH_BRANCHES;
  PatchSolveArgs<float> *d_args = nullptr;  // [k] per-problem patch-solve arguments
  int2 *d_work = nullptr;                    // the global work list
  int nwork = 0;
  size_t multi_smem = 0;
  int *d_active = nullptr;                             // [k] 1 while a problem iterates
  cudaGraphConditionalHandle *d_ifh = nullptr;         // [3 k] its segments' IF handles
  std::vector<size_t> seg_kernels;                     // kernel nodes per problem and iteration
  void release_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
  }
  ~fdm_batch() {
    release_graph();
    if (cap) cudaStreamDestroy(cap);
    if (d_times) cudaFree(d_times);
    for (void *ptr : {(void *)d_args, (void *)d_work, (void *)d_active, (void *)d_ifh})
      if (ptr) cudaFree(ptr);
  }
};

namespace {

// dynamic shared memory a CTA may use on sm_103 (227 KB)
constexpr size_t kScfSmemCap = 227 * 1024;

// whether the warp-per-patch solve takes this context's classes with
// `threads` / 32 patches per CTA: top blocks within its register column sums,
// per-warp work space within shared memory
bool scw_fits(const fdm_ctx *c, bool fp32, int threads) {
  const size_t ws = (size_t)patch_scw_ws(c->maxG, c->maxN0, c->maxN1) * (fp32 ? 4 : 8) * (threads / 32);
  return c->maxN2 <= patch_scw_max_n2(4) && ws <= kScfSmemCap;
}

// ---------------------------------------------------------------- helpers
__global__ void k_mask_dirichlet(Grid g, double *v) {
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ndof; id += (int64_t)gridDim.x * blockDim.x) {
    int x = int(id % g.N[0]), y = int((id / g.N[0]) % g.N[1]), z = int(id / ((int64_t)g.N[0] * g.N[1]));
    if (node_dirichlet(g, x, y, z)) v[id] = 0.0;
  }
}
void mask_dirichlet(const Grid &g, double *v, cudaStream_t st) {
  int64_t b = std::min<int64_t>((g.ndof + 255) / 256, 152 * 32);
  k_mask_dirichlet<<<(int)std::max<int64_t>(b, 1), 256, 0, st>>>(g, v);
}
__global__ void k_fill(int64_t n, double v, double *x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}
__global__ void k_copy(int64_t n, const double *__restrict__ a, double *__restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) b[i] = a[i];
}
int vec_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }
void fill(int64_t n, double v, double *x, cudaStream_t st) { k_fill<<<vec_blocks(n), 256, 0, st>>>(n, v, x); }
void copy(int64_t n, const double *a, double *b, cudaStream_t st) { k_copy<<<vec_blocks(n), 256, 0, st>>>(n, a, b); }

template <typename T>
StreamArgs<T> stream_args(fdm_ctx *c) {
  StreamArgs<T> s;
  s.g = c->g;
  s.cls = c->d_cls;
  s.patches = c->d_patches;
  s.order = c->d_order_nz;
  s.npatch = c->nsolve_nz;
  s.E = c->E<T>();
  s.L = c->L<T>();
  s.X = c->X<T>();
  s.maxG = c->maxG;
  s.maxN0 = c->maxN0;
  s.maxN1 = c->maxN1;
  // scratch of the transposed products: slices * row length <= 4 * consumer threads
  s.tmpcap = std::max({4 * std::max(c->patch_threads, 128), (c->maxN1 + 3) & ~3, (c->maxN2 + 3) & ~3});
  s.nbuf = c->nbuf;
  s.buf_bytes = c->buf_bytes;
  s.ctas_per_sm = c->opt.patch_ctas_per_sm;
  s.timeout_ns = (uint64_t)(std::max(c->opt.wait_timeout_s, 0.0) * 1e9);
  s.inject_stall = c->opt.inject_stall;
  s.status = c->status;
  return s;
}

// One relaxation sweep in three phases: the per-cell restriction to the FDM
// basis with the Schur condensation (E), the star solves (X), and the
// back-substitution and basis change back (z).  The batched lockstep solve runs
// the middle phase of every problem in one launch.
template <typename T, typename Tin>
void asm_restrict(fdm_ctx *c, const Tin *r, cudaStream_t st) {
  c->tmark(FDM_T_RESTRICT, true, st);
  launch_restrict_fdm<T, Tin>(c->g, r, c->tab<T>(), c->mu, c->E<T>(), st);
  c->tmark(FDM_T_RESTRICT, false, st);
  c->launches += 1;
}

template <typename T, typename Tout>
void asm_interp(fdm_ctx *c, Tout *z, double omega, cudaStream_t st, const T *addv) {
  c->tmark(FDM_T_INTERP, true, st);
  InterpArgs<T> ia{c->g, c->d_patches, c->d_cls, c->X<T>(), c->E<T>(), c->mu, c->tab<T>(), c->cmap, addv};
  launch_interp_fdm<T, Tout>(ia, omega, z, st);
  c->tmark(FDM_T_INTERP, false, st);
  c->launches += 1;
}

template <typename T>
void asm_patch(fdm_ctx *c, cudaStream_t st) {
  c->tmark(FDM_T_PATCH, true, st);
  const bool resident = sizeof(T) == 4 ? c->res32 : c->res64;
  if (c->scform) {
    PatchSolveArgs<T> a{c->g, c->d_cls, c->d_patches, c->d_order, c->E<T>(), c->mu, c->tab<T>(), c->L<T>(),
                        c->X<T>(), patch_sc_tmp(c->maxN1, c->maxN2, c->patch_threads), 0,
                        (uint64_t)(std::max(c->opt.wait_timeout_s, 0.0) * 1e9), c->status, 0, 0, 0};
    a.rows8 = c->rows8;  // Schur-coupling form: four rows per warp in the W product (else two)
    a.inject_stall = c->opt.inject_stall;
    if (c->sc_warp) {  // one warp per patch, patch_threads / 32 patches per CTA
      launch_patch_scw<T>(a, c->nsolve, patch_scw_ws(c->maxG, c->maxN0, c->maxN1), c->patch_threads / 32, c->maxN2, st);
    } else if (c->sc_full) {  // persistent: each patch's whole operator staged, two buffers
      a.stage_st = 1;
      a.tmpcap = patch_sc_tmp(c->maxN1, c->maxN2, c->patch_threads);
      a.headcap = c->fcap_sc;
      launch_patch_scf<T>(a, c->nsolve, patch_sc_smem<T>(c->maxG, c->maxN1, c->maxN2, c->patch_threads, 2 * a.headcap),
                          c->patch_threads, st);
    } else if (c->sc_persist) {  // persistent (256 threads): two buffers for the lower block's values, S_TB and W via L2
      a.stage_st = 0;
      a.tmpcap = patch_sc_tmp(c->maxN1, c->maxN2, 256);  // the scratch the kernel zeroes, sized for its threads
      a.headcap = sizeof(T) == 4 ? c->bcap32 : c->bcap64;
      launch_patch_scp<T>(a, c->nsolve, patch_sc_smem<T>(c->maxG, c->maxN1, c->maxN2, 256, 2 * a.headcap), st);
    } else {
      // 128 threads, or 256 with rows8 = 2: only the lower block's values are staged (eight or
      // six CTAs per SM)
      a.stage_st = (c->patch_threads <= 128 || c->rows8 >= 2) ? 0 : 1;
      a.headcap = a.stage_st ? (sizeof(T) == 4 ? c->headcap32 : c->headcap64) : (sizeof(T) == 4 ? c->bcap32 : c->bcap64);
      if (c->rows8 == 3) {  // nothing staged: the whole value block prefetched into L2 at the start
        a.headcap = 0;
        a.prefetch = 1;
      }
      launch_patch_sc<T>(a, c->nsolve, patch_sc_smem<T>(c->maxG, c->maxN1, c->maxN2, c->patch_threads, a.headcap),
                         c->patch_threads, st);
    }
  } else if (c->stream) {
    if (launch_patch_stream<T>(stream_args<T>(c), c->patch_threads, st) != 0)
      fail(FDM_ECUDA, "streamed patch solve: launch configuration rejected");
  } else if (resident) {
    PatchSolveArgs<T> a{c->g, c->d_cls, c->d_patches, c->d_order, c->E<T>(), c->mu, c->tab<T>(), c->L<T>(), c->X<T>(),
                        c->res_tmp, 0, (uint64_t)(std::max(c->opt.wait_timeout_s, 0.0) * 1e9), c->status,
                        c->opt.inject_stall, 0, 0};
    launch_patch_resident<T>(a, c->nsolve, c->fcap, sizeof(T) == 4 ? c->rsmem32 : c->rsmem64, c->res_threads, st);
  } else {
    const bool clus = sizeof(T) == 4 ? c->cl32 : c->cl64;
    const int skip = clus ? c->n_heavy : 0;
    if (clus) {
      ClusterArgs<T> ca = cluster_args<T>(c);
      ca.cls = c->d_cls;
      ca.patches = c->d_patches;
      ca.order = c->d_order;
      ca.E = c->E<T>();
      ca.L = c->L<T>();
      ca.X = c->X<T>();
      ca.status = c->status;
      launch_patch_cluster<T>(ca, c->cl_threads, st);
    }
    PatchSolveArgs<T> a{c->g, c->d_cls, c->d_patches, c->d_order + skip, c->E<T>(), c->mu, c->tab<T>(), c->L<T>(),
                        c->X<T>(), patch_tmp_elems(c->maxN1, c->maxN2),
                        c->opt.patch_prefetch > 0 ? c->opt.patch_prefetch : 3, 0, c->status, 0,
                        c->opt.patch_l2_hints != 2 ? 1 : 0, c->rows8};
    launch_patch_solve<T>(a, c->nsolve - skip, c->smem<T>(), c->patch_threads, st);
  }
  c->tmark(FDM_T_PATCH, false, st);
  c->launches += 1;
}

template <typename T, typename Tin, typename Tout>
void run_asm(fdm_ctx *c, const Tin *r, Tout *z, double omega, cudaStream_t st, const T *addv = nullptr) {
  asm_restrict<T, Tin>(c, r, st);
  asm_patch<T>(c, st);
  asm_interp<T, Tout>(c, z, omega, st, addv);
}

// one V-cycle of the geometric multigrid on level l: out = V(b) from a zero
// start (min(nu, 2) Jacobi sweeps in one kernel, the rest one kernel each)
template <typename T>
void gmg_level(fdm_ctx *c, int l, const T *b, T *out, cudaStream_t st) {
  auto &G = c->gmg<T>();
  if (l == c->gmg_L) {
    launch_dense_symv<T>(c->nc_dense, c->Acinv<T>(), b, out, st);
    c->launches += 1;
    return;
  }
  const GmgDev<T> &F = G.lev[l], &C = G.lev[l + 1];
  const int nu = c->gmg_nu;
  T *cur = G.xa[l], *oth = G.xb[l];
  launch_gmg_pre<T>(F, nu, b, cur, st);
  for (int s = 2; s < nu; ++s) {
    launch_gmg_sweep<T>(F, b, cur, oth, st);
    std::swap(cur, oth);
  }
  launch_gmg_resid<T>(F, b, cur, G.r[l], st);
  launch_gmg_restrict<T>(F, C, G.r[l], G.b[l + 1], st);
  gmg_level<T>(c, l + 1, G.b[l + 1], G.out[l + 1], st);
  launch_gmg_prolong<T>(F, C, G.out[l + 1], cur, st);
  for (int s = 0; s < nu; ++s) {
    T *dst = s == nu - 1 ? out : oth;
    launch_gmg_sweep<T>(F, b, cur, dst, st);
    std::swap(cur, oth);
  }
  c->launches += (nu >= 2 ? nu - 1 : 1) + 3 + nu;
}

// restriction to the Q1 vertices, the Q1 solve (exact, or one multigrid
// V-cycle), prolongation added to x
template <typename T>
void coarse_correct(fdm_ctx *c, const T *r1, T *x, cudaStream_t st) {
  c->tmark(FDM_T_COARSE, true, st);
  launch_coarse_restrict<T, T>(c->g, r1, c->tab<T>(), c->cfree, c->rc<T>(), c->cb<T>(), st);
  if (c->nc > 0) {
    if (c->gmg_L > 0) gmg_level<T>(c, 0, c->rc<T>(), c->xc<T>(), st);
    else {
      launch_dense_symv<T>(c->nc, c->Acinv<T>(), c->rc<T>(), c->xc<T>(), st);
      c->launches += 1;
    }
  }
  launch_coarse_prolong<T, T>(c->g, c->xc<T>(), c->tab<T>(), c->cfree, x, true, st);
  c->tmark(FDM_T_COARSE, false, st);
  c->launches += 3;
}

// y = A u with the FP64 operator (PCG residual) or the FP32 one (inside the preconditioner)
template <typename T>
void apply_op(fdm_ctx *c, const T *u, T *y, cudaStream_t st) {
  const int tag = sizeof(T) == 4 ? FDM_T_OP32 : FDM_T_OP64;
  c->tmark(tag, true, st);
  launch_operator<T, T, T>(c->op_args(sizeof(T) == 4), false, u, y, c->E<T>(), st);
  c->tmark(tag, false, st);
  c->launches += 2;
}

__global__ void k_rsub(int64_t n, const double *__restrict__ r, float *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = float(r[i]) - y[i];
}
__global__ void k_rsub(int64_t n, const double *__restrict__ r, double *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = r[i] - y[i];
}

// r1 = r - A u in precision T (r: the FP64 preconditioner input, Dirichlet
// entries 0); on box cells fused into the node gather of the stiffness apply
template <typename T>
void apply_residual(fdm_ctx *c, const T *u, const double *r, T *r1, cudaStream_t st) {
  const int tag = sizeof(T) == 4 ? FDM_T_OP32 : FDM_T_OP64;
  c->tmark(tag, true, st);
  if (!launch_box_op_fast<T, T, T>(c->op_args(sizeof(T) == 4), u, r1, c->E<T>(), st, r)) {
    launch_operator<T, T, T>(c->op_args(sizeof(T) == 4), false, u, r1, c->E<T>(), st);
    k_rsub<<<vec_blocks(c->g.ndof), 256, 0, st>>>(c->g.ndof, r, r1);
    c->launches += 1;
  }
  c->tmark(tag, false, st);
  c->launches += 2;
}

// hybrid multiplicative V(1,1) (Section 2.5) computed in precision T from the
// FP64 input r to the FP64 output z:
//   x1 = omega ASM(r); r1 = r - A x1; x1 += P A_c^{-1} P^T r1; r1 = r - A x1;
//   z = x1 + omega ASM(r1)
// (the conversions, residual subtractions and the final sum are fused into the
// restriction, the node gather and the interpolation)
template <typename T>
void run_vcycle(fdm_ctx *c, const double *r, double *z, T *x1, T *r1, cudaStream_t st) {
  run_asm<T, double, T>(c, r, x1, c->omega, st);  // pre-relaxation
  apply_residual<T>(c, x1, r, r1, st);
  coarse_correct<T>(c, r1, x1, st);  // multiplicative coarse correction
  apply_residual<T>(c, x1, r, r1, st);
  run_asm<T, T, double>(c, r1, z, c->omega, st, x1);  // post-relaxation, z = x1 + omega ASM(r1)
}

void pc_apply_impl(fdm_ctx *c, const double *r, double *z, cudaStream_t st) {
  const int64_t n = c->g.ndof;
  if (c->opt.pc == FDM_PC_NONE) {
    copy(n, r, z, st);
    mask_dirichlet(c->g, z, st);
    c->launches += 2;
    return;
  }
  if (c->opt.precision == FDM_PREC_FP64) {
    if (c->opt.pc == FDM_PC_ASM) run_asm<double, double, double>(c, r, z, c->omega, st);
    else run_vcycle<double>(c, r, z, c->v1, c->v3, st);
  } else {
    if (c->opt.pc == FDM_PC_ASM) {
      run_asm<float, double, double>(c, r, z, c->omega, st);
    } else {
      run_vcycle<float>(c, r, z, c->f1, c->f3, st);
    }
  }
}

// ---------------------------------------------------------------- set-up pieces
void setup_geometry(fdm_ctx *c, const fdm_mesh *mesh, const fdm_coeff *coeff) {
  const int n = c->g.n, p = c->p, ncell = c->g.ncell;
  std::vector<double> xv(mesh->xv, mesh->xv + mesh->nx + 1), yv(mesh->yv, mesh->yv + mesh->ny + 1),
      zv(mesh->zv, mesh->zv + mesh->nz + 1);
  for (auto *v : {&xv, &yv, &zv})
    for (size_t i = 0; i + 1 < v->size(); ++i)
      if (!((*v)[i + 1] > (*v)[i])) fail(FDM_EINVAL, "vertex coordinates must be strictly increasing");
  c->vert[0] = xv;
  c->vert[1] = yv;
  c->vert[2] = zv;
  std::vector<double> mub(3 * ncell);
  for (int cz = 0; cz < c->g.nz; ++cz)
    for (int cy = 0; cy < c->g.ny; ++cy)
      for (int cx = 0; cx < c->g.nx; ++cx) {
        int e = cx + c->g.nx * (cy + c->g.ny * cz);
        double L[3] = {0.5 * (xv[cx + 1] - xv[cx]), 0.5 * (yv[cy + 1] - yv[cy]), 0.5 * (zv[cz + 1] - zv[cz])};
        double vol = L[0] * L[1] * L[2];
        for (int a = 0; a < 3; ++a) mub[3 * e + a] = vol / (L[a] * L[a]);  // Section 2.2
      }
  c->mu_box = c->upload(mub);
  std::vector<double> mu = mub;
  if (mesh->jac) {
    c->general = 1;
    const int nq = n * n * n;
    std::vector<double> Gw((size_t)6 * nq * ncell), dw((size_t)nq * ncell);
    for (int e = 0; e < ncell; ++e) {
      double avg[3] = {0, 0, 0};
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            int q = i + n * (j + n * k);
            const double *J = mesh->jac + ((size_t)e * nq + q) * 9;
            double a00 = J[4] * J[8] - J[5] * J[7], a01 = J[2] * J[7] - J[1] * J[8], a02 = J[1] * J[5] - J[2] * J[4];
            double a10 = J[5] * J[6] - J[3] * J[8], a11 = J[0] * J[8] - J[2] * J[6], a12 = J[2] * J[3] - J[0] * J[5];
            double a20 = J[3] * J[7] - J[4] * J[6], a21 = J[1] * J[6] - J[0] * J[7], a22 = J[0] * J[4] - J[1] * J[3];
            double det = J[0] * a00 + J[1] * a10 + J[2] * a20;
            if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) fail(FDM_EINVAL, "singular Jacobian");
            double Ji[9] = {a00 / det, a01 / det, a02 / det, a10 / det, a11 / det, a12 / det,
                            a20 / det, a21 / det, a22 / det};
            double kap = (coeff && coeff->kappa_q) ? coeff->kappa_q[(size_t)e * nq + q] : 1.0;
            double w = c->basis.wq[i] * c->basis.wq[j] * c->basis.wq[k];
            // Ghat = kappa |det J| J^{-1} J^{-T}   (Section 2.7)
            double G[3][3];
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int r = 0; r < 3; ++r) s += Ji[a * 3 + r] * Ji[b * 3 + r];
                G[a][b] = kap * std::fabs(det) * s;
              }
            double *o = &Gw[((size_t)e * nq + q) * 6];
            o[0] = w * G[0][0]; o[1] = w * G[1][1]; o[2] = w * G[2][2];
            o[3] = w * G[0][1]; o[4] = w * G[0][2]; o[5] = w * G[1][2];
            dw[(size_t)e * nq + q] = w * std::fabs(det);
            for (int a = 0; a < 3; ++a) avg[a] += w * G[a][a];
          }
      for (int a = 0; a < 3; ++a) mu[3 * e + a] = avg[a] / 8.0;  // |K_hat| = 8
    }
    c->Gw64 = c->upload(Gw);
    c->detw64 = c->upload(dw);
    std::vector<float> Gf(Gw.begin(), Gw.end()), df(dw.begin(), dw.end());
    c->Gw32 = c->upload(Gf);
    c->detw32 = c->upload(df);
    c->mubar = c->upload(mu);
    c->wq64 = c->upload(c->basis.wq);
    if (coeff && coeff->samples27) {
      for (size_t i = 0; i < (size_t)ncell * 27; ++i)
        if (!(coeff->samples27[10 * i] > 0.0)) fail(FDM_EINVAL, "samples27: kappa must be positive");
      std::vector<double> s27(coeff->samples27, coeff->samples27 + (size_t)ncell * 270);
      double *d_s27 = c->upload(s27);
      c->feat = c->alloc<float>((size_t)ncell * MLP_NIN);
      const Basis1D b3 = make_basis(2);  // its Gauss rule has 3 points
      launch_surr_features(ncell, d_s27, b3.wq.data(), c->feat, 0);
      FDM_CUDA(cudaDeviceSynchronize());
    }
  } else if (coeff && coeff->samples27) {
    fail(FDM_EINVAL, "samples27 needs curved cells (mesh->jac)");
  }
  if (coeff && coeff->mu) {  // separable coefficients of the relaxation supplied by the caller
    for (int64_t i = 0; i < 3 * (int64_t)ncell; ++i)
      if (!(coeff->mu[i] > 0.0) || !std::isfinite(coeff->mu[i])) fail(FDM_EINVAL, "coeff->mu must be positive");
    mu.assign(coeff->mu, coeff->mu + 3 * (size_t)ncell);
  }
  c->mu = c->upload(mu);
  (void)p;
}

void setup_tables(fdm_ctx *c) {
  const Basis1D &b = c->basis;
  const int n = b.n;
  std::vector<double> t(tab_size(n), 0.0);
  auto put = [&](int which, const std::vector<double> &M) { std::copy(M.begin(), M.end(), t.begin() + tab_off(which, n)); };
  put(TAB_A, b.A);
  put(TAB_B, b.B);
  put(TAB_AF, b.Af);
  put(TAB_BF, b.Bf);
  put(TAB_T, b.T);
  put(TAB_VQ, b.Vq);
  put(TAB_DQ, b.Dq);
  std::copy(b.xi.begin(), b.xi.end(), t.begin() + tab_off(TAB_XI, n));
  put(TAB_VE, b.Ve);
  std::copy(b.lame.begin(), b.lame.end(), t.begin() + tab_off(TAB_LE, n));
  c->tab64 = c->upload(t);
  std::vector<float> tf(t.begin(), t.end());
  c->tab32 = c->upload(tf);
}

// Cluster patch solve: the patches of the classes with n1 > 0 and n2 > 0 come
// first in the order (heaviest first); the smallest cluster (2, 4, 8 or 16 CTAs)
// whose share of L21 rows fits in shared memory is used, if the GPU can host it.
template <typename T>
bool cluster_config(fdm_ctx *c, ClusterArgs<T> &a) {
  int n2max = 0, ldmax = 0;
  for (const PatchClass &C : c->classes)
    if (C.n1 > 0 && C.n2 > 0) {
      n2max = std::max(n2max, C.n2);
      ldmax = std::max(ldmax, C.ld21);
    }
  if (c->n_heavy == 0 || n2max == 0) return false;
  const int thr = c->cl_threads;
  a.g = c->g;
  a.npatch = c->n_heavy;
  a.ld_cap = ldmax;
  a.n2_cap = (n2max + 3) & ~3;
  a.maxG = c->maxG;
  a.tmpcap = std::max({4 * thr, a.n2_cap, a.ld_cap});
  if (a.n2_cap / 4 > thr || a.ld_cap / 4 > thr) return false;  // one thread per 4-column group
  a.timeout_ns = (uint64_t)(std::max(c->opt.wait_timeout_s, 0.0) * 1e9);
  a.inject_stall = c->opt.inject_stall;
  for (int cs : {2, 4, 8, 16}) {
    a.cs = cs;
    a.rows_cap = (n2max + cs - 1) / cs;
    if (patch_cluster_smem<T>(a) > 224 * 1024) continue;
    return patch_cluster_fits<T>(a, thr) > 0;
  }
  return false;
}

void setup_cluster(fdm_ctx *c) {
  // the prefix of the order with a dense top level; the rest must have none
  int nh = 0;
  std::vector<int> order(c->nsolve);
  FDM_CUDA(cudaMemcpy(order.data(), c->d_order, sizeof(int) * c->nsolve, cudaMemcpyDeviceToHost));
  while (nh < c->nsolve) {
    const PatchClass &C = c->classes[c->h_patches[order[nh]].cls];
    if (!(C.n1 > 0 && C.n2 > 0)) break;
    ++nh;
  }
  for (int i = nh; i < c->nsolve; ++i)
    if (c->classes[c->h_patches[order[i]].cls].n2 > 0) nh = 0;
  c->n_heavy = nh;
  int n2max = 0;
  for (const PatchClass &C : c->classes) n2max = std::max(n2max, C.n2);
  c->cl_threads = n2max > 400 ? 512 : 256;
  const bool want = c->opt.patch_kernel == 4;
  c->cl32 = want && cluster_config<float>(c, c->cla32);
  c->cl64 = want && cluster_config<double>(c, c->cla64);
}

void setup_patches(fdm_ctx *c) {
  const int p = c->p;
  // factor form: the Schur-coupling form serves the one-CTA-per-patch solve;
  // the streamed, resident and cluster kernels read the L form
  const bool l_kernel = c->opt.patch_kernel >= 2 && c->opt.patch_kernel <= 4;
  if (c->opt.patch_form == 2 && l_kernel) fail(FDM_EINVAL, "patch_form 2 needs patch_kernel 0, 1 or 5");
  if (c->opt.patch_form == 1 && c->opt.patch_kernel >= 5)
    fail(FDM_EINVAL, "patch_kernel 5, 6 and 7 need the Schur-coupling form");
  if (c->opt.patch_kernel < 0 || c->opt.patch_kernel > 7) fail(FDM_EINVAL, "patch_kernel out of range");
  c->scform = c->opt.patch_form == 2 || (c->opt.patch_form == 0 && !l_kernel);
  c->sc_persist = c->scform && c->opt.patch_kernel == 5;
  c->sc_full = c->scform && c->opt.patch_kernel == 6;
  c->sc_warp = c->scform && c->opt.patch_kernel == 7;
  c->classes = build_classes(p, c->scform);
  c->nbuf = c->opt.stream_buffers > 0 ? c->opt.stream_buffers : 4;
  c->buf_bytes = 1024 * (c->opt.stream_buffer_kb > 0 ? c->opt.stream_buffer_kb : 16);
  // default: one CTA per patch reading the factor directly (measured fastest on
  // GB300 for p <= 15); the streamed ring (patch_kernel = 2) reads the factor
  // from DRAM once but is latency-bound per chunk
  c->stream = c->opt.patch_kernel == 2;
  if (c->nbuf < 2 || c->nbuf > 16 || c->buf_bytes > 96 * 1024) fail(FDM_EINVAL, "stream buffers out of range");
  c->h_cls.resize(8);
  for (int id = 0; id < 8; ++id) {
    const PatchClass &C = c->classes[id];
    ClassDev &D = c->h_cls[id];
    D.nd = C.nd; D.nI = C.nI; D.nG = C.nG; D.n0 = C.n0; D.n1 = C.n1; D.n2 = C.n2;
    D.nlines = C.nlines; D.K0 = C.K0; D.nrow0 = C.nrow0; D.ldr0 = C.ldr0; D.ld21 = C.ld21;
    for (int a = 0; a < 3; ++a) { D.dim[a] = C.dim[a]; D.full[a] = C.full[a]; }
    D.off_dinv0 = C.off_dinv0; D.off_ell = C.off_ell; D.off_lines = C.off_lines;
    D.off_l21 = C.off_l21; D.off_z = C.off_z; D.nval = C.nval;
    D.gpos = c->upload(C.gpos);
    D.line_start = c->upload(C.line_start);
    D.line_len = c->upload(C.line_len);
    D.line_off = c->upload(C.line_off);
    D.ell_col = c->upload(C.ell_col);
    D.c0_ptr = c->upload(C.c0_ptr);
    D.c0_pos = c->upload(C.c0_pos);
    D.r0_ptr = c->upload(C.r0_ptr);
    D.r0_idx = c->upload(C.r0_idx);
    D.zoff = c->upload(C.zoff);
    D.ginv = c->upload(C.ginv);
    D.line_of = c->upload(C.line_of);
    D.gsrc = c->upload(C.gsrc);
    D.sc = C.sc ? 1 : 0;
    D.KT = C.KT;
    D.ldT = C.ldT;
    D.off_st = C.off_st;
    D.st_col = c->upload(C.st_col);
    D.ct_ptr = c->upload(C.ct_ptr);
    D.ct_pos = c->upload(C.ct_pos);
    D.cB_ptr = c->upload(C.cB_ptr);
    D.cB_pos = c->upload(C.cB_pos);
    {
      std::vector<ChunkDev> s32 = build_schedule(C, 4, c->buf_bytes), s64 = build_schedule(C, 8, c->buf_bytes);
      D.sched32 = c->upload(s32);
      D.sched64 = c->upload(s64);
      D.nsched32 = (int)s32.size();
      D.nsched64 = (int)s64.size();
    }
    c->maxG = std::max(c->maxG, C.nG);
    c->maxN0 = std::max(c->maxN0, C.n0);
    c->maxN1 = std::max(c->maxN1, C.n1);
    c->maxN2 = std::max(c->maxN2, C.n2);
  }
  c->d_cls = c->upload(c->h_cls);
  {  // cell-to-star map: node (i, j, k) of a cell in the star of its corner o
    const int n = c->g.n, n3 = n * n * n, p1 = c->p - 1;
    std::vector<int> cm((size_t)64 * n3, -1);
    for (int id = 0; id < 8; ++id) {
      const PatchClass &C = c->classes[id];
      for (int o = 0; o < 8; ++o)
        for (int idx = 0; idx < n3; ++idx) {
          const int li[3] = {idx % n, (idx / n) % n, idx / (n * n)};
          int t[3];
          bool ok = true;
          for (int ax = 0; ax < 3; ++ax) {
            const int side = (o >> ax) & 1, i = li[ax];
            if (C.full[ax]) {
              if (side == 0) { ok = ok && i <= c->p - 1; t[ax] = i + p1; }
              else { ok = ok && i >= 1; t[ax] = i - 1; }
            } else {
              ok = ok && i >= 1 && i <= c->p - 1;
              t[ax] = i - 1;
            }
          }
          if (ok && C.nd > 0) cm[((size_t)id * 8 + o) * n3 + idx] = C.ginv[t[0] + C.dim[0] * (t[1] + C.dim[1] * t[2])];
        }
    }
    c->cmap = c->upload(cm);
  }
  const int nvx = c->g.nx + 1, nvy = c->g.ny + 1, nvz = c->g.nz + 1;
  c->npatch = nvx * nvy * nvz;
  c->h_patches.resize(c->npatch);
  int64_t voff = 0, xoff = 0;
  std::vector<int> order;
  for (int vz = 0; vz < nvz; ++vz)
    for (int vy = 0; vy < nvy; ++vy)
      for (int vx = 0; vx < nvx; ++vx) {
        int pid = vx + nvx * (vy + nvy * vz);
        int v[3] = {vx, vy, vz}, nc[3] = {c->g.nx, c->g.ny, c->g.nz}, cls = 0;
        for (int a = 0; a < 3; ++a)
          if (v[a] >= 1 && v[a] <= nc[a] - 1) cls |= 1 << a;
        PatchDev &P = c->h_patches[pid];
        P.cls = cls;
        P.v[0] = vx; P.v[1] = vy; P.v[2] = vz;
        P.voff = voff;
        P.xoff = xoff;
        voff += c->classes[cls].nval;
        xoff += c->classes[cls].nG;  // the stars' interface solutions
        if (c->classes[cls].nd > 0) order.push_back(pid);
      }
  // heaviest patches first (one CTA each) for load balance
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return c->classes[c->h_patches[a].cls].nval > c->classes[c->h_patches[b].cls].nval;
  });
  c->nsolve = (int)order.size();
  std::vector<int> order_nz;
  for (int pid : order)
    if (c->classes[c->h_patches[pid].cls].nG > 0) order_nz.push_back(pid);
  c->nsolve_nz = (int)order_nz.size();
  c->d_order_nz = c->upload(order_nz);
  c->status = c->alloc<int>(1);
  FDM_CUDA(cudaMemset(c->status, 0, sizeof(int)));
  c->nval_total = voff;
  c->nstar_total = xoff;
  c->d_patches = c->upload(c->h_patches);
  c->d_order = c->upload(order);
  c->L64 = c->alloc<double>(voff);
  c->L32 = c->alloc<float>(voff);
  c->X64 = c->alloc<double>(xoff);
  c->X32 = c->alloc<float>(xoff);
  const int64_t ne = (int64_t)c->g.ncell * c->g.n * c->g.n * c->g.n;
  c->E64 = c->alloc<double>(ne);
  c->E32 = c->alloc<float>(ne);
  c->smem64 = patch_smem_bytes<double>(c->g.n, c->maxG, c->maxN1, c->maxN2);
  c->smem32 = patch_smem_bytes<float>(c->g.n, c->maxG, c->maxN1, c->maxN2);
  c->patch_threads = c->opt.patch_threads > 0 ? c->opt.patch_threads : (c->maxG > 1000 ? 1024 : 256);
  if (c->scform) {  // 256 or 512 threads
    c->patch_threads = c->opt.patch_threads > 0 ? (c->opt.patch_threads >= 512 ? 512 : c->opt.patch_threads <= 128 ? 128 : 256)
                                                : (c->maxG > 1000 ? 512 : 256);
    if (patch_sc_smem<double>(c->maxG, c->maxN1, c->maxN2, 512, 0) > 224 * 1024)
      fail(FDM_EINVAL, "patch interface too large for shared memory (Schur-coupling form)");
    // the variant of the 256-thread kernel (rows8 holds its code): 0 = two rows of W per warp,
    // all values before W staged; 1 = four rows; 2 = two rows, lower block staged only
    if (c->opt.sc_variant < 0 || c->opt.sc_variant > 4) fail(FDM_EINVAL, "sc_variant out of range");
    c->rows8 = c->opt.sc_variant > 0 ? c->opt.sc_variant - 1 : 0;
    // stage the values before W in shared memory where the largest class's fit in 48 KB
    int64_t head = 0, bhead = 0;
    for (const PatchClass &C : c->classes) {
      head = std::max<int64_t>(head, C.off_z);
      bhead = std::max<int64_t>(bhead, C.off_st);
    }
    c->headcap32 = head * 4 <= 48 * 1024 ? (int)head : 0;
    c->headcap64 = head * 8 <= 48 * 1024 ? (int)head : 0;
    c->bcap32 = bhead * 4 <= 24 * 1024 ? (int)bhead : 0;
    c->bcap64 = bhead * 8 <= 24 * 1024 ? (int)bhead : 0;
    int64_t nvmax = 0;  // the fully staged kernel's buffers: the largest class's values
    for (const PatchClass &C : c->classes) nvmax = std::max<int64_t>(nvmax, C.nval);
    c->fcap_sc = (int)((nvmax + 3) & ~3);
    if (c->sc_warp) {
      if (c->opt.patch_threads > 0 && c->opt.patch_threads != 128 && c->opt.patch_threads != 256)
        fail(FDM_EINVAL, "patch_kernel 7: patch_threads must be 128 or 256 (4 or 8 patches per CTA)");
      c->patch_threads = c->opt.patch_threads > 0 ? c->opt.patch_threads : 256;
      if (!scw_fits(c, c->opt.precision == FDM_PREC_FP32, c->patch_threads))
        fail(FDM_EINVAL, "patch_kernel 7: the interface is too large for one warp per patch");
    }
    if (c->sc_full) {
      const size_t need = c->opt.precision == FDM_PREC_FP32
                              ? patch_sc_smem<float>(c->maxG, c->maxN1, c->maxN2, c->patch_threads, 2 * c->fcap_sc)
                              : patch_sc_smem<double>(c->maxG, c->maxN1, c->maxN2, c->patch_threads, 2 * c->fcap_sc);
      if (need > kScfSmemCap)
        fail(FDM_EINVAL, "patch_kernel 6: two patch operators do not fit in shared memory (" + std::to_string(need) +
                             " bytes)");
    }
  }
  // eight rows per warp in flight pay off for long L21 rows with 256 threads (measured:
  // 10 % at Q8, neutral at Q7, slower with 1024 threads at Q15)
  {
    int ld21 = 0;
    for (const PatchClass &C : c->classes) ld21 = std::max(ld21, C.ld21);
    c->rows8 = c->opt.patch_rows_per_warp == 8   ? 1
               : c->opt.patch_rows_per_warp == 4 ? 0
                                                   : (c->patch_threads == 256 && ld21 >= 200 ? 1 : 0);
  }
  setup_cluster(c);
  c->smem64 = patch_smem_for_occupancy<double>(c->smem64, c->opt.patch_ctas_per_sm);
  c->smem32 = patch_smem_for_occupancy<float>(c->smem32, c->opt.patch_ctas_per_sm);
  if (c->smem64 > 200 * 1024) fail(FDM_EINVAL, "patch interface too large for shared memory");
  // resident variant (patch_kernel = 3) where one patch's whole factor fits in
  // shared memory; not the default: with one 184 KB factor per SM (Q7) no other
  // patch overlaps the latency of the solve phases, and it measured slower
  // than the one-CTA-per-patch kernel
  int64_t maxval = 0;
  for (const PatchClass &C : c->classes) maxval = std::max<int64_t>(maxval, C.nval);
  c->fcap = (int)((maxval + 3) & ~3);
  c->res_threads = c->opt.patch_threads > 0 ? c->opt.patch_threads : 512;
  c->res_tmp = patch_resident_tmp(c->maxN1, c->maxN2, c->res_threads);
  c->rsmem32 = patch_resident_smem<float>(c->fcap, c->maxG, c->res_tmp);
  c->rsmem64 = patch_resident_smem<double>(c->fcap, c->maxG, c->res_tmp);
  const bool want_res = !c->stream && c->opt.patch_kernel == 3;
  const size_t res_cap = 225 * 1024;
  c->res32 = want_res && c->rsmem32 <= res_cap;
  c->res64 = want_res && c->rsmem64 <= res_cap;
  if (c->stream) {
    size_t need = std::max(stream_smem_bytes<double>(stream_args<double>(c)), stream_smem_bytes<float>(stream_args<float>(c)));
    if (need > 220 * 1024) fail(FDM_EINVAL, "streamed patch solve needs too much shared memory; use fewer or smaller buffers");
  }
}

// numeric factorisation of every patch (FP64 with an FP32 copy)
void factor_all(fdm_ctx *c, cudaStream_t st) {
  const int64_t per = (int64_t)c->maxG * c->maxG;
  if (per == 0) return;
  std::vector<int> ids;
  for (int pid = 0; pid < c->npatch; ++pid)
    if (c->classes[c->h_patches[pid].cls].nG > 0 || c->classes[c->h_patches[pid].cls].n0 >= 0) ids.push_back(pid);
  const int64_t budget = (int64_t)6 << 30;  // bytes of dense workspace
  int batch = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)ids.size(), budget / (per * 8)));
  double *S = c->alloc<double>((size_t)batch * per);
  int *status = c->alloc<int>(1);
  int *plist = c->alloc<int>(batch);
  FDM_CUDA(cudaMemsetAsync(status, 0, sizeof(int), st));
  for (size_t b0 = 0; b0 < ids.size(); b0 += batch) {
    int cnt = (int)std::min<size_t>(batch, ids.size() - b0);
    FDM_CUDA(cudaMemcpyAsync(plist, ids.data() + b0, cnt * sizeof(int), cudaMemcpyHostToDevice, st));
    FactorArgs a{c->g, c->d_cls, c->d_patches, plist, c->mu, c->tab64, S, per, c->L64, c->L32, status};
    launch_factor_batch(a, cnt, st);
    FDM_CUDA(cudaStreamSynchronize(st));
  }
  FDM_CUDA(cudaGetLastError());
  int hs = 0;
  FDM_CUDA(cudaMemcpy(&hs, status, sizeof(int), cudaMemcpyDeviceToHost));
  // workspace is released with the context; free it now to return memory early
  cudaFree(S);
  c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), (void *)S));
  if (hs) fail(FDM_ENOTSPD, "a patch Schur complement has a nonpositive pivot");
}

// in-place Cholesky of a banded SPD matrix in lower storage Lb[i][k] = A[i][i-k]
void banded_cholesky(int m, int bw, std::vector<double> &Lb) {
  for (int i = 0; i < m; ++i)
    for (int k = std::max(0, i - bw); k <= i; ++k) {
      double s = Lb[(size_t)i * (bw + 1) + (i - k)];
      for (int j = std::max(0, std::max(i - bw, k - bw)); j < k; ++j)
        s -= Lb[(size_t)i * (bw + 1) + (i - j)] * Lb[(size_t)k * (bw + 1) + (k - j)];
      if (k == i) {
        if (!(s > 0.0)) fail(FDM_ENOTSPD, "coarse operator is not positive definite");
        Lb[(size_t)i * (bw + 1)] = std::sqrt(s);
      } else {
        Lb[(size_t)i * (bw + 1) + (i - k)] = s / Lb[(size_t)k * (bw + 1)];
      }
    }
}

// device copies of one multigrid level in precision T
template <typename T>
GmgDev<T> upload_level(fdm_ctx *c, const GmgHostLevel &H, double omega) {
  GmgDev<T> d;
  for (int a = 0; a < 3; ++a) d.m[a] = H.m[a];
  d.nf = H.nf;
  std::vector<T> A(H.A.begin(), H.A.end()), dw(H.nf);
  for (int i = 0; i < H.nf; ++i) dw[i] = (T)(omega / H.A[(size_t)13 * H.nf + i]);
  d.A = c->upload(A);
  d.dw = c->upload(dw);
  for (int a = 0; a < 3; ++a)
    if (!H.t[a].empty()) d.t[a] = c->upload(std::vector<T>(H.t[a].begin(), H.t[a].end()));
  return d;
}

template <typename T>
void alloc_gmg_vectors(fdm_ctx *c, T *rc, T *xc) {
  auto &G = c->gmg<T>();
  const int L = c->gmg_L;
  G.lev.clear();
  for (int l = 0; l <= L; ++l) G.lev.push_back(upload_level<T>(c, c->gmg_host[l], c->gmg_omega));
  G.b.assign(L + 1, nullptr);
  G.out.assign(L + 1, nullptr);
  G.xa.assign(L + 1, nullptr);
  G.xb.assign(L + 1, nullptr);
  G.r.assign(L + 1, nullptr);
  for (int l = 0; l <= L; ++l) {
    const int nf = c->gmg_host[l].nf;
    G.b[l] = l == 0 ? rc : c->alloc<T>(nf);
    G.out[l] = l == 0 ? xc : c->alloc<T>(nf);
    if (l < L) {
      G.xa[l] = c->alloc<T>(nf);
      G.xb[l] = c->alloc<T>(nf);
      G.r[l] = c->alloc<T>(nf);
    }
  }
}

// The Q1 coarse space (Section 3): the Galerkin operator of the p-coarse
// problem, assembled from the cells' 8 x 8 matrices as a 27-point stencil over
// the free vertices, then either inverted densely (from a banded Cholesky
// factor) or handed to the geometric multigrid, whose coarsest level is
// inverted the same way.
void setup_coarse(fdm_ctx *c, cudaStream_t st) {
  const int nvx = c->g.nx + 1, nvy = c->g.ny + 1, nvz = c->g.nz + 1, nv = nvx * nvy * nvz;
  std::vector<int> cfree(nv, -1);
  int nc = 0;
  for (int vz = 0; vz < nvz; ++vz)
    for (int vy = 0; vy < nvy; ++vy)
      for (int vx = 0; vx < nvx; ++vx)
        if (vx > 0 && vy > 0 && vz > 0 && vx < nvx - 1 && vy < nvy - 1 && vz < nvz - 1)
          cfree[vx + nvx * (vy + nvy * vz)] = nc++;
  c->nc = nc;
  c->cfree = c->upload(cfree);
  c->cb64 = c->alloc<double>((size_t)8 * c->g.ncell);
  c->cb32 = c->alloc<float>((size_t)8 * c->g.ncell);
  c->rc64 = c->alloc<double>(nc);
  c->xc64 = c->alloc<double>(nc);
  c->rc32 = c->alloc<float>(nc);
  c->xc32 = c->alloc<float>(nc);
  c->gmg_L = 0;
  c->gmg_host.clear();
  if (nc == 0) return;
  double *Ac = c->alloc<double>((size_t)64 * c->g.ncell);
  launch_coarse_cell_matrices(c->op_args(false), Ac, st);
  FDM_CUDA(cudaGetLastError());
  std::vector<double> hAc((size_t)64 * c->g.ncell);
  FDM_CUDA(cudaMemcpyAsync(hAc.data(), Ac, hAc.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  FDM_CUDA(cudaStreamSynchronize(st));
  // level 0: the Q1 operator as a 27-point stencil (cell contributions in cell order)
  std::vector<GmgHostLevel> &lev = c->gmg_host;
  lev.emplace_back();
  {
    GmgHostLevel &L0 = lev[0];
    const int ncell[3] = {c->g.nx, c->g.ny, c->g.nz};
    for (int a = 0; a < 3; ++a) {
      L0.n[a] = ncell[a];
      L0.m[a] = ncell[a] - 1;
      L0.x[a] = c->vert[a];
    }
    L0.nf = nc;
    L0.A.assign((size_t)27 * nc, 0.0);
    for (int cz = 0; cz < c->g.nz; ++cz)
      for (int cy = 0; cy < c->g.ny; ++cy)
        for (int cx = 0; cx < c->g.nx; ++cx) {
          const int e = cx + c->g.nx * (cy + c->g.ny * cz);
          int f[8];
          for (int s = 0; s < 8; ++s)
            f[s] = cfree[(cx + (s & 1)) + nvx * ((cy + ((s >> 1) & 1)) + nvy * (cz + (s >> 2)))];
          for (int t = 0; t < 8; ++t)
            for (int s = 0; s < 8; ++s)
              if (f[t] >= 0 && f[s] >= 0) {
                const int k = ((s & 1) - (t & 1) + 1) + 3 * (((s >> 1) & 1) - ((t >> 1) & 1) + 1) + 9 * ((s >> 2) - (t >> 2) + 1);
                L0.A[(size_t)k * nc + f[t]] += hAc[(size_t)e * 64 + t * 8 + s];
              }
        }
  }
  int want = c->opt.coarse_levels;
  if (want < 0) want = nc > 4096 ? 64 : 0;
  c->gmg_nu = c->opt.gmg_nu > 0 ? c->opt.gmg_nu : 2;
  c->gmg_omega = c->opt.gmg_omega > 0.0 ? c->opt.gmg_omega : 2.0 / 3.0;
  gmg_coarsen(lev, want);
  c->gmg_L = (int)lev.size() - 1;
  // the dense inverse of the coarsest level, from its banded Cholesky factor
  // (lexicographic order: the band reaches the (+1, +1, +1) neighbour)
  const GmgHostLevel &B = lev.back();
  const int m = B.nf;
  const int bw = 1 + B.m[0] + B.m[0] * B.m[1];
  std::vector<double> Lb((size_t)m * (bw + 1), 0.0);
  for (int i = 0; i < m; ++i) {
    const int ix = i % B.m[0], iy = (i / B.m[0]) % B.m[1], iz = i / (B.m[0] * B.m[1]);
    for (int k = 0; k < 27; ++k) {
      const int jx = ix + k % 3 - 1, jy = iy + (k / 3) % 3 - 1, jz = iz + k / 9 - 1;
      if (jx < 0 || jy < 0 || jz < 0 || jx >= B.m[0] || jy >= B.m[1] || jz >= B.m[2]) continue;
      const int j = jx + B.m[0] * (jy + B.m[1] * jz);
      if (j <= i) Lb[(size_t)i * (bw + 1) + (i - j)] = B.A[(size_t)k * m + i];
    }
  }
  banded_cholesky(m, bw, Lb);
  double *dLb = c->upload(Lb);
  c->nc_dense = m;
  c->Acinv64 = c->alloc<double>((size_t)m * m);
  c->Acinv32 = c->alloc<float>((size_t)m * m);
  launch_banded_inverse(m, bw, dLb, c->Acinv64, st);
  launch_convert<double, float>((int64_t)m * m, c->Acinv64, c->Acinv32, st);
  if (c->gmg_L > 0) {
    alloc_gmg_vectors<double>(c, c->rc64, c->xc64);
    alloc_gmg_vectors<float>(c, c->rc32, c->xc32);
  }
  FDM_CUDA(cudaStreamSynchronize(st));
  FDM_CUDA(cudaGetLastError());
}

// extreme eigenvalues of the symmetric tridiagonal matrix (d, e) by bisection
void tridiag_extremes(const std::vector<double> &d, const std::vector<double> &e, double &lo, double &hi) {
  const int m = (int)d.size();
  auto below = [&](double x) {
    int cnt = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      q = d[i] - x - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++cnt;
    }
    return cnt;
  };
  double a = d[0], b = d[0];
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(e[i]) : 0.0);
    a = std::min(a, d[i] - r);
    b = std::max(b, d[i] + r);
  }
  auto kth = [&](int k) {
    double l = a, h = b;
    for (int it = 0; it < 300 && h - l > 1e-15 * std::max(std::fabs(l), std::fabs(h)); ++it) {
      double mid = 0.5 * (l + h);
      if (below(mid) > k) h = mid; else l = mid;
    }
    return 0.5 * (l + h);
  };
  lo = kth(0);
  hi = kth(m - 1);
}

// splitmix64 + Box-Muller: the library's own seeded N(0,1) stream
void normal_vector(uint64_t seed, int64_t n, std::vector<double> &out) {
  out.resize(n);
  uint64_t s = seed;
  auto next = [&]() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (int64_t i = 0; i < n; i += 2) {
    double u1 = ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double u2 = ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    double rr = std::sqrt(-2.0 * std::log(u1)), th = 2.0 * M_PI * u2;
    out[i] = rr * std::cos(th);
    if (i + 1 < n) out[i + 1] = rr * std::sin(th);
  }
}

// omega from k CG-Lanczos steps on P_ASM^{-1} A (Section 2.5), FP64
void lanczos_omega(fdm_ctx *c, const double *start_host, cudaStream_t st) {
  const int64_t n = c->g.ndof;
  std::vector<double> b0;
  if (start_host) b0.assign(start_host, start_host + n);
  else normal_vector(c->opt.lanczos_seed, n, b0);
  FDM_CUDA(cudaMemcpyAsync(c->r, b0.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
  mask_dirichlet(c->g, c->r, st);
  run_asm<double, double, double>(c, c->r, c->z, 1.0, st);
  FDM_CUDA(cudaMemcpyAsync(c->d, c->z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double h[2];
  launch_dot(n, c->r, c->z, c->partial, c->dots, st);
  FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
  FDM_CUDA(cudaStreamSynchronize(st));
  double rz = h[0];
  std::vector<double> al, be;
  for (int k = 0; k < c->opt.lanczos_steps; ++k) {
    if (!(rz > 0.0)) break;
    launch_operator<double, double, double>(c->op_args(false), false, c->d, c->q, c->E64, st);
    launch_dot(n, c->d, c->q, c->partial, c->dots, st);
    FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    if (!(h[0] > 0.0)) break;
    double alpha = rz / h[0];
    al.push_back(alpha);
    launch_axpby<double>(n, -alpha, c->q, 1.0, c->r, c->r, st);
    run_asm<double, double, double>(c, c->r, c->z, 1.0, st);
    launch_dot(n, c->r, c->z, c->partial, c->dots, st);
    FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    double beta = h[0] / rz;
    be.push_back(beta);
    rz = h[0];
    launch_axpby<double>(n, 1.0, c->z, beta, c->d, c->d, st);
  }
  const int m = (int)al.size();
  if (m < 1) fail(FDM_EINVAL, "Lanczos: no steps could be taken");
  std::vector<double> dd(m), ee(std::max(m - 1, 1), 0.0);
  for (int j = 0; j < m; ++j) {
    dd[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < m) ee[j] = std::sqrt(be[j]) / al[j];
  }
  tridiag_extremes(dd, ee, c->lmin, c->lmax);
  const double alpha = 0.25;
  c->omega = 2.0 / ((1.0 + alpha) * c->lmax + (1.0 - alpha) * c->lmin);
}

// ---- autotuner: the patch-solve variant with the shortest relaxation sweep
// Candidates: one CTA per patch with 256 threads (four or eight rows per warp
// in the forward products), 512 or 1024 threads, and the resident kernel where
// a patch factor fits in shared memory.  Each is timed with CUDA events over
// `reps` sweeps in the context's preconditioner precision after two untimed
// ones, on the set-up's work vectors; the fastest is kept.
void autotune_patch(fdm_ctx *c, cudaStream_t st) {
  struct Cand { int kernel, threads, rows8; };
  std::vector<Cand> cands = {{1, 256, 0}, {1, 256, 1}, {1, 512, 0}, {1, 1024, 0}};
  const bool fp32 = c->opt.precision == FDM_PREC_FP32;
  const size_t rs = fp32 ? c->rsmem32 : c->rsmem64;
  if (c->scform) {  // the layout fixes the kernel
    cands = {{5, 128, 0}, {5, 256, 0}, {5, 256, 1}, {5, 256, 2}, {5, 512, 0}, {6, 256, 0}};
    for (int t : {256, 512, 1024}) {  // fully staged persistent kernel, where two patch operators fit
      const size_t need = fp32 ? patch_sc_smem<float>(c->maxG, c->maxN1, c->maxN2, t, 2 * c->fcap_sc)
                               : patch_sc_smem<double>(c->maxG, c->maxN1, c->maxN2, t, 2 * c->fcap_sc);
      if (need <= kScfSmemCap) cands.push_back({7, t, 0});
    }
    for (int t : {128, 256})  // one warp per patch, 4 or 8 patches per CTA
      if (scw_fits(c, fp32, t)) cands.push_back({8, t, 0});
  }
  else if (rs <= 225 * 1024) cands.push_back({3, 512, 0});
  const int64_t n = c->g.ndof;
  fill(n, 1.0, c->r, st);
  mask_dirichlet(c->g, c->r, st);
  cudaEvent_t e0, e1;
  FDM_CUDA(cudaEventCreate(&e0));
  FDM_CUDA(cudaEventCreate(&e1));
  const int reps = 5;
  double best = 1e300;
  Cand pick = {1, c->patch_threads, c->rows8};
  const int rthreads = c->res_threads;
  for (const Cand &k : cands) {
    c->patch_threads = k.threads;
    c->rows8 = k.rows8;
    c->res32 = fp32 && k.kernel == 3;
    c->res64 = !fp32 && k.kernel == 3;
    c->res_threads = k.threads;
    c->sc_persist = k.kernel == 6;
    c->sc_full = k.kernel == 7;
    c->sc_warp = k.kernel == 8;
    auto sweep = [&]() {
      if (fp32) run_asm<float, double, double>(c, c->r, c->z, c->omega, st);
      else run_asm<double, double, double>(c, c->r, c->z, c->omega, st);
    };
    sweep();
    sweep();
    FDM_CUDA(cudaEventRecord(e0, st));
    for (int i = 0; i < reps; ++i) sweep();
    FDM_CUDA(cudaEventRecord(e1, st));
    FDM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FDM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    const double us = 1e3 * ms / reps;
    if (us < best) {
      best = us;
      pick = k;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->patch_threads = pick.threads;
  c->rows8 = pick.rows8;
  c->res32 = fp32 && pick.kernel == 3;
  c->res64 = !fp32 && pick.kernel == 3;
  c->res_threads = pick.kernel == 3 ? pick.threads : rthreads;
  c->sc_persist = pick.kernel == 6;
  c->sc_full = pick.kernel == 7;
  c->sc_warp = pick.kernel == 8;
  c->tuning[0] = pick.kernel;
  c->tuning[1] = pick.threads;
  c->tuning[2] = pick.rows8;
  c->tuning[3] = best;
  c->tuning[4] = (double)cands.size();
}

// ---- batched solves: one CUDA graph, a device-driven PCG loop per problem
// Scalars of a problem in c->sc: [0] r.z, [1] alpha, [2] beta, [3] d.q, [4] true-residual checks,
// [7] flexible beta, [8] non-finite flag, [9] first iteration, [10] rtol^2, [11] maxit, [12] ||b||^2,
// [13] iterations, [14] ||r||^2, [15] converged.  c->dots: [0] r.z, [1] r.z_prev, [2] r.r, [3] d.q.
// Convergence is declared on the true residual: when the recursive residual
// meets the test, r is replaced by b - A x (FP64) and the test is repeated on
// it; if that fails the iteration continues from the replaced residual.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__global__ void k_btime(unsigned long long *t) {
  if (threadIdx.x == 0) t[0] = global_ns();
}
__global__ void k_bconst(double *sc, double flex, double rtol2, double maxit) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < 16; ++i) sc[i] = 0.0;
  sc[7] = flex;
  sc[10] = rtol2;
  sc[11] = maxit;
}
// ||b||^2 is in dots[2]: start the loop unless b = 0 (or maxit = 0)
__global__ void k_bstart(double *sc, const double *dots, cudaGraphConditionalHandle h) {
  if (threadIdx.x != 0) return;
  const double bb = dots[2];
  sc[12] = bb;
  sc[14] = bb;
  sc[9] = 1.0;
  sc[13] = 0.0;
  sc[15] = bb == 0.0 ? 1.0 : 0.0;
  if (!isfinite(bb)) sc[8] = 1.0;
  cudaGraphSetConditional(h, (bb > 0.0 && isfinite(bb) && sc[11] > 0.0) ? 1u : 0u);
}
// beta = (r.z - flex r.z_prev) / (r.z)_prev, 0 in the first iteration
__global__ void k_bbeta(double *sc, const double *dots) {
  if (threadIdx.x != 0) return;
  const double rz = dots[0];
  double b = 0.0;
  if (sc[9] == 0.0) {
    b = (sc[7] != 0.0 ? rz - dots[1] : rz) / sc[0];
    if (!isfinite(b)) {
      sc[8] = 1.0;
      b = 0.0;
    }
  }
  if (!isfinite(rz)) sc[8] = 1.0;
  sc[9] = 0.0;
  sc[2] = b;
  sc[0] = rz;
}
// end of an iteration: when the recursive residual meets ||r||^2 <= rtol^2 ||b||^2
// the true-residual check runs (hv = 1) and decides; otherwise stop at maxit or
// on a non-finite value
__global__ void k_bcheck(double *sc, const double *dots, cudaGraphConditionalHandle h,
                         cudaGraphConditionalHandle hv, unsigned long long *tend) {
  if (threadIdx.x != 0) return;
  const double rr = dots[2];
  const double it = sc[13] + 1.0;
  sc[13] = it;
  sc[14] = rr;
  if (!isfinite(rr)) sc[8] = 1.0;
  const bool conv = rr <= sc[10] * sc[12] && sc[8] == 0.0;
  sc[15] = 0.0;
  const bool stop = it >= sc[11] || sc[8] != 0.0;
  if (!conv && stop) *tend = global_ns();
  cudaGraphSetConditional(hv, conv ? 1u : 0u);
  cudaGraphSetConditional(h, (conv || stop) ? 0u : 1u);
}
// after r = b - A x: converged if the true residual meets the test, else
// continue from it (within maxit)
__global__ void k_bverify(double *sc, const double *dots, cudaGraphConditionalHandle h, unsigned long long *tend) {
  if (threadIdx.x != 0) return;
  const double rr = dots[2];
  sc[4] += 1.0;
  sc[14] = rr;
  if (!isfinite(rr)) sc[8] = 1.0;
  const bool conv = rr <= sc[10] * sc[12] && sc[8] == 0.0;
  sc[15] = conv ? 1.0 : 0.0;
  const bool done = conv || sc[13] >= sc[11] || sc[8] != 0.0;
  if (done) *tend = global_ns();
  cudaGraphSetConditional(h, done ? 0u : 1u);
}

void capture_iteration(fdm_ctx *c, double *x, cudaGraphConditionalHandle h, cudaGraphConditionalHandle hv,
                       unsigned long long *tend, cudaStream_t st) {
  const int64_t n = c->g.ndof;
  launch_dot(n, c->r, c->z, c->partial, c->dots + 1, st);  // r . z_prev (flexible beta)
  pc_apply_impl(c, c->r, c->z, st);
  launch_dot(n, c->r, c->z, c->partial, c->dots, st);
  k_bbeta<<<1, 32, 0, st>>>(c->sc, c->dots);
  launch_pcg_update_d(n, c->sc, c->z, c->d, st);
  apply_op<double>(c, c->d, c->q, st);
  launch_dot(n, c->d, c->q, c->partial, c->dots + 3, st);
  launch_pcg_scalars(0, c->sc, c->dots + 3, st);
  launch_pcg_update_xr(n, c->sc, c->d, c->q, x, c->r, st);
  launch_dot(n, c->r, c->r, c->partial, c->dots + 2, st);
  k_bcheck<<<1, 32, 0, st>>>(c->sc, c->dots, h, hv, tend);
  FDM_CUDA(cudaGetLastError());
}

// the true-residual check: r = b - A x (FP64, Dirichlet entries 0), ||r||^2, decide
void capture_verify(fdm_ctx *c, const double *b, const double *x, cudaGraphConditionalHandle h,
                    unsigned long long *tend, cudaStream_t st) {
  const int64_t n = c->g.ndof;
  apply_op<double>(c, x, c->q, st);
  launch_sub<double>(n, b, c->q, c->r, st);
  mask_dirichlet(c->g, c->r, st);
  launch_dot(n, c->r, c->r, c->partial, c->dots + 2, st);
  k_bverify<<<1, 32, 0, st>>>(c->sc, c->dots, h, tend);
  FDM_CUDA(cudaGetLastError());
}

// the single node of a captured (linear) graph that no other node depends on
cudaGraphNode_t graph_leaf(cudaGraph_t g) {
  size_t nn = 0;
  FDM_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  FDM_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
  cudaGraphNode_t leaf = nullptr;
  int leaves = 0;
  for (cudaGraphNode_t v : nodes) {
    size_t nd = 0;
    FDM_CUDA(cudaGraphNodeGetDependentNodes(v, nullptr, nullptr, &nd));
    if (nd == 0) {
      leaf = v;
      ++leaves;
    }
  }
  if (leaves != 1) fail(FDM_ECUDA, "captured PCG iteration does not end in a single node");
  return leaf;
}

// the scheduling priority of every kernel node of a captured graph
void set_kernel_priority(cudaGraph_t g, int prio) {
  size_t nn = 0;
  FDM_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  FDM_CUDA(cudaGraphGetNodes(g, nodes.data(), &nn));
  cudaKernelNodeAttrValue v{};
  v.priority = prio;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    FDM_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t == cudaGraphNodeTypeKernel) FDM_CUDA(cudaGraphKernelNodeSetAttribute(nd, cudaLaunchAttributePriority, &v));
  }
}

// per problem its kernels' priority: the smaller a problem (free dofs), the
// higher, so that small problems finish early while the larger ones fill the
// SMs they leave; the device's priority levels are spread over the size ranks
std::vector<int> batch_priorities(const std::vector<fdm_ctx *> &ctxs) {
  const int k = (int)ctxs.size();
  int least = 0, greatest = 0;
  FDM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  std::vector<int> order(k), prio(k, least);
  for (int i = 0; i < k; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctxs[a]->g.ndof < ctxs[b]->g.ndof; });
  const int levels = least - greatest + 1;
  for (int r = 0; r < k; ++r) prio[order[r]] = greatest + (int)((int64_t)r * levels / k);
  return prio;
}

void build_batch_graph(fdm_batch *B, const double *const *bv, double *const *xv, double rtol, int maxit) {
  B->release_graph();
  B->init_kernels.clear();
  B->body_kernels.clear();
  B->verify_kernels.clear();
  const int k = (int)B->ctxs.size();
  if (!B->cap) FDM_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  if (!B->d_times) FDM_CUDA(cudaMalloc(&B->d_times, sizeof(unsigned long long) * (k + 1)));
  cudaGraph_t G;
  FDM_CUDA(cudaGraphCreate(&G, 0));
  B->graph = G;
  cudaGraphNode_t t0;
  {
    cudaKernelNodeParams kp{};
    void *args[] = {&B->d_times};
    kp.func = (void *)k_btime;
    kp.gridDim = dim3(1);
    kp.blockDim = dim3(32);
    kp.kernelParams = args;
    FDM_CUDA(cudaGraphAddKernelNode(&t0, G, nullptr, 0, &kp));
  }
  const std::vector<int> prio = batch_priorities(B->ctxs);
  for (int i = 0; i < k; ++i) {
    fdm_ctx *c = B->ctxs[i];
    const int64_t n = c->g.ndof;
    const int64_t counted = c->launches;  // captured launches do not run now
    c->capturing = true;
    try {
      // x = 0, r = b (Dirichlet entries 0), z = d = 0, ||b||^2
      cudaGraph_t gi;
      FDM_CUDA(cudaGraphCreate(&gi, 0));
      FDM_CUDA(cudaStreamBeginCaptureToGraph(B->cap, gi, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      k_bconst<<<1, 32, 0, B->cap>>>(c->sc, c->opt.flexible_beta ? 1.0 : 0.0, rtol * rtol, (double)maxit);
      fill(n, 0.0, xv[i], B->cap);
      fill(n, 0.0, c->z, B->cap);
      fill(n, 0.0, c->d, B->cap);
      copy(n, bv[i], c->r, B->cap);
      mask_dirichlet(c->g, c->r, B->cap);
      launch_dot(n, c->r, c->r, c->partial, c->dots + 2, B->cap);
      FDM_CUDA(cudaStreamEndCapture(B->cap, &gi));
      cudaGraphNode_t ni, nb, nw;
      size_t nk = 0;
      FDM_CUDA(cudaGraphGetNodes(gi, nullptr, &nk));
      B->init_kernels.push_back(nk + 1);  // + the start kernel below
      set_kernel_priority(gi, prio[i]);
      FDM_CUDA(cudaGraphAddChildGraphNode(&ni, G, &t0, 1, gi));
      FDM_CUDA(cudaGraphDestroy(gi));
      cudaGraphConditionalHandle h;
      FDM_CUDA(cudaGraphConditionalHandleCreate(&h, G, 0, cudaGraphCondAssignDefault));
      {
        cudaKernelNodeParams kp{};
        double *sc = c->sc, *dots = c->dots;
        void *args[] = {&sc, &dots, &h};
        kp.func = (void *)k_bstart;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = args;
        FDM_CUDA(cudaGraphAddKernelNode(&nb, G, &ni, 1, &kp));
        cudaKernelNodeAttrValue v{};
        v.priority = prio[i];
        FDM_CUDA(cudaGraphKernelNodeSetAttribute(nb, cudaLaunchAttributePriority, &v));
      }
      cudaGraphNodeParams cp{};
      cp.type = cudaGraphNodeTypeConditional;
      cp.conditional.handle = h;
      cp.conditional.type = cudaGraphCondTypeWhile;
      cp.conditional.size = 1;
      FDM_CUDA(cudaGraphAddNode(&nw, G, &nb, nullptr, 1, &cp));
      cudaGraph_t body = cp.conditional.phGraph_out[0];
      cudaGraphConditionalHandle hv;
      FDM_CUDA(cudaGraphConditionalHandleCreate(&hv, body, 0, cudaGraphCondAssignDefault));
      FDM_CUDA(cudaStreamBeginCaptureToGraph(B->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      capture_iteration(c, xv[i], h, hv, B->d_times + 1 + i, B->cap);
      FDM_CUDA(cudaStreamEndCapture(B->cap, &body));
      size_t nbk = 0;
      FDM_CUDA(cudaGraphGetNodes(body, nullptr, &nbk));
      B->body_kernels.push_back(nbk);
      set_kernel_priority(body, prio[i]);
      // the true-residual check, run when the recursive residual has converged
      cudaGraphNode_t leaf = graph_leaf(body), nv;
      cudaGraphNodeParams vp{};
      vp.type = cudaGraphNodeTypeConditional;
      vp.conditional.handle = hv;
      vp.conditional.type = cudaGraphCondTypeIf;
      vp.conditional.size = 1;
      FDM_CUDA(cudaGraphAddNode(&nv, body, &leaf, nullptr, 1, &vp));
      cudaGraph_t vbody = vp.conditional.phGraph_out[0];
      FDM_CUDA(cudaStreamBeginCaptureToGraph(B->cap, vbody, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      capture_verify(c, bv[i], xv[i], h, B->d_times + 1 + i, B->cap);
      FDM_CUDA(cudaStreamEndCapture(B->cap, &vbody));
      size_t nvk = 0;
      FDM_CUDA(cudaGraphGetNodes(vbody, nullptr, &nvk));
      B->verify_kernels.push_back(nvk);
      set_kernel_priority(vbody, prio[i]);
    } catch (...) {
      c->capturing = false;
      cudaStreamCaptureStatus cs;
      if (cudaStreamIsCapturing(B->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
        cudaGraph_t junk = nullptr;
        cudaStreamEndCapture(B->cap, &junk);
        if (junk && junk != G) cudaGraphDestroy(junk);
      }
      cudaGetLastError();
      throw;
    }
    c->capturing = false;
    c->launches = counted;
  }
  FDM_CUDA(cudaGraphInstantiate(&B->exec, G, cudaGraphInstantiateFlagUseNodePriority));
  B->key_b.assign(bv, bv + k);
  B->key_x.assign(xv, xv + k);
  B->key_rtol = rtol;
  B->key_maxit = maxit;
}

// ---- lockstep batched solves: one device-driven loop for all problems
// ||b||^2 in dots[2]: the problem iterates unless b = 0 (or maxit = 0)
__global__ void k_lstart(double *sc, const double *dots, int *active) {
  if (threadIdx.x != 0) return;
  const double bb = dots[2];
  sc[12] = bb;
  sc[14] = bb;
  sc[9] = 1.0;
  sc[13] = 0.0;
  sc[15] = bb == 0.0 ? 1.0 : 0.0;
  if (!isfinite(bb)) sc[8] = 1.0;
  *active = (bb > 0.0 && isfinite(bb) && sc[11] > 0.0) ? 1 : 0;
}
// the three segment conditions of every problem from its flag, at the start of a pass
__global__ void k_lset(int k, const int *active, const cudaGraphConditionalHandle *h) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * k; t += gridDim.x * blockDim.x)
    cudaGraphSetConditional(h[t], active[t / 3] ? 1u : 0u);
}
// as k_bcheck, with the problem's flag in place of its own loop condition
__global__ void k_lcheck(double *sc, const double *dots, int *active, cudaGraphConditionalHandle hv,
                         unsigned long long *tend) {
  if (threadIdx.x != 0) return;
  const double rr = dots[2];
  const double it = sc[13] + 1.0;
  sc[13] = it;
  sc[14] = rr;
  if (!isfinite(rr)) sc[8] = 1.0;
  const bool conv = rr <= sc[10] * sc[12] && sc[8] == 0.0;
  sc[15] = 0.0;
  const bool stop = it >= sc[11] || sc[8] != 0.0;
  if (!conv && stop) *tend = global_ns();
  cudaGraphSetConditional(hv, conv ? 1u : 0u);
  *active = (conv || stop) ? 0 : 1;
}
// as k_bverify, with the problem's flag in place of its own loop condition
__global__ void k_lverify(double *sc, const double *dots, int *active, unsigned long long *tend) {
  if (threadIdx.x != 0) return;
  const double rr = dots[2];
  sc[4] += 1.0;
  sc[14] = rr;
  if (!isfinite(rr)) sc[8] = 1.0;
  const bool conv = rr <= sc[10] * sc[12] && sc[8] == 0.0;
  sc[15] = conv ? 1.0 : 0.0;
  const bool done = conv || sc[13] >= sc[11] || sc[8] != 0.0;
  if (done) *tend = global_ns();
  *active = done ? 0 : 1;
}
// the loop goes on while any problem iterates
__global__ void k_lany(int k, const int *active, cudaGraphConditionalHandle hw) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int i = 0; i < k; ++i) any |= active[i];
  cudaGraphSetConditional(hw, any ? 1u : 0u);
}

// the kernels of one problem's PCG iteration around the two star-solve launches
// (FP32 V(1,1)): segment 0 up to the first restriction, segment 1 from the first
// interpolation to the second restriction, segment 2 the rest of the iteration
void capture_segment(fdm_ctx *c, int seg, double *x, int *active, cudaGraphConditionalHandle hv,
                     unsigned long long *tend, cudaStream_t st) {
  const int64_t n = c->g.ndof;
  float *x1 = c->f1, *r1 = c->f3;
  if (seg == 0) {
    launch_dot(n, c->r, c->z, c->partial, c->dots + 1, st);  // r . z_prev (flexible beta)
    asm_restrict<float, double>(c, c->r, st);
  } else if (seg == 1) {
    asm_interp<float, float>(c, x1, c->omega, st, nullptr);  // x1 = omega ASM(r)
    apply_residual<float>(c, x1, c->r, r1, st);
    coarse_correct<float>(c, r1, x1, st);
    apply_residual<float>(c, x1, c->r, r1, st);
    asm_restrict<float, float>(c, r1, st);
  } else {
    asm_interp<float, double>(c, c->z, c->omega, st, x1);  // z = x1 + omega ASM(r1)
    launch_dot(n, c->r, c->z, c->partial, c->dots, st);
    k_bbeta<<<1, 32, 0, st>>>(c->sc, c->dots);
    launch_pcg_update_d(n, c->sc, c->z, c->d, st);
    apply_op<double>(c, c->d, c->q, st);
    launch_dot(n, c->d, c->q, c->partial, c->dots + 3, st);
    launch_pcg_scalars(0, c->sc, c->dots + 3, st);
    launch_pcg_update_xr(n, c->sc, c->d, c->q, x, c->r, st);
    launch_dot(n, c->r, c->r, c->partial, c->dots + 2, st);
    k_lcheck<<<1, 32, 0, st>>>(c->sc, c->dots, active, hv, tend);
  }
  FDM_CUDA(cudaGetLastError());
}

// the set-up of the global star-solve list: per problem the arguments of the
// 256-thread Schur-coupling kernel, and (problem, position) pairs by patch size
void setup_lockstep(fdm_batch *B) {
  const int k = (int)B->ctxs.size();
  std::vector<PatchSolveArgs<float>> args(k);
  struct Item {
    int64_t cost;
    int prob, slot;
  };
  std::vector<Item> items;
  size_t smem = 0;
  for (int i = 0; i < k; ++i) {
    fdm_ctx *c = B->ctxs[i];
    if (c->opt.precision != FDM_PREC_FP32 || c->opt.pc != FDM_PC_VCYCLE || !c->scform)
      fail(FDM_EINVAL, "lockstep batch: every context needs the FP32 V(1,1) and the Schur-coupling form");
    PatchSolveArgs<float> a{c->g, c->d_cls, c->d_patches, c->d_order, c->E<float>(), c->mu, c->tab<float>(),
                            c->L<float>(), c->X<float>(), patch_sc_tmp(c->maxN1, c->maxN2, 256), 0,
                            (uint64_t)(std::max(c->opt.wait_timeout_s, 0.0) * 1e9), c->status, 0, 0, 0};
    a.rows8 = 1;
    a.stage_st = 1;
    a.headcap = c->headcap32;
    args[i] = a;
    smem = std::max(smem, patch_sc_smem<float>(c->maxG, c->maxN1, c->maxN2, 256, a.headcap));
    std::vector<int> order(c->nsolve);
    if (c->nsolve > 0)
      FDM_CUDA(cudaMemcpy(order.data(), c->d_order, sizeof(int) * c->nsolve, cudaMemcpyDeviceToHost));
    for (int slot = 0; slot < c->nsolve; ++slot)
      items.push_back({c->classes[c->h_patches[order[slot]].cls].nval, i, slot});
  }
  if (smem > 224 * 1024) fail(FDM_EINVAL, "lockstep batch: a patch does not fit the shared memory of one CTA");
  std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
  std::vector<int2> work(items.size());
  for (size_t t = 0; t < items.size(); ++t) work[t] = make_int2(items[t].prob, items[t].slot);
  B->nwork = (int)work.size();
  B->multi_smem = smem;
  FDM_CUDA(cudaMalloc(&B->d_args, sizeof(PatchSolveArgs<float>) * std::max(k, 1)));
  FDM_CUDA(cudaMalloc(&B->d_work, sizeof(int2) * std::max<size_t>(work.size(), 1)));
  FDM_CUDA(cudaMalloc(&B->d_active, sizeof(int) * std::max(k, 1)));
  FDM_CUDA(cudaMalloc(&B->d_ifh, sizeof(cudaGraphConditionalHandle) * std::max(3 * k, 1)));
  if (k > 0) FDM_CUDA(cudaMemcpy(B->d_args, args.data(), sizeof(PatchSolveArgs<float>) * k, cudaMemcpyHostToDevice));
  if (!work.empty()) FDM_CUDA(cudaMemcpy(B->d_work, work.data(), sizeof(int2) * work.size(), cudaMemcpyHostToDevice));
}

// the launches of `launch`, captured into a child graph added to g after the given nodes
template <typename F>
cudaGraphNode_t capture_after(fdm_batch *B, cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, F &&launch) {
  cudaGraph_t child;
  FDM_CUDA(cudaGraphCreate(&child, 0));
  FDM_CUDA(cudaStreamBeginCaptureToGraph(B->cap, child, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  launch(B->cap);
  FDM_CUDA(cudaStreamEndCapture(B->cap, &child));
  cudaGraphNode_t node;
  FDM_CUDA(cudaGraphAddChildGraphNode(&node, g, deps.empty() ? nullptr : deps.data(), deps.size(), child));
  FDM_CUDA(cudaGraphDestroy(child));
  return node;
}

// a conditional node of the given type on handle h in g after deps; its body graph in *body
cudaGraphNode_t add_conditional(cudaGraph_t g, const std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                                cudaGraphConditionalNodeType type, cudaGraph_t *body) {
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = type;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  FDM_CUDA(cudaGraphAddNode(&node, g, deps.empty() ? nullptr : deps.data(), nullptr, deps.size(), &cp));
  *body = cp.conditional.phGraph_out[0];
  return node;
}

size_t graph_nodes(cudaGraph_t g) {
  size_t nn = 0;
  FDM_CUDA(cudaGraphGetNodes(g, nullptr, &nn));
  return nn;
}

// The lockstep graph: per problem its set-up (x = 0, r = b, ||b||^2, the flag),
// then one WHILE loop whose body is: the segment conditions from the flags;
// segment 0 of every problem (each in an IF node); the star solves of all
// active problems; segment 1; the star solves; segment 2 (ending with the
// problem's convergence check, and its true-residual check in a nested IF);
// the loop condition from the flags.
void build_lockstep_graph(fdm_batch *B, const double *const *bv, double *const *xv, double rtol, int maxit) {
  B->release_graph();
  B->init_kernels.clear();
  B->body_kernels.clear();
  B->verify_kernels.clear();
  const int k = (int)B->ctxs.size();
  if (!B->cap) FDM_CUDA(cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking));
  if (!B->d_times) FDM_CUDA(cudaMalloc(&B->d_times, sizeof(unsigned long long) * (k + 1)));
  if (!B->d_args) setup_lockstep(B);
  cudaGraph_t G;
  FDM_CUDA(cudaGraphCreate(&G, 0));
  B->graph = G;
  for (fdm_ctx *c : B->ctxs) c->capturing = true;
  std::vector<int64_t> counted(k);
  for (int i = 0; i < k; ++i) counted[i] = B->ctxs[i]->launches;
  try {
    unsigned long long *dt = B->d_times;
    cudaGraphNode_t t0 = capture_after(B, G, {}, [&](cudaStream_t st) { k_btime<<<1, 32, 0, st>>>(dt); });
    std::vector<cudaGraphNode_t> starts;
    for (int i = 0; i < k; ++i) {
      fdm_ctx *c = B->ctxs[i];
      const int64_t n = c->g.ndof;
      int *act = B->d_active + i;
      cudaGraphNode_t ni = capture_after(B, G, {t0}, [&](cudaStream_t st) {
        k_bconst<<<1, 32, 0, st>>>(c->sc, c->opt.flexible_beta ? 1.0 : 0.0, rtol * rtol, (double)maxit);
        fill(n, 0.0, xv[i], st);
        fill(n, 0.0, c->z, st);
        fill(n, 0.0, c->d, st);
        copy(n, bv[i], c->r, st);
        mask_dirichlet(c->g, c->r, st);
        launch_dot(n, c->r, c->r, c->partial, c->dots + 2, st);
        k_lstart<<<1, 32, 0, st>>>(c->sc, c->dots, act);
      });
      starts.push_back(ni);
    }
    cudaGraphConditionalHandle hw;
    FDM_CUDA(cudaGraphConditionalHandleCreate(&hw, G, 1, cudaGraphCondAssignDefault));
    cudaGraph_t body;
    add_conditional(G, starts, hw, cudaGraphCondTypeWhile, &body);
    std::vector<cudaGraphConditionalHandle> hif(3 * (size_t)k);
    for (auto &h : hif) FDM_CUDA(cudaGraphConditionalHandleCreate(&h, body, 0, cudaGraphCondAssignDefault));
    FDM_CUDA(cudaMemcpy(B->d_ifh, hif.data(), sizeof(cudaGraphConditionalHandle) * hif.size(),
                        cudaMemcpyHostToDevice));
    int *dact = B->d_active;
    cudaGraphConditionalHandle *difh = B->d_ifh;
    std::vector<cudaGraphNode_t> prev = {capture_after(B, body, {}, [&](cudaStream_t st) {
      k_lset<<<1, 256, 0, st>>>(k, dact, difh);
    })};
    B->seg_kernels.assign(k, 0);
    for (int seg = 0; seg < 3; ++seg) {
      std::vector<cudaGraphNode_t> ifs;
      for (int i = 0; i < k; ++i) {
        fdm_ctx *c = B->ctxs[i];
        cudaGraph_t sb;
        ifs.push_back(add_conditional(body, prev, hif[3 * i + seg], cudaGraphCondTypeIf, &sb));
        cudaGraphConditionalHandle hv = 0;
        if (seg == 2) FDM_CUDA(cudaGraphConditionalHandleCreate(&hv, sb, 0, cudaGraphCondAssignDefault));
        FDM_CUDA(cudaStreamBeginCaptureToGraph(B->cap, sb, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        capture_segment(c, seg, xv[i], B->d_active + i, hv, B->d_times + 1 + i, B->cap);
        FDM_CUDA(cudaStreamEndCapture(B->cap, &sb));
        B->seg_kernels[i] += graph_nodes(sb);
        if (seg == 2) {  // the true-residual check, when the recursive residual has converged
          cudaGraph_t vb;
          add_conditional(sb, {graph_leaf(sb)}, hv, cudaGraphCondTypeIf, &vb);
          FDM_CUDA(cudaStreamBeginCaptureToGraph(B->cap, vb, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
          const int64_t n = c->g.ndof;
          const double *b = bv[i];
          const double *x = xv[i];
          apply_op<double>(c, x, c->q, B->cap);
          launch_sub<double>(n, b, c->q, c->r, B->cap);
          mask_dirichlet(c->g, c->r, B->cap);
          launch_dot(n, c->r, c->r, c->partial, c->dots + 2, B->cap);
          k_lverify<<<1, 32, 0, B->cap>>>(c->sc, c->dots, B->d_active + i, B->d_times + 1 + i);
          FDM_CUDA(cudaStreamEndCapture(B->cap, &vb));
          B->verify_kernels.push_back(graph_nodes(vb));
        }
      }
      if (seg < 2) {
        PatchSolveArgs<float> *da = B->d_args;
        int2 *dw = B->d_work;
        const int nw = B->nwork;
        const size_t sm = B->multi_smem;
        prev = {capture_after(B, body, ifs, [&](cudaStream_t st) {
          launch_patch_sc_multi<float>(da, dw, nw, dact, sm, st);
        })};
      } else {
        capture_after(B, body, ifs, [&](cudaStream_t st) { k_lany<<<1, 32, 0, st>>>(k, dact, hw); });
      }
    }
    for (int i = 0; i < k; ++i) B->init_kernels.push_back(1);
  } catch (...) {
    for (fdm_ctx *c : B->ctxs) c->capturing = false;
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(B->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(B->cap, &junk);
    }
    cudaGetLastError();
    throw;
  }
  for (int i = 0; i < k; ++i) {
    B->ctxs[i]->capturing = false;
    B->ctxs[i]->launches = counted[i];
  }
  FDM_CUDA(cudaGraphInstantiate(&B->exec, G, 0));
  B->key_b.assign(bv, bv + k);
  B->key_x.assign(xv, xv + k);
  B->key_rtol = rtol;
  B->key_maxit = maxit;
}

int handle(fdm_ctx *c, const Error &e);

// the captured batched solve (one graph, a device-driven PCG loop per problem)
int solve_batch(fdm_batch *b, const double *const *bv, double *const *xv, double rtol, int maxit,
                fdm_solve_info *infos, cudaStream_t st) {
  const int k = (int)b->ctxs.size();
  fdm_ctx *c0 = b->ctxs[0];
  try {
    const bool same = b->exec && b->key_rtol == rtol && b->key_maxit == maxit &&
                      std::equal(b->key_b.begin(), b->key_b.end(), bv) && std::equal(b->key_x.begin(), b->key_x.end(), xv);
    if (!same) {
      if (b->mode == FDM_BATCH_LOCKSTEP) build_lockstep_graph(b, bv, xv, rtol, maxit);
      else build_batch_graph(b, bv, xv, rtol, maxit);
    }
    FDM_CUDA(cudaGraphLaunch(b->exec, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    std::vector<unsigned long long> t(k + 1);
    FDM_CUDA(cudaMemcpy(t.data(), b->d_times, sizeof(unsigned long long) * (k + 1), cudaMemcpyDeviceToHost));
    int worst = FDM_OK;
    for (int i = 0; i < k; ++i) {
      fdm_ctx *c = b->ctxs[i];
      double hsc[16];
      FDM_CUDA(cudaMemcpy(hsc, c->sc, sizeof hsc, cudaMemcpyDeviceToHost));
      // kernels this problem ran inside the graph (the timer kernel counts for the first;
      // in lockstep the shared kernels of every pass count for the first too)
      if (b->mode == FDM_BATCH_LOCKSTEP) {
        int64_t passes = 0;
        if (i == 0) {
          for (fdm_ctx *cc : b->ctxs) {
            double h13 = 0.0;
            FDM_CUDA(cudaMemcpy(&h13, cc->sc + 13, sizeof(double), cudaMemcpyDeviceToHost));
            passes = std::max<int64_t>(passes, (int64_t)h13);
          }
        }
        c->launches += 7 + (int64_t)hsc[13] * (int64_t)b->seg_kernels[i] +
                       (int64_t)hsc[4] * (int64_t)b->verify_kernels[i] + (i == 0) * (1 + 4 * passes);
      } else {
        c->launches += (int64_t)b->init_kernels[i] + (int64_t)hsc[13] * (int64_t)b->body_kernels[i] +
                       (int64_t)hsc[4] * (int64_t)b->verify_kernels[i] + (i == 0);
      }
      int hstat = 0;
      FDM_CUDA(cudaMemcpy(&hstat, c->status, sizeof(int), cudaMemcpyDeviceToHost));
      int rc = FDM_OK;
      if (hstat) {
        FDM_CUDA(cudaMemset(c->status, 0, sizeof(int)));
        c->err = "a bounded device-side wait of the patch solve ran out";
        rc = FDM_ETIMEOUT;
      } else if (hsc[8] != 0.0) {
        c->err = "non-finite scalar in PCG";
        rc = FDM_ENAN;
      } else if (hsc[15] == 0.0) {
        c->err = "PCG reached maxit";
        rc = FDM_ENOCONV;
      }
      if (infos) {
        fdm_solve_info &f = infos[i];
        f.iterations = (int)hsc[13];
        f.converged = hsc[15] != 0.0;
        f.rnorm0 = std::sqrt(hsc[12]);
        f.rnorm = std::sqrt(hsc[14]);
        f.seconds = hsc[13] > 0 && t[1 + i] > t[0] ? (double)(t[1 + i] - t[0]) * 1e-9 : 0.0;
        if (hsc[15] != 0.0 && hsc[13] > 0) {
          f.true_rnorm = f.rnorm;  // the converged residual is the true one (checked in the graph)
        } else {
          const int64_t n = c->g.ndof;  // true residual ||b - A x||, outside the timed graph
          launch_operator<double, double, double>(c->op_args(false), false, xv[i], c->q, c->E64, st);
          launch_sub<double>(n, bv[i], c->q, c->v1, st);
          mask_dirichlet(c->g, c->v1, st);
          launch_dot(n, c->v1, c->v1, c->partial, c->dots, st);
          double h = 0.0;
          FDM_CUDA(cudaMemcpyAsync(&h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
          FDM_CUDA(cudaStreamSynchronize(st));
          f.true_rnorm = std::sqrt(h);
        }
      }
      if (rc < worst) worst = rc;
    }
    if (worst != FDM_OK) g_last_error = "pcg_solve_batched: a problem did not converge (see its context)";
    return worst;
  } catch (const Error &e) { return handle(c0, e); }
}


// ---- learned surrogate helpers
void need_surrogate_data(const fdm_ctx *c) {
  if (!c->general || !c->feat) fail(FDM_EINVAL, "the learned surrogate needs curved cells and samples27");
}

// per-cell Theorem 1 labels, computed once per context
void ensure_labels(fdm_ctx *c, cudaStream_t st) {
  if (c->cstar) return;
  const int ncell = c->g.ncell;
  double *cs = c->alloc<double>(3 * (size_t)ncell);
  c->F0 = c->alloc<double>(ncell);
  c->F1 = c->alloc<double>(ncell);
  c->label32 = c->alloc<float>(3 * (size_t)ncell);
  launch_surr_label(ncell, c->g.n, c->Gw64, c->wq64, c->mubar, cs, c->F0, c->F1, st);
  launch_convert<double, float>(3 * (int64_t)ncell, cs, c->label32, st);
  FDM_CUDA(cudaStreamSynchronize(st));
  c->launches += 2;
  c->cstar = cs;
}

// labels scored by the Lanczos condition number of each cell's interior patch,
// computed once per context
void ensure_kappa_labels(fdm_ctx *c, cudaStream_t st) {
  if (c->ckap) return;
  const int ncell = c->g.ncell, p = c->p;
  if (p < 2 || p > PATCH_KAPPA_PMAX) fail(FDM_EINVAL, "patch-condition labels need p in 2..8");
  c->S64 = c->upload(c->basis.S);
  c->lam64 = c->upload(c->basis.lam);
  double *ck = c->alloc<double>(3 * (size_t)ncell);
  c->Fkap = c->alloc<double>(2 * (size_t)ncell);
  c->label32k = c->alloc<float>(3 * (size_t)ncell);
  launch_surr_patch_label(ncell, p, c->Gw64, c->tab64, c->S64, c->lam64, c->mubar, ck, c->Fkap, nullptr, st);
  launch_convert<double, float>(3 * (int64_t)ncell, ck, c->label32k, st);
  FDM_CUDA(cudaStreamSynchronize(st));
  FDM_CUDA(cudaGetLastError());
  c->launches += 2;
  c->ckap = ck;
}

// the training labels the context has selected
const float *train_labels(fdm_ctx *c, cudaStream_t st) {
  if (c->label_kind == FDM_LABEL_PATCH_KAPPA) {
    ensure_kappa_labels(c, st);
    return c->label32k;
  }
  ensure_labels(c, st);
  return c->label32;
}

// device buffers of one training run, released on every exit path
struct DevScratch {
  std::vector<void *> p;
  size_t bytes = 0;
  template <typename T>
  T *get(size_t n) {
    void *ptr = device_alloc(std::max<size_t>(n, 1) * sizeof(T), bytes);
    p.push_back(ptr);
    return static_cast<T *>(ptr);
  }
  ~DevScratch() {
    for (void *x : p) cudaFree(x);
  }
};

int handle(fdm_ctx *c, const Error &e) {
  if (c) c->err = e.msg;
  g_last_error = e.msg;
  return e.code;
}

}  // namespace

namespace fdm {
// accessors used by other translation units of the library
OpArgs ctx_op_args64(const fdm_ctx *c) { return c->op_args(false); }
void ctx_count_launches(fdm_ctx *c, int k) { c->launches += k; }
int ctx_device(const fdm_ctx *c) { return c->device; }
int ctx_fail(fdm_ctx *c, int code, const std::string &msg) { return handle(c, Error{code, msg}); }
void ctx_mask_dirichlet(const Grid &g, double *v, cudaStream_t st) { mask_dirichlet(g, v, st); }
void ctx_copy(int64_t n, const double *a, double *b, cudaStream_t st) { copy(n, a, b, st); }
int ctx_vec_blocks(int64_t n) { return vec_blocks(n); }
void ctx_banded_cholesky(int m, int bw, std::vector<double> &Lb) { banded_cholesky(m, bw, Lb); }
void ctx_tridiag_extremes(const std::vector<double> &d, const std::vector<double> &e, double &lo, double &hi) {
  tridiag_extremes(d, e, lo, hi);
}
void ctx_normal_vector(uint64_t seed, int64_t n, std::vector<double> &out) { normal_vector(seed, n, out); }
std::string &ctx_last_error() { return g_last_error; }
template <typename T, typename Tin, typename Tout>
void ctx_run_asm(fdm_ctx *c, const Tin *r, Tout *z, double omega, cudaStream_t st, const T *addv) {
  run_asm<T, Tin, Tout>(c, r, z, omega, st, addv);
}
template void ctx_run_asm<double, double, double>(fdm_ctx *, const double *, double *, double, cudaStream_t,
                                                  const double *);
template void ctx_run_asm<float, double, float>(fdm_ctx *, const double *, float *, double, cudaStream_t, const float *);
template void ctx_run_asm<float, float, double>(fdm_ctx *, const float *, double *, double, cudaStream_t, const float *);
template void ctx_run_asm<float, double, double>(fdm_ctx *, const double *, double *, double, cudaStream_t,
                                                 const float *);
template <typename T>
void ctx_coarse_solve(fdm_ctx *c, cudaStream_t st) {
  if (c->nc == 0) return;
  if (c->gmg_L > 0) gmg_level<T>(c, 0, c->rc<T>(), c->xc<T>(), st);
  else {
    launch_dense_symv<T>(c->nc, c->Acinv<T>(), c->rc<T>(), c->xc<T>(), st);
    c->launches += 1;
  }
}
template void ctx_coarse_solve<double>(fdm_ctx *, cudaStream_t);
template void ctx_coarse_solve<float>(fdm_ctx *, cudaStream_t);
}  // namespace fdm

// ====================================================================== C-ABI
extern "C" {

int fdm_default_options(fdm_options *opt) {
  if (!opt) return FDM_EINVAL;
  std::memset(opt, 0, sizeof *opt);
  opt->precision = FDM_PREC_FP32;
  opt->pc = FDM_PC_VCYCLE;
  opt->surrogate = FDM_SURR_AVERAGED;
  opt->lanczos_steps = 20;
  opt->omega = 0.0;
  opt->lanczos_seed = 12345;
  opt->flexible_beta = -1;
  opt->wait_timeout_s = 1.0;
  opt->lanczos_start = nullptr;
  opt->kernel_timing = 0;
  opt->patch_ctas_per_sm = 0;
  opt->patch_threads = 0;
  opt->patch_kernel = 0;
  opt->stream_buffers = 0;
  opt->stream_buffer_kb = 0;
  opt->inject_stall = 0;
  opt->pcg_graph = 1;
  opt->patch_l2_hints = 0;
  opt->autotune = 0;
  opt->patch_rows_per_warp = 0;
  opt->coarse_levels = -1;
  opt->gmg_nu = 2;
  opt->gmg_omega = 2.0 / 3.0;
  return FDM_OK;
}

int fdm_setup(const fdm_mesh *mesh, int p, const fdm_coeff *coeff, const fdm_options *opt, fdm_ctx **out,
              void *stream) {
  if (!mesh || !out || !mesh->xv || !mesh->yv || !mesh->zv || mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1) {
    g_last_error = "fdm_setup: invalid mesh";
    return FDM_EINVAL;
  }
  if (p < 1 || p > 15) {
    g_last_error = "fdm_setup: the CUDA path supports 1 <= p <= 15";
    return FDM_EINVAL;
  }
  *out = nullptr;
  fdm_ctx *c = new fdm_ctx();
  cudaGetDevice(&c->device);
  cudaStream_t st = (cudaStream_t)stream;
  try {
    if (opt) c->opt = *opt;
    else fdm_default_options(&c->opt);
    if (c->opt.lanczos_steps <= 0) c->opt.lanczos_steps = 20;
    if (c->opt.flexible_beta < 0) c->opt.flexible_beta = c->opt.precision == FDM_PREC_FP32 ? 1 : 0;
    c->p = p;
    Grid &g = c->g;
    g.p = p;
    g.n = p + 1;
    g.nx = mesh->nx; g.ny = mesh->ny; g.nz = mesh->nz;
    g.N[0] = g.nx * p + 1; g.N[1] = g.ny * p + 1; g.N[2] = g.nz * p + 1;
    g.ndof = (int64_t)g.N[0] * g.N[1] * g.N[2];
    g.ncell = g.nx * g.ny * g.nz;
    double t0 = now_s();
    c->basis = make_basis(p);
    setup_tables(c);
    setup_geometry(c, mesh, coeff);
    setup_patches(c);
    // work vectors
    const int64_t n = g.ndof;
    for (double **v : {&c->r, &c->z, &c->zold, &c->d, &c->q, &c->v1, &c->v2, &c->v3}) *v = c->alloc<double>(n);
    for (float **v : {&c->f_in, &c->f_out, &c->f1, &c->f2, &c->f3}) *v = c->alloc<float>(n);
    c->partial = c->alloc<double>(2 * DOT_BLOCKS);
    c->dots = c->alloc<double>(4);
    c->sc = c->alloc<double>(16);
    double t1 = now_s();
    factor_all(c, st);
    double t2 = now_s();
    setup_coarse(c, st);
    double t3 = now_s();
    if (c->opt.omega > 0.0) c->omega = c->opt.omega;
    else {
      lanczos_omega(c, c->opt.lanczos_start, st);
      c->kappa_avg = c->lmax / c->lmin;
    }
    // one preconditioner application (on r = 0) so that every kernel of the
    // solve has been launched once, with its attributes set, before any capture
    if (c->opt.autotune && !c->opt.inject_stall && !c->stream) autotune_patch(c, st);
    if (!c->opt.inject_stall) {
      fill(g.ndof, 0.0, c->r, st);
      pc_apply_impl(c, c->r, c->z, st);
    }
    FDM_CUDA(cudaStreamSynchronize(st));
    FDM_CUDA(cudaGetLastError());
    double t4 = now_s();
    c->t_setup[0] = t1 - t0;
    c->t_setup[1] = t2 - t1;
    c->t_setup[2] = t3 - t2;
    c->t_setup[3] = t4 - t3;
  } catch (const Error &e) {
    int rc = handle(c, e);
    delete c;
    return rc;
  }
  *out = c;
  return FDM_OK;
}

int stiffness_apply(fdm_ctx *c, const double *u, double *y, void *stream) {
  if (!c || !u || !y) return FDM_EINVAL;
  try {
    apply_op<double>(c, u, y, (cudaStream_t)stream);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int mass_apply(fdm_ctx *c, const double *f, double *b, void *stream) {
  if (!c || !f || !b) return FDM_EINVAL;
  try {
    launch_operator<double, double, double>(c->op_args(false), true, f, b, c->E64, (cudaStream_t)stream);
    c->launches += 2;
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int asm_apply(fdm_ctx *c, const double *r, double *z, void *stream) {
  if (!c || !r || !z) return FDM_EINVAL;
  try {
    cudaStream_t st = (cudaStream_t)stream;
    if (c->opt.precision == FDM_PREC_FP64) run_asm<double, double, double>(c, r, z, c->omega, st);
    else run_asm<float, double, double>(c, r, z, c->omega, st);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int pc_apply(fdm_ctx *c, const double *r, double *z, void *stream) {
  if (!c || !r || !z) return FDM_EINVAL;
  try {
    pc_apply_impl(c, r, z, (cudaStream_t)stream);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int pcg_solve(fdm_ctx *c, const double *b, double *x, double rtol, int maxit, fdm_solve_info *info, void *stream) {
  if (!c || !b || !x || maxit < 0 || !(rtol >= 0.0)) return FDM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (c->opt.pcg_graph && !c->opt.kernel_timing) {
    // the device-driven loop of the batched solve, for a batch of one (its
    // graph is kept and reused while b, x, rtol and maxit stay the same)
    if (!c->solo) {
      c->solo = new fdm_batch();
      c->solo->ctxs.push_back(c);
    }
    const double *bv[1] = {b};
    double *xv[1] = {x};
    return solve_batch(c->solo, bv, xv, rtol, maxit, info, st);
  }
  const int64_t n = c->g.ndof;
  try {
    cudaEvent_t e0, e1;
    FDM_CUDA(cudaEventCreate(&e0));
    FDM_CUDA(cudaEventCreate(&e1));
    FDM_CUDA(cudaEventRecord(e0, st));
    const double flex = c->opt.flexible_beta ? 1.0 : 0.0;
    double hsc[16] = {0};
    hsc[7] = flex;
    FDM_CUDA(cudaMemcpyAsync(c->sc, hsc, sizeof hsc, cudaMemcpyHostToDevice, st));
    FDM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    FDM_CUDA(cudaMemcpyAsync(c->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    mask_dirichlet(c->g, c->r, st);
    double h[2];
    launch_dot(n, c->r, c->r, c->partial, c->dots, st);
    c->launches += 3;
    FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    const double nb = std::sqrt(h[0]);
    double nr = nb;
    int it = 0, conv = nb == 0.0, bad = 0;
    double *z = c->z, *zold = c->zold;
    if (!conv) {
      pc_apply_impl(c, c->r, z, st);
      launch_dot(n, c->r, z, c->partial, c->dots, st);
      launch_pcg_scalars(2, c->sc, c->dots, st);
      FDM_CUDA(cudaMemcpyAsync(c->d, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      c->launches += 6;
      while (it < maxit) {
        apply_op<double>(c, c->d, c->q, st);
        c->tmark(FDM_T_VEC, true, st);
        launch_dot(n, c->d, c->q, c->partial, c->dots, st);
        launch_pcg_scalars(0, c->sc, c->dots, st);
        launch_pcg_update_xr(n, c->sc, c->d, c->q, x, c->r, st);
        ++it;
        launch_dot(n, c->r, c->r, c->partial, c->dots + 2, st);
        c->tmark(FDM_T_VEC, false, st);
        c->launches += 6;
        FDM_CUDA(cudaMemcpyAsync(h, c->dots + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
        FDM_CUDA(cudaStreamSynchronize(st));
        nr = std::sqrt(h[0]);
        if (!std::isfinite(nr)) { bad = 1; break; }
        if (nr <= rtol * nb) {
          // converged on the recursive residual: replace it by the true one,
          // r = b - A x, and stop only if that meets the test too
          apply_op<double>(c, x, c->q, st);
          launch_sub<double>(n, b, c->q, c->r, st);
          mask_dirichlet(c->g, c->r, st);
          launch_dot(n, c->r, c->r, c->partial, c->dots + 2, st);
          c->launches += 4;
          FDM_CUDA(cudaMemcpyAsync(h, c->dots + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
          FDM_CUDA(cudaStreamSynchronize(st));
          nr = std::sqrt(h[0]);
          if (!std::isfinite(nr)) { bad = 1; break; }
          if (nr <= rtol * nb) { conv = 1; break; }
          if (it >= maxit) break;
        }
        std::swap(z, zold);
        pc_apply_impl(c, c->r, z, st);
        c->tmark(FDM_T_VEC, true, st);
        launch_dot2(n, c->r, z, zold, c->partial, c->dots, st);
        launch_pcg_scalars(1, c->sc, c->dots, st);
        launch_pcg_update_d(n, c->sc, z, c->d, st);
        c->tmark(FDM_T_VEC, false, st);
        c->launches += 4;
      }
    }
    FDM_CUDA(cudaEventRecord(e1, st));
    FDM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FDM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    FDM_CUDA(cudaMemcpy(hsc, c->sc, sizeof hsc, cudaMemcpyDeviceToHost));
    if (hsc[8] != 0.0) bad = 1;
    int hstat = 0;
    FDM_CUDA(cudaMemcpy(&hstat, c->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (hstat) {
      FDM_CUDA(cudaMemset(c->status, 0, sizeof(int)));
      fail(FDM_ETIMEOUT, "a bounded device-side wait of the patch solve ran out");
    }
    if (info) {
      info->iterations = it;
      info->converged = conv;
      info->rnorm0 = nb;
      info->rnorm = nr;
      info->seconds = ms * 1e-3;
      // true residual ||b - A x||
      launch_operator<double, double, double>(c->op_args(false), false, x, c->q, c->E64, st);
      launch_sub<double>(n, b, c->q, c->v1, st);
      mask_dirichlet(c->g, c->v1, st);
      c->launches += 6;
      launch_dot(n, c->v1, c->v1, c->partial, c->dots, st);
      FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
      FDM_CUDA(cudaStreamSynchronize(st));
      info->true_rnorm = std::sqrt(h[0]);
    }
    FDM_CUDA(cudaGetLastError());
    if (bad) { c->err = "non-finite scalar in PCG"; return FDM_ENAN; }
    if (!conv) { c->err = "PCG reached maxit"; return FDM_ENOCONV; }
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int fdm_batch_setup(int k, fdm_ctx *const *ctxs, fdm_batch **out) {
  return fdm_batch_setup_mode(k, ctxs, FDM_BATCH_BRANCHES, out);
}

int fdm_batch_setup_mode(int k, fdm_ctx *const *ctxs, int mode, fdm_batch **out) {
  if (k < 0 || !out || (k > 0 && !ctxs) || (mode != FDM_BATCH_BRANCHES && mode != FDM_BATCH_LOCKSTEP))
    return FDM_EINVAL;
  *out = nullptr;
  fdm_batch *b = new fdm_batch();
  b->mode = mode;
  for (int i = 0; i < k; ++i) {
    if (!ctxs[i]) { delete b; return FDM_EINVAL; }
    b->ctxs.push_back(ctxs[i]);
  }
  if (mode == FDM_BATCH_LOCKSTEP) {
    try {
      setup_lockstep(b);
    } catch (const Error &e) {
      g_last_error = e.msg;
      delete b;
      return e.code;
    }
  }
  *out = b;
  return FDM_OK;
}

int pcg_solve_batched(fdm_batch *b, const double *const *bv, double *const *xv, double rtol, int maxit,
                      fdm_solve_info *infos, void *stream) {
  if (!b || !bv || !xv || maxit < 0 || !(rtol >= 0.0)) return FDM_EINVAL;
  const int k = (int)b->ctxs.size();
  if (k == 0) return FDM_OK;
  for (int i = 0; i < k; ++i)
    if (!bv[i] || !xv[i]) return FDM_EINVAL;
  return solve_batch(b, bv, xv, rtol, maxit, infos, (cudaStream_t)stream);
}

void fdm_batch_destroy(fdm_batch *b) { delete b; }

int fdm_surrogate_load(fdm_ctx *c, const double *mu_host, void *stream) {
  if (!c || !mu_host) return FDM_EINVAL;
  try {
    cudaStream_t st = (cudaStream_t)stream;
    for (int64_t i = 0; i < 3 * (int64_t)c->g.ncell; ++i)
      if (!(mu_host[i] > 0.0) || !std::isfinite(mu_host[i])) fail(FDM_EINVAL, "surrogate coefficients must be positive");
    FDM_CUDA(cudaMemcpyAsync(c->mu, mu_host, 3 * sizeof(double) * c->g.ncell, cudaMemcpyHostToDevice, st));
    factor_all(c, st);
    if (c->opt.omega <= 0.0) lanczos_omega(c, c->opt.lanczos_start, st);
    FDM_CUDA(cudaStreamSynchronize(st));
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int fdm_surrogate_grad(fdm_ctx *c, const float *w_host, float *grad_host, double *loss, void *stream) {
  if (!c || !w_host || !grad_host) return FDM_EINVAL;
  try {
    need_surrogate_data(c);
    cudaStream_t st = (cudaStream_t)stream;
    const float *lab = train_labels(c, st);
    const int ncell = c->g.ncell, nblk = mlp_blocks(ncell);
    DevScratch s;
    float *P = s.get<float>(MLP_NPARAM), *g = s.get<float>(MLP_NPARAM), *out = s.get<float>(3 * (size_t)ncell);
    float *partial = s.get<float>((size_t)nblk * MLP_NPARAM), *lossp = s.get<float>(nblk);
    double *dl = s.get<double>(1);
    FDM_CUDA(cudaMemcpyAsync(P, w_host, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, st));
    launch_mlp(ncell, P, c->feat, lab, out, partial, lossp, st);
    launch_mlp_reduce(nblk, partial, lossp, g, dl, st);
    c->launches += 2;
    FDM_CUDA(cudaMemcpyAsync(grad_host, g, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, st));
    double l = 0.0;
    FDM_CUDA(cudaMemcpyAsync(&l, dl, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = l;
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int fdm_surrogate_labels(fdm_ctx *c, int kind, double *labels_host, double *score_host, void *stream) {
  if (!c || (kind != FDM_LABEL_THEOREM1 && kind != FDM_LABEL_PATCH_KAPPA)) return FDM_EINVAL;
  try {
    need_surrogate_data(c);
    cudaStream_t st = (cudaStream_t)stream;
    const int ncell = c->g.ncell;
    const double *lab, *F0, *F1;
    if (kind == FDM_LABEL_PATCH_KAPPA) {
      ensure_kappa_labels(c, st);
      lab = c->ckap;
    } else {
      ensure_labels(c, st);
      lab = c->cstar;
    }
    c->label_kind = kind;
    if (labels_host)
      FDM_CUDA(cudaMemcpy(labels_host, lab, sizeof(double) * 3 * (size_t)ncell, cudaMemcpyDeviceToHost));
    if (score_host) {
      std::vector<double> h(2 * (size_t)ncell);
      if (kind == FDM_LABEL_PATCH_KAPPA) {
        FDM_CUDA(cudaMemcpy(h.data(), c->Fkap, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (int e = 0; e < ncell; ++e) {
          score_host[e] = h[2 * (size_t)e];
          score_host[ncell + e] = h[2 * (size_t)e + 1];
        }
      } else {
        F0 = c->F0;
        F1 = c->F1;
        FDM_CUDA(cudaMemcpy(score_host, F0, sizeof(double) * ncell, cudaMemcpyDeviceToHost));
        FDM_CUDA(cudaMemcpy(score_host + ncell, F1, sizeof(double) * ncell, cudaMemcpyDeviceToHost));
      }
    }
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int fdm_surrogate_train(int k, fdm_ctx *const *ctxs, const float *w_init, int steps, double lr, double weight_decay,
                        float *w_out, double *loss_hist, void *stream) {
  if (k < 1 || !ctxs || !w_init || !w_out || steps < 0 || !(lr > 0.0) || !(weight_decay >= 0.0)) {
    g_last_error = "fdm_surrogate_train: invalid arguments";
    return FDM_EINVAL;
  }
  fdm_ctx *c0 = ctxs[0];
  try {
    cudaStream_t st = (cudaStream_t)stream;
    int64_t ntot = 0;
    for (int i = 0; i < k; ++i) {
      if (!ctxs[i]) fail(FDM_EINVAL, "fdm_surrogate_train: null context");
      need_surrogate_data(ctxs[i]);
      train_labels(ctxs[i], st);
      ntot += ctxs[i]->g.ncell;
    }
    if (ntot > (int64_t)1 << 26) fail(FDM_EINVAL, "fdm_surrogate_train: too many cells");
    const int ncell = (int)ntot, nblk = mlp_blocks(ncell);
    DevScratch s;
    float *X = s.get<float>((size_t)ncell * MLP_NIN), *Y = s.get<float>(3 * (size_t)ncell);
    int64_t off = 0;
    for (int i = 0; i < k; ++i) {  // the training set: every cell of every context
      const int nc = ctxs[i]->g.ncell;
      FDM_CUDA(cudaMemcpyAsync(X + off * MLP_NIN, ctxs[i]->feat, sizeof(float) * MLP_NIN * nc,
                               cudaMemcpyDeviceToDevice, st));
      FDM_CUDA(cudaMemcpyAsync(Y + off * 3, train_labels(ctxs[i], st), sizeof(float) * 3 * nc,
                               cudaMemcpyDeviceToDevice, st));
      off += nc;
    }
    float *P = s.get<float>(MLP_NPARAM), *g = s.get<float>(MLP_NPARAM), *m = s.get<float>(MLP_NPARAM),
          *v = s.get<float>(MLP_NPARAM), *out = s.get<float>(3 * (size_t)ncell);
    float *partial = s.get<float>((size_t)nblk * MLP_NPARAM), *lossp = s.get<float>(nblk);
    double *hist = s.get<double>((size_t)steps + 1);
    FDM_CUDA(cudaMemcpyAsync(P, w_init, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, st));
    FDM_CUDA(cudaMemsetAsync(m, 0, sizeof(float) * MLP_NPARAM, st));
    FDM_CUDA(cudaMemsetAsync(v, 0, sizeof(float) * MLP_NPARAM, st));
    // full-batch Adam: loss and gradient over all cells, then one update
    for (int t = 1; t <= steps; ++t) {
      launch_mlp(ncell, P, X, Y, out, partial, lossp, st);
      launch_mlp_reduce(nblk, partial, lossp, g, hist + (t - 1), st);
      launch_adam(P, g, m, v, t, lr, weight_decay, st);
    }
    launch_mlp(ncell, P, X, Y, out, partial, lossp, st);
    launch_mlp_reduce(nblk, partial, lossp, g, hist + steps, st);
    c0->launches += 3 * (int64_t)steps + 2;
    FDM_CUDA(cudaMemcpyAsync(w_out, P, sizeof(float) * MLP_NPARAM, cudaMemcpyDeviceToHost, st));
    std::vector<double> h((size_t)steps + 1);
    FDM_CUDA(cudaMemcpyAsync(h.data(), hist, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    if (loss_hist) std::copy(h.begin(), h.end(), loss_hist);
  } catch (const Error &e) { return handle(c0, e); }
  return FDM_OK;
}

int fdm_surrogate_apply(fdm_ctx *c, const float *w_host, int judge, int *nfallback, int *kept, void *stream) {
  if (!c || !w_host) return FDM_EINVAL;
  try {
    need_surrogate_data(c);
    if (judge && !(c->kappa_avg > 0.0))
      fail(FDM_EINVAL, "fdm_surrogate_apply: judging needs the Lanczos estimate (omega must not be fixed)");
    cudaStream_t st = (cudaStream_t)stream;
    const int ncell = c->g.ncell;
    if (!c->surr_c) c->surr_c = c->alloc<float>(3 * (size_t)ncell);
    if (!c->d_count) c->d_count = c->alloc<int>(4);
    DevScratch s;
    float *P = s.get<float>(MLP_NPARAM);
    FDM_CUDA(cudaMemcpyAsync(P, w_host, sizeof(float) * MLP_NPARAM, cudaMemcpyHostToDevice, st));
    FDM_CUDA(cudaMemsetAsync(c->d_count, 0, sizeof(int), st));
    launch_mlp(ncell, P, c->feat, nullptr, c->surr_c, nullptr, nullptr, st);
    launch_surr_apply(ncell, c->surr_c, c->mubar, c->mu, c->d_count, st);
    c->launches += 2;
    int nf = 0;
    FDM_CUDA(cudaMemcpyAsync(&nf, c->d_count, sizeof(int), cudaMemcpyDeviceToHost, st));
    factor_all(c, st);
    if (c->opt.omega <= 0.0) lanczos_omega(c, c->opt.lanczos_start, st);
    FDM_CUDA(cudaStreamSynchronize(st));
    int keep = 1;
    if (judge && c->lmax / c->lmin > c->kappa_avg) {
      // the averaged surrogate judges: keep the network's scalings only if the
      // Lanczos estimate of the preconditioned condition number did not grow
      keep = 0;
      FDM_CUDA(cudaMemcpyAsync(c->mu, c->mubar, 3 * sizeof(double) * ncell, cudaMemcpyDeviceToDevice, st));
      factor_all(c, st);
      lanczos_omega(c, c->opt.lanczos_start, st);
      FDM_CUDA(cudaStreamSynchronize(st));
    }
    if (nfallback) *nfallback = nf;
    if (kept) *kept = keep;
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

int fdm_query(fdm_ctx *c, int what, void *out, size_t *len) {
  if (!c || !out || !len) return FDM_EINVAL;
  try {
    auto put = [&](const void *src, size_t bytes) {
      if (*len < bytes) fail(FDM_EINVAL, "fdm_query: buffer too small (" + std::to_string(bytes) + " bytes needed)");
      std::memcpy(out, src, bytes);
      *len = bytes;
    };
    switch (what) {
      case FDM_Q_NDOF: { int64_t v = c->g.ndof; put(&v, sizeof v); break; }
      case FDM_Q_OMEGA: put(&c->omega, sizeof(double)); break;
      case FDM_Q_LAMBDA: { double v[2] = {c->lmin, c->lmax}; put(v, sizeof v); break; }
      case FDM_Q_MU: {
        std::vector<double> h(3 * (size_t)c->g.ncell);
        FDM_CUDA(cudaMemcpy(h.data(), c->mu, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
        put(h.data(), h.size() * sizeof(double));
        break;
      }
      case FDM_Q_NPATCH: put(&c->npatch, sizeof(int)); break;
      case FDM_Q_PATCH_CLASS: {
        std::vector<int> h(c->npatch);
        for (int i = 0; i < c->npatch; ++i) h[i] = c->h_patches[i].cls;
        put(h.data(), h.size() * sizeof(int));
        break;
      }
      case FDM_Q_CLASS_INFO: {
        std::vector<int> h(64, 0);
        for (int i = 0; i < 8; ++i) {
          const PatchClass &C = c->classes[i];
          int v[8] = {C.nd, C.nI, C.nG, C.n0, C.n1, C.n2, C.nlines, (int)C.nnzL};
          std::copy(v, v + 8, h.begin() + 8 * i);
        }
        put(h.data(), h.size() * sizeof(int));
        break;
      }
      case FDM_Q_GAMMA_ORDER: {
        std::vector<int> h;
        for (int i = 0; i < 8; ++i) h.insert(h.end(), c->classes[i].gpos.begin(), c->classes[i].gpos.end());
        put(h.data(), h.size() * sizeof(int));
        break;
      }
      case FDM_Q_FACTOR_NNZ: {
        int64_t s = 0;
        for (int i = 0; i < c->npatch; ++i) s += c->classes[c->h_patches[i].cls].nnzL;
        put(&s, sizeof s);
        break;
      }
      case FDM_Q_PATTERN: {
        int cls = *(const int *)out;
        if (cls < 0 || cls > 7) fail(FDM_EINVAL, "class id");
        const auto &pt = c->classes[cls].pattern;
        put(pt.data(), pt.size());
        break;
      }
      case FDM_Q_FACTOR: {
        int pid = *(const int *)out;
        if (pid < 0 || pid >= c->npatch) fail(FDM_EINVAL, "patch id");
        const int nG = c->classes[c->h_patches[pid].cls].nG;
        if (*len < (size_t)nG * nG * sizeof(double)) fail(FDM_EINVAL, "fdm_query: buffer too small");
        double *S = c->alloc<double>((size_t)c->maxG * c->maxG);
        int *plist = c->alloc<int>(1);
        int *status = c->alloc<int>(1);
        FDM_CUDA(cudaMemcpy(plist, &pid, sizeof(int), cudaMemcpyHostToDevice));
        FactorArgs a{c->g, c->d_cls, c->d_patches, plist, c->mu, c->tab64, S, (int64_t)c->maxG * c->maxG,
                     nullptr, nullptr, status};
        launch_assemble_factor_only(a, 1, 0);
        FDM_CUDA(cudaDeviceSynchronize());
        std::vector<double> h((size_t)nG * nG);
        FDM_CUDA(cudaMemcpy(h.data(), S, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
        for (void *ptr : {(void *)S, (void *)plist, (void *)status}) {
          cudaFree(ptr);
          c->allocs.erase(std::find(c->allocs.begin(), c->allocs.end(), ptr));
        }
        for (int i = 0; i < nG; ++i)
          for (int j = i + 1; j < nG; ++j) h[(size_t)i * nG + j] = 0.0;
        put(h.data(), h.size() * sizeof(double));
        break;
      }
      case FDM_Q_BASIS: {
        const Basis1D &b = c->basis;
        std::vector<double> h;
        for (auto *M : {&b.A, &b.B, &b.T, &b.Af, &b.Bf}) h.insert(h.end(), M->begin(), M->end());
        put(h.data(), h.size() * sizeof(double));
        break;
      }
      case FDM_Q_FACTOR_BYTES: {
        int64_t v[2] = {c->nval_total * 8, c->nval_total * 4};
        put(v, sizeof v);
        break;
      }
      case FDM_Q_SETUP_SECONDS: put(c->t_setup, sizeof c->t_setup); break;
      case FDM_Q_SURR_FEATURES: {
        need_surrogate_data(c);
        std::vector<float> h((size_t)c->g.ncell * MLP_NIN);
        FDM_CUDA(cudaMemcpy(h.data(), c->feat, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
        put(h.data(), h.size() * sizeof(float));
        break;
      }
      case FDM_Q_SURR_LABELS: {
        need_surrogate_data(c);
        ensure_labels(c, 0);
        std::vector<double> h(3 * (size_t)c->g.ncell);
        FDM_CUDA(cudaMemcpy(h.data(), c->cstar, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
        put(h.data(), h.size() * sizeof(double));
        break;
      }
      case FDM_Q_SURR_BOUNDS: {
        if (!c->general) fail(FDM_EINVAL, "bounds need curved cells");
        const int ncell = c->g.ncell;
        std::vector<double> h(3 * (size_t)ncell);
        if (!c->Fcur) c->Fcur = c->alloc<double>(ncell);
        double *Fc = c->Fcur;
        if (c->feat) {
          ensure_labels(c, 0);
          FDM_CUDA(cudaMemcpy(h.data(), c->F0, ncell * sizeof(double), cudaMemcpyDeviceToHost));
          FDM_CUDA(cudaMemcpy(h.data() + ncell, c->F1, ncell * sizeof(double), cudaMemcpyDeviceToHost));
        } else {
          launch_surr_bound(ncell, c->g.n, c->Gw64, c->wq64, c->mubar, Fc, 0);
          FDM_CUDA(cudaMemcpy(h.data(), Fc, ncell * sizeof(double), cudaMemcpyDeviceToHost));
          for (int e = 0; e < ncell; ++e) h[ncell + e] = NAN;
        }
        launch_surr_bound(ncell, c->g.n, c->Gw64, c->wq64, c->mu, Fc, 0);
        FDM_CUDA(cudaMemcpy(h.data() + 2 * (size_t)ncell, Fc, ncell * sizeof(double), cudaMemcpyDeviceToHost));
        put(h.data(), h.size() * sizeof(double));
        break;
      }
      case FDM_Q_MUBAR: {
        if (!c->general) fail(FDM_EINVAL, "the averaged surrogate is defined on curved cells");
        std::vector<double> h(3 * (size_t)c->g.ncell);
        FDM_CUDA(cudaMemcpy(h.data(), c->mubar, h.size() * sizeof(double), cudaMemcpyDeviceToHost));
        put(h.data(), h.size() * sizeof(double));
        break;
      }
      case FDM_Q_SURR_OUTPUT: {
        if (!c->surr_c) fail(FDM_EINVAL, "no network output yet (call fdm_surrogate_apply)");
        std::vector<float> h(3 * (size_t)c->g.ncell);
        FDM_CUDA(cudaMemcpy(h.data(), c->surr_c, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
        put(h.data(), h.size() * sizeof(float));
        break;
      }
      case FDM_Q_TUNING: put(c->tuning, sizeof c->tuning); break;
      case FDM_Q_GMG_LEVELS: {
        std::vector<int> v{c->gmg_L};
        for (const GmgHostLevel &H : c->gmg_host) v.insert(v.end(), {H.n[0], H.n[1], H.n[2], H.nf});
        put(v.data(), v.size() * sizeof(int));
        break;
      }
      case FDM_Q_GMG_STENCIL: {
        std::vector<double> v;
        for (const GmgHostLevel &H : c->gmg_host) v.insert(v.end(), H.A.begin(), H.A.end());
        put(v.data(), v.size() * sizeof(double));
        break;
      }
      case FDM_Q_STATUS: {
        int v = 0;
        FDM_CUDA(cudaMemcpy(&v, c->status, sizeof(int), cudaMemcpyDeviceToHost));
        FDM_CUDA(cudaMemset(c->status, 0, sizeof(int)));
        put(&v, sizeof v);
        break;
      }
      case FDM_Q_KERNEL_TIMES: {
        std::vector<double> h(2 * FDM_NTIMER, 0.0);
        if (c->ev_used > 0) FDM_CUDA(cudaEventSynchronize(c->ev_pool[c->ev_used - 1]));
        for (size_t i = 0; i < c->ev_used / 2; ++i) {
          float ms = 0.f;
          FDM_CUDA(cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]));
          h[2 * c->ev_tag[i]] += 1.0;
          h[2 * c->ev_tag[i] + 1] += ms;
        }
        c->ev_used = 0;
        c->ev_tag.clear();
        put(h.data(), h.size() * sizeof(double));
        break;
      }
      case FDM_Q_LAUNCHES: {
        int64_t v = c->launches;
        c->launches = 0;
        put(&v, sizeof v);
        break;
      }
      case FDM_Q_ALGO_BYTES: {
        // one patch-solve launch reads every stored nonzero of every patch's
        // solve operator once (L form: the structurally nonzero entries of
        // L_Gamma; Schur-coupling form: level-0 pivots, L10, the line blocks,
        // S_TB and the lower triangle of W), reads the cell-local FDM residual
        // once and writes every star solution once; one asm_apply adds the FP64
        // input and output vectors and the 3 surrogate coefficients per cell.
        double nnz = 0.0, nd = 0.0;
        for (int i = 0; i < c->npatch; ++i) {
          const PatchClass &K = c->classes[c->h_patches[i].cls];
          nnz += (double)(c->scform ? K.nnzSC : K.nnzL);
          nd += (double)c->classes[c->h_patches[i].cls].nd;
        }
        double ne = (double)c->g.ncell * c->g.n * c->g.n * c->g.n;
        double v[4];
        for (int s = 0; s < 2; ++s) {
          double w = s == 0 ? 8.0 : 4.0;
          v[s] = w * (nnz + ne + nd);
          v[2 + s] = v[s] + 16.0 * (double)c->g.ndof + 24.0 * c->g.ncell;
        }
        put(v, sizeof v);
        break;
      }
      case FDM_Q_ALGO_BYTES_LFORM: {  // the same count for the L form (whichever form is in use)
        double nnz = 0.0, nd = 0.0;
        for (int i = 0; i < c->npatch; ++i) {
          nnz += (double)c->classes[c->h_patches[i].cls].nnzL;
          nd += (double)c->classes[c->h_patches[i].cls].nd;
        }
        const double ne = (double)c->g.ncell * c->g.n * c->g.n * c->g.n;
        double v[2] = {8.0 * (nnz + ne + nd), 4.0 * (nnz + ne + nd)};
        put(v, sizeof v);
        break;
      }
      default: fail(FDM_EINVAL, "fdm_query: unknown quantity");
    }
  } catch (const Error &e) { return handle(c, e); }
  return FDM_OK;
}

const char *fdm_last_error(const fdm_ctx *c) { return c ? c->err.c_str() : g_last_error.c_str(); }

void fdm_destroy(fdm_ctx *c) {
  if (!c) return;
  delete c->solo;
  delete c;
}

}  // extern "C"
