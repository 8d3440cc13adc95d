// Symmetric interior penalty DG (SIPG) for the Poisson equation on DQ_p box
// cells (Section 5): the context and its C-ABI entry points (declared in
// include/fdmpc.h).
//
// Relaxation: additive Schwarz over the vertex stars of the interior vertices,
// each star holding all (2p+2)^3 values of its 8 cells, solved exactly.  On a
// Cartesian star the star matrix (the principal submatrix of A) is a
// Kronecker sum of 1D two-cell pencils, so the exact solve is the
// fast-diagonalisation product of their eigendecompositions, set up here on
// the host in FP64.  Coarse space: the conforming Q1 functions vanishing on
// the boundary; their jumps vanish, so the Galerkin operator is the Q1
// stiffness, which the Q1 context of the same mesh holds and solves (exactly,
// or by one multigrid V-cycle).  Preconditioner: the hybrid V(1,1) of the
// conforming problem (Section 2.5).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ctx.h"

struct fdm_sipg {
  fdm_ctx *q1 = nullptr;  // the Q1 problem of the same mesh: coarse space and its solver
  fdm_options opt;
  int p = 0, n = 0, nc[3] = {0, 0, 0};
  double eta = 0.0, omega = 1.0, lmin = 0.0, lmax = 0.0;
  int64_t ndof = 0;
  std::string err;
  std::vector<void *> allocs;
  SipgDev<double> d64;
  SipgDev<float> d32;
  int color_blocks[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  double *F64 = nullptr, *cb64 = nullptr;
  float *F32 = nullptr, *cb32 = nullptr;
  double *r = nullptr, *z = nullptr, *zold = nullptr, *d = nullptr, *q = nullptr, *v1 = nullptr, *v3 = nullptr;
  float *f1 = nullptr, *f3 = nullptr, *zp32 = nullptr;
  double *partial = nullptr, *dots = nullptr, *sc = nullptr;
  int *vlist = nullptr;
  int *status = nullptr;  // 1 when a bounded wait of the tensor-core star solve ran out
  int *vall = nullptr;    // all interior vertices, lexicographic: the stars of the one-launch sweep
  int nstar_all = 0;
  bool one_launch = true;  // every star in one launch into zpa, then a per-value gather
  double *zpa64 = nullptr;
  float *zpa32 = nullptr;
  bool tc = false;        // star solves of the FP32 preconditioner on the tensor cores
  int vcap = 0;
  int64_t zcap = 0;
  int64_t launches = 0;
  size_t alloc_bytes = 0;  // device bytes allocated through alloc()
  template <typename T>
  T *alloc(size_t k) {
    void *ptr = device_alloc(std::max<size_t>(k, 1) * sizeof(T), alloc_bytes);
    allocs.push_back(ptr);
    return static_cast<T *>(ptr);
  }
  template <typename T>
  T *upload(const std::vector<T> &h) {
    T *ptr = alloc<T>(h.size());
    if (!h.empty()) FDM_CUDA(cudaMemcpy(ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return ptr;
  }
  template <typename T> const SipgDev<T> &dev() const;
  template <typename T> T *F() const;
  template <typename T> T *cb() const;
  ~fdm_sipg() {
    fdm_destroy(q1);
    for (void *ptr : allocs) cudaFree(ptr);
  }
};
template <> const SipgDev<double> &fdm_sipg::dev<double>() const { return d64; }
template <> const SipgDev<float> &fdm_sipg::dev<float>() const { return d32; }
template <> double *fdm_sipg::F<double>() const { return F64; }
template <> float *fdm_sipg::F<float>() const { return F32; }
template <> double *fdm_sipg::cb<double>() const { return cb64; }
template <> float *fdm_sipg::cb<float>() const { return cb32; }

namespace {

int handle_sipg(fdm_sipg *s, const Error &err) {
  if (s) s->err = err.msg;
  ctx_last_error() = err.msg;
  return err.code;
}

// y = A u (rsub == nullptr) or y = rsub - A u, in precision T
template <typename T, typename Tin>
void sipg_op(fdm_sipg *s, const Tin *u, T *y, const double *rsub, cudaStream_t st) {
  launch_sipg_op<T, Tin>(s->dev<T>(), u, s->F<T>(), rsub, y, st);
  s->launches += 2;
}

uint64_t sipg_timeout_ns(const fdm_sipg *s) { return (uint64_t)(std::max(s->opt.wait_timeout_s, 0.0) * 1e9); }

// the status word of the bounded waits: FDM_ETIMEOUT (and cleared) when set
void sipg_check_status(fdm_sipg *s) {
  if (!s->status) return;
  int h = 0;
  FDM_CUDA(cudaMemcpy(&h, s->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) {
    FDM_CUDA(cudaMemset(s->status, 0, sizeof(int)));
    fail(FDM_ETIMEOUT, "a bounded wait of the tensor-core star solve ran out");
  }
}

// z = omega ASM(r) (+ addv): the 8 vertex parity classes in a fixed order
template <typename T>
T *sipg_zpa(fdm_sipg *s) {
  if constexpr (sizeof(T) == 8) {
    if (!s->zpa64) s->zpa64 = s->alloc<double>((size_t)s->nstar_all * 8 * s->n * s->n * s->n);
    return s->zpa64;
  } else {
    if (!s->zpa32) s->zpa32 = s->alloc<float>((size_t)s->nstar_all * 8 * s->n * s->n * s->n);
    return s->zpa32;
  }
}

template <typename T, typename Tin, typename Tout>
void sipg_asm(fdm_sipg *s, const Tin *r, Tout *z, double omega, cudaStream_t st, const T *addv = nullptr) {
  if (s->one_launch && s->nstar_all > 0 &&
      (std::is_same<T, Tout>::value || std::is_same<Tout, double>::value)) {
    // every star in one launch into its own output, then a deterministic gather per value
    T *zpa = sipg_zpa<T>(s);
    bool done = false;
    if constexpr (std::is_same<T, float>::value) {
      if (s->tc) {
        launch_sipg_patch_tc<Tin, float>(s->d32, 0, s->nstar_all, s->vall, r, nullptr, zpa, 1.0, sipg_timeout_ns(s),
                                         s->status, st);
        done = true;
      }
    }
    if (!done) launch_sipg_patch<T, Tin, T>(s->dev<T>(), 0, s->nstar_all, s->vall, r, nullptr, zpa, 1.0, st);
    launch_sipg_star_gather<T, Tout>(s->dev<T>(), zpa, omega, addv, z, st);
    s->launches += 2;
    return;
  }
  if (addv) {
    if constexpr (std::is_same<T, double>::value && std::is_same<Tout, double>::value) ctx_copy(s->ndof, addv, z, st);
    else if constexpr (!std::is_same<T, Tout>::value) launch_convert<T, Tout>(s->ndof, addv, z, st);
    else fail(FDM_EINVAL, "SIPG relaxation: no FP32 to FP32 accumulation");
    s->launches += 1;
  } else {
    FDM_CUDA(cudaMemsetAsync(z, 0, s->ndof * sizeof(Tout), st));
  }
  for (int color = 0; color < 8; ++color)
    if (s->color_blocks[color] > 0) {
      if constexpr (std::is_same<T, float>::value) {
        if (s->tc) {
          launch_sipg_patch_tc<Tin, Tout>(s->d32, color, s->color_blocks[color], nullptr, r, z, nullptr, omega,
                                          sipg_timeout_ns(s), s->status, st);
          s->launches += 1;
          continue;
        }
      }
      launch_sipg_patch<T, Tin, Tout>(s->dev<T>(), color, s->color_blocks[color], nullptr, r, z, nullptr, omega, st);
      s->launches += 1;
    }
}

// x1 += P A_c^{-1} P^T r1
template <typename T>
void sipg_coarse(fdm_sipg *s, const T *r1, T *x1, cudaStream_t st) {
  fdm_ctx *c = s->q1;
  launch_sipg_restrict<T, T>(s->dev<T>(), r1, c->cfree, s->cb<T>(), c->rc<T>(), st);
  c->launches = 0;
  ctx_coarse_solve<T>(c, st);
  launch_sipg_prolong<T>(s->dev<T>(), c->cfree, c->xc<T>(), x1, st);
  s->launches += 3 + c->launches;
}

// the hybrid V(1,1), FP64 r to FP64 z, computed in T:
//   x1 = omega ASM(r); r1 = r - A x1; x1 += P A_c^{-1} P^T r1; r1 = r - A x1;
//   z = x1 + omega ASM(r1)
template <typename T>
void sipg_vcycle(fdm_sipg *s, const double *r, double *z, T *x1, T *r1, cudaStream_t st) {
  sipg_asm<T, double, T>(s, r, x1, s->omega, st);
  sipg_op<T, T>(s, x1, r1, r, st);
  if (s->q1->nc > 0) sipg_coarse<T>(s, r1, x1, st);
  sipg_op<T, T>(s, x1, r1, r, st);
  sipg_asm<T, T, double>(s, r1, z, s->omega, st, x1);
}

void sipg_pc(fdm_sipg *s, const double *r, double *z, cudaStream_t st) {
  const bool fp64 = s->opt.precision == FDM_PREC_FP64;
  if (s->opt.pc == FDM_PC_NONE) {
    ctx_copy(s->ndof, r, z, st);
    s->launches += 1;
  } else if (s->opt.pc == FDM_PC_ASM) {
    if (fp64) sipg_asm<double, double, double>(s, r, z, s->omega, st);
    else sipg_asm<float, double, double>(s, r, z, s->omega, st);
  } else {
    if (fp64) sipg_vcycle<double>(s, r, z, s->v1, s->v3, st);
    else sipg_vcycle<float>(s, r, z, s->f1, s->f3, st);
  }
}

// omega from k CG-Lanczos steps on ASM^{-1} A (undamped relaxation), FP64
void sipg_lanczos(fdm_sipg *s, const double *start_host, cudaStream_t st) {
  const int64_t n = s->ndof;
  std::vector<double> b0;
  if (start_host) b0.assign(start_host, start_host + n);
  else ctx_normal_vector(s->opt.lanczos_seed, n, b0);
  FDM_CUDA(cudaMemcpyAsync(s->r, b0.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
  sipg_asm<double, double, double>(s, s->r, s->z, 1.0, st);
  FDM_CUDA(cudaMemcpyAsync(s->d, s->z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double h[2];
  launch_dot(n, s->r, s->z, s->partial, s->dots, st);
  FDM_CUDA(cudaMemcpyAsync(h, s->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
  FDM_CUDA(cudaStreamSynchronize(st));
  double rz = h[0];
  std::vector<double> al, be;
  for (int k = 0; k < s->opt.lanczos_steps; ++k) {
    if (!(rz > 0.0)) break;
    sipg_op<double, double>(s, s->d, s->q, nullptr, st);
    launch_dot(n, s->d, s->q, s->partial, s->dots, st);
    FDM_CUDA(cudaMemcpyAsync(h, s->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    if (!(h[0] > 0.0)) break;
    const double alpha = rz / h[0];
    al.push_back(alpha);
    launch_axpby<double>(n, -alpha, s->q, 1.0, s->r, s->r, st);
    sipg_asm<double, double, double>(s, s->r, s->z, 1.0, st);
    launch_dot(n, s->r, s->z, s->partial, s->dots, st);
    FDM_CUDA(cudaMemcpyAsync(h, s->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    const double beta = h[0] / rz;
    be.push_back(beta);
    rz = h[0];
    launch_axpby<double>(n, 1.0, s->z, beta, s->d, s->d, st);
  }
  const int m = (int)al.size();
  if (m < 1) fail(FDM_EINVAL, "Lanczos: no steps could be taken");
  std::vector<double> dd(m), ee(std::max(m - 1, 1), 0.0);
  for (int j = 0; j < m; ++j) {
    dd[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < m) ee[j] = std::sqrt(be[j]) / al[j];
  }
  ctx_tridiag_extremes(dd, ee, s->lmin, s->lmax);
  s->omega = 2.0 / (1.25 * s->lmax + 0.75 * s->lmin);
}

template <typename T>
SipgDev<T> make_dev(const fdm_sipg *s, const double *hx, const double *hy, const double *hz, const T *tab,
                    const T *S, const T *lam, const int64_t soff[3], const int64_t loff[3]) {
  SipgDev<T> d;
  d.p = s->p;
  d.n = s->n;
  d.nx = s->nc[0];
  d.ny = s->nc[1];
  d.nz = s->nc[2];
  d.ncell = s->nc[0] * s->nc[1] * s->nc[2];
  d.eta = s->eta;
  d.hx = hx;
  d.hy = hy;
  d.hz = hz;
  d.tab = tab;
  d.S = S;
  d.lam = lam;
  for (int a = 0; a < 3; ++a) {
    d.soff[a] = soff[a];
    d.loff[a] = loff[a];
  }
  return d;
}

}  // namespace


// ====================================================================== C-ABI
extern "C" {

int fdm_sipg_setup(const fdm_mesh *mesh, int p, double eta, const fdm_options *opt, fdm_sipg **out, void *stream) {
  if (!out) return FDM_EINVAL;
  *out = nullptr;
  if (!mesh || !mesh->xv || !mesh->yv || !mesh->zv || mesh->nx < 2 || mesh->ny < 2 || mesh->nz < 2 || p < 1 ||
      p > SIPG_MAX_N - 1 || !std::isfinite(eta)) {
    ctx_last_error() = "fdm_sipg_setup: invalid mesh (at least 2 cells per axis), degree (1.." +
                       std::to_string(SIPG_MAX_N - 1) + ") or penalty";
    return FDM_EINVAL;
  }
  if (mesh->jac) {
    ctx_last_error() = "fdm_sipg_setup: box cells only (mesh->jac must be NULL)";
    return FDM_EINVAL;
  }
  const double *vv[3] = {mesh->xv, mesh->yv, mesh->zv};
  const int ncs[3] = {mesh->nx, mesh->ny, mesh->nz};
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < ncs[a]; ++i)
      if (!(vv[a][i + 1] > vv[a][i]) || !std::isfinite(vv[a][i + 1] - vv[a][i])) {
        ctx_last_error() = "fdm_sipg_setup: vertex coordinates must increase strictly";
        return FDM_EINVAL;
      }
  fdm_sipg *s = new fdm_sipg();
  try {
    cudaStream_t st = (cudaStream_t)stream;
    if (opt) s->opt = *opt;
    else fdm_default_options(&s->opt);
    if (s->opt.lanczos_steps <= 0) s->opt.lanczos_steps = 20;
    if (s->opt.flexible_beta < 0) s->opt.flexible_beta = s->opt.precision == FDM_PREC_FP32 ? 1 : 0;
    s->p = p;
    s->n = p + 1;
    s->eta = eta > 0.0 ? eta : p * (p + 1.0);
    if (s->opt.tensor_core && p != 7)
      fail(FDM_EINVAL, "fdm_sipg_setup: the tensor-core star solve covers DQ_7 (p = 7) only");
    s->tc = s->opt.tensor_core != 0;
    for (int a = 0; a < 3; ++a) s->nc[a] = ncs[a];
    const int n = s->n, m = 2 * n, ncell = ncs[0] * ncs[1] * ncs[2];
    s->ndof = (int64_t)ncell * n * n * n;
    // the Q1 context of the same mesh: only its coarse space is used
    fdm_options copt = s->opt;
    copt.pc = FDM_PC_VCYCLE;
    copt.omega = 1.0;
    copt.lanczos_start = nullptr;
    copt.pcg_graph = 0;
    copt.kernel_timing = 0;
    copt.autotune = 0;
    const int rc = fdm_setup(mesh, 1, nullptr, &copt, &s->q1, stream);
    if (rc != FDM_OK) fail(rc, "Q1 coarse space: " + ctx_last_error());
    // tables: A_hat, B_hat, l'(-1), l'(+1), GLL nodes
    const Basis1D b = make_basis(p);
    std::vector<double> dm, dp;
    sipg_end_derivatives(b.xi, dm, dp);
    std::vector<double> tab;
    tab.insert(tab.end(), b.A.begin(), b.A.end());
    tab.insert(tab.end(), b.B.begin(), b.B.end());
    tab.insert(tab.end(), dm.begin(), dm.end());
    tab.insert(tab.end(), dp.begin(), dp.end());
    tab.insert(tab.end(), b.xi.begin(), b.xi.end());
    // half-widths per axis and the stars' pencils
    std::vector<double> h[3], S64, L64;
    int64_t soff[3], loff[3];
    std::vector<double> A(m * m), M(m * m), Sv(m * m), lv(m);
    for (int a = 0; a < 3; ++a) {
      for (int i = 0; i < ncs[a]; ++i) h[a].push_back(0.5 * (vv[a][i + 1] - vv[a][i]));
      soff[a] = (int64_t)S64.size();
      loff[a] = (int64_t)L64.size();
      for (int k = 1; k < ncs[a]; ++k) {
        const double hl = k >= 2 ? h[a][k - 2] : -1.0, hr = k + 1 < ncs[a] ? h[a][k + 1] : -1.0;
        sipg_star_pencil(n, b.A.data(), b.B.data(), dm.data(), dp.data(), s->eta, h[a][k - 1], h[a][k], hl, hr,
                         A.data(), M.data());
        sym_gen_eig(m, A.data(), M.data(), Sv.data(), lv.data());
        S64.insert(S64.end(), Sv.begin(), Sv.end());
        L64.insert(L64.end(), lv.begin(), lv.end());
      }
    }
    const double *hx = s->upload(h[0]), *hy = s->upload(h[1]), *hz = s->upload(h[2]);
    auto f32 = [](const std::vector<double> &v) { return std::vector<float>(v.begin(), v.end()); };
    s->d64 = make_dev<double>(s, hx, hy, hz, s->upload(tab), s->upload(S64), s->upload(L64), soff, loff);
    s->d32 = make_dev<float>(s, hx, hy, hz, s->upload(f32(tab)), s->upload(f32(S64)), s->upload(f32(L64)), soff,
                             loff);
    for (int color = 0; color < 8; ++color) {
      int cnt = 1;
      for (int a = 0; a < 3; ++a) {
        const int first = ((color >> a) & 1) ? 1 : 2;
        cnt *= first <= ncs[a] - 1 ? (ncs[a] - 1 - first) / 2 + 1 : 0;
      }
      s->color_blocks[color] = cnt;
    }
    const size_t fn = (size_t)ncell * 12 * n * n;
    s->status = s->alloc<int>(1);
    FDM_CUDA(cudaMemset(s->status, 0, sizeof(int)));
    {  // the interior vertices, lexicographic (the stars of the one-launch sweep)
      std::vector<int> va;
      for (int vz = 1; vz < ncs[2]; ++vz)
        for (int vy = 1; vy < ncs[1]; ++vy)
          for (int vx = 1; vx < ncs[0]; ++vx) va.push_back(vx + (ncs[0] + 1) * (vy + (ncs[1] + 1) * vz));
      s->nstar_all = (int)va.size();
      if (!va.empty()) s->vall = s->upload(va);
      s->one_launch = s->opt.patch_kernel != 1;
    }
    s->F64 = s->alloc<double>(fn);
    s->cb64 = s->alloc<double>(8 * (size_t)ncell);
    s->cb32 = s->alloc<float>(8 * (size_t)ncell);
    if (s->opt.precision == FDM_PREC_FP32) {
      s->F32 = s->alloc<float>(fn);
      s->f1 = s->alloc<float>(s->ndof);
      s->f3 = s->alloc<float>(s->ndof);
    }
    for (double **v : {&s->r, &s->z, &s->zold, &s->d, &s->q, &s->v1, &s->v3}) *v = s->alloc<double>(s->ndof);
    s->partial = s->alloc<double>(2 * DOT_BLOCKS);
    s->dots = s->alloc<double>(4);
    s->sc = s->alloc<double>(16);
    if (s->opt.omega > 0.0) s->omega = s->opt.omega;
    else sipg_lanczos(s, s->opt.lanczos_start, st);
    FDM_CUDA(cudaStreamSynchronize(st));
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &err) {
    ctx_last_error() = err.msg;
    delete s;
    return err.code;
  }
  *out = s;
  return FDM_OK;
}

int sipg_apply(fdm_sipg *s, const double *u, double *y, void *stream) {
  if (!s || !u || !y) return FDM_EINVAL;
  try {
    sipg_op<double, double>(s, u, y, nullptr, (cudaStream_t)stream);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &err) { return handle_sipg(s, err); }
  return FDM_OK;
}

int sipg_asm_apply(fdm_sipg *s, const double *r, double *z, void *stream) {
  if (!s || !r || !z) return FDM_EINVAL;
  try {
    cudaStream_t st = (cudaStream_t)stream;
    if (s->opt.precision == FDM_PREC_FP64) sipg_asm<double, double, double>(s, r, z, s->omega, st);
    else sipg_asm<float, double, double>(s, r, z, s->omega, st);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &err) { return handle_sipg(s, err); }
  return FDM_OK;
}

int sipg_pc_apply(fdm_sipg *s, const double *r, double *z, void *stream) {
  if (!s || !r || !z) return FDM_EINVAL;
  try {
    sipg_pc(s, r, z, (cudaStream_t)stream);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &err) { return handle_sipg(s, err); }
  return FDM_OK;
}

int sipg_patch_solve(fdm_sipg *s, const double *r, int nv, const int *vertices, double *out, void *stream) {
  if (!s || !r || !out || nv < 0 || (nv > 0 && !vertices)) return FDM_EINVAL;
  if (nv == 0) return FDM_OK;
  const int nvx = s->nc[0] + 1, nvy = s->nc[1] + 1;
  for (int i = 0; i < nv; ++i) {
    const int v = vertices[i], vx = v % nvx, vy = (v / nvx) % nvy, vz = v / (nvx * nvy);
    if (v < 0 || vx < 1 || vy < 1 || vz < 1 || vx >= s->nc[0] || vy >= s->nc[1] || vz >= s->nc[2]) {
      s->err = "sipg_patch_solve: vertex " + std::to_string(v) + " is not an interior vertex";
      return FDM_EINVAL;
    }
  }
  try {
    cudaStream_t st = (cudaStream_t)stream;
    if (nv > s->vcap) {
      s->vlist = s->alloc<int>(nv);
      s->vcap = nv;
    }
    FDM_CUDA(cudaMemcpyAsync(s->vlist, vertices, nv * sizeof(int), cudaMemcpyHostToDevice, st));
    const int64_t m3 = 8 * (int64_t)s->n * s->n * s->n;
    if (s->opt.precision == FDM_PREC_FP64) {
      launch_sipg_patch<double, double, double>(s->d64, 0, nv, s->vlist, r, s->z, out, 1.0, st);
    } else {
      if ((int64_t)nv * m3 > s->zcap) {
        s->zp32 = s->alloc<float>((size_t)nv * m3);
        s->zcap = (int64_t)nv * m3;
      }
      if (s->tc)
        launch_sipg_patch_tc<double, float>(s->d32, 0, nv, s->vlist, r, s->f1, s->zp32, 1.0, sipg_timeout_ns(s),
                                            s->status, st);
      else launch_sipg_patch<float, double, float>(s->d32, 0, nv, s->vlist, r, s->f1, s->zp32, 1.0, st);
      launch_convert<float, double>((int64_t)nv * m3, s->zp32, out, st);
    }
    s->launches += 1;
    FDM_CUDA(cudaStreamSynchronize(st));
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &err) { return handle_sipg(s, err); }
  return FDM_OK;
}

int sipg_pcg_solve(fdm_sipg *s, const double *b, double *x, double rtol, int maxit, fdm_solve_info *info,
                   void *stream) {
  if (!s || !b || !x || maxit < 0 || !(rtol >= 0.0)) return FDM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = s->ndof;
  try {
    cudaEvent_t e0, e1;
    FDM_CUDA(cudaEventCreate(&e0));
    FDM_CUDA(cudaEventCreate(&e1));
    FDM_CUDA(cudaEventRecord(e0, st));
    double hsc[16] = {0};
    hsc[7] = s->opt.flexible_beta ? 1.0 : 0.0;
    FDM_CUDA(cudaMemcpyAsync(s->sc, hsc, sizeof hsc, cudaMemcpyHostToDevice, st));
    FDM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    FDM_CUDA(cudaMemcpyAsync(s->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    double h[2];
    launch_dot(n, s->r, s->r, s->partial, s->dots, st);
    s->launches += 2;
    FDM_CUDA(cudaMemcpyAsync(h, s->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    const double nb = std::sqrt(h[0]);
    double nr = nb;
    int it = 0, conv = nb == 0.0, bad = 0;
    double *z = s->z, *zold = s->zold;
    if (!conv) {
      sipg_pc(s, s->r, z, st);
      launch_dot(n, s->r, z, s->partial, s->dots, st);
      launch_pcg_scalars(2, s->sc, s->dots, st);
      FDM_CUDA(cudaMemcpyAsync(s->d, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      s->launches += 3;
      while (it < maxit) {
        sipg_op<double, double>(s, s->d, s->q, nullptr, st);
        launch_dot(n, s->d, s->q, s->partial, s->dots, st);
        launch_pcg_scalars(0, s->sc, s->dots, st);
        launch_pcg_update_xr(n, s->sc, s->d, s->q, x, s->r, st);
        ++it;
        launch_dot(n, s->r, s->r, s->partial, s->dots + 2, st);
        s->launches += 6;
        FDM_CUDA(cudaMemcpyAsync(h, s->dots + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
        FDM_CUDA(cudaStreamSynchronize(st));
        nr = std::sqrt(h[0]);
        if (!std::isfinite(nr)) { bad = 1; break; }
        if (nr <= rtol * nb) {
          // converged on the recursive residual: replace it by the true one,
          // r = b - A x, and stop only if that meets the test too
          sipg_op<double, double>(s, x, s->r, b, st);
          launch_dot(n, s->r, s->r, s->partial, s->dots + 2, st);
          s->launches += 3;
          FDM_CUDA(cudaMemcpyAsync(h, s->dots + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
          FDM_CUDA(cudaStreamSynchronize(st));
          nr = std::sqrt(h[0]);
          if (!std::isfinite(nr)) { bad = 1; break; }
          if (nr <= rtol * nb) { conv = 1; break; }
          if (it >= maxit) break;
        }
        std::swap(z, zold);
        sipg_pc(s, s->r, z, st);
        launch_dot2(n, s->r, z, zold, s->partial, s->dots, st);
        launch_pcg_scalars(1, s->sc, s->dots, st);
        launch_pcg_update_d(n, s->sc, z, s->d, st);
        s->launches += 4;
      }
    }
    FDM_CUDA(cudaEventRecord(e1, st));
    FDM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FDM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    FDM_CUDA(cudaMemcpy(hsc, s->sc, sizeof hsc, cudaMemcpyDeviceToHost));
    if (hsc[8] != 0.0) bad = 1;
    sipg_check_status(s);
    if (info) {
      info->iterations = it;
      info->converged = conv;
      info->rnorm0 = nb;
      info->rnorm = nr;
      info->seconds = ms * 1e-3;
      sipg_op<double, double>(s, x, s->v1, b, st);  // b - A x
      launch_dot(n, s->v1, s->v1, s->partial, s->dots, st);
      s->launches += 3;
      FDM_CUDA(cudaMemcpyAsync(h, s->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
      FDM_CUDA(cudaStreamSynchronize(st));
      info->true_rnorm = std::sqrt(h[0]);
    }
    FDM_CUDA(cudaGetLastError());
    if (bad) { s->err = "non-finite scalar in PCG"; return FDM_ENAN; }
    if (!conv) { s->err = "PCG reached maxit"; return FDM_ENOCONV; }
  } catch (const Error &err) { return handle_sipg(s, err); }
  return FDM_OK;
}

int fdm_sipg_query(fdm_sipg *s, int what, void *out, size_t *len) {
  if (!s || !out || !len) return FDM_EINVAL;
  try {
    auto put = [&](const void *src, size_t bytes) {
      if (*len < bytes) fail(FDM_EINVAL, "fdm_sipg_query: buffer too small (" + std::to_string(bytes) + " bytes needed)");
      std::memcpy(out, src, bytes);
      *len = bytes;
    };
    switch (what) {
      case FDM_Q_NDOF: { int64_t v = s->ndof; put(&v, sizeof v); break; }
      case FDM_Q_STATUS: {  // the tensor-core star solve's status word (read and cleared)
        int v = 0;
        FDM_CUDA(cudaMemcpy(&v, s->status, sizeof(int), cudaMemcpyDeviceToHost));
        FDM_CUDA(cudaMemset(s->status, 0, sizeof(int)));
        put(&v, sizeof v);
        break;
      }
      case FDM_Q_OMEGA: put(&s->omega, sizeof(double)); break;
      case FDM_Q_LAMBDA: { double v[2] = {s->lmin, s->lmax}; put(v, sizeof v); break; }
      case FDM_Q_LAUNCHES: { int64_t v = s->launches; s->launches = 0; put(&v, sizeof v); break; }
      case FDM_Q_NPATCH: {
        int v = (s->nc[0] - 1) * (s->nc[1] - 1) * (s->nc[2] - 1);
        put(&v, sizeof v);
        break;
      }
      default: fail(FDM_EINVAL, "fdm_sipg_query: unknown quantity");
    }
  } catch (const Error &err) { return handle_sipg(s, err); }
  return FDM_OK;
}

const char *fdm_sipg_last_error(const fdm_sipg *s) { return s ? s->err.c_str() : ctx_last_error().c_str(); }

void fdm_sipg_destroy(fdm_sipg *s) { delete s; }

}  // extern "C"
