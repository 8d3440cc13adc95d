// The scalar context shared by the library's translation units (not part of
// the C-ABI): problem data on the device, patch factors, coarse space, work
// vectors and instrumentation, with per-precision accessors.
#pragma once
#include <algorithm>
#include <string>
#include <vector>

#include "factor.h"
#include "internal.h"
#include "kernels.h"

using namespace fdm;

struct fdm_ctx {
  Grid g{};
  int p = 0;
  int device = 0;  // the CUDA device current at set-up, which holds all of the context's data
  fdm_options opt{};
  Basis1D basis;
  std::vector<PatchClass> classes;
  int general = 0;
  std::vector<void *> allocs;
  std::string err;

  // device data
  double *tab64 = nullptr;
  float *tab32 = nullptr;
  double *mu_box = nullptr, *mu = nullptr;
  double *Gw64 = nullptr, *detw64 = nullptr;
  float *Gw32 = nullptr, *detw32 = nullptr;
  ClassDev *d_cls = nullptr;
  int *cmap = nullptr;  // cell node -> star interface index per (class, corner)
  std::vector<ClassDev> h_cls;
  std::vector<PatchDev> h_patches;
  PatchDev *d_patches = nullptr;
  int *d_order = nullptr;
  int npatch = 0, nsolve = 0;
  int maxG = 0, maxN0 = 0, maxN1 = 0, maxN2 = 0;
  int patch_threads = 256;
  // streamed patch solve
  bool stream = true;
  int nbuf = 4, buf_bytes = 16384;
  int *status = nullptr;
  int *d_order_nz = nullptr;  // patches with an interface, heaviest first
  int nsolve_nz = 0;
  int64_t nval_total = 0, nstar_total = 0;
  double *L64 = nullptr;
  float *L32 = nullptr;
  double *X64 = nullptr, *E64 = nullptr;
  float *X32 = nullptr, *E32 = nullptr;
  size_t smem64 = 0, smem32 = 0;
  // resident patch solve (whole factor of a patch in shared memory), per precision
  bool res64 = false, res32 = false;
  int fcap = 0, res_threads = 512, res_tmp = 0;
  int rows8 = 0;  // forward products of the classic patch solve: eight rows per warp
  bool scform = false;  // Schur-coupling form of the patch factors and solve
  int headcap32 = 0, headcap64 = 0;  // its staged values before W, per precision (elements)
  int bcap32 = 0, bcap64 = 0;        // the same before S_TB (lower block only)
  bool sc_persist = false;           // persistent Schur-coupling kernel (patch_kernel = 5)
  bool sc_full = false;              // persistent, whole patch staged (patch_kernel = 6)
  bool sc_warp = false;              // one warp per patch (patch_kernel = 7)
  int fcap_sc = 0;                   // its buffer size: the largest class's value count
  // cluster patch solve for the classes with a dense top level (a prefix of the order)
  int n_heavy = 0, cl_threads = 256;
  bool cl32 = false, cl64 = false;
  ClusterArgs<float> cla32{};
  ClusterArgs<double> cla64{};
  double tuning[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // autotuner: kernel, threads, rows8, best us, candidates tried
  size_t rsmem64 = 0, rsmem32 = 0;
  // coarse
  int nc = 0;
  int nc_dense = 0;  // order of the dense inverse: the Q1 problem, or the coarsest multigrid level
  // geometric multigrid on the Q1 problem: gmg_L coarsenings (0 = exact solve)
  int gmg_L = 0, gmg_nu = 2;
  double gmg_omega = 2.0 / 3.0;
  std::vector<GmgHostLevel> gmg_host;
  template <typename T>
  struct GmgVecs {
    std::vector<GmgDev<T>> lev;
    std::vector<T *> b, out, xa, xb, r;  // per level: right-hand side, result, two iterates, residual
  };
  GmgVecs<double> gmg64;
  GmgVecs<float> gmg32;
  template <typename T> GmgVecs<T> &gmg();
  std::vector<double> vert[3];  // mesh vertex coordinates per axis
  int *cfree = nullptr;
  double *Acinv64 = nullptr, *rc64 = nullptr, *xc64 = nullptr, *cb64 = nullptr;
  float *Acinv32 = nullptr, *rc32 = nullptr, *xc32 = nullptr, *cb32 = nullptr;
  // work vectors
  double *r = nullptr, *z = nullptr, *zold = nullptr, *d = nullptr, *q = nullptr;
  double *v1 = nullptr, *v2 = nullptr, *v3 = nullptr;
  float *f_in = nullptr, *f_out = nullptr, *f1 = nullptr, *f2 = nullptr, *f3 = nullptr;
  double *partial = nullptr, *dots = nullptr, *sc = nullptr;
  double omega = 1.0, lmin = 0.0, lmax = 0.0;
  double t_setup[4] = {0, 0, 0, 0};
  // learned surrogate (curved cells)
  double *mubar = nullptr;      // averaged surrogate of Section 2.7, [ncell][3]
  double *wq64 = nullptr;       // Gauss weights (n)
  float *feat = nullptr;        // network inputs [ncell][189] (with samples27)
  double *cstar = nullptr, *F0 = nullptr, *F1 = nullptr;  // labels and bound ratios (on first use)
  float *label32 = nullptr;
  // labels scored by the interior patch's Lanczos condition number (on request)
  int label_kind = 0;  // FDM_LABEL_*: the labels fdm_surrogate_grad / _train use
  double *ckap = nullptr, *Fkap = nullptr, *S64 = nullptr, *lam64 = nullptr;
  float *label32k = nullptr;
  float *surr_c = nullptr;      // network outputs of the last fdm_surrogate_apply
  int *d_count = nullptr;
  double *Fcur = nullptr;       // bound ratios at the current mu (queries)
  double kappa_avg = 0.0;       // Lanczos lmax / lmin with the averaged surrogate (0: not run)
  // instrumentation: launch counter and optional per-group CUDA-event timers
  int64_t launches = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_tag;  // tag of each recorded (begin, end) pair
  size_t ev_used = 0;
  bool capturing = false;  // building a CUDA graph: no event timers
  struct fdm_batch *solo = nullptr;  // one-problem batch of the graph-driven pcg_solve
  void tmark(int tag, bool begin, cudaStream_t st) {
    if (!opt.kernel_timing || capturing) return;
    if (begin) {
      if (ev_used + 2 > ev_pool.size()) {
        for (int i = 0; i < 256; ++i) {
          cudaEvent_t e;
          FDM_CUDA(cudaEventCreate(&e));
          ev_pool.push_back(e);
        }
      }
      ev_tag.push_back(tag);
      FDM_CUDA(cudaEventRecord(ev_pool[ev_used], st));
    } else {
      FDM_CUDA(cudaEventRecord(ev_pool[ev_used + 1], st));
      ev_used += 2;
    }
  }

  size_t alloc_bytes = 0;  // device bytes allocated through alloc()
  template <typename T>
  T *alloc(size_t n) {
    void *ptr = device_alloc(std::max<size_t>(n, 1) * sizeof(T), alloc_bytes);
    allocs.push_back(ptr);
    return static_cast<T *>(ptr);
  }
  template <typename T>
  T *upload(const std::vector<T> &h) {
    T *ptr = alloc<T>(h.size());
    if (!h.empty()) FDM_CUDA(cudaMemcpy(ptr, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return ptr;
  }
  ~fdm_ctx() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    for (void *ptr : allocs) cudaFree(ptr);
  }

  template <typename T> const T *tab() const;
  template <typename T> T *E() const;
  template <typename T> T *X() const;
  template <typename T> const T *L() const;
  template <typename T> size_t smem() const;
  template <typename T> T *rc() const;
  template <typename T> T *xc() const;
  template <typename T> T *cb() const;
  template <typename T> const T *Acinv() const;
  OpArgs op_args(bool fp32) const {
    OpArgs a;
    a.g = g;
    a.general = general;
    a.mu_box = mu_box;
    a.Gw = fp32 ? (const void *)Gw32 : (const void *)Gw64;
    a.detw = fp32 ? (const void *)detw32 : (const void *)detw64;
    a.tab = fp32 ? (const void *)tab32 : (const void *)tab64;
    return a;
  }
};
template <> inline fdm_ctx::GmgVecs<double> &fdm_ctx::gmg<double>() { return gmg64; }
template <> inline fdm_ctx::GmgVecs<float> &fdm_ctx::gmg<float>() { return gmg32; }
template <> inline const double *fdm_ctx::tab<double>() const { return tab64; }
template <> inline const float *fdm_ctx::tab<float>() const { return tab32; }
template <> inline double *fdm_ctx::E<double>() const { return E64; }
template <> inline float *fdm_ctx::E<float>() const { return E32; }
template <> inline double *fdm_ctx::X<double>() const { return X64; }
template <> inline float *fdm_ctx::X<float>() const { return X32; }
template <> inline const double *fdm_ctx::L<double>() const { return L64; }
template <> inline const float *fdm_ctx::L<float>() const { return L32; }
template <> inline size_t fdm_ctx::smem<double>() const { return smem64; }
template <typename T> ClusterArgs<T> cluster_args(const fdm_ctx *c);
template <> inline ClusterArgs<float> cluster_args<float>(const fdm_ctx *c) { return c->cla32; }
template <> inline ClusterArgs<double> cluster_args<double>(const fdm_ctx *c) { return c->cla64; }
template <> inline size_t fdm_ctx::smem<float>() const { return smem32; }
template <> inline double *fdm_ctx::rc<double>() const { return rc64; }
template <> inline float *fdm_ctx::rc<float>() const { return rc32; }
template <> inline double *fdm_ctx::xc<double>() const { return xc64; }
template <> inline float *fdm_ctx::xc<float>() const { return xc32; }
template <> inline double *fdm_ctx::cb<double>() const { return cb64; }
template <> inline float *fdm_ctx::cb<float>() const { return cb32; }
template <> inline const double *fdm_ctx::Acinv<double>() const { return Acinv64; }
template <> inline const float *fdm_ctx::Acinv<float>() const { return Acinv32; }

namespace fdm {
// internals of the scalar path that other translation units use
void ctx_mask_dirichlet(const Grid &g, double *v, cudaStream_t st);
void ctx_copy(int64_t n, const double *a, double *b, cudaStream_t st);
int ctx_vec_blocks(int64_t n);
void ctx_banded_cholesky(int m, int bw, std::vector<double> &Lb);
void ctx_tridiag_extremes(const std::vector<double> &d, const std::vector<double> &e, double &lo, double &hi);
void ctx_normal_vector(uint64_t seed, int64_t n, std::vector<double> &out);
std::string &ctx_last_error();
// one relaxation sweep z = omega ASM(r) (+ addv) in precision T
template <typename T, typename Tin, typename Tout>
void ctx_run_asm(fdm_ctx *c, const Tin *r, Tout *z, double omega, cudaStream_t st, const T *addv);
// xc = A_c^{-1} rc on the context's Q1 vectors (exact, or one multigrid V-cycle), precision T
template <typename T>
void ctx_coarse_solve(fdm_ctx *c, cudaStream_t st);
}  // namespace fdm
