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
};
int patch_tmp_elems(int maxN1, int maxN2);

template <typename T>
struct InterpArgs {
  Grid g;
  const PatchDev *patches;
  const ClassDev *cls;
  const T *X;       // interface solutions of all stars
  const T *E;       // condensed cell-local FDM residual (interior entries unchanged)
  const double *mu; // surrogate coefficients
  const T *tab;
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
// per-cell Galerkin coarse matrices P_K^T A^K P_K (FP64), [ncell][8][8]
void launch_coarse_cell_matrices(const OpArgs &a, double *Ac, cudaStream_t st);

// context accessors (defined with the C-ABI)
OpArgs ctx_op_args64(const fdm_ctx *c);
void ctx_count_launches(fdm_ctx *c, int k);
int ctx_fail(fdm_ctx *c, int code, const std::string &msg);

// coarse space
template <typename T, typename Tin>
void launch_coarse_restrict(const Grid &g, const Tin *r, const T *tab, const int *cfree, T *rc, T *cellbuf,
                            cudaStream_t st);
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

}  // namespace fdm
