// Surrogate labels scored by the condition number of each cell's interior
// patch (Section 2.7): for candidate scalings mu, the Lanczos estimate of
// kappa(A~_P(mu)^{-1} A_P) with A_P the true cell stiffness on the interior
// functions (sum factorisation on the Gauss points) and A~_P(mu) the separable
// surrogate's interior block, diagonal in the interior FDM basis:
// A~_P = S^{-T} D S^{-1} with S = S_1 (x) S_1 (x) S_1 and D = mu_x lam_i +
// mu_y lam_j + mu_z lam_k.  The estimate runs Lanczos with full
// reorthogonalisation on the symmetric form D^{-1/2} S^T A_P S D^{-1/2}, its
// vectors in shared memory.  One CTA per cell runs the compass search over the
// two scaling ratios and centres the labelled spectrum.  FP64 throughout.
#include <cmath>
#include <cstdint>

#include "cellop.cuh"
#include "device.cuh"
#include "kernels.h"

namespace fdm {
namespace {

constexpr int PK_THREADS = 256;

struct PatchKappaArgs {
  int ncell, p, n, m1;
  const double *Gw;     // [cell][n^3][6] w_q kappa Ghat
  const double *tab;    // 1D tables (Gauss values and derivatives at TAB_VQ, TAB_DQ)
  const double *S;      // interior eigenvectors (m1 x m1, column i = vector i)
  const double *lam;    // interior eigenvalues (m1)
  const double *mubar;  // [cell][3]
};

// the CTA's sum of a[i] b[i], i < m, in a fixed order (each thread a fixed
// stride, then the warps, then the warp sums in order); every thread gets it
__device__ double block_dot(const double *a, const double *b, int m, double *red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += a[i] * b[i];
  s = warp_sum(s);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

// eigenvalues of the symmetric tridiagonal (d[k], e[k-1]) below x (Sturm count)
__device__ int sturm_count(const double *d, const double *e, int k, double x) {
  int c = 0;
  double q = d[0] - x;
  if (q < 0.0) ++c;
  for (int j = 1; j < k; ++j) {
    if (q == 0.0) q = 1e-300;
    q = d[j] - x - e[j - 1] * e[j - 1] / q;
    if (q < 0.0) ++c;
  }
  return c;
}

// the eigenvalue of index idx (ascending) by bisection on the Gershgorin interval
__device__ double tridiag_eig(const double *d, const double *e, int k, int idx) {
  double lo = INFINITY, hi = -INFINITY;
  for (int j = 0; j < k; ++j) {
    const double r = (j > 0 ? fabs(e[j - 1]) : 0.0) + (j + 1 < k ? fabs(e[j]) : 0.0);
    lo = fmin(lo, d[j] - r);
    hi = fmax(hi, d[j] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;  // the interval cannot shrink further
    if (sturm_count(d, e, k, mid) > idx) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

struct PkSmem {
  double *V, *D, *S, *lam, *Dm;         // Gauss tables, interior FDM basis, D^{-1/2}
  double *U, *B1, *B2, *B3, *B4, *OUT;  // cell cubes n^3
  double *Q;                            // Lanczos vectors [K + 1][m]
  double *w, *t1, *t2;                  // patch vectors m
  double *red, *c, *al, *be, *tri;      // reduction scratch, projections, Lanczos coefficients
};

// q = A_P x: zero-extended to the cell, the cell stiffness, restricted back
__device__ void apply_true(const PatchKappaArgs &a, const PkSmem &s, const double *Gw, const double *x, double *q) {
  const int n = a.n, m1 = a.m1, n3 = n * n * n, m = m1 * m1 * m1;
  for (int i = threadIdx.x; i < n3; i += blockDim.x) s.U[i] = 0.0;
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int ix = i % m1, iy = (i / m1) % m1, iz = i / (m1 * m1);
    s.U[(ix + 1) + n * ((iy + 1) + n * (iz + 1))] = x[i];
  }
  __syncthreads();
  cell_stiffness_gen<double>(s.V, s.D, Gw, n, s.U, s.B1, s.B2, s.B3, s.B4, s.OUT);
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int ix = i % m1, iy = (i / m1) % m1, iz = i / (m1 * m1);
    q[i] = s.OUT[(ix + 1) + n * ((iy + 1) + n * (iz + 1))];
  }
  __syncthreads();
}

// w = C y with C = D^{-1/2} S^T A_P S D^{-1/2} (S = S_1 (x) S_1 (x) S_1): similar
// to A~_P(mu)^{-1} A_P, since A~_P = S^{-T} D S^{-1} in the interior FDM basis
__device__ void apply_symmetric(const PatchKappaArgs &a, const PkSmem &s, const double *Gw, const double *y,
                                double *w) {
  const int m1 = a.m1, m = m1 * m1 * m1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s.t1[i] = s.Dm[i] * y[i];
  __syncthreads();
  contract(s.t1, s.t2, s.S, false, 2, m1, 1.0, false);
  __syncthreads();
  contract(s.t2, s.t1, s.S, false, 1, m1, 1.0, false);
  __syncthreads();
  contract(s.t1, s.t2, s.S, false, 0, m1, 1.0, false);
  __syncthreads();
  apply_true(a, s, Gw, s.t2, s.t1);
  contract(s.t1, s.t2, s.S, true, 0, m1, 1.0, false);
  __syncthreads();
  contract(s.t2, s.t1, s.S, true, 1, m1, 1.0, false);
  __syncthreads();
  contract(s.t1, w, s.S, true, 2, m1, 1.0, false);
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) w[i] *= s.Dm[i];
  __syncthreads();
}

// one classical Gram-Schmidt pass of w against the nv stored Lanczos vectors:
// all projections from the same w (per-thread strided sums, warp sums, then
// the warps in order), then one update
__device__ void cgs_pass(const PkSmem &s, int nv, int m) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < nv; ++j) {
    double t = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) t += s.w[i] * s.Q[(size_t)j * m + i];
    t = warp_sum(t);
    if (lane == 0) s.red[warp * (PATCH_KAPPA_STEPS + 1) + j] = t;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < nw; ++q) t += s.red[q * (PATCH_KAPPA_STEPS + 1) + j];
    s.c[j] = t;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    double t = s.w[i];
    for (int j = 0; j < nv; ++j) t -= s.c[j] * s.Q[(size_t)j * m + i];
    s.w[i] = t;
  }
  __syncthreads();
}

// Lanczos extremes of A~(mu)^{-1} A: K = min(PATCH_KAPPA_STEPS, m) steps of
// Lanczos with full reorthogonalisation (two passes) on C from the fixed
// golden-ratio start vector, ended early when the next vector's norm is below
// PATCH_KAPPA_BREAKDOWN times the largest diagonal entry; returns log(hi / lo)
__device__ double patch_log_kappa(const PatchKappaArgs &a, const PkSmem &s, const double *Gw, const double mu[3],
                                  double &lo, double &hi) {
  const int m1 = a.m1, m = m1 * m1 * m1;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    const int ix = i % m1, iy = (i / m1) % m1, iz = i / (m1 * m1);
    s.Dm[i] = 1.0 / sqrt(mu[0] * s.lam[ix] + mu[1] * s.lam[iy] + mu[2] * s.lam[iz]);
    s.Q[i] = (double)(((uint64_t)i * 2654435769ull) & 0xffffffffull) / 4294967296.0 - 0.5;
  }
  __syncthreads();
  const double r0n = sqrt(block_dot(s.Q, s.Q, m, s.red));
  for (int i = threadIdx.x; i < m; i += blockDim.x) s.Q[i] /= r0n;
  __syncthreads();
  const int K = PATCH_KAPPA_STEPS < m ? PATCH_KAPPA_STEPS : m;
  int nal = 0;
  double amax = 0.0;
  for (int k = 0; k < K; ++k) {
    const double *qk = s.Q + (size_t)k * m;
    apply_symmetric(a, s, Gw, qk, s.w);
    const double alpha = block_dot(s.w, qk, m, s.red);
    amax = fmax(amax, fabs(alpha));
    const double bprev = k > 0 ? s.be[k - 1] : 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      s.w[i] -= alpha * qk[i] + (k > 0 ? bprev * s.Q[(size_t)(k - 1) * m + i] : 0.0);
    __syncthreads();
    cgs_pass(s, k + 1, m);
    cgs_pass(s, k + 1, m);
    const double b = sqrt(block_dot(s.w, s.w, m, s.red));
    if (threadIdx.x == 0) s.al[k] = alpha;
    nal = k + 1;
    if (k == K - 1 || !(b > PATCH_KAPPA_BREAKDOWN * amax)) break;
    if (threadIdx.x == 0) s.be[k] = b;
    double *qn = s.Q + (size_t)(k + 1) * m;
    for (int i = threadIdx.x; i < m; i += blockDim.x) qn[i] = s.w[i] / b;
    __syncthreads();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double *dd = s.tri, *ee = s.tri + PATCH_KAPPA_STEPS;
    for (int j = 0; j < nal; ++j) {
      dd[j] = s.al[j];
      if (j + 1 < nal) ee[j] = s.be[j];
    }
    s.red[0] = tridiag_eig(dd, ee, nal, 0);
    s.red[1] = tridiag_eig(dd, ee, nal, nal - 1);
  }
  __syncthreads();
  lo = s.red[0];
  hi = s.red[1];
  __syncthreads();
  return log(hi / lo);
}

__global__ void __launch_bounds__(PK_THREADS) k_surr_patch_label(PatchKappaArgs a, double *cout, double *fout,
                                                                 int *evals_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = a.n, m1 = a.m1, n3 = n * n * n, m = m1 * m1 * m1;
  PkSmem s;
  double *ptr = reinterpret_cast<double *>(smem_raw);
  s.V = ptr; ptr += n * n;
  s.D = ptr; ptr += n * n;
  s.S = ptr; ptr += m1 * m1;
  s.lam = ptr; ptr += m1;
  s.Dm = ptr; ptr += m;
  s.U = ptr; ptr += n3;
  s.B1 = ptr; ptr += n3;
  s.B2 = ptr; ptr += n3;
  s.B3 = ptr; ptr += n3;
  s.B4 = ptr; ptr += n3;
  s.OUT = ptr; ptr += n3;
  s.Q = ptr; ptr += (size_t)(PATCH_KAPPA_STEPS + 1) * m;
  s.w = ptr; ptr += m;
  s.t1 = ptr; ptr += m;
  s.t2 = ptr; ptr += m;
  s.red = ptr; ptr += (PK_THREADS / 32) * (PATCH_KAPPA_STEPS + 1);
  s.c = ptr; ptr += PATCH_KAPPA_STEPS + 1;
  s.al = ptr; ptr += PATCH_KAPPA_STEPS;
  s.be = ptr; ptr += PATCH_KAPPA_STEPS;
  s.tri = ptr;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    s.V[i] = a.tab[tab_off(TAB_VQ, n) + i];
    s.D[i] = a.tab[tab_off(TAB_DQ, n) + i];
  }
  for (int i = threadIdx.x; i < m1 * m1; i += blockDim.x) s.S[i] = a.S[i];
  for (int i = threadIdx.x; i < m1; i += blockDim.x) s.lam[i] = a.lam[i];
  __syncthreads();
  const int e = blockIdx.x;
  const double *Gw = a.Gw + (size_t)e * n3 * 6;
  const double mb[3] = {a.mubar[3 * e], a.mubar[3 * e + 1], a.mubar[3 * e + 2]};
  double lo, hi;
  // compass search over (t1, t2), mu = mubar exp((0, t1, t2))
  double t0 = 0.0, t1 = 0.0;
  double f = patch_log_kappa(a, s, Gw, mb, lo, hi);
  const double f0 = f;
  double step = PATCH_KAPPA_S0;
  int evals = 1;
  for (int round = 0; round < PATCH_KAPPA_ROUNDS && step >= PATCH_KAPPA_SMIN; ++round) {
    double best = f, b0 = t0, b1 = t1;
    bool moved = false;
    for (int k = 0; k < 4; ++k) {
      const double u0 = t0 + (k == 0 ? step : (k == 1 ? -step : 0.0));
      const double u1 = t1 + (k == 2 ? step : (k == 3 ? -step : 0.0));
      const double mu[3] = {mb[0], mb[1] * exp(u0), mb[2] * exp(u1)};
      const double ft = patch_log_kappa(a, s, Gw, mu, lo, hi);
      ++evals;
      if (ft < best - PATCH_KAPPA_IMPROVE) {
        best = ft;
        b0 = u0;
        b1 = u1;
        moved = true;
      }
    }
    if (moved) {
      t0 = b0;
      t1 = b1;
      f = best;
    } else {
      step *= 0.5;
    }
  }
  const double mu[3] = {mb[0], mb[1] * exp(t0), mb[2] * exp(t1)};
  const double f1 = patch_log_kappa(a, s, Gw, mu, lo, hi);
  if (threadIdx.x == 0) {
    const double g = 0.5 * log(lo * hi);  // centre: lambda_min lambda_max = 1
    cout[3 * e] = g;
    cout[3 * e + 1] = t0 + g;
    cout[3 * e + 2] = t1 + g;
    fout[2 * e] = f0;
    fout[2 * e + 1] = f1;
    if (evals_out) evals_out[e] = evals;
  }
}

size_t patch_label_smem(int n, int m1) {
  const size_t n3 = (size_t)n * n * n, m = (size_t)m1 * m1 * m1, K = PATCH_KAPPA_STEPS;
  return sizeof(double) * (2 * (size_t)n * n + (size_t)m1 * m1 + m1 + m + 6 * n3 + (K + 1) * m + 3 * m +
                           (PK_THREADS / 32) * (K + 1) + (K + 1) + 4 * K);
}

}  // namespace

void launch_surr_patch_label(int ncell, int p, const double *Gw, const double *tab, const double *S,
                             const double *lam, const double *mubar, double *cstar, double *F, int *evals,
                             cudaStream_t st) {
  if (p < 2 || p > PATCH_KAPPA_PMAX) fail(FDM_EINVAL, "patch-condition labels: degree 2..8");
  if (ncell == 0) return;
  PatchKappaArgs a{ncell, p, p + 1, p - 1, Gw, tab, S, lam, mubar};
  const size_t sm = patch_label_smem(p + 1, p - 1);
  if (sm > 227 * 1024) fail(FDM_EINVAL, "patch-condition labels: shared memory");
  FDM_CUDA(cudaFuncSetAttribute(k_surr_patch_label, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  k_surr_patch_label<<<ncell, PK_THREADS, sm, st>>>(a, cstar, F, evals);
}

}  // namespace fdm
