// Primal linear elasticity (Section 4.1) with the SDC/FDM/sparse relaxation:
// the elasticity context and its C-ABI entry points (declared in
// include/fdmpc.h).  The three scalar contexts of the SDC blocks come from
// fdm_setup; their relaxation is driven through the scalar path's internals
// (ctx.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"

// ====================================================================== linear elasticity (Section 4.1)
// Primal formulation on box cells, clamped on the faces of a mask (the others
// traction-free: the natural condition); vectors are component-major
// [3][ndof].  The SDC relaxation is block-Jacobi over the displacement
// components: block j is the scalar operator with per-axis coefficients
// c_a = mu + (mu + lam) delta_aj, separable on box cells.  With every face
// clamped each block is a scalar context whose vertex-star FDM/sparse
// relaxation uses the exact surrogate mu_a^(j) = c_a vol / L_a^2; otherwise (or
// on request) the star solves use the star-local fast diagonalisation, exact
// for the block's constant coefficient, with the stars of vertices on
// traction-free faces keeping their boundary nodes.  Both invert the same star
// matrices.  The V(1,1) cycle uses the elasticity residual and the vector Q1
// Galerkin coarse problem over the vertices off the clamped faces, which on box
// cells is the Q1 elasticity stiffness (exactly integrated by 2 Gauss points
// per axis), solved through its dense inverse.
struct fdm_elast {
  fdm_ctx *comp[3] = {nullptr, nullptr, nullptr};
  fdm_options opt;
  double mu = 1.0, lam = 0.0, omega = 1.0, lmin = 0.0, lmax = 0.0;
  Grid g{};
  int64_t n = 0;  // grid nodes per component
  bool star = false;  // SDC star solves by the star-local FDM (else the scalar contexts)
  std::string err;
  std::vector<void *> allocs;
  double *Lc = nullptr;
  double *tab64 = nullptr;
  float *tab32 = nullptr;
  double *wq64 = nullptr;
  float *wq32 = nullptr;
  int *cfree = nullptr;  // [nv] coarse vertex of each vertex or -1
  double *cb64 = nullptr;
  float *cb32 = nullptr;
  StarFdmDev<double> sf64;
  StarFdmDev<float> sf32;
  double *X64 = nullptr;
  float *X32 = nullptr;
  double *G64 = nullptr, *E64 = nullptr;
  float *G32 = nullptr, *E32 = nullptr;
  int nq = 0, m = 0;  // free Q1 vertices, coarse unknowns 3 nq
  double *Ainv64 = nullptr, *rc64 = nullptr, *xc64 = nullptr;
  float *Ainv32 = nullptr, *rc32 = nullptr, *xc32 = nullptr;
  double *r = nullptr, *z = nullptr, *zold = nullptr, *d = nullptr, *q = nullptr, *v1 = nullptr, *v3 = nullptr;
  float *f1 = nullptr, *f3 = nullptr;
  double *partial = nullptr, *dots = nullptr, *sc = nullptr;
  int64_t launches = 0;
  int rec_its = -1, rec_misses = 0;  // the last solve's first recursive convergence, failed true checks
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
  template <typename T> T *G() const;
  template <typename T> T *E() const;
  template <typename T> const T *tab() const;
  template <typename T> T *cb() const;
  template <typename T> const StarFdmDev<T> &sf() const;
  template <typename T> T *X() const;
  template <typename T> const T *wq() const;
  template <typename T> const T *Ainv() const;
  template <typename T> T *rc() const;
  template <typename T> T *xc() const;
  ~fdm_elast() {
    for (fdm_ctx *c : comp) fdm_destroy(c);
    for (void *ptr : allocs) cudaFree(ptr);
  }
};
template <> const double *fdm_elast::tab<double>() const { return tab64; }
template <> const float *fdm_elast::tab<float>() const { return tab32; }
template <> double *fdm_elast::cb<double>() const { return cb64; }
template <> float *fdm_elast::cb<float>() const { return cb32; }
template <> const StarFdmDev<double> &fdm_elast::sf<double>() const { return sf64; }
template <> const StarFdmDev<float> &fdm_elast::sf<float>() const { return sf32; }
template <> double *fdm_elast::X<double>() const { return X64; }
template <> float *fdm_elast::X<float>() const { return X32; }
template <> double *fdm_elast::G<double>() const { return G64; }
template <> float *fdm_elast::G<float>() const { return G32; }
template <> double *fdm_elast::E<double>() const { return E64; }
template <> float *fdm_elast::E<float>() const { return E32; }
template <> const double *fdm_elast::wq<double>() const { return wq64; }
template <> const float *fdm_elast::wq<float>() const { return wq32; }
template <> const double *fdm_elast::Ainv<double>() const { return Ainv64; }
template <> const float *fdm_elast::Ainv<float>() const { return Ainv32; }
template <> double *fdm_elast::rc<double>() const { return rc64; }
template <> float *fdm_elast::rc<float>() const { return rc32; }
template <> double *fdm_elast::xc<double>() const { return xc64; }
template <> float *fdm_elast::xc<float>() const { return xc32; }

namespace {

int handle_elast(fdm_elast *e, const Error &err) {
  if (e) e->err = err.msg;
  ctx_last_error() = err.msg;
  return err.code;
}

void mask3(const fdm_elast *e, double *v, cudaStream_t st) {
  for (int a = 0; a < 3; ++a) ctx_mask_dirichlet(e->g, v + a * e->n, st);
}

// y = A u (rsub == nullptr) or y = rsub - A u, in precision T
template <typename T, typename Tin>
void elast_op(fdm_elast *e, const Tin *u, T *y, const double *rsub, cudaStream_t st) {
  launch_elast_cells<T, Tin>(e->g, u, e->tab<T>(), e->wq<T>(), e->Lc, e->mu, e->lam, e->G<T>(), e->E<T>(), st);
  const int64_t cn = (int64_t)e->g.ncell * e->g.n * e->g.n * e->g.n;
  for (int a = 0; a < 3; ++a)
    launch_gather_cells<T, T>(e->g, e->E<T>() + a * cn, rsub ? rsub + a * e->n : nullptr, y + a * e->n, st);
  e->launches += 5;
}

// z = omega S(r): the three scalar relaxations (precision T inside)
template <typename T, typename Tin, typename Tout>
void elast_sdc(fdm_elast *e, const Tin *r, Tout *z, double omega, cudaStream_t st, const T *addv = nullptr) {
  if (e->star) {
    launch_star_fdm_solve<T, Tin>(e->sf<T>(), r, e->X<T>(), 3, st);
    launch_star_fdm_gather<T, Tout>(e->sf<T>(), e->X<T>(), omega, addv, z, 3, st);
    e->launches += 2;
    return;
  }
  for (int a = 0; a < 3; ++a) {
    fdm_ctx *c = e->comp[a];
    c->launches = 0;
    ctx_run_asm<T, Tin, Tout>(c, r + a * e->n, z + a * e->n, omega, st, addv ? addv + a * e->n : nullptr);
    e->launches += c->launches;
  }
}

template <typename T>
void elast_coarse(fdm_elast *e, const T *r1, T *x1, cudaStream_t st) {
  for (int a = 0; a < 3; ++a)
    launch_coarse_restrict<T, T>(e->g, r1 + a * e->n, e->tab<T>(), e->cfree, e->rc<T>() + a * e->nq, e->cb<T>(), st);
  launch_dense_symv<T>(e->m, e->Ainv<T>(), e->rc<T>(), e->xc<T>(), st);
  for (int a = 0; a < 3; ++a)
    launch_coarse_prolong<T, T>(e->g, e->xc<T>() + a * e->nq, e->tab<T>(), e->cfree, x1 + a * e->n, true, st);
  e->launches += 10;
}

// the hybrid V(1,1) with the SDC relaxation, FP64 r to FP64 z, computed in T
template <typename T>
void elast_vcycle(fdm_elast *e, const double *r, double *z, T *x1, T *r1, cudaStream_t st) {
  elast_sdc<T, double, T>(e, r, x1, e->omega, st);
  elast_op<T, T>(e, x1, r1, r, st);
  if (e->m > 0) elast_coarse<T>(e, r1, x1, st);
  elast_op<T, T>(e, x1, r1, r, st);
  elast_sdc<T, T, double>(e, r1, z, e->omega, st, x1);
}

void elast_pc(fdm_elast *e, const double *r, double *z, cudaStream_t st) {
  const bool fp64 = e->opt.precision == FDM_PREC_FP64;
  if (e->opt.pc == FDM_PC_NONE) {
    ctx_copy(3 * e->n, r, z, st);
    mask3(e, z, st);
    e->launches += 4;
  } else if (e->opt.pc == FDM_PC_ASM) {
    if (fp64) elast_sdc<double, double, double>(e, r, z, e->omega, st);
    else elast_sdc<float, double, double>(e, r, z, e->omega, st);
  } else {
    if (fp64) elast_vcycle<double>(e, r, z, e->v1, e->v3, st);
    else elast_vcycle<float>(e, r, z, e->f1, e->f3, st);
  }
}

__global__ void k_permute_sym(int m, int nq, const double *__restrict__ in, double *__restrict__ out) {
  // out is component-major (a nq + v), in interleaved (3 v + a)
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)m * m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / m), j = (int)(t % m);
    const int pi = 3 * (i % nq) + i / nq, pj = 3 * (j % nq) + j / nq;
    out[t] = in[(int64_t)pi * m + pj];
  }
}

// vector Q1 coarse problem: cell stiffness of Q1 elasticity by 2-point Gauss
// (exact on box cells), banded Cholesky in vertex-interleaved order, dense
// inverse on the device, permuted to component-major order
void elast_setup_coarse(fdm_elast *e, const std::vector<double> *vert, cudaStream_t st) {
  const int nx = e->g.nx, ny = e->g.ny, nz = e->g.nz, nvx = nx + 1, nvy = ny + 1, nv = nvx * nvy * (nz + 1);
  // the coarse unknowns: the vertices off the clamped faces, in vertex order
  std::vector<int> cfree(nv, -1);
  int nq = 0;
  for (int v = 0; v < nv; ++v) {
    const int vx = v % nvx, vy = (v / nvx) % nvy, vz = v / (nvx * nvy);
    if (!node_dirichlet(e->g, vx * e->g.p, vy * e->g.p, vz * e->g.p)) cfree[v] = nq++;
  }
  e->cfree = e->upload(cfree);
  e->cb64 = e->alloc<double>((size_t)8 * e->g.ncell);
  e->cb32 = e->alloc<float>((size_t)8 * e->g.ncell);
  e->nq = nq;
  e->m = 3 * e->nq;
  e->rc64 = e->alloc<double>(e->m);
  e->xc64 = e->alloc<double>(e->m);
  e->rc32 = e->alloc<float>(e->m);
  e->xc32 = e->alloc<float>(e->m);
  if (e->m == 0) return;
  // half-bandwidth of the vertex-interleaved numbering: the widest index span of a cell
  int span = 0;
  for (int c = 0; c < e->g.ncell; ++c) {
    const int cx = c % nx, cy = (c / nx) % ny, cz = c / (nx * ny);
    int lo = nq, hi = -1;
    for (int s = 0; s < 8; ++s) {
      const int f = cfree[(cx + (s & 1)) + nvx * ((cy + ((s >> 1) & 1)) + nvy * (cz + (s >> 2)))];
      if (f >= 0) lo = std::min(lo, f), hi = std::max(hi, f);
    }
    if (hi >= 0) span = std::max(span, hi - lo);
  }
  const int m = e->m, bw = 3 * span + 2;
  std::vector<double> Lb((size_t)m * (bw + 1), 0.0);
  const double gp = 1.0 / std::sqrt(3.0);
  for (int cz = 0; cz < nz; ++cz)
    for (int cy = 0; cy < ny; ++cy)
      for (int cx = 0; cx < nx; ++cx) {
        const double L[3] = {0.5 * (vert[0][cx + 1] - vert[0][cx]), 0.5 * (vert[1][cy + 1] - vert[1][cy]),
                             0.5 * (vert[2][cz + 1] - vert[2][cz])};
        const double vol = L[0] * L[1] * L[2];
        int f[8];
        for (int s = 0; s < 8; ++s)
          f[s] = cfree[(cx + (s & 1)) + nvx * ((cy + ((s >> 1) & 1)) + nvy * (cz + (s >> 2)))];
        double K[24][24] = {};
        for (int qp = 0; qp < 8; ++qp) {
          const double xi[3] = {(qp & 1) ? gp : -gp, ((qp >> 1) & 1) ? gp : -gp, (qp >> 2) ? gp : -gp};
          double dphi[8][3];
          for (int s = 0; s < 8; ++s) {
            const double sg[3] = {(s & 1) ? 1.0 : -1.0, ((s >> 1) & 1) ? 1.0 : -1.0, (s >> 2) ? 1.0 : -1.0};
            const double h[3] = {0.5 * (1 + sg[0] * xi[0]), 0.5 * (1 + sg[1] * xi[1]), 0.5 * (1 + sg[2] * xi[2])};
            dphi[s][0] = 0.5 * sg[0] * h[1] * h[2] / L[0];
            dphi[s][1] = 0.5 * sg[1] * h[0] * h[2] / L[1];
            dphi[s][2] = 0.5 * sg[2] * h[0] * h[1] / L[2];
          }
          for (int s = 0; s < 8; ++s)
            for (int a = 0; a < 3; ++a)
              for (int t = 0; t < 8; ++t)
                for (int b = 0; b < 3; ++b) {
                  double v = e->mu * dphi[s][b] * dphi[t][a] + e->lam * dphi[s][a] * dphi[t][b];
                  if (a == b) v += e->mu * (dphi[s][0] * dphi[t][0] + dphi[s][1] * dphi[t][1] + dphi[s][2] * dphi[t][2]);
                  K[3 * s + a][3 * t + b] += vol * v;
                }
        }
        for (int s = 0; s < 8; ++s)
          for (int t = 0; t < 8; ++t) {
            if (f[s] < 0 || f[t] < 0) continue;
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) {
                const int i = 3 * f[s] + a, j = 3 * f[t] + b;
                if (j <= i) Lb[(size_t)i * (bw + 1) + (i - j)] += K[3 * s + a][3 * t + b];
              }
          }
      }
  ctx_banded_cholesky(m, bw, Lb);
  double *dLb = e->upload(Lb);
  double *inv_il = e->alloc<double>((size_t)m * m);
  e->Ainv64 = e->alloc<double>((size_t)m * m);
  e->Ainv32 = e->alloc<float>((size_t)m * m);
  launch_banded_inverse(m, bw, dLb, inv_il, st);
  k_permute_sym<<<ctx_vec_blocks((int64_t)m * m), 256, 0, st>>>(m, e->nq, inv_il, e->Ainv64);
  launch_convert<double, float>((int64_t)m * m, e->Ainv64, e->Ainv32, st);
  FDM_CUDA(cudaStreamSynchronize(st));
  FDM_CUDA(cudaGetLastError());
}

// The star-local FDM of the SDC blocks: per axis a and vertex coordinate v the
// 1D star (the free nodes within p - 1 of the vertex: strictly between the
// neighbouring vertices, with the boundary node at a traction-free end and
// without it at a clamped one), its stiffness and mass assembled from
// A_e = A_hat / L_e and M_e = L_e B_hat over its cells and their generalised
// eigenpairs; per vertex (the vertices on clamped faces included, as in the
// FDM/sparse relaxation) a star with its block of the star-solution buffer.
void setup_star_fdm(fdm_elast *e, const Basis1D &b, const std::vector<double> *vert) {
  const Grid &g = e->g;
  const int p = g.p, n = g.n;
  const int ncell[3] = {g.nx, g.ny, g.nz};
  std::vector<double> tab;
  std::vector<int> lo[3], len[3], soff[3];
  int maxlen = 0;
  for (int a = 0; a < 3; ++a) {
    const int na = ncell[a];
    const bool nat_lo = !(g.dmask & (1 << (2 * a))), nat_hi = !(g.dmask & (1 << (2 * a + 1)));
    lo[a].assign(na + 1, 0);
    len[a].assign(na + 1, 0);
    soff[a].assign(na + 1, 0);
    for (int v = 0; v <= na; ++v) {
      // the free nodes within p - 1 of the vertex
      const int l0 = v == 0 ? (nat_lo ? 0 : 1) : (v - 1) * p + 1;
      const int l1 = v == na ? (nat_hi ? na * p : na * p - 1) : (v + 1) * p - 1;
      const int m = l1 - l0 + 1;
      if (m <= 0) continue;  // p = 1 at a clamped end
      std::vector<double> A((size_t)m * m, 0.0), M((size_t)m * m, 0.0), S((size_t)m * m), lam(m);
      for (int c = v - 1; c <= v; ++c) {
        if (c < 0 || c >= na) continue;
        const double L = 0.5 * (vert[a][c + 1] - vert[a][c]);
        for (int i = 0; i < n; ++i)
          for (int k = 0; k < n; ++k) {
            const int gi = c * p + i - l0, gk = c * p + k - l0;
            if (gi < 0 || gi >= m || gk < 0 || gk >= m) continue;
            A[(size_t)gi * m + gk] += b.A[i * n + k] / L;
            M[(size_t)gi * m + gk] += L * b.B[i * n + k];
          }
      }
      sym_gen_eig(m, A.data(), M.data(), S.data(), lam.data());
      lo[a][v] = l0;
      len[a][v] = m;
      soff[a][v] = (int)tab.size();
      tab.insert(tab.end(), S.begin(), S.end());
      tab.insert(tab.end(), lam.begin(), lam.end());
      maxlen = std::max(maxlen, m);
    }
  }
  const int nvx = g.nx + 1, nvy = g.ny + 1, nv = nvx * nvy * (g.nz + 1);
  std::vector<int> vstar(nv, -1), svert;
  std::vector<int64_t> off;
  int64_t tot = 0;
  for (int v = 0; v < nv; ++v) {
    const int vc[3] = {v % nvx, (v / nvx) % nvy, v / (nvx * nvy)};
    const int64_t sz = (int64_t)len[0][vc[0]] * len[1][vc[1]] * len[2][vc[2]];
    if (sz == 0) continue;
    vstar[v] = (int)svert.size();
    svert.push_back(v);
    off.push_back(tot);
    tot += sz;
  }
  StarFdmDev<double> d;
  d.g = g;
  for (int a = 0; a < 3; ++a) {
    d.ax[a].lo = e->upload(lo[a]);
    d.ax[a].len = e->upload(len[a]);
    d.ax[a].soff = e->upload(soff[a]);
  }
  d.vstar = e->upload(vstar);
  d.svert = e->upload(svert);
  d.off = e->upload(off);
  d.xstride = tot;
  d.nstar = (int)svert.size();
  d.maxlen = maxlen;
  for (int j = 0; j < 3; ++j)
    for (int a = 0; a < 3; ++a) d.c[j][a] = e->mu + (a == j ? e->mu + e->lam : 0.0);
  if (star_fdm_smem(maxlen, sizeof(double)) > 227 * 1024)
    fail(FDM_EINVAL, "fdm_elast_setup: star larger than the shared memory of one CTA");
  e->sf64 = d;
  e->sf64.tab = e->upload(tab);
  e->X64 = e->alloc<double>((size_t)3 * tot);
  e->sf32.g = d.g;
  for (int a = 0; a < 3; ++a) e->sf32.ax[a] = d.ax[a];
  e->sf32.vstar = d.vstar;
  e->sf32.svert = d.svert;
  e->sf32.off = d.off;
  e->sf32.xstride = d.xstride;
  e->sf32.nstar = d.nstar;
  e->sf32.maxlen = d.maxlen;
  std::memcpy(e->sf32.c, d.c, sizeof d.c);
  e->sf32.tab = e->upload(std::vector<float>(tab.begin(), tab.end()));
  if (e->opt.precision == FDM_PREC_FP32) e->X32 = e->alloc<float>((size_t)3 * tot);
}

// omega from k CG-Lanczos steps on A_SDC^{-1} A (undamped SDC relaxation), FP64
void elast_lanczos(fdm_elast *e, const double *start_host, cudaStream_t st) {
  const int64_t n3 = 3 * e->n;
  std::vector<double> b0;
  if (start_host) b0.assign(start_host, start_host + n3);
  else ctx_normal_vector(e->opt.lanczos_seed, n3, b0);
  FDM_CUDA(cudaMemcpyAsync(e->r, b0.data(), n3 * sizeof(double), cudaMemcpyHostToDevice, st));
  mask3(e, e->r, st);
  elast_sdc<double, double, double>(e, e->r, e->z, 1.0, st);
  FDM_CUDA(cudaMemcpyAsync(e->d, e->z, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double h[2];
  launch_dot(n3, e->r, e->z, e->partial, e->dots, st);
  FDM_CUDA(cudaMemcpyAsync(h, e->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
  FDM_CUDA(cudaStreamSynchronize(st));
  double rz = h[0];
  std::vector<double> al, be;
  for (int k = 0; k < e->opt.lanczos_steps; ++k) {
    if (!(rz > 0.0)) break;
    elast_op<double, double>(e, e->d, e->q, nullptr, st);
    launch_dot(n3, e->d, e->q, e->partial, e->dots, st);
    FDM_CUDA(cudaMemcpyAsync(h, e->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    if (!(h[0] > 0.0)) break;
    const double alpha = rz / h[0];
    al.push_back(alpha);
    launch_axpby<double>(n3, -alpha, e->q, 1.0, e->r, e->r, st);
    elast_sdc<double, double, double>(e, e->r, e->z, 1.0, st);
    launch_dot(n3, e->r, e->z, e->partial, e->dots, st);
    FDM_CUDA(cudaMemcpyAsync(h, e->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    const double beta = h[0] / rz;
    be.push_back(beta);
    rz = h[0];
    launch_axpby<double>(n3, 1.0, e->z, beta, e->d, e->d, st);
  }
  const int m = (int)al.size();
  if (m < 1) fail(FDM_EINVAL, "Lanczos: no steps could be taken");
  std::vector<double> dd(m), ee(std::max(m - 1, 1), 0.0);
  for (int j = 0; j < m; ++j) {
    dd[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < m) ee[j] = std::sqrt(be[j]) / al[j];
  }
  ctx_tridiag_extremes(dd, ee, e->lmin, e->lmax);
  e->omega = 2.0 / (1.25 * e->lmax + 0.75 * e->lmin);
}

}  // namespace


// ====================================================================== C-ABI
extern "C" {

// ---------------------------------------------------------------- linear elasticity (Section 4.1)
int fdm_elast_setup(const fdm_mesh *mesh, int p, double mu, double lam, const fdm_options *opt, fdm_elast **out,
                    void *stream) {
  return fdm_elast_setup_bc(mesh, p, mu, lam, 63, FDM_SDC_AUTO, opt, out, stream);
}

int fdm_elast_setup_bc(const fdm_mesh *mesh, int p, double mu, double lam, int dirichlet_faces, int sdc_form,
                       const fdm_options *opt, fdm_elast **out, void *stream) {
  if (!out) return FDM_EINVAL;
  *out = nullptr;
  if (!mesh || !mesh->xv || !mesh->yv || !mesh->zv || mesh->nx < 1 || mesh->ny < 1 || mesh->nz < 1 || p < 1 ||
      p > 15 || !(mu > 0.0) || !(lam >= 0.0) || !std::isfinite(mu) || !std::isfinite(lam)) {
    ctx_last_error() = "fdm_elast_setup: invalid mesh, degree (1..15) or Lame parameters (mu > 0, lambda >= 0)";
    return FDM_EINVAL;
  }
  if (dirichlet_faces < 1 || dirichlet_faces > 63 || sdc_form < FDM_SDC_AUTO || sdc_form > FDM_SDC_STAR_FDM ||
      (sdc_form == FDM_SDC_FDM_SPARSE && dirichlet_faces != 63)) {
    ctx_last_error() = "fdm_elast_setup: dirichlet_faces must be 1..63 (some face clamped) and the FDM/sparse form "
                       "needs every face clamped";
    return FDM_EINVAL;
  }
  if (mesh->jac) {
    ctx_last_error() = "fdm_elast_setup: box cells only (mesh->jac must be NULL)";
    return FDM_EINVAL;
  }
  fdm_elast *e = new fdm_elast();
  try {
    cudaStream_t st = (cudaStream_t)stream;
    if (opt) e->opt = *opt;
    else fdm_default_options(&e->opt);
    if (e->opt.lanczos_steps <= 0) e->opt.lanczos_steps = 20;
    if (e->opt.flexible_beta < 0) e->opt.flexible_beta = e->opt.precision == FDM_PREC_FP32 ? 1 : 0;
    e->mu = mu;
    e->lam = lam;
    e->star = sdc_form == FDM_SDC_STAR_FDM || (sdc_form == FDM_SDC_AUTO && dirichlet_faces != 63);
    const int nx = mesh->nx, ny = mesh->ny, nz = mesh->nz, ncell = nx * ny * nz;
    std::vector<double> vert[3] = {std::vector<double>(mesh->xv, mesh->xv + nx + 1),
                                   std::vector<double>(mesh->yv, mesh->yv + ny + 1),
                                   std::vector<double>(mesh->zv, mesh->zv + nz + 1)};
    for (int a = 0; a < 3; ++a)
      for (size_t v = 0; v + 1 < vert[a].size(); ++v)
        if (!(vert[a][v + 1] > vert[a][v])) fail(FDM_EINVAL, "fdm_elast_setup: vertex coordinates must increase");
    Grid &g = e->g;
    g.p = p;
    g.n = p + 1;
    g.nx = nx; g.ny = ny; g.nz = nz;
    g.N[0] = nx * p + 1; g.N[1] = ny * p + 1; g.N[2] = nz * p + 1;
    g.ndof = (int64_t)g.N[0] * g.N[1] * g.N[2];
    g.ncell = ncell;
    g.dmask = dirichlet_faces;
    e->n = g.ndof;
    const Basis1D basis = make_basis(p);
    std::vector<double> L(3 * (size_t)ncell);
    for (int cz = 0; cz < nz; ++cz)
      for (int cy = 0; cy < ny; ++cy)
        for (int cx = 0; cx < nx; ++cx) {
          const int c = cx + nx * (cy + ny * cz);
          L[3 * c] = 0.5 * (mesh->xv[cx + 1] - mesh->xv[cx]);
          L[3 * c + 1] = 0.5 * (mesh->yv[cy + 1] - mesh->yv[cy]);
          L[3 * c + 2] = 0.5 * (mesh->zv[cz + 1] - mesh->zv[cz]);
        }
    // the scalar contexts of the SDC blocks: exact separable coefficients
    fdm_options copt = e->opt;
    copt.pc = FDM_PC_ASM;
    copt.omega = 1.0;
    copt.lanczos_start = nullptr;
    copt.pcg_graph = 0;
    copt.kernel_timing = 0;
    for (int a = 0; a < 3 && !e->star; ++a) {
      std::vector<double> mua(3 * (size_t)ncell);
      for (int c = 0; c < ncell; ++c) {
        const double vol = L[3 * c] * L[3 * c + 1] * L[3 * c + 2];
        for (int d = 0; d < 3; ++d)
          mua[3 * c + d] = (mu + (d == a ? mu + lam : 0.0)) * vol / (L[3 * c + d] * L[3 * c + d]);
      }
      fdm_coeff cf{nullptr, nullptr, mua.data()};
      const int rc = fdm_setup(mesh, p, &cf, &copt, &e->comp[a], stream);
      if (rc != FDM_OK) fail(rc, "SDC block " + std::to_string(a) + ": " + ctx_last_error());
    }
    if (e->star) setup_star_fdm(e, basis, vert);
    // the 1D tables (layout of tab_off) and the Gauss weights of the operator
    std::vector<double> t(tab_size(g.n), 0.0);
    auto put = [&](int which, const std::vector<double> &M) {
      std::copy(M.begin(), M.end(), t.begin() + tab_off(which, g.n));
    };
    put(TAB_A, basis.A);
    put(TAB_B, basis.B);
    put(TAB_AF, basis.Af);
    put(TAB_BF, basis.Bf);
    put(TAB_T, basis.T);
    put(TAB_VQ, basis.Vq);
    put(TAB_DQ, basis.Dq);
    std::copy(basis.xi.begin(), basis.xi.end(), t.begin() + tab_off(TAB_XI, g.n));
    put(TAB_VE, basis.Ve);
    std::copy(basis.lame.begin(), basis.lame.end(), t.begin() + tab_off(TAB_LE, g.n));
    e->tab64 = e->upload(t);
    e->tab32 = e->upload(std::vector<float>(t.begin(), t.end()));
    e->Lc = e->upload(L);
    e->wq64 = e->upload(basis.wq);
    e->wq32 = e->upload(std::vector<float>(basis.wq.begin(), basis.wq.end()));
    const size_t cn = (size_t)ncell * e->g.n * e->g.n * e->g.n;
    e->G64 = e->alloc<double>(9 * cn);
    e->E64 = e->alloc<double>(3 * cn);
    if (e->opt.precision == FDM_PREC_FP32) {
      e->G32 = e->alloc<float>(9 * cn);
      e->E32 = e->alloc<float>(3 * cn);
      e->f1 = e->alloc<float>(3 * e->n);
      e->f3 = e->alloc<float>(3 * e->n);
    }
    for (double **v : {&e->r, &e->z, &e->zold, &e->d, &e->q, &e->v1, &e->v3}) *v = e->alloc<double>(3 * e->n);
    e->partial = e->alloc<double>(2 * DOT_BLOCKS);
    e->dots = e->alloc<double>(4);
    e->sc = e->alloc<double>(16);
    elast_setup_coarse(e, vert, st);
    if (e->opt.omega > 0.0) e->omega = e->opt.omega;
    else elast_lanczos(e, e->opt.lanczos_start, st);
    FDM_CUDA(cudaStreamSynchronize(st));
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &err) {
    ctx_last_error() = err.msg;
    delete e;
    return err.code;
  }
  *out = e;
  return FDM_OK;
}

int elast_apply(fdm_elast *e, const double *u, double *y, void *stream) {
  if (!e || !u || !y) return FDM_EINVAL;
  try {
    elast_op<double, double>(e, u, y, nullptr, (cudaStream_t)stream);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &err) { return handle_elast(e, err); }
  return FDM_OK;
}

int elast_pc_apply(fdm_elast *e, const double *r, double *z, void *stream) {
  if (!e || !r || !z) return FDM_EINVAL;
  try {
    elast_pc(e, r, z, (cudaStream_t)stream);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &err) { return handle_elast(e, err); }
  return FDM_OK;
}

int elast_pcg_solve(fdm_elast *e, const double *b, double *x, double rtol, int maxit, fdm_solve_info *info,
                    void *stream) {
  if (!e || !b || !x || maxit < 0 || !(rtol >= 0.0)) return FDM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n3 = 3 * e->n;
  try {
    cudaEvent_t e0, e1;
    FDM_CUDA(cudaEventCreate(&e0));
    FDM_CUDA(cudaEventCreate(&e1));
    FDM_CUDA(cudaEventRecord(e0, st));
    double hsc[16] = {0};
    hsc[7] = e->opt.flexible_beta ? 1.0 : 0.0;
    FDM_CUDA(cudaMemcpyAsync(e->sc, hsc, sizeof hsc, cudaMemcpyHostToDevice, st));
    FDM_CUDA(cudaMemsetAsync(x, 0, n3 * sizeof(double), st));
    FDM_CUDA(cudaMemcpyAsync(e->r, b, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    mask3(e, e->r, st);
    double h[2];
    launch_dot(n3, e->r, e->r, e->partial, e->dots, st);
    e->launches += 5;
    FDM_CUDA(cudaMemcpyAsync(h, e->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    const double nb = std::sqrt(h[0]);
    double nr = nb;
    int it = 0, conv = nb == 0.0, bad = 0;
    e->rec_its = conv ? 0 : -1;
    e->rec_misses = 0;
    double *z = e->z, *zold = e->zold;
    if (!conv) {
      elast_pc(e, e->r, z, st);
      launch_dot(n3, e->r, z, e->partial, e->dots, st);
      launch_pcg_scalars(2, e->sc, e->dots, st);
      FDM_CUDA(cudaMemcpyAsync(e->d, z, n3 * sizeof(double), cudaMemcpyDeviceToDevice, st));
      e->launches += 3;
      while (it < maxit) {
        elast_op<double, double>(e, e->d, e->q, nullptr, st);
        launch_dot(n3, e->d, e->q, e->partial, e->dots, st);
        launch_pcg_scalars(0, e->sc, e->dots, st);
        launch_pcg_update_xr(n3, e->sc, e->d, e->q, x, e->r, st);
        ++it;
        launch_dot(n3, e->r, e->r, e->partial, e->dots + 2, st);
        e->launches += 6;
        FDM_CUDA(cudaMemcpyAsync(h, e->dots + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
        FDM_CUDA(cudaStreamSynchronize(st));
        nr = std::sqrt(h[0]);
        if (!std::isfinite(nr)) { bad = 1; break; }
        if (nr <= rtol * nb) {
          // converged on the recursive residual: replace it by the true one,
          // r = b - A x, and stop only if that meets the test too
          if (e->rec_its < 0) e->rec_its = it;
          elast_op<double, double>(e, x, e->r, b, st);
          mask3(e, e->r, st);
          launch_dot(n3, e->r, e->r, e->partial, e->dots + 2, st);
          e->launches += 4;
          FDM_CUDA(cudaMemcpyAsync(h, e->dots + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
          FDM_CUDA(cudaStreamSynchronize(st));
          nr = std::sqrt(h[0]);
          if (!std::isfinite(nr)) { bad = 1; break; }
          if (nr <= rtol * nb) { conv = 1; break; }
          ++e->rec_misses;
          if (it >= maxit) break;
        }
        std::swap(z, zold);
        elast_pc(e, e->r, z, st);
        launch_dot2(n3, e->r, z, zold, e->partial, e->dots, st);
        launch_pcg_scalars(1, e->sc, e->dots, st);
        launch_pcg_update_d(n3, e->sc, z, e->d, st);
        e->launches += 4;
      }
    }
    FDM_CUDA(cudaEventRecord(e1, st));
    FDM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    FDM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    FDM_CUDA(cudaMemcpy(hsc, e->sc, sizeof hsc, cudaMemcpyDeviceToHost));
    if (hsc[8] != 0.0) bad = 1;
    for (fdm_ctx *c : e->comp) {
      if (!c) continue;
      int hstat = 0;
      FDM_CUDA(cudaMemcpy(&hstat, c->status, sizeof(int), cudaMemcpyDeviceToHost));
      if (hstat) {
        FDM_CUDA(cudaMemset(c->status, 0, sizeof(int)));
        fail(FDM_ETIMEOUT, "a bounded device-side wait of the patch solve ran out");
      }
    }
    if (info) {
      info->iterations = it;
      info->converged = conv;
      info->rnorm0 = nb;
      info->rnorm = nr;
      info->seconds = ms * 1e-3;
      elast_op<double, double>(e, x, e->v1, b, st);  // b - A x
      mask3(e, e->v1, st);
      launch_dot(n3, e->v1, e->v1, e->partial, e->dots, st);
      e->launches += 4;
      FDM_CUDA(cudaMemcpyAsync(h, e->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
      FDM_CUDA(cudaStreamSynchronize(st));
      info->true_rnorm = std::sqrt(h[0]);
    }
    FDM_CUDA(cudaGetLastError());
    if (bad) { e->err = "non-finite scalar in PCG"; return FDM_ENAN; }
    if (!conv) { e->err = "PCG reached maxit"; return FDM_ENOCONV; }
  } catch (const Error &err) { return handle_elast(e, err); }
  return FDM_OK;
}

int fdm_elast_query(fdm_elast *e, int what, void *out, size_t *len) {
  if (!e || !out || !len) return FDM_EINVAL;
  try {
    auto put = [&](const void *src, size_t bytes) {
      if (*len < bytes) fail(FDM_EINVAL, "fdm_elast_query: buffer too small (" + std::to_string(bytes) + " bytes needed)");
      std::memcpy(out, src, bytes);
      *len = bytes;
    };
    switch (what) {
      case FDM_Q_NDOF: { int64_t v = e->n; put(&v, sizeof v); break; }
      case FDM_Q_OMEGA: put(&e->omega, sizeof(double)); break;
      case FDM_Q_LAMBDA: { double v[2] = {e->lmin, e->lmax}; put(v, sizeof v); break; }
      case FDM_Q_LAUNCHES: { int64_t v = e->launches; e->launches = 0; put(&v, sizeof v); break; }
      case FDM_Q_RECURSIVE_ITS: { int32_t v[2] = {e->rec_its, e->rec_misses}; put(v, sizeof v); break; }
      default: fail(FDM_EINVAL, "fdm_elast_query: unknown quantity");
    }
  } catch (const Error &err) { return handle_elast(e, err); }
  return FDM_OK;
}

const char *fdm_elast_last_error(const fdm_elast *e) { return e ? e->err.c_str() : ctx_last_error().c_str(); }

void fdm_elast_destroy(fdm_elast *e) { delete e; }

}  // extern "C"
