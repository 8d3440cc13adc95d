// GPU context for general hexahedral meshes (fdm_hex_*): the stiffness apply,
// the vertex-star relaxation, the hybrid V(1,1) with the Q1 coarse space and
// PCG on the device, from the host set-up of an fdm_hexmesh (Sections 2.4-2.8
// on the meshes of the paper's unstructured experiments, Sec. 3).
//
// Set-up (host, once): the hexmesh's cell maps, inverse maps, geometry factors
// and Schur-coupling factors are uploaded in FP64 and FP32; the sparse lower
// factor L_BB of every class gets level schedules for its forward and
// backward solves (rows grouped by their depth in the dependency graph, so a
// level's rows are solved in parallel); the Q1 Galerkin operator is inverted
// densely (host Cholesky); omega comes from CG-Lanczos on the device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "hexdev.h"
#include "hexmesh_host.h"
#include "internal.h"
#include "kernels.h"

using namespace fdm;

struct fdm_hexgpu {
  fdm_options opt{};
  int p = 0, n = 0, nc = 0, nv = 0, nstar = 0, nco = 0, maxG = 0;
  int *bin_list = nullptr;  // dense form: star indices by interface-size bin, largest first in each
  int bin_count[3] = {0, 0, 0}, bin_maxg[3] = {0, 0, 0};
  // the largest bin runs on a second stream beside the others (it has too few
  // stars to fill the GPU alone); fork and join events
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  int64_t nnode = 0, nxtot = 0, nval = 0;
  bool dense = true;  // interface solves with the dense S_G^{-1} (else the Schur-coupling form)
  std::vector<void *> allocs;
  size_t alloc_bytes = 0;
  HexDev<double> d64;
  HexDev<float> d32;
  double *E64 = nullptr, *rc64 = nullptr, *X64 = nullptr, *zf64 = nullptr, *Y64 = nullptr;
  float *E32 = nullptr, *rc32 = nullptr, *X32 = nullptr, *zf32 = nullptr, *Y32 = nullptr;
  double *x1_64 = nullptr, *t64 = nullptr, *w64 = nullptr, *cr64 = nullptr, *cx64 = nullptr;
  float *r32 = nullptr, *x1_32 = nullptr, *t32 = nullptr, *w32 = nullptr, *cr32 = nullptr, *cx32 = nullptr;
  double *r = nullptr, *z = nullptr, *zold = nullptr, *d = nullptr, *q = nullptr, *v1 = nullptr;
  double *partial = nullptr, *dots = nullptr, *sc = nullptr;
  double omega = 0.0, lmin = 0.0, lmax = 0.0;
  int64_t launches = 0;
  std::string err;

  template <typename T>
  T *alloc(size_t n) {
    void *ptr = device_alloc(std::max<size_t>(n, 1) * sizeof(T), alloc_bytes);
    allocs.push_back(ptr);
    return static_cast<T *>(ptr);
  }
  template <typename T>
  T *upload(const std::vector<T> &v) {
    T *p = alloc<T>(v.size());
    if (!v.empty()) FDM_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return p;
  }
  template <typename T>
  const HexDev<T> &dev() const;
  template <typename T>
  T *E() { return pick<T>(E64, E32); }
  template <typename T>
  T *rc() { return pick<T>(rc64, rc32); }
  template <typename T>
  T *X() { return pick<T>(X64, X32); }
  template <typename T>
  T *zf() { return pick<T>(zf64, zf32); }
  template <typename T>
  T *Y() { return pick<T>(Y64, Y32); }
  template <typename T>
  static T *pick(double *a, float *b) {
    if constexpr (sizeof(T) == 8) return reinterpret_cast<T *>(a);
    else return reinterpret_cast<T *>(b);
  }
  ~fdm_hexgpu() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (aux) cudaStreamDestroy(aux);
    for (void *p : allocs) cudaFree(p);
  }
};
template <>
const HexDev<double> &fdm_hexgpu::dev<double>() const { return d64; }
template <>
const HexDev<float> &fdm_hexgpu::dev<float>() const { return d32; }

namespace {

thread_local std::string g_hex_err;

int handle_hexgpu(fdm_hexgpu *c, const Error &e) {
  if (c) c->err = e.msg;
  g_hex_err = e.msg;
  cudaGetLastError();
  return e.code;
}

template <typename T>
std::vector<T> conv(const std::vector<double> &v) {
  return std::vector<T>(v.begin(), v.end());
}

// dense inverse of the SPD matrix A (m x m, row-major) by Cholesky
std::vector<double> spd_inverse(const std::vector<double> &A, int m) {
  std::vector<double> L(A);
  for (int j = 0; j < m; ++j) {
    double s = L[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) s -= L[(size_t)j * m + k] * L[(size_t)j * m + k];
    if (!(s > 0.0)) fail(FDM_ENOTSPD, "fdm_hex_setup: the Q1 coarse operator is not positive definite");
    const double djj = std::sqrt(s);
    L[(size_t)j * m + j] = djj;
    for (int i = j + 1; i < m; ++i) {
      double t = L[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) t -= L[(size_t)i * m + k] * L[(size_t)j * m + k];
      L[(size_t)i * m + j] = t / djj;
    }
  }
  // columns of A^{-1} = L^{-T} L^{-1} e_c, independent: on host threads
  std::vector<double> inv((size_t)m * m);
  std::atomic<int> next{0};
  auto work = [&]() {
    std::vector<double> y(m);
    for (int c = next++; c < m; c = next++) {
      for (int i = 0; i < m; ++i) {
        double s = i == c ? 1.0 : 0.0;
        for (int k = 0; k < i; ++k) s -= L[(size_t)i * m + k] * y[k];
        y[i] = s / L[(size_t)i * m + i];
      }
      for (int i = m - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < m; ++k) s -= L[(size_t)k * m + i] * y[k];
        y[i] = s / L[(size_t)i * m + i];
      }
      for (int i = 0; i < m; ++i) inv[(size_t)i * m + c] = y[i];
    }
  };
  const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), 64));
  std::vector<std::thread> pool;
  for (int i = 1; i < nt && m > 256; ++i) pool.emplace_back(work);
  work();
  for (std::thread &t : pool) t.join();
  return inv;
}

// the lower triangle of S^{-1} = L^{-T} L^{-1} by rows (row r at zoff[r],
// padded with zeros to zoff[r + 1]) from the Cholesky factor L (m x m, dense,
// row-major): Z = L^{-1} by row updates, then S^{-1} = Z^T Z
void dense_inverse_rows(const std::vector<double> &L, int m, const std::vector<int> &zoff, double *out) {
  std::vector<double> Z((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) {
    double *zi = Z.data() + (size_t)i * m;
    zi[i] = 1.0;
    for (int k = 0; k < i; ++k) {
      const double l = L[(size_t)i * m + k];
      if (l == 0.0) continue;
      const double *zk = Z.data() + (size_t)k * m;
      for (int j = 0; j <= k; ++j) zi[j] -= l * zk[j];
    }
    const double inv = 1.0 / L[(size_t)i * m + i];
    for (int j = 0; j <= i; ++j) zi[j] *= inv;
  }
  for (int r = 0; r < m; ++r)
    for (int q = zoff[r]; q < zoff[r + 1]; ++q) out[q] = 0.0;
  for (int k = 0; k < m; ++k) {  // S^{-1}[i][j] = sum_{k >= i} Z[k][i] Z[k][j], j <= i
    const double *zk = Z.data() + (size_t)k * m;
    for (int i = 0; i <= k; ++i) {
      const double a = zk[i];
      if (a == 0.0) continue;
      double *row = out + zoff[i];
      for (int j = 0; j <= i; ++j) row[j] += a * zk[j];
    }
  }
}

// the dense interface inverses of all stars (host threads), values in star
// order at voff; per class the row offsets appended to ct
void build_dense(fdm_hexgpu *c, const fdm_hexmesh *h, std::vector<HexStarDev> &stars, std::vector<HexClassDev> &classes,
                 const std::vector<int> &cls_nG, std::vector<int> &ct, std::vector<double> &vals) {
  const int ncls = (int)classes.size();
  std::vector<std::vector<int>> zoff(ncls);
  for (int cl = 0; cl < ncls; ++cl) {
    const int m = std::max(cls_nG[cl], 0);
    zoff[cl].assign(m + 1, 0);
    for (int r = 0; r < m; ++r) zoff[cl][r + 1] = zoff[cl][r] + ((r + 1 + 3) & ~3);
    classes[cl].zoff = (int)ct.size();
    ct.insert(ct.end(), zoff[cl].begin(), zoff[cl].end());
  }
  int64_t off = 0;
  for (HexStarDev &S : stars) {
    S.voff = off;
    off += zoff[S.cls].back();
  }
  vals.assign((size_t)std::max<int64_t>(off, 1), 0.0);
  std::atomic<int> next{0};
  std::vector<std::string> errs(stars.size());
  auto work = [&]() {
    for (int k = next++; k < (int)stars.size(); k = next++) {
      const HexStarDev &S = stars[k];
      const int m = S.nG;
      if (m == 0) continue;
      const int64_t *rp = h->fill_rowptr.data() + h->fill_ptr[S.cls];
      const int32_t *cols = h->fill_cols.data() + h->fill_colptr[S.cls];
      const double *fv = h->factor.data() + h->factor_ptr[k];
      if (h->factor_ptr[k + 1] - h->factor_ptr[k] != rp[m]) {
        errs[k] = "fdm_hex_setup: star " + std::to_string(k) + " has a factor of another pattern";
        continue;
      }
      std::vector<double> L((size_t)m * m, 0.0);
      for (int r = 0; r < m; ++r)
        for (int64_t q = rp[r]; q < rp[r + 1]; ++q) L[(size_t)r * m + cols[q]] = fv[q];
      dense_inverse_rows(L, m, zoff[S.cls], vals.data() + S.voff);
    }
  };
  const int nt = std::max(1, std::min<int>((int)std::thread::hardware_concurrency(), 64));
  std::vector<std::thread> pool;
  for (int i = 1; i < nt; ++i) pool.emplace_back(work);
  work();
  for (std::thread &t : pool) t.join();
  for (const std::string &e : errs)
    if (!e.empty()) fail(FDM_EINVAL, e);
  c->nval = off;
}

// the class tables of the stars' interface solves, concatenated into ct
void build_class(const fdm_hexmesh *h, int cl, int nG, std::vector<int> &ct, HexClassDev &D) {
  const int t = h->sc_t[cl], nB = nG - t;
  const int64_t *rp = h->sc_rowptr.data() + h->sc_ptr[cl];
  const int32_t *cols = h->sc_cols.data() + h->sc_colptr[cl];
  if (h->sc_ptr[cl + 1] - h->sc_ptr[cl] != (int64_t)nB + 1 + t + 1)
    fail(FDM_EINVAL, "fdm_hex_setup: inconsistent Schur-coupling row pointers of class " + std::to_string(cl));
  const int64_t *rb = rp, *rt = rp + nB + 1;
  const int nnzL = (int)rb[nB];
  const int32_t *cst = cols + nnzL;
  auto put = [&](const std::vector<int> &v) {
    const int off = (int)ct.size();
    ct.insert(ct.end(), v.begin(), v.end());
    return off;
  };
  D.nB = nB;
  D.t = t;
  // rows of L_BB: the diagonal and the strictly lower entries; forward levels
  std::vector<int> ldiag(nB, -1), lptr(nB + 1, 0), lcol, lpos, lev(nB, 0);
  std::vector<std::vector<std::pair<int, int>>> colent(nB);  // column c: (row, value position)
  for (int r = 0; r < nB; ++r) {
    for (int64_t q = rb[r]; q < rb[r + 1]; ++q) {
      const int c = cols[q];
      if (c == r) ldiag[r] = (int)q;
      else if (c >= 0 && c < r) {
        lcol.push_back(c);
        lpos.push_back((int)q);
        lev[r] = std::max(lev[r], lev[c] + 1);
        colent[c].push_back({r, (int)q});
      } else {
        fail(FDM_EINVAL, "fdm_hex_setup: L_BB entry above the diagonal in class " + std::to_string(cl));
      }
    }
    if (ldiag[r] < 0) fail(FDM_EINVAL, "fdm_hex_setup: L_BB row without a diagonal in class " + std::to_string(cl));
    lptr[r + 1] = (int)lcol.size();
  }
  auto levels = [&](const std::vector<int> &lv, std::vector<int> &ptr, std::vector<int> &rows) {
    int nl = 0;
    for (int x : lv) nl = std::max(nl, x + 1);
    ptr.assign(nl + 1, 0);
    for (int x : lv) ++ptr[x + 1];
    for (int l = 0; l < nl; ++l) ptr[l + 1] += ptr[l];
    rows.assign(lv.size(), 0);
    std::vector<int> at(ptr.begin(), ptr.end() - 1);
    for (int r = 0; r < (int)lv.size(); ++r) rows[at[lv[r]]++] = r;
    return nl;
  };
  std::vector<int> levf_ptr, rows_f;
  D.nlf = nB ? levels(lev, levf_ptr, rows_f) : 0;
  // columns of L_BB (rows of L_BB^T), backward levels
  std::vector<int> tptr(nB + 1, 0), trow, tpos, blev(nB, 0);
  for (int c = nB - 1; c >= 0; --c)
    for (const auto &e : colent[c]) blev[c] = std::max(blev[c], blev[e.first] + 1);
  for (int c = 0; c < nB; ++c) {
    for (const auto &e : colent[c]) {
      trow.push_back(e.first);
      tpos.push_back(e.second);
    }
    tptr[c + 1] = (int)trow.size();
  }
  std::vector<int> levb_ptr, rows_b;
  D.nlb = nB ? levels(blev, levb_ptr, rows_b) : 0;
  // S_TB by rows, and by B columns
  D.off_st = nnzL;
  std::vector<int> stptr(t + 1, 0), stcol;
  std::vector<std::vector<std::pair<int, int>>> bcol(nB);
  for (int r = 0; r < t; ++r) {
    for (int64_t q = rt[r]; q < rt[r + 1]; ++q) {
      const int c = cst[q];
      if (c < 0 || c >= nB) fail(FDM_EINVAL, "fdm_hex_setup: S_TB column out of range in class " + std::to_string(cl));
      stcol.push_back(c);
      bcol[c].push_back({r, nnzL + (int)q});
    }
    stptr[r + 1] = (int)stcol.size();
  }
  std::vector<int> sbtptr(nB + 1, 0), sbtrow, sbtpos;
  for (int c = 0; c < nB; ++c) {
    for (const auto &e : bcol[c]) {
      sbtrow.push_back(e.first);
      sbtpos.push_back(e.second);
    }
    sbtptr[c + 1] = (int)sbtrow.size();
  }
  D.off_w = nnzL + (int)rt[t];
  D.lev_f = put(levf_ptr.empty() ? std::vector<int>{0} : levf_ptr);
  D.rows_f = put(rows_f);
  D.lptr = put(lptr);
  D.lcol = put(lcol);
  D.lpos = put(lpos);
  D.ldiag = put(ldiag);
  D.lev_b = put(levb_ptr.empty() ? std::vector<int>{0} : levb_ptr);
  D.rows_b = put(rows_b);
  D.tptr = put(tptr);
  D.trow = put(trow);
  D.tpos = put(tpos);
  D.stptr = put(stptr);
  D.stcol = put(stcol);
  D.sbtptr = put(sbtptr);
  D.sbtrow = put(sbtrow);
  D.sbtpos = put(sbtpos);
}

}  // namespace

namespace fdm {
void ctx_tridiag_extremes(const std::vector<double> &d, const std::vector<double> &e, double &lo, double &hi);
void ctx_normal_vector(uint64_t seed, int64_t n, std::vector<double> &out);
}  // namespace fdm

namespace {

__global__ void k_hex_mask(int64_t n, const uint8_t *__restrict__ dir, double *__restrict__ v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (dir[i]) v[i] = 0.0;
}
int vblocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }
void hex_mask(fdm_hexgpu *c, double *v, cudaStream_t st) {
  k_hex_mask<<<vblocks(c->nnode), 256, 0, st>>>(c->nnode, c->d64.dirichlet, v);
  c->launches += 1;
}

// the device view in precision T of the host tables (integer maps shared)
template <typename T>
void fill_dev(fdm_hexgpu *c, const fdm_hexmesh *h, HexDev<T> &d, const HexDev<double> &base,
              const std::vector<double> &tab, const std::vector<double> &inv_mult, const std::vector<double> &Ainv,
              const std::vector<double> &vals) {
  d = HexDev<T>();
  d.p = base.p;
  d.n = base.n;
  d.nc = base.nc;
  d.nstar = base.nstar;
  d.nco = base.nco;
  d.nnode = base.nnode;
  d.cell_nodes = base.cell_nodes;
  d.cell_fdm = base.cell_fdm;
  d.cell_sign = base.cell_sign;
  d.dirichlet = base.dirichlet;
  d.cell_m = base.cell_m;
  d.slot_cells_ptr = base.slot_cells_ptr;
  d.slot_cells = base.slot_cells;
  d.slot_stars_ptr = base.slot_stars_ptr;
  d.slot_stars = base.slot_stars;
  d.node_owner = base.node_owner;
  d.node_cells_ptr = base.node_cells_ptr;
  d.node_cells = base.node_cells;
  d.stars = base.stars;
  d.classes = base.classes;
  d.ct = base.ct;
  d.star_nodes = base.star_nodes;
  d.cells8 = base.cells8;
  d.coarse_of = base.coarse_of;
  d.vcell_ptr = base.vcell_ptr;
  d.vcell = base.vcell;
  d.coarse_vertex = base.coarse_vertex;
  d.inv_mult = c->upload(conv<T>(inv_mult));
  d.mu = c->upload(conv<T>(h->mu));
  d.tab = c->upload(conv<T>(tab));
  d.geom = c->upload(conv<T>(h->geom));
  d.vals = c->upload(conv<T>(vals));
  d.Acinv = c->upload(conv<T>(Ainv));
}

void setup(fdm_hexgpu *c, const fdm_hexmesh *h, cudaStream_t st) {
  const int p = h->p, n = h->n, n3 = n * n * n, nc = h->nc;
  if ((int64_t)h->mu.size() != 3LL * nc || (int64_t)h->geom.size() != 6LL * nc * n3)
    fail(FDM_EINVAL, "fdm_hex_setup: the mesh has no numeric set-up (call fdm_hexmesh_factor first)");
  c->p = p;
  c->n = n;
  c->nc = nc;
  c->nv = h->nv;
  c->nnode = h->nnode;
  HexDev<double> &b = c->d64;
  b.p = p;
  b.n = n;
  b.nc = nc;
  b.nnode = h->nnode;
  // 1D tables: T, Af, Bf, Vq, Dq (n x n), GLL nodes
  const Basis1D B1 = make_basis(p);
  std::vector<double> tab;
  for (const std::vector<double> *v : {&B1.T, &B1.Af, &B1.Bf, &B1.Vq, &B1.Dq}) tab.insert(tab.end(), v->begin(), v->end());
  tab.insert(tab.end(), B1.xi.begin(), B1.xi.end());
  // multiplicities, stars holding each cell's interior
  std::vector<double> inv_mult(h->nnode);
  for (int64_t g = 0; g < h->nnode; ++g) {
    const int64_t m = h->node_cells_ptr[g + 1] - h->node_cells_ptr[g];
    if (m < 1) fail(FDM_EINVAL, "fdm_hex_setup: a node belongs to no cell");
    inv_mult[g] = 1.0 / (double)m;
  }
  std::vector<int> cell_m(nc, 0);
  if (p >= 2)
    for (int e = 0; e < nc; ++e) {
      const int slot = h->cell_fdm[(size_t)e * n3 + 1 + n + n * n];
      cell_m[e] = (int)(h->slot_stars_ptr[slot + 1] - h->slot_stars_ptr[slot]);
    }
  // stars and classes
  const int nstar = (int)h->star_vertex.size(), ncls = (int)h->class_star.size();
  std::vector<HexStarDev> stars(nstar);
  std::vector<int> cls_nG(ncls, -1);
  int64_t xo = 0;
  for (int k = 0; k < nstar; ++k) {
    HexStarDev &S = stars[k];
    S.cls = h->star_class[k];
    S.ni = h->star_nint[k];
    S.nG = (int)(h->star_ptr[k + 1] - h->star_ptr[k]) - S.ni;
    S.nodes_off = h->star_ptr[k];
    S.voff = h->sc_values_ptr.empty() ? 0 : h->sc_values_ptr[k];
    S.xoff = xo;
    xo += S.nG;
    c->maxG = std::max(c->maxG, S.nG);
    if (cls_nG[S.cls] < 0) cls_nG[S.cls] = S.nG;
    else if (cls_nG[S.cls] != S.nG) fail(FDM_EINVAL, "fdm_hex_setup: stars of one class differ in size");
  }
  if ((int64_t)h->sc_values_ptr.size() != (int64_t)nstar + 1)
    fail(FDM_EINVAL, "fdm_hex_setup: the mesh has no Schur-coupling factors (call fdm_hexmesh_factor first)");
  c->nxtot = xo;
  c->nstar = nstar;
  {  // size bins of the dense interface solves, each largest first
    std::vector<int> order(nstar);
    for (int k = 0; k < nstar; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return stars[a].nG > stars[b].nG; });
    std::vector<int> bins[3];
    for (int k : order) {
      const int nG = stars[k].nG, b = nG <= 256 ? 0 : (nG <= 512 ? 1 : 2);
      bins[b].push_back(k);
      c->bin_maxg[b] = std::max(c->bin_maxg[b], nG);
    }
    std::vector<int> all;
    for (int b = 0; b < 3; ++b) {
      c->bin_count[b] = (int)bins[b].size();
      all.insert(all.end(), bins[b].begin(), bins[b].end());
    }
    c->bin_list = c->upload(all);
    if (c->dense && c->bin_count[2] > 0 && c->bin_count[0] + c->bin_count[1] > 0) {
      FDM_CUDA(cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking));
      FDM_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
      FDM_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    }
  }
  std::vector<int> ct;
  std::vector<HexClassDev> classes(ncls);
  for (int cl = 0; cl < ncls; ++cl) build_class(h, cl, std::max(cls_nG[cl], 0), ct, classes[cl]);
  for (int k = 0; k < nstar; ++k) {  // every star's values match its class's layout
    const HexClassDev &D = classes[stars[k].cls];
    const int64_t need = stars[k].nG ? (int64_t)D.off_w + (int64_t)D.t * (D.t + 1) / 2 : 0;
    if (h->sc_values_ptr[k + 1] - h->sc_values_ptr[k] != need)
      fail(FDM_EINVAL, "fdm_hex_setup: star " + std::to_string(k) + " has values of another layout");
  }
  c->nval = (int64_t)h->sc_values.size();
  c->dense = c->opt.patch_form != 2;
  std::vector<double> dvals;
  if (c->dense) build_dense(c, h, stars, classes, cls_nG, ct, dvals);
  // coarse space: unknowns, their vertices and cells, the dense inverse
  int nco = 0;
  for (int v = 0; v < h->nv; ++v) nco = std::max(nco, h->coarse_of[v] + 1);
  if ((int64_t)h->coarse.size() != (int64_t)nco * nco) fail(FDM_EINVAL, "fdm_hex_setup: no Q1 coarse operator");
  std::vector<int> coarse_vertex(std::max(nco, 1), -1);
  for (int v = 0; v < h->nv; ++v)
    if (h->coarse_of[v] >= 0) coarse_vertex[h->coarse_of[v]] = v;
  std::vector<std::vector<int>> vc(nco);
  for (int e = 0; e < nc; ++e)
    for (int k = 0; k < 8; ++k) {
      const int u = h->coarse_of[h->cells[8 * e + k]];
      if (u >= 0) vc[u].push_back(8 * e + k);
    }
  std::vector<int64_t> vcell_ptr(nco + 1, 0);
  std::vector<int> vcell;
  for (int u = 0; u < nco; ++u) {
    vcell.insert(vcell.end(), vc[u].begin(), vc[u].end());
    vcell_ptr[u + 1] = (int64_t)vcell.size();
  }
  const std::vector<double> Ainv = nco > 0 ? spd_inverse(h->coarse, nco) : std::vector<double>();
  c->nco = nco;
  // integer maps (shared by both precisions)
  b.nstar = nstar;
  b.nco = nco;
  b.cell_nodes = c->upload(h->cell_nodes);
  b.cell_fdm = c->upload(h->cell_fdm);
  b.cell_sign = c->upload(h->cell_sign);
  b.dirichlet = c->upload(h->dirichlet);
  b.cell_m = c->upload(cell_m);
  b.slot_cells_ptr = c->upload(h->slot_cells_ptr);
  b.slot_cells = c->upload(h->slot_cells);
  b.slot_stars_ptr = c->upload(h->slot_stars_ptr);
  b.slot_stars = c->upload(h->slot_stars);
  b.node_owner = c->upload(h->node_owner);
  b.node_cells_ptr = c->upload(h->node_cells_ptr);
  b.node_cells = c->upload(h->node_cells);
  b.stars = c->upload(stars);
  b.classes = c->upload(classes);
  b.ct = c->upload(ct.empty() ? std::vector<int>{0} : ct);
  b.star_nodes = c->upload(h->star_nodes);
  b.cells8 = c->upload(h->cells);
  b.coarse_of = c->upload(h->coarse_of);
  b.vcell_ptr = c->upload(vcell_ptr);
  b.vcell = c->upload(vcell.empty() ? std::vector<int>{0} : vcell);
  b.coarse_vertex = c->upload(coarse_vertex);
  const HexDev<double> base = b;
  const std::vector<double> &vals = c->dense ? dvals : h->sc_values;
  fill_dev<double>(c, h, c->d64, base, tab, inv_mult, Ainv, vals);
  fill_dev<float>(c, h, c->d32, base, tab, inv_mult, Ainv, vals);
  // work vectors
  const int64_t ne = (int64_t)nc * n3, nn = h->nnode, nx = std::max<int64_t>(c->nxtot, 1);
  const bool fp32 = c->opt.precision == FDM_PREC_FP32;
  c->E64 = c->alloc<double>(ne);
  c->Y64 = c->alloc<double>(ne);
  c->rc64 = c->alloc<double>(nn);
  c->zf64 = c->alloc<double>(nn);
  c->X64 = c->alloc<double>(nx);
  c->x1_64 = c->alloc<double>(nn);
  c->t64 = c->alloc<double>(nn);
  c->w64 = c->alloc<double>(nn);
  c->cr64 = c->alloc<double>(std::max(nco, 1));
  c->cx64 = c->alloc<double>(std::max(nco, 1));
  if (fp32) {
    c->E32 = c->alloc<float>(ne);
    c->Y32 = c->alloc<float>(ne);
    c->rc32 = c->alloc<float>(nn);
    c->zf32 = c->alloc<float>(nn);
    c->X32 = c->alloc<float>(nx);
    c->r32 = c->alloc<float>(nn);
    c->x1_32 = c->alloc<float>(nn);
    c->t32 = c->alloc<float>(nn);
    c->w32 = c->alloc<float>(nn);
    c->cr32 = c->alloc<float>(std::max(nco, 1));
    c->cx32 = c->alloc<float>(std::max(nco, 1));
  }
  for (double **v : {&c->r, &c->z, &c->zold, &c->d, &c->q, &c->v1}) *v = c->alloc<double>(nn);
  c->partial = c->alloc<double>(2 * DOT_BLOCKS);
  c->dots = c->alloc<double>(8);
  c->sc = c->alloc<double>(16);
  FDM_CUDA(cudaStreamSynchronize(st));
}

// y = A u (precision T, cell-local results in Y, summed per node); rsub: y = rsub - A u
template <typename T>
void hex_op(fdm_hexgpu *c, const T *u, const T *rsub, T *y, cudaStream_t st) {
  launch_hex_op_cells<T, T>(c->dev<T>(), u, c->Y<T>(), st);
  launch_hex_gather<T, T>(c->dev<T>(), c->Y<T>(), rsub, y, st);
  c->launches += 2;
}

// z = omega sum_v R_v^T A~_v^{-1} R_v r in precision T
template <typename T>
void hex_asm(fdm_hexgpu *c, const T *r, T *z, double omega, cudaStream_t st) {
  const HexDev<T> &d = c->dev<T>();
  launch_hex_restrict<T, T>(d, r, c->E<T>(), st);
  launch_hex_assemble<T>(d, c->E<T>(), c->rc<T>(), st);
  if (c->dense && c->aux && c->bin_count[2] > 0 && c->bin_count[0] + c->bin_count[1] > 0) {
    FDM_CUDA(cudaEventRecord(c->ev_fork, st));
    FDM_CUDA(cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    launch_hex_star_dense<T>(d, c->rc<T>(), c->X<T>(), c->bin_list, c->bin_count, c->bin_maxg, 4u, c->aux);
    FDM_CUDA(cudaEventRecord(c->ev_join, c->aux));
    launch_hex_star_dense<T>(d, c->rc<T>(), c->X<T>(), c->bin_list, c->bin_count, c->bin_maxg, 3u, st);
    FDM_CUDA(cudaStreamWaitEvent(st, c->ev_join, 0));
  } else if (c->dense) {
    launch_hex_star_dense<T>(d, c->rc<T>(), c->X<T>(), c->bin_list, c->bin_count, c->bin_maxg, 7u, st);
  } else {
    launch_hex_star_solve<T>(d, c->rc<T>(), c->X<T>(), c->maxG, st);
  }
  launch_hex_slot_stars<T>(d, c->X<T>(), c->zf<T>(), st);
  launch_hex_interp<T, T>(d, c->E<T>(), c->zf<T>(), omega, z, st);
  const int solves = c->dense ? (c->bin_count[0] > 0) + (c->bin_count[1] > 0) + (c->bin_count[2] > 0) : 1;
  c->launches += 4 + solves;
}

// hybrid V(1,1) in precision T: x1 = w S r, x1 += P Ac^{-1} P^T (r - A x1), z = x1 + w S (r - A x1)
template <typename T>
void hex_vcycle(fdm_hexgpu *c, const T *r, T *z, T *x1, T *t, T *w, T *cr, T *cx, cudaStream_t st) {
  const int64_t nn = c->nnode;
  hex_asm<T>(c, r, x1, c->omega, st);
  hex_op<T>(c, x1, r, t, st);
  if (c->nco > 0) {
    launch_hex_coarse_restrict<T>(c->dev<T>(), t, c->Y<T>(), cr, st);  // Y: scratch of the corner sums
    launch_dense_symv<T>(c->nco, c->dev<T>().Acinv, cr, cx, st);
    launch_hex_coarse_prolong<T>(c->dev<T>(), cx, x1, st);
    c->launches += 4;
  }
  hex_op<T>(c, x1, r, t, st);
  hex_asm<T>(c, t, w, c->omega, st);
  launch_axpby<T>(nn, T(1), x1, T(1), w, z, st);
  c->launches += 1;
}

void hex_pc(fdm_hexgpu *c, const double *r, double *z, cudaStream_t st) {
  const int64_t nn = c->nnode;
  if (c->opt.pc == FDM_PC_NONE) {
    FDM_CUDA(cudaMemcpyAsync(z, r, nn * sizeof(double), cudaMemcpyDeviceToDevice, st));
    hex_mask(c, z, st);
    return;
  }
  if (c->opt.precision == FDM_PREC_FP32) {
    launch_convert<double, float>(nn, r, c->r32, st);
    c->launches += 1;
    if (c->opt.pc == FDM_PC_ASM) hex_asm<float>(c, c->r32, c->w32, c->omega, st);
    else hex_vcycle<float>(c, c->r32, c->w32, c->x1_32, c->t32, c->w32, c->cr32, c->cx32, st);
    launch_convert<float, double>(nn, c->w32, z, st);
    c->launches += 1;
  } else {
    if (c->opt.pc == FDM_PC_ASM) hex_asm<double>(c, r, z, c->omega, st);
    else hex_vcycle<double>(c, r, z, c->x1_64, c->t64, c->w64, c->cr64, c->cx64, st);
  }
}

void hex_lanczos(fdm_hexgpu *c, const double *start_host, cudaStream_t st) {
  const int64_t n = c->nnode;
  std::vector<double> b0;
  if (start_host) b0.assign(start_host, start_host + n);
  else ctx_normal_vector(c->opt.lanczos_seed, n, b0);
  FDM_CUDA(cudaMemcpyAsync(c->r, b0.data(), n * sizeof(double), cudaMemcpyHostToDevice, st));
  hex_mask(c, c->r, st);
  hex_asm<double>(c, c->r, c->z, 1.0, st);
  FDM_CUDA(cudaMemcpyAsync(c->d, c->z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  double h[2];
  launch_dot(n, c->r, c->z, c->partial, c->dots, st);
  FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
  FDM_CUDA(cudaStreamSynchronize(st));
  double rz = h[0];
  std::vector<double> al, be;
  const int steps = c->opt.lanczos_steps > 0 ? c->opt.lanczos_steps : 20;
  for (int k = 0; k < steps; ++k) {
    if (!(rz > 0.0)) break;
    hex_op<double>(c, c->d, nullptr, c->q, st);
    launch_dot(n, c->d, c->q, c->partial, c->dots, st);
    FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    if (!(h[0] > 0.0)) break;
    const double alpha = rz / h[0];
    al.push_back(alpha);
    launch_axpby<double>(n, -alpha, c->q, 1.0, c->r, c->r, st);
    hex_asm<double>(c, c->r, c->z, 1.0, st);
    launch_dot(n, c->r, c->z, c->partial, c->dots, st);
    FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    const double beta = h[0] / rz;
    be.push_back(beta);
    rz = h[0];
    launch_axpby<double>(n, 1.0, c->z, beta, c->d, c->d, st);
  }
  const int m = (int)al.size();
  if (m < 1) fail(FDM_EINVAL, "fdm_hex_setup: Lanczos took no step (zero start vector?)");
  std::vector<double> dd(m), ee(std::max(m - 1, 1), 0.0);
  for (int j = 0; j < m; ++j) {
    dd[j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
    if (j + 1 < m) ee[j] = std::sqrt(be[j]) / al[j];
  }
  ctx_tridiag_extremes(dd, ee, c->lmin, c->lmax);
  c->omega = 2.0 / (1.25 * c->lmax + 0.75 * c->lmin);
}

}  // namespace

extern "C" {

int fdm_hex_setup(const fdm_hexmesh *h, const fdm_options *opt, fdm_hexgpu **out, void *stream) {
  if (!h || !out) return FDM_EINVAL;
  *out = nullptr;
  fdm_hexgpu *c = new fdm_hexgpu();
  cudaStream_t st = (cudaStream_t)stream;
  try {
    if (opt) c->opt = *opt;
    else fdm_default_options(&c->opt);
    if (c->opt.flexible_beta < 0) c->opt.flexible_beta = c->opt.precision == FDM_PREC_FP32 ? 1 : 0;
    if (c->opt.precision != FDM_PREC_FP32 && c->opt.precision != FDM_PREC_FP64)
      fail(FDM_EINVAL, "fdm_hex_setup: precision must be FDM_PREC_FP64 or FDM_PREC_FP32");
    setup(c, h, st);
    if (c->opt.omega > 0.0) c->omega = c->opt.omega;
    else if (c->opt.pc != FDM_PC_NONE) hex_lanczos(c, c->opt.lanczos_start, st);
    FDM_CUDA(cudaStreamSynchronize(st));
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &e) {
    const int rc = handle_hexgpu(nullptr, e);
    delete c;
    return rc;
  }
  *out = c;
  return FDM_OK;
}

int hex_stiffness_apply(fdm_hexgpu *c, const double *u, double *y, void *stream) {
  if (!c || !u || !y) return FDM_EINVAL;
  try {
    hex_op<double>(c, u, nullptr, y, (cudaStream_t)stream);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &e) { return handle_hexgpu(c, e); }
  return FDM_OK;
}

int hex_asm_apply(fdm_hexgpu *c, const double *r, double *z, void *stream) {
  if (!c || !r || !z) return FDM_EINVAL;
  try {
    cudaStream_t st = (cudaStream_t)stream;
    if (c->opt.precision == FDM_PREC_FP32) {
      launch_convert<double, float>(c->nnode, r, c->r32, st);
      hex_asm<float>(c, c->r32, c->w32, c->omega, st);
      launch_convert<float, double>(c->nnode, c->w32, z, st);
      c->launches += 2;
    } else {
      hex_asm<double>(c, r, z, c->omega, st);
    }
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &e) { return handle_hexgpu(c, e); }
  return FDM_OK;
}

int hex_pc_apply(fdm_hexgpu *c, const double *r, double *z, void *stream) {
  if (!c || !r || !z) return FDM_EINVAL;
  try {
    hex_pc(c, r, z, (cudaStream_t)stream);
    FDM_CUDA(cudaGetLastError());
  } catch (const Error &e) { return handle_hexgpu(c, e); }
  return FDM_OK;
}

int hex_pcg_solve(fdm_hexgpu *c, const double *b, double *x, double rtol, int maxit, fdm_solve_info *info,
                  void *stream) {
  if (!c || !b || !x || maxit < 0 || !(rtol >= 0.0)) return FDM_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = c->nnode;
  try {
    cudaEvent_t e0, e1;
    FDM_CUDA(cudaEventCreate(&e0));
    FDM_CUDA(cudaEventCreate(&e1));
    FDM_CUDA(cudaEventRecord(e0, st));
    double hsc[16] = {0};
    hsc[7] = c->opt.flexible_beta ? 1.0 : 0.0;
    FDM_CUDA(cudaMemcpyAsync(c->sc, hsc, sizeof hsc, cudaMemcpyHostToDevice, st));
    FDM_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    FDM_CUDA(cudaMemcpyAsync(c->r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
    hex_mask(c, c->r, st);
    double h[2];
    launch_dot(n, c->r, c->r, c->partial, c->dots, st);
    c->launches += 2;
    FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
    FDM_CUDA(cudaStreamSynchronize(st));
    const double nb = std::sqrt(h[0]);
    double nr = nb;
    int it = 0, conv = nb == 0.0, bad = 0;
    double *z = c->z, *zold = c->zold;
    if (!conv) {
      hex_pc(c, c->r, z, st);
      launch_dot(n, c->r, z, c->partial, c->dots, st);
      launch_pcg_scalars(2, c->sc, c->dots, st);
      FDM_CUDA(cudaMemcpyAsync(c->d, z, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
      c->launches += 3;
      while (it < maxit) {
        hex_op<double>(c, c->d, nullptr, c->q, st);
        launch_dot(n, c->d, c->q, c->partial, c->dots, st);
        launch_pcg_scalars(0, c->sc, c->dots, st);
        launch_pcg_update_xr(n, c->sc, c->d, c->q, x, c->r, st);
        ++it;
        launch_dot(n, c->r, c->r, c->partial, c->dots + 2, st);
        c->launches += 6;
        FDM_CUDA(cudaMemcpyAsync(h, c->dots + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
        FDM_CUDA(cudaStreamSynchronize(st));
        nr = std::sqrt(h[0]);
        if (!std::isfinite(nr)) { bad = 1; break; }
        if (nr <= rtol * nb) {
          // converged on the recursive residual: replace it by the true one,
          // r = b - A x, and stop only if that meets the test too
          hex_op<double>(c, x, b, c->r, st);
          launch_dot(n, c->r, c->r, c->partial, c->dots + 2, st);
          c->launches += 2;
          FDM_CUDA(cudaMemcpyAsync(h, c->dots + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
          FDM_CUDA(cudaStreamSynchronize(st));
          nr = std::sqrt(h[0]);
          if (!std::isfinite(nr)) { bad = 1; break; }
          if (nr <= rtol * nb) { conv = 1; break; }
          if (it >= maxit) break;
        }
        std::swap(z, zold);
        hex_pc(c, c->r, z, st);
        launch_dot2(n, c->r, z, zold, c->partial, c->dots, st);
        launch_pcg_scalars(1, c->sc, c->dots, st);
        launch_pcg_update_d(n, c->sc, z, c->d, st);
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
    if (info) {
      info->iterations = it;
      info->converged = conv;
      info->rnorm0 = nb;
      info->rnorm = nr;
      info->seconds = ms * 1e-3;
      hex_op<double>(c, x, b, c->v1, st);  // b - A x (0 on Dirichlet nodes)
      launch_dot(n, c->v1, c->v1, c->partial, c->dots, st);
      c->launches += 2;
      FDM_CUDA(cudaMemcpyAsync(h, c->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
      FDM_CUDA(cudaStreamSynchronize(st));
      info->true_rnorm = std::sqrt(h[0]);
    }
    FDM_CUDA(cudaGetLastError());
    if (bad) { c->err = "non-finite scalar in PCG"; return FDM_ENAN; }
    if (!conv) { c->err = "PCG reached maxit"; return FDM_ENOCONV; }
  } catch (const Error &e) { return handle_hexgpu(c, e); }
  return FDM_OK;
}

int fdm_hex_query(fdm_hexgpu *c, int what, void *out, size_t *len) {
  if (!c || !out || !len) return FDM_EINVAL;
  auto put = [&](const void *src, size_t bytes) {
    if (*len < bytes) {
      c->err = "fdm_hex_query: buffer too small (" + std::to_string(bytes) + " bytes needed)";
      return FDM_EINVAL;
    }
    std::memcpy(out, src, bytes);
    *len = bytes;
    return FDM_OK;
  };
  switch (what) {
    case FDM_XQ_NNODE: return put(&c->nnode, sizeof c->nnode);
    case FDM_XQ_OMEGA: return put(&c->omega, sizeof c->omega);
    case FDM_XQ_LAMBDA: { double v[2] = {c->lmin, c->lmax}; return put(v, sizeof v); }
    case FDM_XQ_LAUNCHES: { const int64_t v = c->launches; c->launches = 0; return put(&v, sizeof v); }
    case FDM_XQ_SIZES: {
      const int64_t v[6] = {c->nc, c->nstar, c->nxtot, c->nval, c->nco, c->maxG};
      return put(v, sizeof v);
    }
    case FDM_XQ_ALGO_BYTES: {
      // one relaxation sweep reads every stored value of the stars' interface
      // solves and the per-cell data once (map, signs, surrogate), writes and
      // reads the cell-local residual, the slot values and the star solutions,
      // and reads r and writes z (FP64): the bytes of an ideal single pass
      double v[2];
      for (int s = 0; s < 2; ++s) {
        const double w = s == 0 ? 8.0 : 4.0;
        const double ne = (double)c->nc * c->n * c->n * c->n;
        v[s] = w * ((double)c->nval + 2.0 * ne + 2.0 * (double)c->nnode + 2.0 * (double)c->nxtot + 3.0 * c->nc) +
               ne * (4.0 + 4.0 + 1.0) + 16.0 * (double)c->nnode;
      }
      return put(v, sizeof v);
    }
    default: c->err = "fdm_hex_query: unknown quantity"; return FDM_EINVAL;
  }
}

const char *fdm_hex_last_error(const fdm_hexgpu *c) { return c ? c->err.c_str() : g_hex_err.c_str(); }

void fdm_hex_destroy(fdm_hexgpu *c) { delete c; }

}  // extern "C"
