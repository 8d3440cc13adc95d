// Matrix-free operators (Sections 2.2, 2.7, 2.8 of the paper), the Q1 coarse
// space (Section 2.5) and the PCG vector kernels.
#include "cellop.cuh"
#include "device.cuh"
#include "kernels.h"

namespace fdm {

// ------------------------------------------------------------------ cell operators
// Sum-factorised y_K = A^K u_K on one cell, everything in shared memory.
// Box cells, eq. (kron): mu1 (B (x) B (x) A) + mu2 (B (x) A (x) B) + mu3 (A (x) B (x) B)
// in 7 one-dimensional contractions.  buf: 4 n^3 scratch; result in out.
template <typename T>
__device__ void cell_stiffness_box(const T *sA, const T *sB, const T mu[3], int n, T *u, T *b1, T *b2, T *b3,
                                   T *out) {
  contract(u, b1, sB, false, 0, n, T(1), false);  // Bx u
  contract(u, b2, sA, false, 0, n, T(1), false);  // Ax u
  __syncthreads();
  contract(b1, u, sB, false, 1, n, T(1), false);      // By Bx u
  contract(b1, b3, sA, false, 1, n, mu[1], false);    // mu2 Ay Bx u
  __syncthreads();
  contract(b2, b3, sB, false, 1, n, mu[0], true);     // + mu1 By Ax u
  __syncthreads();
  contract(b3, out, sB, false, 2, n, T(1), false);    // Bz (...)
  __syncthreads();
  contract(u, out, sA, false, 2, n, mu[2], true);     // + mu3 Az By Bx u
  __syncthreads();
}

template <typename T>
__device__ void cell_mass(const OpArgs &a, int cell, const T *sB, const T *sV, int n, T *u, T *b1, T *out) {
  if (!a.general) {
    const double *m = a.mu_box + 3 * cell;
    T vol = T(m[0] * m[1] * m[2]);  // mu1 mu2 mu3 = L1 L2 L3
    contract(u, b1, sB, false, 0, n, T(1), false);
    __syncthreads();
    contract(b1, u, sB, false, 1, n, T(1), false);
    __syncthreads();
    contract(u, out, sB, false, 2, n, vol, false);
    __syncthreads();
  } else {
    const int n3 = n * n * n;
    const T *dw = reinterpret_cast<const T *>(a.detw) + (int64_t)cell * n3;
    contract(u, b1, sV, false, 0, n, T(1), false);
    __syncthreads();
    contract(b1, u, sV, false, 1, n, T(1), false);
    __syncthreads();
    contract(u, b1, sV, false, 2, n, T(1), false);
    __syncthreads();
    for (int q = threadIdx.x; q < n3; q += blockDim.x) b1[q] *= dw[q];
    __syncthreads();
    contract(b1, u, sV, true, 2, n, T(1), false);
    __syncthreads();
    contract(u, b1, sV, true, 1, n, T(1), false);
    __syncthreads();
    contract(b1, out, sV, true, 0, n, T(1), false);
    __syncthreads();
  }
}

template <typename T, typename Tin>
__global__ void __launch_bounds__(256) k_operator_cells(OpArgs a, int mass, const Tin *__restrict__ u, T *__restrict__ E) {
  extern __shared__ unsigned char smem_[];
  const Grid &g = a.g;
  const int n = g.n, p = g.p, n3 = n * n * n;
  const T *tab = reinterpret_cast<const T *>(a.tab);
  T *s1 = reinterpret_cast<T *>(smem_);  // A or V
  T *s2 = s1 + n * n;                    // B or D
  T *s3 = s2 + n * n;                    // B (general mass)
  // b5 exists only for curved cells (the launcher sizes shared memory accordingly)
  T *b0 = s3 + n * n, *b1 = b0 + n3, *b2 = b1 + n3, *b3 = b2 + n3, *b4 = b3 + n3, *b5 = b4 + n3;
  const int cell = blockIdx.x;
  const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    if (!a.general) {
      s1[i] = tab[tab_off(TAB_A, n) + i];
      s2[i] = tab[tab_off(TAB_B, n) + i];
    } else {
      s1[i] = tab[tab_off(TAB_VQ, n) + i];
      s2[i] = tab[tab_off(TAB_DQ, n) + i];
    }
    s3[i] = tab[tab_off(TAB_B, n) + i];
  }
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
    int gx = cx * p + i, gy = cy * p + j, gz = cz * p + k;
    bool dir = node_dirichlet(g, gx, gy, gz);
    b0[idx] = dir ? T(0) : T(u[gidx(g, gx, gy, gz)]);
  }
  __syncthreads();
  T *out = E + (int64_t)cell * n3;
  if (mass) {
    cell_mass<T>(a, cell, s3, s1, n, b0, b1, b2);
    for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) out[idx] = b2[idx];
  } else if (!a.general) {
    T mu[3] = {T(a.mu_box[3 * cell]), T(a.mu_box[3 * cell + 1]), T(a.mu_box[3 * cell + 2])};
    cell_stiffness_box<T>(s1, s2, mu, n, b0, b1, b2, b3, b4);
    for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) out[idx] = b4[idx];
  } else {
    const T *Gw = reinterpret_cast<const T *>(a.Gw) + (int64_t)cell * n3 * 6;
    cell_stiffness_gen<T>(s1, s2, Gw, n, b0, b1, b2, b3, b4, b5);
    for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) out[idx] = b5[idx];
  }
}

// direct stiffness summation: y(node) = sum over the cells containing it, in
// a fixed order (deterministic); Dirichlet rows set to 0.
template <typename T, typename Tout>
__global__ void k_gather_nodes(Grid g, const T *__restrict__ E, Tout *__restrict__ y) {
  const int n = g.n, p = g.p, n3 = n * n * n;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ndof; id += (int64_t)gridDim.x * blockDim.x) {
    int gc[3] = {int(id % g.N[0]), int((id / g.N[0]) % g.N[1]), int(id / ((int64_t)g.N[0] * g.N[1]))};
    const bool dir = node_dirichlet(g, gc[0], gc[1], gc[2]);
    int cA[3][2], lA[3][2], cnt[3];
    const int ncl[3] = {g.nx, g.ny, g.nz};
    for (int ax = 0; ax < 3; ++ax) {
      int v = gc[ax];
      cnt[ax] = 0;
      if (v % p == 0) {
        int vv = v / p;
        if (vv > 0) { cA[ax][cnt[ax]] = vv - 1; lA[ax][cnt[ax]++] = p; }
        if (vv < ncl[ax]) { cA[ax][cnt[ax]] = vv; lA[ax][cnt[ax]++] = 0; }
      } else {
        cA[ax][0] = v / p;
        lA[ax][0] = v % p;
        cnt[ax] = 1;
      }
    }
    if (dir) { y[id] = Tout(0); continue; }
    T s = 0;
    for (int a2 = 0; a2 < cnt[2]; ++a2)
      for (int a1 = 0; a1 < cnt[1]; ++a1)
        for (int a0 = 0; a0 < cnt[0]; ++a0) {
          int cell = cA[0][a0] + g.nx * (cA[1][a1] + g.ny * cA[2][a2]);
          s += E[(int64_t)cell * n3 + lA[0][a0] + n * (lA[1][a1] + n * lA[2][a2])];
        }
    y[id] = Tout(s);
  }
}

inline int gs_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 4 * 152 * 8 ? (b > 0 ? b : 1) : 4 * 152 * 8);
}

template <typename T, typename Tin, typename Tout>
void launch_operator(const OpArgs &a, bool mass, const Tin *u, Tout *y, T *E, cudaStream_t st) {
  if (!mass && launch_box_op_fast<T, Tin, Tout>(a, u, y, E, st)) return;
  const int n = a.g.n, n3 = n * n * n;
  // box cells use 5 n^3 buffers, curved cells 6
  size_t sm = sizeof(T) * (3 * n * n + (a.general ? 6 : 5) * n3);
  cudaFuncSetAttribute(k_operator_cells<T, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_operator_cells<T, Tin><<<a.g.ncell, 256, sm, st>>>(a, mass ? 1 : 0, u, E);
  k_gather_nodes<T, Tout><<<gs_blocks(a.g.ndof), 256, 0, st>>>(a.g, E, y);
}

// ------------------------------------------------------------------ coarse space
// Galerkin cell matrices A_c^K = P_K^T A^K P_K (FP64) with P_K the trilinear
// interpolation of the 8 cell vertices at the GLL nodes.
__global__ void __launch_bounds__(256) k_coarse_cells(OpArgs a, double *__restrict__ Ac) {
  extern __shared__ unsigned char smem_[];
  const Grid &g = a.g;
  const int n = g.n, n3 = n * n * n;
  const double *tab = reinterpret_cast<const double *>(a.tab);
  double *s1 = reinterpret_cast<double *>(smem_);
  double *s2 = s1 + n * n;
  double *xi = s2 + n * n;
  // red[64] first, then 5 (box) or 6 (curved) n^3 buffers
  double *red = xi + n;
  double *b0 = red + 64, *b1 = b0 + n3, *b2 = b1 + n3, *b3 = b2 + n3, *b4 = b3 + n3, *b5 = b4 + n3;
  const int cell = blockIdx.x;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    s1[i] = a.general ? tab[tab_off(TAB_VQ, n) + i] : tab[tab_off(TAB_A, n) + i];
    s2[i] = a.general ? tab[tab_off(TAB_DQ, n) + i] : tab[tab_off(TAB_B, n) + i];
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) xi[i] = tab[tab_off(TAB_XI, n) + i];
  __syncthreads();
  auto hat = [&](int i, int s) { return s ? 0.5 * (1.0 + xi[i]) : 0.5 * (1.0 - xi[i]); };
  for (int s = 0; s < 8; ++s) {
    for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
      int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
      b0[idx] = hat(i, s & 1) * hat(j, (s >> 1) & 1) * hat(k, s >> 2);
    }
    __syncthreads();
    double *res;
    if (!a.general) {
      double mu[3] = {a.mu_box[3 * cell], a.mu_box[3 * cell + 1], a.mu_box[3 * cell + 2]};
      cell_stiffness_box<double>(s1, s2, mu, n, b0, b1, b2, b3, b4);
      res = b4;
    } else {
      const double *Gw = reinterpret_cast<const double *>(a.Gw) + (int64_t)cell * n3 * 6;
      cell_stiffness_gen<double>(s1, s2, Gw, n, b0, b1, b2, b3, b4, b5);
      res = b5;
    }
    // Ac[t][s] = P(:,t) . y
    for (int t = 0; t < 8; ++t) {
      double acc = 0.0;
      for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
        int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
        acc += hat(i, t & 1) * hat(j, (t >> 1) & 1) * hat(k, t >> 2) * res[idx];
      }
      acc = warp_sum(acc);
      if ((threadIdx.x & 31) == 0) red[t * 8 + (threadIdx.x >> 5)] = acc;
    }
    __syncthreads();
    if (threadIdx.x < 8) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += red[threadIdx.x * 8 + w];
      Ac[(int64_t)cell * 64 + threadIdx.x * 8 + s] = v;
    }
    __syncthreads();
  }
}

void launch_coarse_cell_matrices(const OpArgs &a, double *Ac, cudaStream_t st) {
  const int n = a.g.n, n3 = n * n * n;
  size_t sm = sizeof(double) * (2 * n * n + n + 64 + (a.general ? 6 : 5) * n3);
  cudaFuncSetAttribute(k_coarse_cells, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_coarse_cells<<<a.g.ncell, 256, sm, st>>>(a, Ac);
}

// r_c = P^T r: per cell the 8 corner sums of P_K^T (W_K r_K) (W = 1/multiplicity),
// then per coarse vertex the sum over its cells in a fixed order.
template <typename T, typename Tin>
__global__ void __launch_bounds__(256) k_coarse_restrict_cells(Grid g, const Tin *__restrict__ r, const T *__restrict__ tab,
                                                                T *__restrict__ cellbuf) {
  __shared__ T red[8][8];
  const int n = g.n, p = g.p, n3 = n * n * n;
  const int cell = blockIdx.x;
  const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
  const T *xi = tab + tab_off(TAB_XI, n);
  T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
    int gx = cx * p + i, gy = cy * p + j, gz = cz * p + k;
    bool dir = node_dirichlet(g, gx, gy, gz);
    if (dir) continue;
    int mult = ((i == 0 && cx > 0) || (i == p && cx < g.nx - 1) ? 2 : 1) *
               ((j == 0 && cy > 0) || (j == p && cy < g.ny - 1) ? 2 : 1) *
               ((k == 0 && cz > 0) || (k == p && cz < g.nz - 1) ? 2 : 1);
    T v = T(r[gidx(g, gx, gy, gz)]) / T(mult);
    T hx[2] = {T(0.5) * (T(1) - xi[i]), T(0.5) * (T(1) + xi[i])};
    T hy[2] = {T(0.5) * (T(1) - xi[j]), T(0.5) * (T(1) + xi[j])};
    T hz[2] = {T(0.5) * (T(1) - xi[k]), T(0.5) * (T(1) + xi[k])};
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[s] += hx[s & 1] * hy[(s >> 1) & 1] * hz[s >> 2] * v;
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    T v = warp_sum(acc[s]);
    if ((threadIdx.x & 31) == 0) red[s][threadIdx.x >> 5] = v;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    T v = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v += red[threadIdx.x][w];
    cellbuf[(int64_t)cell * 8 + threadIdx.x] = v;
  }
}

template <typename T>
__global__ void k_coarse_restrict_vertices(Grid g, const int *__restrict__ cfree, const T *__restrict__ cellbuf,
                                           T *__restrict__ rc) {
  const int nvx = g.nx + 1, nvy = g.ny + 1, nv = nvx * nvy * (g.nz + 1);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    int f = cfree[v];
    if (f < 0) continue;
    int vx = v % nvx, vy = (v / nvx) % nvy, vz = v / (nvx * nvy);
    T s = 0;
    for (int s8 = 0; s8 < 8; ++s8) {  // the cell at offset (-1 + ox, ...) sees v as corner (1 - ox, ...)
      int ox = s8 & 1, oy = (s8 >> 1) & 1, oz = s8 >> 2;
      int cx = vx - 1 + ox, cy = vy - 1 + oy, cz = vz - 1 + oz;
      if (cx < 0 || cy < 0 || cz < 0 || cx >= g.nx || cy >= g.ny || cz >= g.nz) continue;
      int corner = (1 - ox) | ((1 - oy) << 1) | ((1 - oz) << 2);
      s += cellbuf[(int64_t)(cx + g.nx * (cy + g.ny * cz)) * 8 + corner];
    }
    rc[f] = s;
  }
}

template <typename T, typename Tin>
void launch_coarse_restrict(const Grid &g, const Tin *r, const T *tab, const int *cfree, T *rc, T *cellbuf,
                            cudaStream_t st) {
  if (!launch_coarse_restrict_fast<T, Tin>(g, r, tab, cellbuf, st))
    k_coarse_restrict_cells<T, Tin><<<g.ncell, 256, 0, st>>>(g, r, tab, cellbuf);
  int nv = (g.nx + 1) * (g.ny + 1) * (g.nz + 1);
  k_coarse_restrict_vertices<T><<<(nv + 255) / 256, 256, 0, st>>>(g, cfree, cellbuf, rc);
}

// y = A x for a dense symmetric m x m matrix (row-major): one warp per row
template <typename T>
__global__ void k_dense_symv(int m, const T *__restrict__ A, const T *__restrict__ x, T *__restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < m; r += warps) {
    const T *row = A + (int64_t)r * m;
    T s = 0;
    for (int c = lane; c < m; c += 32) s += row[c] * x[c];
    s = warp_sum(s);
    if (lane == 0) y[r] = s;
  }
}

// the same with 16-byte loads: a row starts at an arbitrary element offset r m,
// so each warp reads the unaligned head and the tail element by element and the
// body in 16-byte vectors (VW = 16 / sizeof(T) elements)
template <typename T>
__global__ void k_dense_symv_vec(int m, const T *__restrict__ A, const T *__restrict__ x, T *__restrict__ y) {
  constexpr int VW = 16 / sizeof(T);
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < m; r += warps) {
    const T *row = A + (int64_t)r * m;
    const int head = (int)((VW - ((int64_t)r * m) % VW) % VW);
    const int body = (m - head) / VW;
    T s = 0;
    if (lane < head && lane < m) s += row[lane] * x[lane];
    for (int q = lane; q < body; q += 32) {
      const int c = head + q * VW;
      if constexpr (VW == 4) {
        const float4 v = *reinterpret_cast<const float4 *>(row + c);
        s += v.x * x[c] + v.y * x[c + 1] + v.z * x[c + 2] + v.w * x[c + 3];
      } else {
        const double2 v = *reinterpret_cast<const double2 *>(row + c);
        s += v.x * x[c] + v.y * x[c + 1];
      }
    }
    const int t0 = head + body * VW;
    if (t0 + lane < m) s += row[t0 + lane] * x[t0 + lane];
    s = warp_sum(s);
    if (lane == 0) y[r] = s;
  }
}

template <typename T>
void launch_dense_symv(int m, const T *Ainv, const T *x, T *y, cudaStream_t st) {
  if (m <= 0) return;
  int blocks = (m * 32 + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_dense_symv_vec<T><<<blocks, 256, 0, st>>>(m, Ainv, x, y);
}

// z (+)= P x_c: per cell, trilinear interpolation of the corner values at the
// GLL nodes, written by the owning cell.
template <typename T, typename Tout>
__global__ void k_coarse_prolong(Grid g, const T *__restrict__ xc, const T *__restrict__ tab, const int *__restrict__ cfree,
                                 Tout *__restrict__ z, int accumulate) {
  const int n = g.n, p = g.p, n3 = n * n * n;
  const int cell = blockIdx.x;
  const int ce[3] = {cell % g.nx, (cell / g.nx) % g.ny, cell / (g.nx * g.ny)};
  const T *xi = tab + tab_off(TAB_XI, n);
  T cv[8];
  for (int s = 0; s < 8; ++s) {
    int v = (ce[0] + (s & 1)) + (g.nx + 1) * ((ce[1] + ((s >> 1) & 1)) + (g.ny + 1) * (ce[2] + (s >> 2)));
    int f = cfree[v];
    cv[s] = f >= 0 ? xc[f] : T(0);
  }
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
    if ((i == 0 && ce[0] > 0) || (j == 0 && ce[1] > 0) || (k == 0 && ce[2] > 0)) continue;
    int gx = ce[0] * p + i, gy = ce[1] * p + j, gz = ce[2] * p + k;
    bool dir = node_dirichlet(g, gx, gy, gz);
    T hx[2] = {T(0.5) * (T(1) - xi[i]), T(0.5) * (T(1) + xi[i])};
    T hy[2] = {T(0.5) * (T(1) - xi[j]), T(0.5) * (T(1) + xi[j])};
    T hz[2] = {T(0.5) * (T(1) - xi[k]), T(0.5) * (T(1) + xi[k])};
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += hx[c & 1] * hy[(c >> 1) & 1] * hz[c >> 2] * cv[c];
    int64_t id = gidx(g, gx, gy, gz);
    if (dir) s = 0;
    z[id] = accumulate ? Tout(z[id] + s) : Tout(s);
  }
}

template <typename T, typename Tout>
void launch_coarse_prolong(const Grid &g, const T *xc, const T *tab, const int *cfree, Tout *z, bool accumulate,
                           cudaStream_t st) {
  if (!launch_coarse_prolong_fast<T, Tout>(g, xc, tab, cfree, z, accumulate, st))
    k_coarse_prolong<T, Tout><<<g.ncell, 128, 0, st>>>(g, xc, tab, cfree, z, accumulate ? 1 : 0);
}

// ------------------------------------------------------------------ vectors
// Deterministic dot product: fixed grid, fixed per-thread striding, fixed trees.
template <int K>
__global__ void __launch_bounds__(256) k_dot_partial(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                                                     const double *__restrict__ c, double *__restrict__ partial) {
  __shared__ double red[K][8];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double ai = a[i];
    s0 += ai * b[i];
    if (K == 2) s1 += ai * c[i];
  }
  s0 = warp_sum(s0);
  if (K == 2) s1 = warp_sum(s1);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s0;
    if (K == 2) red[K - 1][threadIdx.x >> 5] = s1;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[threadIdx.x][w];
    partial[threadIdx.x * DOT_BLOCKS + blockIdx.x] = v;
  }
}

template <int K>
__global__ void __launch_bounds__(256) k_dot_final(const double *__restrict__ partial, double *__restrict__ out) {
  __shared__ double red[8];
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    for (int i = threadIdx.x; i < DOT_BLOCKS; i += blockDim.x) s += partial[k * DOT_BLOCKS + i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += red[w];
      out[k] = v;
    }
    __syncthreads();
  }
}

void launch_dot(int64_t n, const double *a, const double *b, double *partial, double *out, cudaStream_t st) {
  k_dot_partial<1><<<DOT_BLOCKS, 256, 0, st>>>(n, a, b, nullptr, partial);
  k_dot_final<1><<<1, 256, 0, st>>>(partial, out);
}

void launch_dot2(int64_t n, const double *a, const double *b, const double *c, double *partial, double *out,
                 cudaStream_t st) {
  k_dot_partial<2><<<DOT_BLOCKS, 256, 0, st>>>(n, a, b, c, partial);
  k_dot_final<2><<<1, 256, 0, st>>>(partial, out);
}

template <typename Ta, typename Tb>
__global__ void k_convert(int64_t n, const Ta *__restrict__ a, Tb *__restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = Tb(a[i]);
}
template <typename Ta, typename Tb>
void launch_convert(int64_t n, const Ta *a, Tb *b, cudaStream_t st) {
  k_convert<Ta, Tb><<<gs_blocks(n), 256, 0, st>>>(n, a, b);
}

template <typename T>
__global__ void k_axpby(int64_t n, T alpha, const T *__restrict__ x, T beta, const T *__restrict__ y, T *__restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = alpha * x[i] + beta * y[i];
}
template <typename T>
void launch_axpby(int64_t n, T alpha, const T *x, T beta, const T *y, T *z, cudaStream_t st) {
  k_axpby<T><<<gs_blocks(n), 256, 0, st>>>(n, alpha, x, beta, y, z);
}
template <typename T>
void launch_sub(int64_t n, const T *x, const T *y, T *z, cudaStream_t st) {
  k_axpby<T><<<gs_blocks(n), 256, 0, st>>>(n, T(1), x, T(-1), y, z);
}
template <typename T>
__global__ void k_add(int64_t n, const T *__restrict__ x, T *__restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}
template <typename T>
void launch_add(int64_t n, const T *x, T *y, cudaStream_t st) {
  k_add<T><<<gs_blocks(n), 256, 0, st>>>(n, x, y);
}

// PCG scalars sc[]: 0 rz, 1 alpha, 2 beta, 3 dq, 4 rr, 5 rz_new, 6 r.z_old, 7 flexible flag, 8 nonfinite flag
__global__ void k_pcg_scalars(int which, double *sc, const double *dots) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (which == 0) {  // alpha = rz / (d.q)
    sc[3] = dots[0];
    double a = sc[0] / sc[3];
    if (!isfinite(a)) sc[8] = 1.0;
    sc[1] = isfinite(a) ? a : 0.0;
  } else if (which == 1) {  // beta = (r.z - flex * r.z_old) / rz_prev
    double rz = dots[0];
    double num = sc[7] != 0.0 ? rz - dots[1] : rz;
    double b = num / sc[0];
    if (!isfinite(b)) sc[8] = 1.0;
    sc[2] = isfinite(b) ? b : 0.0;
    sc[0] = rz;
  } else if (which == 2) {  // initial rz
    sc[0] = dots[0];
    if (!isfinite(sc[0])) sc[8] = 1.0;
  }
}
void launch_pcg_scalars(int which, double *sc, const double *dots, cudaStream_t st) {
  k_pcg_scalars<<<1, 32, 0, st>>>(which, sc, dots);
}

__global__ void k_pcg_update_xr(int64_t n, const double *__restrict__ sc, const double *__restrict__ d,
                                const double *__restrict__ q, double *__restrict__ x, double *__restrict__ r) {
  const double alpha = sc[1];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * d[i];
    r[i] -= alpha * q[i];
  }
}
void launch_pcg_update_xr(int64_t n, const double *sc, const double *d, const double *q, double *x, double *r,
                          cudaStream_t st) {
  k_pcg_update_xr<<<gs_blocks(n), 256, 0, st>>>(n, sc, d, q, x, r);
}
__global__ void k_pcg_update_d(int64_t n, const double *__restrict__ sc, const double *__restrict__ z, double *__restrict__ d) {
  const double beta = sc[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = z[i] + beta * d[i];
}
void launch_pcg_update_d(int64_t n, const double *sc, const double *z, double *d, cudaStream_t st) {
  k_pcg_update_d<<<gs_blocks(n), 256, 0, st>>>(n, sc, z, d);
}

// ------------------------------------------------------------------ instantiations
template void launch_operator<double, double, double>(const OpArgs &, bool, const double *, double *, double *, cudaStream_t);
template void launch_operator<float, float, float>(const OpArgs &, bool, const float *, float *, float *, cudaStream_t);
template void launch_operator<double, double, float>(const OpArgs &, bool, const double *, float *, double *, cudaStream_t);
template void launch_coarse_restrict<double, double>(const Grid &, const double *, const double *, const int *, double *, double *, cudaStream_t);
template void launch_coarse_restrict<float, float>(const Grid &, const float *, const float *, const int *, float *, float *, cudaStream_t);
template void launch_dense_symv<double>(int, const double *, const double *, double *, cudaStream_t);
template void launch_dense_symv<float>(int, const float *, const float *, float *, cudaStream_t);
template void launch_coarse_prolong<double, double>(const Grid &, const double *, const double *, const int *, double *, bool, cudaStream_t);
template void launch_coarse_prolong<float, float>(const Grid &, const float *, const float *, const int *, float *, bool, cudaStream_t);
template void launch_convert<double, float>(int64_t, const double *, float *, cudaStream_t);
template void launch_convert<float, double>(int64_t, const float *, double *, cudaStream_t);
template void launch_axpby<double>(int64_t, double, const double *, double, const double *, double *, cudaStream_t);
template void launch_axpby<float>(int64_t, float, const float *, float, const float *, float *, cudaStream_t);
template void launch_sub<double>(int64_t, const double *, const double *, double *, cudaStream_t);
template void launch_sub<float>(int64_t, const float *, const float *, float *, cudaStream_t);
template void launch_add<double>(int64_t, const double *, double *, cudaStream_t);
template void launch_add<float>(int64_t, const float *, float *, cudaStream_t);

}  // namespace fdm
