// Kernels of the GPU apply on general hexahedral meshes (Sections 2.4-2.7):
// the vertex-star relaxation in the glued FDM basis and the stiffness apply by
// Gauss quadrature with the geometry factors of the trilinear map.
//
// One relaxation sweep z = omega sum_v R_v^T A~_v^{-1} R_v r is five kernels:
//   restrict:  per cell, E_e = (T^T)^{x3} (r / multiplicity)_e in the cell's
//              local FDM basis, then the cell's share of the Schur condensation:
//              every face function c (one vertex index along axis d) gets
//              E_e[c] - sum_m a_d(c, m) E_e[m] / D_e[m] over the interior line
//              through it.  The interior block of a star's surrogate matrix is
//              diagonal and each interior function lies in one cell, so the
//              condensation is the same for every star holding c;
//   assemble:  per FDM slot, the signed sum of its cells' condensed values (by
//              cell: deterministic);
//   star:      per star, the interface solve with the Schur-coupling factors
//              (level-scheduled sparse solves with L_BB, S_TB, the symmetric W);
//   slot sum:  per interface slot, the sum of the star solutions holding it;
//   interp:    per cell, the interface functions from the slot sums (signed),
//              the interior functions by the summed back-substitution
//              z_i = (m_e E_e[i] - sum_j a(i, j) z_j) / D_e[i] (m_e: the stars
//              holding the cell's interior), T^{x3} back to nodal values,
//              omega, and the node written by its owner cell.
// The surrogate couplings a are mu_d Af along axis d times Bf along the
// others (the structural zeros of Bf make the interior block diagonal); D is
// the same sum at the interior function itself.
#include <algorithm>

#include "hexdev.h"
#include "internal.h"

namespace fdm {
namespace {

// out = M' along axis ax of the n^3 tensor in (x fastest): trans ? out[i] =
// sum_m M[m][i] in[m] : out[i] = sum_m M[i][m] in[m]; acc adds to out
template <typename T>
__device__ __forceinline__ void tpass(const T *M, bool trans, int ax, const T *in, T *out, int n, bool acc) {
  const int n3 = n * n * n, s = ax == 0 ? 1 : (ax == 1 ? n : n * n);
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    const int i = (idx / s) % n, base = idx - i * s;
    T a = 0;
    if (trans)
      for (int m = 0; m < n; ++m) a += M[m * n + i] * in[base + m * s];
    else
      for (int m = 0; m < n; ++m) a += M[i * n + m] * in[base + m * s];
    out[idx] = acc ? out[idx] + a : a;
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void load_tab(const HexDev<T> &d, T *st) {
  const int m = 5 * d.n * d.n + d.n;
  for (int i = threadIdx.x; i < m; i += blockDim.x) st[i] = d.tab[i];
  __syncthreads();
}

// D_e at the interior function (i, j, k) and the coupling of the face
// function with index `side` along axis ax to the interior function c
template <typename T>
__device__ __forceinline__ T diag_at(const T *Af, const T *Bf, const T *mu, int n, int i, int j, int k) {
  return mu[0] * Af[i * n + i] * Bf[j * n + j] * Bf[k * n + k] + mu[1] * Bf[i * n + i] * Af[j * n + j] * Bf[k * n + k] +
         mu[2] * Bf[i * n + i] * Bf[j * n + j] * Af[k * n + k];
}

__device__ __forceinline__ int vertex_axis_count(int i, int j, int k, int p, int &ax) {
  int c = 0;
  ax = -1;
  if (i == 0 || i == p) { ++c; ax = 0; }
  if (j == 0 || j == p) { ++c; ax = 1; }
  if (k == 0 || k == p) { ++c; ax = 2; }
  return c;
}

template <typename T, typename Tin>
__global__ void __launch_bounds__(128) k_hex_restrict(HexDev<T> d, const Tin *__restrict__ r, T *__restrict__ CE) {
  extern __shared__ __align__(16) unsigned char smem_[];
  const int n = d.n, p = d.p, n3 = n * n * n, e = blockIdx.x;
  T *tab = reinterpret_cast<T *>(smem_);
  T *A = tab + ((5 * n * n + n + 1) & ~1), *B = A + n3;
  load_tab(d, tab);
  const T *Tm = tab + htab(HTAB_T, n), *Af = tab + htab(HTAB_AF, n), *Bf = tab + htab(HTAB_BF, n);
  const int *cn = d.cell_nodes + (int64_t)e * n3;
  for (int l = threadIdx.x; l < n3; l += blockDim.x) {
    const int g = cn[l];
    A[l] = d.dirichlet[g] ? T(0) : T(r[g]) * d.inv_mult[g];
  }
  __syncthreads();
  tpass(Tm, true, 0, A, B, n, false);
  tpass(Tm, true, 1, B, A, n, false);
  tpass(Tm, true, 2, A, B, n, false);
  const T mu[3] = {d.mu[3 * e], d.mu[3 * e + 1], d.mu[3 * e + 2]};
  T *out = CE + (int64_t)e * n3;
  for (int c = threadIdx.x; c < n3; c += blockDim.x) {
    const int i = c % n, j = (c / n) % n, k = c / (n * n);
    int ax;
    T v = B[c];
    if (p >= 2 && vertex_axis_count(i, j, k, p, ax) == 1) {  // a face function: condense over its line
      const int idx[3] = {i, j, k}, side = idx[ax], o1 = idx[(ax + 1) % 3], o2 = idx[(ax + 2) % 3];
      const int s = ax == 0 ? 1 : (ax == 1 ? n : n * n);
      const T bb = Bf[o1 * n + o1] * Bf[o2 * n + o2];
      T acc = 0;
      for (int m = 1; m < p; ++m) {
        int q[3] = {i, j, k};
        q[ax] = m;
        acc += mu[ax] * Af[side * n + m] * bb * B[c + (m - side) * s] / diag_at(Af, Bf, mu, n, q[0], q[1], q[2]);
      }
      v -= acc;
    }
    out[c] = v;
  }
}

template <typename T>
__global__ void k_hex_assemble(HexDev<T> d, const T *__restrict__ CE, T *__restrict__ rc) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < d.nnode; g += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int64_t t = d.slot_cells_ptr[g]; t < d.slot_cells_ptr[g + 1]; ++t) {
      const int ec = d.slot_cells[t];
      s += d.cell_sign[ec] > 0 ? CE[ec] : -CE[ec];
    }
    rc[g] = s;
  }
}

template <typename T>
__global__ void k_hex_slot_stars(HexDev<T> d, const T *__restrict__ X, T *__restrict__ zf) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < d.nnode; g += (int64_t)gridDim.x * blockDim.x) {
    T s = 0;
    for (int64_t t = d.slot_stars_ptr[g]; t < d.slot_stars_ptr[g + 1]; ++t) {
      const HexStarDev &S = d.stars[d.slot_stars[2 * t]];
      const int pos = d.slot_stars[2 * t + 1];
      if (pos >= S.ni) s += X[S.xoff + pos - S.ni];
    }
    zf[g] = s;
  }
}

template <typename T, typename Tout>
__global__ void __launch_bounds__(128) k_hex_interp(HexDev<T> d, const T *__restrict__ CE, const T *__restrict__ zf,
                                                    T omega, Tout *__restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_[];
  const int n = d.n, p = d.p, n3 = n * n * n, e = blockIdx.x;
  T *tab = reinterpret_cast<T *>(smem_);
  T *A = tab + ((5 * n * n + n + 1) & ~1), *B = A + n3;
  load_tab(d, tab);
  const T *Tm = tab + htab(HTAB_T, n), *Af = tab + htab(HTAB_AF, n), *Bf = tab + htab(HTAB_BF, n);
  const int64_t e0 = (int64_t)e * n3;
  for (int c = threadIdx.x; c < n3; c += blockDim.x) {
    const int i = c % n, j = (c / n) % n, k = c / (n * n);
    int ax;
    if (vertex_axis_count(i, j, k, p, ax) > 0) {
      const T v = zf[d.cell_fdm[e0 + c]];
      A[c] = d.cell_sign[e0 + c] > 0 ? v : -v;
    }
  }
  __syncthreads();
  if (p >= 2) {
    const T mu[3] = {d.mu[3 * e], d.mu[3 * e + 1], d.mu[3 * e + 2]};
    const T me = T(d.cell_m[e]);
    for (int c = threadIdx.x; c < n3; c += blockDim.x) {
      const int idx[3] = {c % n, (c / n) % n, c / (n * n)};
      int ax;
      if (vertex_axis_count(idx[0], idx[1], idx[2], p, ax) > 0) continue;
      T s = me * CE[e0 + c];
      for (int a = 0; a < 3; ++a) {
        const int st = a == 0 ? 1 : (a == 1 ? n : n * n);
        const int o1 = idx[(a + 1) % 3], o2 = idx[(a + 2) % 3];
        const T bb = Bf[o1 * n + o1] * Bf[o2 * n + o2];
        for (int side = 0; side <= p; side += p)
          s -= mu[a] * Af[idx[a] * n + side] * bb * A[c + (side - idx[a]) * st];
      }
      A[c] = s / diag_at(Af, Bf, mu, n, idx[0], idx[1], idx[2]);
    }
    __syncthreads();
  }
  tpass(Tm, false, 0, A, B, n, false);
  tpass(Tm, false, 1, B, A, n, false);
  tpass(Tm, false, 2, A, B, n, false);
  const int *cn = d.cell_nodes + e0;
  for (int l = threadIdx.x; l < n3; l += blockDim.x) {
    const int g = cn[l];
    if (d.node_owner[g] == e0 + l) z[g] = d.dirichlet[g] ? Tout(0) : Tout(omega * B[l]);
  }
}

}  // namespace

template <typename T>
static size_t hex_cell_smem(int n, int buffers) {
  return sizeof(T) * ((size_t)((5 * n * n + n + 1) & ~1) + (size_t)buffers * n * n * n);
}

template <typename K>
static void hex_set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) FDM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

static int hex_blocks(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16)); }

template <typename T, typename Tin>
void launch_hex_restrict(const HexDev<T> &d, const Tin *r, T *CE, cudaStream_t st) {
  const size_t sm = hex_cell_smem<T>(d.n, 2);
  hex_set_smem(k_hex_restrict<T, Tin>, sm);
  k_hex_restrict<T, Tin><<<d.nc, 128, sm, st>>>(d, r, CE);
}

template <typename T>
void launch_hex_assemble(const HexDev<T> &d, const T *CE, T *rc, cudaStream_t st) {
  k_hex_assemble<T><<<hex_blocks(d.nnode), 256, 0, st>>>(d, CE, rc);
}

template <typename T>
void launch_hex_slot_stars(const HexDev<T> &d, const T *X, T *zf, cudaStream_t st) {
  k_hex_slot_stars<T><<<hex_blocks(d.nnode), 256, 0, st>>>(d, X, zf);
}

template <typename T, typename Tout>
void launch_hex_interp(const HexDev<T> &d, const T *CE, const T *zf, double omega, Tout *z, cudaStream_t st) {
  const size_t sm = hex_cell_smem<T>(d.n, 2);
  hex_set_smem(k_hex_interp<T, Tout>, sm);
  k_hex_interp<T, Tout><<<d.nc, 128, sm, st>>>(d, CE, zf, T(omega), z);
}

namespace {

// out = L_BB^{-1} in (forward, by levels) and io = L_BB^{-T} io (backward, by levels)
template <typename T>
__device__ __forceinline__ void lbb_forward(const HexClassDev &C, const int *ct, const T *v, const T *in, T *out) {
  const int *lev = ct + C.lev_f, *rows = ct + C.rows_f, *lptr = ct + C.lptr, *lcol = ct + C.lcol, *lpos = ct + C.lpos,
            *ldiag = ct + C.ldiag;
  for (int lv = 0; lv < C.nlf; ++lv) {
    for (int q = lev[lv] + threadIdx.x; q < lev[lv + 1]; q += blockDim.x) {
      const int r = rows[q];
      T s = in[r];
      for (int e = lptr[r]; e < lptr[r + 1]; ++e) s -= v[lpos[e]] * out[lcol[e]];
      out[r] = s / v[ldiag[r]];
    }
    __syncthreads();
  }
}
template <typename T>
__device__ __forceinline__ void lbb_backward(const HexClassDev &C, const int *ct, const T *v, T *io) {
  const int *lev = ct + C.lev_b, *rows = ct + C.rows_b, *tptr = ct + C.tptr, *trow = ct + C.trow, *tpos = ct + C.tpos,
            *ldiag = ct + C.ldiag;
  for (int lv = 0; lv < C.nlb; ++lv) {
    for (int q = lev[lv] + threadIdx.x; q < lev[lv + 1]; q += blockDim.x) {
      const int r = rows[q];
      T s = io[r];
      for (int e = tptr[r]; e < tptr[r + 1]; ++e) s -= v[tpos[e]] * io[trow[e]];
      io[r] = s / v[ldiag[r]];
    }
    __syncthreads();
  }
}

// one CTA per star: the interface solve S_G x = g in the Schur-coupling form
//   y_B = S_BB^{-1} g_B, x_T = W (g_T - S_TB y_B), x_B = y_B - S_BB^{-1} S_BT x_T
template <typename T>
__global__ void __launch_bounds__(256) k_hex_star(HexDev<T> d, const T *__restrict__ rc, T *__restrict__ X, int cap) {
  extern __shared__ __align__(16) unsigned char smem_[];
  const HexStarDev S = d.stars[blockIdx.x];
  const HexClassDev C = d.classes[S.cls];
  const int nG = S.nG, nB = C.nB, t = C.t;
  if (nG == 0) return;
  T *g = reinterpret_cast<T *>(smem_), *x = g + cap, *y = x + cap;
  const T *v = d.vals + S.voff;
  const int *ct = d.ct;
  const int *nodes = d.star_nodes + S.nodes_off + S.ni;
  for (int j = threadIdx.x; j < nG; j += blockDim.x) g[j] = rc[nodes[j]];
  __syncthreads();
  if (nB > 0) {
    lbb_forward(C, ct, v, g, y);
    lbb_backward(C, ct, v, y);
  }
  const int *stptr = ct + C.stptr, *stcol = ct + C.stcol;
  for (int r = threadIdx.x; r < t; r += blockDim.x) {  // v_T = g_T - S_TB y_B
    T s = g[nB + r];
    for (int q = stptr[r]; q < stptr[r + 1]; ++q) s -= v[C.off_st + q] * y[stcol[q]];
    g[nB + r] = s;
  }
  __syncthreads();
  const T *W = v + C.off_w, *vt = g + nB;
  for (int r = threadIdx.x; r < t; r += blockDim.x) {  // x_T = W v_T (lower triangle by rows)
    const T *row = W + (int64_t)r * (r + 1) / 2;
    T s = 0;
    for (int c = 0; c <= r; ++c) s += row[c] * vt[c];
    for (int c = r + 1; c < t; ++c) s += W[(int64_t)c * (c + 1) / 2 + r] * vt[c];
    x[nB + r] = s;
  }
  __syncthreads();
  if (nB > 0) {
    const int *sbtptr = ct + C.sbtptr, *sbtrow = ct + C.sbtrow, *sbtpos = ct + C.sbtpos;
    for (int c = threadIdx.x; c < nB; c += blockDim.x) {  // r_B = S_BT x_T, over g_B
      T s = 0;
      for (int q = sbtptr[c]; q < sbtptr[c + 1]; ++q) s += v[sbtpos[q]] * x[nB + sbtrow[q]];
      g[c] = s;
    }
    __syncthreads();
    lbb_forward(C, ct, v, g, x);
    lbb_backward(C, ct, v, x);
    for (int c = threadIdx.x; c < nB; c += blockDim.x) x[c] = y[c] - x[c];
    __syncthreads();
  }
  for (int j = threadIdx.x; j < nG; j += blockDim.x) X[S.xoff + j] = x[j];
}

// stiffness per cell: gradients at the Gauss points (V along two axes, D along
// the third), the flux G grad with the six geometry factors, and the
// transposed contractions back to the nodes; cell-local result Y_e
template <typename T, typename Tin>
__global__ void __launch_bounds__(128) k_hex_op(HexDev<T> d, const Tin *__restrict__ u, T *__restrict__ Y) {
  extern __shared__ __align__(16) unsigned char smem_[];
  const int n = d.n, n3 = n * n * n, e = blockIdx.x;
  T *tab = reinterpret_cast<T *>(smem_);
  T *U = tab + ((5 * n * n + n + 1) & ~1), *A = U + n3, *B = A + n3, *Cx = B + n3, *Dy = Cx + n3;
  load_tab(d, tab);
  const T *Vq = tab + htab(HTAB_VQ, n), *Dq = tab + htab(HTAB_DQ, n);
  const int64_t e0 = (int64_t)e * n3;
  const int *cn = d.cell_nodes + e0;
  for (int l = threadIdx.x; l < n3; l += blockDim.x) {
    const int g = cn[l];
    U[l] = d.dirichlet[g] ? T(0) : T(u[g]);
  }
  __syncthreads();
  tpass(Vq, false, 2, U, A, n, false);   // A = Vz U
  tpass(Vq, false, 1, A, B, n, false);   // B = Vy Vz U
  tpass(Dq, false, 0, B, Cx, n, false);  // Cx = grad_x
  tpass(Vq, false, 0, A, B, n, false);   // B = Vx Vz U
  tpass(Dq, false, 1, B, Dy, n, false);  // Dy = grad_y
  tpass(Vq, false, 0, U, A, n, false);   // A = Vx U
  tpass(Vq, false, 1, A, B, n, false);   // B = Vx Vy U
  tpass(Dq, false, 2, B, A, n, false);   // A = grad_z
  const T *G = d.geom + e0 * 6;
  for (int q = threadIdx.x; q < n3; q += blockDim.x) {
    const T gx = Cx[q], gy = Dy[q], gz = A[q];
    const T *Gq = G + 6 * q;
    Cx[q] = Gq[0] * gx + Gq[3] * gy + Gq[4] * gz;
    Dy[q] = Gq[3] * gx + Gq[1] * gy + Gq[5] * gz;
    A[q] = Gq[4] * gx + Gq[5] * gy + Gq[2] * gz;
  }
  __syncthreads();
  tpass(Dq, true, 0, Cx, B, n, false);   // B = Dx^T fx
  tpass(Vq, true, 1, B, U, n, false);    // U = Vy^T Dx^T fx
  tpass(Vq, true, 0, Dy, B, n, false);   // B = Vx^T fy
  tpass(Dq, true, 1, B, U, n, true);     // U += Dy^T Vx^T fy
  tpass(Vq, true, 2, U, Cx, n, false);   // Cx = Vz^T (...)
  tpass(Vq, true, 0, A, B, n, false);    // B = Vx^T fz
  tpass(Vq, true, 1, B, Dy, n, false);   // Dy = Vy^T Vx^T fz
  tpass(Dq, true, 2, Dy, Cx, n, true);   // Cx += Dz^T Vy^T Vx^T fz
  for (int l = threadIdx.x; l < n3; l += blockDim.x) Y[e0 + l] = Cx[l];
}

template <typename T, typename Tout>
__global__ void k_hex_gather(HexDev<T> d, const T *__restrict__ Y, const Tout *__restrict__ rsub, Tout *__restrict__ y) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < d.nnode; g += (int64_t)gridDim.x * blockDim.x) {
    if (d.dirichlet[g]) {
      y[g] = Tout(0);
      continue;
    }
    T s = 0;
    for (int64_t t = d.node_cells_ptr[g]; t < d.node_cells_ptr[g + 1]; ++t) s += Y[d.node_cells[t]];
    y[g] = rsub ? Tout(T(rsub[g]) - s) : Tout(s);
  }
}

template <typename T>
__device__ __forceinline__ T hat_at(const T *xi, int n, int l, int corner) {
  const int i = l % n, j = (l / n) % n, k = l / (n * n);
  const T hx = (corner & 1) ? T(0.5) * (T(1) + xi[i]) : T(0.5) * (T(1) - xi[i]);
  const T hy = ((corner >> 1) & 1) ? T(0.5) * (T(1) + xi[j]) : T(0.5) * (T(1) - xi[j]);
  const T hz = (corner >> 2) ? T(0.5) * (T(1) + xi[k]) : T(0.5) * (T(1) - xi[k]);
  return hx * hy * hz;
}

// rc = P^T r in two deterministic steps: per cell (one CTA) the 8 corner
// sums C_e[c] = sum_l hat_c(l) r_l / multiplicity_l over its nodes (a fixed
// tree over the threads), then per coarse unknown the sum of C over the
// (cell, corner) pairs of its vertex in cell order (r / multiplicity counts
// every node once)
template <typename T>
__global__ void __launch_bounds__(128) k_hex_coarse_cells(HexDev<T> d, const T *__restrict__ r, T *__restrict__ Cc) {
  __shared__ T red[8][128];
  const int n = d.n, n3 = n * n * n, e = blockIdx.x, tid = threadIdx.x;
  const T *xi = d.tab + htab(HTAB_XI, n);
  const int *cn = d.cell_nodes + (int64_t)e * n3;
  T acc[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) acc[c] = 0;
  for (int l = tid; l < n3; l += 128) {
    const int g = cn[l];
    if (d.dirichlet[g]) continue;
    const T v = r[g] * d.inv_mult[g];
    const int i = l % n, j = (l / n) % n, k = l / (n * n);
    const T hx[2] = {T(0.5) * (T(1) - xi[i]), T(0.5) * (T(1) + xi[i])};
    const T hy[2] = {T(0.5) * (T(1) - xi[j]), T(0.5) * (T(1) + xi[j])};
    const T hz[2] = {T(0.5) * (T(1) - xi[k]), T(0.5) * (T(1) + xi[k])};
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += hx[c & 1] * hy[(c >> 1) & 1] * hz[c >> 2] * v;
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) red[c][tid] = acc[c];
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (tid < w)
#pragma unroll
      for (int c = 0; c < 8; ++c) red[c][tid] += red[c][tid + w];
    __syncthreads();
  }
  if (tid < 8) Cc[8 * (int64_t)e + tid] = red[tid][0];
}

template <typename T>
__global__ void k_hex_coarse_sum(HexDev<T> d, const T *__restrict__ Cc, T *__restrict__ rc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.nco) return;
  T s = 0;
  for (int64_t q = d.vcell_ptr[k]; q < d.vcell_ptr[k + 1]; ++q) s += Cc[d.vcell[q]];
  rc[k] = s;
}

// x += P xc at every free node, evaluated in the node's owner cell
template <typename T>
__global__ void k_hex_coarse_prolong(HexDev<T> d, const T *__restrict__ xc, T *__restrict__ x) {
  const int n = d.n, n3 = n * n * n;
  const T *xi = d.tab + htab(HTAB_XI, n);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < d.nnode; g += (int64_t)gridDim.x * blockDim.x) {
    if (d.dirichlet[g]) continue;
    const int own = d.node_owner[g], e = own / n3, l = own % n3;
    T s = 0;
    for (int c = 0; c < 8; ++c) {
      const int k = d.coarse_of[d.cells8[8 * e + c]];
      if (k >= 0) s += hat_at(xi, n, l, c) * xc[k];
    }
    x[g] += s;
  }
}

}  // namespace

template <typename T>
void launch_hex_star_solve(const HexDev<T> &d, const T *rc, T *X, int maxG, cudaStream_t st) {
  if (d.nstar <= 0) return;
  const int cap = (maxG + 3) & ~3;
  const size_t sm = sizeof(T) * 3 * (size_t)cap;
  hex_set_smem(k_hex_star<T>, sm);
  k_hex_star<T><<<d.nstar, 256, sm, st>>>(d, rc, X, cap);
}

template <typename T, typename Tin>
void launch_hex_op_cells(const HexDev<T> &d, const Tin *u, T *Y, cudaStream_t st) {
  const size_t sm = hex_cell_smem<T>(d.n, 5);
  hex_set_smem(k_hex_op<T, Tin>, sm);
  k_hex_op<T, Tin><<<d.nc, 128, sm, st>>>(d, u, Y);
}

template <typename T, typename Tout>
void launch_hex_gather(const HexDev<T> &d, const T *Y, const Tout *rsub, Tout *y, cudaStream_t st) {
  k_hex_gather<T, Tout><<<hex_blocks(d.nnode), 256, 0, st>>>(d, Y, rsub, y);
}

template <typename T>
void launch_hex_coarse_restrict(const HexDev<T> &d, const T *r, T *Cc, T *rc, cudaStream_t st) {
  if (d.nco <= 0) return;
  k_hex_coarse_cells<T><<<d.nc, 128, 0, st>>>(d, r, Cc);
  k_hex_coarse_sum<T><<<(d.nco + 127) / 128, 128, 0, st>>>(d, Cc, rc);
}

template <typename T>
void launch_hex_coarse_prolong(const HexDev<T> &d, const T *xc, T *x, cudaStream_t st) {
  if (d.nco <= 0) return;
  k_hex_coarse_prolong<T><<<hex_blocks(d.nnode), 256, 0, st>>>(d, xc, x);
}

#define FDM_HEX_INST(T)                                                                                   \
  template void launch_hex_restrict<T, T>(const HexDev<T> &, const T *, T *, cudaStream_t);               \
  template void launch_hex_assemble<T>(const HexDev<T> &, const T *, T *, cudaStream_t);                   \
  template void launch_hex_star_solve<T>(const HexDev<T> &, const T *, T *, int, cudaStream_t);           \
  template void launch_hex_slot_stars<T>(const HexDev<T> &, const T *, T *, cudaStream_t);                 \
  template void launch_hex_interp<T, T>(const HexDev<T> &, const T *, const T *, double, T *, cudaStream_t); \
  template void launch_hex_op_cells<T, T>(const HexDev<T> &, const T *, T *, cudaStream_t);               \
  template void launch_hex_gather<T, T>(const HexDev<T> &, const T *, const T *, T *, cudaStream_t);       \
  template void launch_hex_coarse_restrict<T>(const HexDev<T> &, const T *, T *, T *, cudaStream_t);       \
  template void launch_hex_coarse_prolong<T>(const HexDev<T> &, const T *, T *, cudaStream_t);
FDM_HEX_INST(double)
FDM_HEX_INST(float)

}  // namespace fdm

namespace fdm {
namespace {

template <typename T> struct H4 { T x, y, z, w; };
__device__ __forceinline__ H4<float> ld4g(const float *p) {
  const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ H4<double> ld4g(const double *p) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  return {a.x, a.y, b.x, b.y};
}
__device__ __forceinline__ H4<float> ld4s(const float *p) {
  const float4 v = *reinterpret_cast<const float4 *>(p);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ H4<double> ld4s(const double *p) {
  const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
  return {a.x, a.y, b.x, b.y};
}

// one CTA of 8 warps per star: x = S^{-1} g with the lower triangle of the
// symmetric S^{-1} by rows.  Warp w takes the row blocks w, w + 8, ... (RB
// rows each); lane l owns the column groups q4 = l + 32 q (q < NQ), reads them
// for each row, adds the row dot (warp sum) and keeps the strictly lower
// entries times g_r as column sums in registers; the warps' column sums are
// added in warp order after the row dots (deterministic).
template <typename T, int NQ, int RB>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2) k_hex_star_dense(HexDev<T> d, const T *__restrict__ rc,
                                                                              T *__restrict__ X,
                                                                              const int *__restrict__ list, int cap) {
  extern __shared__ __align__(16) unsigned char smem_[];
  const HexStarDev S = d.stars[list[blockIdx.x]];
  const int nG = S.nG;
  if (nG == 0) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T *g = reinterpret_cast<T *>(smem_), *x = g + cap, *colbuf = x + cap;  // colbuf [8][cap]
  const int *zoff = d.ct + d.classes[S.cls].zoff;
  const T *Wv = d.vals + S.voff;
  const int *nodes = d.star_nodes + S.nodes_off + S.ni;
  for (int j = threadIdx.x; j < cap; j += blockDim.x) g[j] = j < nG ? rc[nodes[j]] : T(0);
  __syncthreads();
  T cacc[NQ][4];
#pragma unroll
  for (int q = 0; q < NQ; ++q)
#pragma unroll
    for (int i = 0; i < 4; ++i) cacc[q][i] = 0;
  for (int r0 = warp * RB; r0 < nG; r0 += 8 * RB) {
    H4<T> wr[RB][NQ];
    T gr[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int r = r0 + u < nG ? r0 + u : nG - 1;
      const int z0 = __ldg(zoff + r), ng = r0 + u < nG ? (__ldg(zoff + r + 1) - z0) / 4 : 0;
      gr[u] = r0 + u < nG ? g[r] : T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int q4 = lane + 32 * q;
        wr[u][q] = q4 < ng ? ld4g(Wv + z0 + 4 * q4) : H4<T>{0, 0, 0, 0};
      }
    }
    T rs[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int r = r0 + u;
      T s = 0;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int cb = 4 * (lane + 32 * q);
        const H4<T> &w = wr[u][q];
        if (cb < cap) {
          const H4<T> v = ld4s(g + cb);
          s += w.x * v.x + w.y * v.y + w.z * v.z + w.w * v.w;
        }
        cacc[q][0] += (cb < r ? w.x : T(0)) * gr[u];
        cacc[q][1] += (cb + 1 < r ? w.y : T(0)) * gr[u];
        cacc[q][2] += (cb + 2 < r ? w.z : T(0)) * gr[u];
        cacc[q][3] += (cb + 3 < r ? w.w : T(0)) * gr[u];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      rs[u] = s;
    }
    if (lane < RB && r0 + lane < nG) {
      T s = rs[0];
#pragma unroll
      for (int u = 1; u < RB; ++u) s = lane == u ? rs[u] : s;
      x[r0 + lane] = s;
    }
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int cb = 4 * (lane + 32 * q);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (cb + i < cap) colbuf[warp * cap + cb + i] = cacc[q][i];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < nG; c += blockDim.x) {
    T s = x[c];
    for (int w = 0; w < 8; ++w) s += colbuf[w * cap + c];
    X[S.xoff + c] = s;
  }
}

}  // namespace

template <typename T, int NQ, int RB>
void star_dense_bin(const HexDev<T> &d, const T *rc, T *X, const int *list, int count, int maxg, cudaStream_t st) {
  if (count <= 0) return;
  const int cap = (maxg + 3) & ~3;
  const size_t sm = sizeof(T) * 10 * (size_t)cap;
  hex_set_smem(k_hex_star_dense<T, NQ, RB>, sm);
  k_hex_star_dense<T, NQ, RB><<<count, 256, sm, st>>>(d, rc, X, list, cap);
}

// the stars in three launches by interface size (at most 256, 512, 1024 values),
// each with the column groups per lane that its rows need and more rows in
// flight per warp where the rows are short
template <typename T>
void launch_hex_star_dense(const HexDev<T> &d, const T *rc, T *X, const int *list, const int count[3],
                           const int maxg[3], unsigned bins, cudaStream_t st) {
  if (d.nstar <= 0) return;
  if (maxg[2] > 1024) fail(FDM_EINVAL, "dense star solve: interface larger than 1024");
  if (bins & 4u) star_dense_bin<T, 8, 2>(d, rc, X, list + count[0] + count[1], count[2], maxg[2], st);
  if (bins & 2u) star_dense_bin<T, 4, 4>(d, rc, X, list + count[0], count[1], maxg[1], st);
  if (bins & 1u) star_dense_bin<T, 2, 8>(d, rc, X, list, count[0], maxg[0], st);
}
template void launch_hex_star_dense<double>(const HexDev<double> &, const double *, double *, const int *,
                                            const int[3], const int[3], unsigned, cudaStream_t);
template void launch_hex_star_dense<float>(const HexDev<float> &, const float *, float *, const int *, const int[3],
                                           const int[3], unsigned, cudaStream_t);

}  // namespace fdm
