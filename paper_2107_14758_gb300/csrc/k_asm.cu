// Additive vertex-star relaxation kernels (Sections 2.4-2.6 of the paper):
//   restrict: per cell, E_K = (T^T (x) T^T (x) T^T)(W_K r_K)  (FDM-basis residual)
//   patch:    per vertex star, gather + Schur condensation + sparse Cholesky
//             forward/backward solves + interior back-substitution
//   interp:   per cell, sum of the star solutions covering each node (fixed
//             order), z_K = (T (x) T (x) T) z_fdm, omega scaling, owner write.
#include "device.cuh"
#include "kernels.h"

namespace fdm {

// ------------------------------------------------------------------ helpers
template <typename T>
__device__ __forceinline__ void contract_axis(const T *__restrict__ in, T *__restrict__ out,
                                              const T *__restrict__ M, bool transpose, int axis, int n,
                                              int tid, int nt) {
  // out[.., i, ..] = sum_m M'[i][m] in[.., m, ..] along `axis`, with
  // M' = M (transpose = false) or M^T (transpose = true); M row-major n x n.
  const int n3 = n * n * n;
  const int stride = axis == 0 ? 1 : (axis == 1 ? n : n * n);
  for (int idx = tid; idx < n3; idx += nt) {
    int i = (idx / stride) % n;
    int base = idx - i * stride;
    T acc = 0;
    if (transpose) {
      for (int m = 0; m < n; ++m) acc += M[m * n + i] * in[base + m * stride];
    } else {
      for (int m = 0; m < n; ++m) acc += M[i * n + m] * in[base + m * stride];
    }
    out[idx] = acc;
  }
}

// ------------------------------------------------------------------ restrict
template <typename T, typename Tin>
__global__ void __launch_bounds__(256) k_restrict_fdm(Grid g, const Tin *__restrict__ r, const T *__restrict__ tab,
                                                      T *__restrict__ E) {
  extern __shared__ unsigned char smem_[];
  T *sT = reinterpret_cast<T *>(smem_);
  const int n = g.n, p = g.p, n3 = n * n * n;
  T *b0 = sT + n * n, *b1 = b0 + n3;
  const int cell = blockIdx.x;
  const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) sT[i] = tab[tab_off(TAB_T, n) + i];
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
    int gx = cx * p + i, gy = cy * p + j, gz = cz * p + k;
    bool dir = gx == 0 || gy == 0 || gz == 0 || gx == g.N[0] - 1 || gy == g.N[1] - 1 || gz == g.N[2] - 1;
    int mult = ((i == 0 && cx > 0) || (i == p && cx < g.nx - 1) ? 2 : 1) *
               ((j == 0 && cy > 0) || (j == p && cy < g.ny - 1) ? 2 : 1) *
               ((k == 0 && cz > 0) || (k == p && cz < g.nz - 1) ? 2 : 1);
    b0[idx] = dir ? T(0) : T(r[gidx(g, gx, gy, gz)]) / T(mult);
  }
  __syncthreads();
  contract_axis(b0, b1, sT, true, 0, n, threadIdx.x, blockDim.x);
  __syncthreads();
  contract_axis(b1, b0, sT, true, 1, n, threadIdx.x, blockDim.x);
  __syncthreads();
  contract_axis(b0, b1, sT, true, 2, n, threadIdx.x, blockDim.x);
  __syncthreads();
  T *out = E + (int64_t)cell * n3;
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) out[idx] = b1[idx];
}

// ------------------------------------------------------------------ patch solve
// cell and cell-local index of star coordinate t along one axis for a side
__device__ __forceinline__ bool star_local(int full, int p, int t, int side, int &loc) {
  const int c = p - 1;
  if (!full) {
    if (side != 0) return false;
    loc = t + 1;
    return true;
  }
  if (side == 0) {
    if (t > c) return false;
    loc = t + 1;
  } else {
    if (t < c) return false;
    loc = t - c;
  }
  return true;
}

template <typename T>
__device__ __forceinline__ T interior_diag(const T *sAf, const T *sBf, const T *mu, int n, int i, int j, int k) {
  T ai = sAf[i * n + i], aj = sAf[j * n + j], ak = sAf[k * n + k];
  T bi = sBf[i * n + i], bj = sBf[j * n + j], bk = sBf[k * n + k];
  return mu[0] * ai * bj * bk + mu[1] * bi * aj * bk + mu[2] * bi * bj * ak;
}

template <typename T>
__global__ void __launch_bounds__(PATCH_THREADS) k_patch_solve(PatchSolveArgs<T> a) {
  extern __shared__ unsigned char smem_[];
  constexpr int NT = PATCH_THREADS, NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const PatchDev P = a.patches[a.order[blockIdx.x]];
  const ClassDev &C = a.cls[P.cls];
  const Grid &g = a.g;
  const int p = g.p, n = g.n, n3 = n * n * n, c = p - 1;
  const int nG = C.nG, n0 = C.n0, n1 = C.n1, n2 = C.n2;
  const int dim0 = C.dim[0], dim1 = C.dim[1];
  T *sAf = reinterpret_cast<T *>(smem_);
  T *sBf = sAf + n * n;
  T *sMu = sBf + n * n;   // [8][3]
  int *sCell = reinterpret_cast<int *>(sMu + 24);  // [8]
  T *gv = reinterpret_cast<T *>(sCell + 8);
  T *yv = gv + nG, *xv = yv + nG, *tmp = xv + nG;  // tmp: max(n1, NW*32)
  for (int i = tid; i < n * n; i += NT) {
    sAf[i] = a.tab[tab_off(TAB_AF, n) + i];
    sBf[i] = a.tab[tab_off(TAB_BF, n) + i];
  }
  if (tid < 8) {
    int s[3] = {tid & 1, (tid >> 1) & 1, tid >> 2};
    int ncl[3] = {g.nx, g.ny, g.nz};
    int cc[3];
    bool ok = true;
    for (int ax = 0; ax < 3; ++ax) {
      if (!C.full[ax] && s[ax]) ok = false;
      cc[ax] = star_cell_along(C.full[ax], P.v[ax], ncl[ax], s[ax]);
    }
    int cell = ok ? cc[0] + g.nx * (cc[1] + g.ny * cc[2]) : -1;
    sCell[tid] = cell;
    for (int q = 0; q < 3; ++q) sMu[tid * 3 + q] = ok ? T(a.mu[3 * cell + q]) : T(0);
  }
  __syncthreads();
  const T *E = a.E;
  const T *Lv = a.L + P.voff;

  // ---- gather the FDM residual on the interface and condense the interior
  for (int k = tid; k < nG; k += NT) {
    int pos = C.gpos[k];
    int t[3] = {pos % dim0, (pos / dim0) % dim1, pos / (dim0 * dim1)};
    T r = 0;
    for (int sd = 0; sd < 8; ++sd) {
      int s[3] = {sd & 1, (sd >> 1) & 1, sd >> 2};
      int l[3];
      bool ok = sCell[sd] >= 0;
      for (int ax = 0; ax < 3 && ok; ++ax) ok = star_local(C.full[ax], p, t[ax], s[ax], l[ax]);
      if (ok) r += E[(int64_t)sCell[sd] * n3 + l[0] + n * (l[1] + n * l[2])];
    }
    int nc = 0, an = -1;
    for (int ax = 0; ax < 3; ++ax)
      if (C.full[ax] && t[ax] == c) { ++nc; an = ax; }
    if (nc == 1) {  // face dof with normal an: A_GI A_II^{-1} r_I from both cells
      for (int s = 0; s < 2; ++s) {
        int sd = 0, l[3];
        for (int ax = 0; ax < 3; ++ax) {
          int side = ax == an ? s : ((C.full[ax] && t[ax] > c) ? 1 : 0);
          sd |= side << ax;
          if (ax != an) star_local(C.full[ax], p, t[ax], side, l[ax]);
        }
        const T *mu = sMu + 3 * sd;
        const T *Ek = E + (int64_t)sCell[sd] * n3;
        int lf = s == 0 ? p : 0;
        int b1 = an == 0 ? 1 : 0, b2 = an == 2 ? 1 : 2;
        T tang = sBf[l[b1] * n + l[b1]] * sBf[l[b2] * n + l[b2]];
        for (int ii = 1; ii < p; ++ii) {
          l[an] = ii;
          T coef = mu[an] * sAf[lf * n + ii] * tang;
          T D = interior_diag(sAf, sBf, mu, n, l[0], l[1], l[2]);
          r -= coef * Ek[l[0] + n * (l[1] + n * l[2])] / D;
        }
      }
    }
    gv[k] = r;
  }
  __syncthreads();

  // ---- forward solve L y = g
  const T *dinv0 = Lv + C.off_dinv0;
  const T *ell = Lv + C.off_ell;
  for (int j = tid; j < n0; j += NT) yv[j] = gv[j] * dinv0[j];
  __syncthreads();
  for (int r = tid; r < C.nrow0; r += NT) {
    T acc = 0;
    for (int e = 0; e < C.K0; ++e) {
      int col = C.ell_col[e * C.nrow0 + r];
      if (col >= 0) acc += ell[e * C.nrow0 + r] * yv[col];
    }
    gv[n0 + r] -= acc;
  }
  __syncthreads();
  for (int i = tid; i < n1; i += NT) {
    int b = C.line_of[i], s0 = C.line_start[b], w = C.line_len[b];
    const T *Li = Lv + C.off_lines + C.line_off[b] + (int64_t)(i - s0) * w;
    T acc = 0;
    for (int cc = 0; cc <= i - s0; ++cc) acc += Li[cc] * gv[n0 + s0 + cc];
    yv[n0 + i] = acc;
  }
  __syncthreads();
  if (n2 > 0) {
    const T *L21 = Lv + C.off_l21;
    for (int r = warp; r < n2; r += NW) {
      const T *row = L21 + (int64_t)r * C.ld21;
      T acc = 0;
      for (int cc = lane; cc < n1; cc += 32) acc += row[cc] * yv[n0 + cc];
      acc = warp_sum(acc);
      if (lane == 0) gv[n0 + n1 + r] -= acc;
    }
    __syncthreads();
    for (int q = 0; q < C.npanel; ++q) {
      const int base = n0 + n1 + q * PANEL, w = min(PANEL, n2 - q * PANEL), rows = n2 - q * PANEL;
      const T *pan = Lv + C.off_pan + C.pan_off[q];
      for (int i = tid; i < w; i += NT) {
        T acc = 0;
        for (int cc = 0; cc <= i; ++cc) acc += pan[i * PANEL + cc] * gv[base + cc];
        yv[base + i] = acc;
      }
      __syncthreads();
      for (int r = w + warp; r < rows; r += NW) {
        T v = lane < w ? pan[(int64_t)r * PANEL + lane] * yv[base + lane] : T(0);
        v = warp_sum(v);
        if (lane == 0) gv[base + r] -= v;
      }
      __syncthreads();
    }
    // ---- backward solve L^T x = y, top level
    for (int q = C.npanel - 1; q >= 0; --q) {
      const int base = n0 + n1 + q * PANEL, w = min(PANEL, n2 - q * PANEL), rows = n2 - q * PANEL;
      const T *pan = Lv + C.off_pan + C.pan_off[q];
      T acc = 0;
      for (int r = w + warp; r < rows; r += NW) acc += pan[(int64_t)r * PANEL + lane] * xv[base + r];
      tmp[warp * 32 + lane] = acc;
      __syncthreads();
      if (tid < w) {
        T s = 0;
        for (int ww = 0; ww < NW; ++ww) s += tmp[ww * 32 + tid];
        tmp[NW * 32 + tid] = yv[base + tid] - s;
      }
      __syncthreads();
      if (tid < w) {
        T s = 0;
        for (int cc = tid; cc < w; ++cc) s += pan[cc * PANEL + tid] * tmp[NW * 32 + cc];
        xv[base + tid] = s;
      }
      __syncthreads();
    }
    // t1 = L21^T x2
    for (int cc = tid; cc < n1; cc += NT) {
      T s = 0;
      for (int r = 0; r < n2; ++r) s += L21[(int64_t)r * C.ld21 + cc] * xv[n0 + n1 + r];
      tmp[cc] = s;
    }
    __syncthreads();
  } else {
    for (int cc = tid; cc < n1; cc += NT) tmp[cc] = 0;
    __syncthreads();
  }
  for (int i = tid; i < n1; i += NT) {
    int b = C.line_of[i], s0 = C.line_start[b], w = C.line_len[b];
    const T *Lb = Lv + C.off_lines + C.line_off[b];
    T s = 0;
    for (int cc = i - s0; cc < w; ++cc) s += Lb[cc * w + (i - s0)] * (yv[n0 + s0 + cc] - tmp[s0 + cc]);
    xv[n0 + i] = s;
  }
  __syncthreads();
  for (int j = tid; j < n0; j += NT) {
    T s = yv[j];
    for (int q = C.c0_ptr[j]; q < C.c0_ptr[j + 1]; ++q) {
      int pos = C.c0_pos[q];
      s -= ell[pos] * xv[n0 + pos % C.nrow0];
    }
    xv[j] = s * dinv0[j];
  }
  __syncthreads();

  // ---- write the star solution: interface values and back-substituted interior
  T *X = a.X + P.xoff;
  for (int k = tid; k < nG; k += NT) X[C.gpos[k]] = xv[k];
  for (int pos = tid; pos < C.nd; pos += NT) {
    if (C.ginv[pos] >= 0) continue;
    int t[3] = {pos % dim0, (pos / dim0) % dim1, pos / (dim0 * dim1)};
    int sd = 0, l[3];
    for (int ax = 0; ax < 3; ++ax) {
      int side = (C.full[ax] && t[ax] > c) ? 1 : 0;
      sd |= side << ax;
      star_local(C.full[ax], p, t[ax], side, l[ax]);
    }
    const T *mu = sMu + 3 * sd;
    T r = E[(int64_t)sCell[sd] * n3 + l[0] + n * (l[1] + n * l[2])];
    for (int ax = 0; ax < 3; ++ax) {
      if (!C.full[ax]) continue;
      int tt[3] = {t[0], t[1], t[2]};
      tt[ax] = c;
      int fk = C.ginv[tt[0] + dim0 * (tt[1] + dim1 * tt[2])];
      int lf = ((sd >> ax) & 1) ? 0 : p;
      int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
      T coef = mu[ax] * sAf[lf * n + l[ax]] * sBf[l[b1] * n + l[b1]] * sBf[l[b2] * n + l[b2]];
      r -= coef * xv[fk];
    }
    X[pos] = r / interior_diag(sAf, sBf, mu, n, l[0], l[1], l[2]);
  }
}

// ------------------------------------------------------------------ interpolate
template <typename T, typename Tout>
__global__ void __launch_bounds__(256) k_interp_fdm(Grid g, const PatchDev *__restrict__ patches,
                                                    const ClassDev *__restrict__ cls, const T *__restrict__ X,
                                                    const T *__restrict__ tab, double omega, Tout *__restrict__ z) {
  extern __shared__ unsigned char smem_[];
  T *sT = reinterpret_cast<T *>(smem_);
  const int n = g.n, p = g.p, n3 = n * n * n, c = p - 1;
  T *b0 = sT + n * n, *b1 = b0 + n3;
  const int cell = blockIdx.x;
  const int ce[3] = {cell % g.nx, (cell / g.nx) % g.ny, cell / (g.nx * g.ny)};
  const int ncl[3] = {g.nx, g.ny, g.nz};
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) sT[i] = tab[tab_off(TAB_T, n) + i];
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int li[3] = {idx % n, (idx / n) % n, idx / (n * n)};
    T acc = 0;
    for (int o = 0; o < 8; ++o) {
      int oo[3] = {o & 1, (o >> 1) & 1, o >> 2};
      int v[3], t[3];
      bool ok = true;
      for (int ax = 0; ax < 3 && ok; ++ax) {
        v[ax] = ce[ax] + oo[ax];
        bool full = v[ax] >= 1 && v[ax] <= ncl[ax] - 1;
        int i = li[ax];
        if (full) {
          if (oo[ax] == 0) { ok = i <= p - 1; t[ax] = i + c; }
          else { ok = i >= 1; t[ax] = i - 1; }
        } else {
          ok = i >= 1 && i <= p - 1;
          t[ax] = i - 1;
        }
      }
      if (!ok) continue;
      int pid = v[0] + (g.nx + 1) * (v[1] + (g.ny + 1) * v[2]);
      const PatchDev P = patches[pid];
      const ClassDev &C = cls[P.cls];
      acc += X[P.xoff + t[0] + C.dim[0] * (t[1] + C.dim[1] * t[2])];
    }
    b0[idx] = acc;
  }
  __syncthreads();
  contract_axis(b0, b1, sT, false, 0, n, threadIdx.x, blockDim.x);
  __syncthreads();
  contract_axis(b1, b0, sT, false, 1, n, threadIdx.x, blockDim.x);
  __syncthreads();
  contract_axis(b0, b1, sT, false, 2, n, threadIdx.x, blockDim.x);
  __syncthreads();
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
    if ((i == 0 && ce[0] > 0) || (j == 0 && ce[1] > 0) || (k == 0 && ce[2] > 0)) continue;  // not owner
    int gx = ce[0] * p + i, gy = ce[1] * p + j, gz = ce[2] * p + k;
    bool dir = gx == 0 || gy == 0 || gz == 0 || gx == g.N[0] - 1 || gy == g.N[1] - 1 || gz == g.N[2] - 1;
    z[gidx(g, gx, gy, gz)] = dir ? Tout(0) : Tout(omega * b1[idx]);
  }
}

// ------------------------------------------------------------------ launchers
template <typename T, typename Tin>
void launch_restrict_fdm(const Grid &g, const Tin *r, const T *tab, T *E, cudaStream_t st) {
  size_t sm = sizeof(T) * (g.n * g.n + 2 * g.n * g.n * g.n);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_restrict_fdm<T, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_restrict_fdm<T, Tin><<<g.ncell, 256, sm, st>>>(g, r, tab, E);
}

template <typename T, typename Tout>
void launch_interp_fdm(const Grid &g, const PatchDev *patches, const ClassDev *cls, const T *X, const T *tab,
                       double omega, Tout *z, cudaStream_t st) {
  size_t sm = sizeof(T) * (g.n * g.n + 2 * g.n * g.n * g.n);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_interp_fdm<T, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_interp_fdm<T, Tout><<<g.ncell, 256, sm, st>>>(g, patches, cls, X, tab, omega, z);
}

template <typename T>
size_t patch_smem_bytes(int n, int maxG, int maxN1) {
  int tmpn = maxN1 > (PATCH_THREADS / 32) * 32 + PANEL ? maxN1 : (PATCH_THREADS / 32) * 32 + PANEL;
  return sizeof(T) * (2 * n * n + 24) + sizeof(int) * 8 + sizeof(T) * (3 * maxG + tmpn) + 64;
}

template <typename T>
void launch_patch_solve(const PatchSolveArgs<T> &a, int npatch, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_patch_solve<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  if (npatch > 0) k_patch_solve<T><<<npatch, PATCH_THREADS, smem, st>>>(a);
}

#define INST(T)                                                                                          \
  template void launch_restrict_fdm<T, double>(const Grid &, const double *, const T *, T *, cudaStream_t); \
  template void launch_restrict_fdm<T, float>(const Grid &, const float *, const T *, T *, cudaStream_t);   \
  template void launch_interp_fdm<T, double>(const Grid &, const PatchDev *, const ClassDev *, const T *,    \
                                             const T *, double, double *, cudaStream_t);                     \
  template void launch_interp_fdm<T, float>(const Grid &, const PatchDev *, const ClassDev *, const T *,     \
                                            const T *, double, float *, cudaStream_t);                       \
  template size_t patch_smem_bytes<T>(int, int, int);                                                       \
  template void launch_patch_solve<T>(const PatchSolveArgs<T> &, int, size_t, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace fdm
