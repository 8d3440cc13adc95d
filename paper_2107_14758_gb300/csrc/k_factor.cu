// Set-up kernels (FP64): per-patch assembly of the interface Schur
// complement S_G = A_GG - A_GI A_II^{-1} A_IG in the FDM basis (Section 2.6,
// eq:LDLT; A_II is diagonal there), its Cholesky factor with the class's
// level structure (diagonal bottom level eliminated sparsely, dense blocked
// right-looking factorisation of the rest), and packing into the solve
// layout in FP64 and FP32.  Also the banded-Cholesky inverse of the coarse
// operator.
#include "device.cuh"
#include "factor.h"

namespace fdm {

__device__ __forceinline__ int star_from_local(int full, int p, int side, int l) {
  // inverse of the star-local map: returns t or -1 if the node is not in the star
  const int c = p - 1;
  if (!full) return (l >= 1 && l <= p - 1) ? l - 1 : -1;
  if (side == 0) return l >= 1 ? l - 1 : -1;
  return l <= p - 1 ? l + c : -1;
}

// block-wide exclusive scan of 0/1 flags (blockDim.x multiple of 32, <= 1024)
__device__ int block_scan(int flag, int *sw, int &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned b = __ballot_sync(0xffffffffu, flag);
  int pre = __popc(b & ((1u << lane) - 1u));
  if (lane == 0) sw[warp] = __popc(b);
  __syncthreads();
  int off = 0;
  total = 0;
  for (int w = 0; w < nw; ++w) {
    if (w < warp) off += sw[w];
    total += sw[w];
  }
  __syncthreads();
  return off + pre;
}

__global__ void __launch_bounds__(256) k_assemble_schur(FactorArgs a) {
  extern __shared__ unsigned char smem_[];
  const int slot = blockIdx.x;
  const PatchDev P = a.patches[a.plist[slot]];
  const ClassDev &C = a.cls[P.cls];
  const Grid &g = a.g;
  const int p = g.p, n = g.n, c = p - 1, nG = C.nG;
  double *S = a.S + (int64_t)slot * a.ldS;
  double *sAf = reinterpret_cast<double *>(smem_);
  double *sBf = sAf + n * n;
  double *sMu = sBf + n * n;
  int *sCell = reinterpret_cast<int *>(sMu + 24);
  int *sw = sCell + 8;
  int *lst = sw + 32;  // [2 * maxclosure]: interface index, packed local index
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    sAf[i] = a.tab[tab_off(TAB_AF, n) + i];
    sBf[i] = a.tab[tab_off(TAB_BF, n) + i];
  }
  if (threadIdx.x < 8) {
    int s[3] = {(int)(threadIdx.x & 1), (int)((threadIdx.x >> 1) & 1), (int)threadIdx.x >> 2};
    int ncl[3] = {g.nx, g.ny, g.nz}, cc[3];
    bool ok = true;
    for (int ax = 0; ax < 3; ++ax) {
      if (!C.full[ax] && s[ax]) ok = false;
      cc[ax] = star_cell_along(C.full[ax], P.v[ax], ncl[ax], s[ax]);
    }
    int cell = ok ? cc[0] + g.nx * (cc[1] + g.ny * cc[2]) : -1;
    sCell[threadIdx.x] = cell;
    for (int q = 0; q < 3; ++q) sMu[threadIdx.x * 3 + q] = ok ? a.mu[3 * cell + q] : 0.0;
  }
  for (int64_t i = threadIdx.x; i < (int64_t)nG * nG; i += blockDim.x) S[i] = 0.0;
  __syncthreads();
  const int dim0 = C.dim[0], dim1 = C.dim[1];
  for (int sd = 0; sd < 8; ++sd) {
    if (sCell[sd] < 0) continue;
    const int side[3] = {sd & 1, (sd >> 1) & 1, sd >> 2};
    const double *mu = sMu + 3 * sd;
    // list the interface dofs in the closure of this cell (deterministic order)
    int cnt = 0;
    const int n3 = n * n * n;
    for (int base = 0; base < n3; base += blockDim.x) {
      int idx = base + threadIdx.x;
      int gi = -1;
      if (idx < n3) {
        int l[3] = {idx % n, (idx / n) % n, idx / (n * n)}, t[3];
        bool ok = true;
        for (int ax = 0; ax < 3 && ok; ++ax) {
          t[ax] = star_from_local(C.full[ax], p, side[ax], l[ax]);
          ok = t[ax] >= 0;
        }
        if (ok) gi = C.ginv[t[0] + dim0 * (t[1] + dim1 * t[2])];
      }
      int tot;
      int pos = block_scan(gi >= 0, sw, tot);
      if (gi >= 0) {
        lst[2 * (cnt + pos)] = gi;
        lst[2 * (cnt + pos) + 1] = idx;
      }
      cnt += tot;
      __syncthreads();
    }
    // A_GG: separable cell matrix in the FDM basis
    for (int64_t q = threadIdx.x; q < (int64_t)cnt * cnt; q += blockDim.x) {
      int u = (int)(q / cnt), v = (int)(q % cnt);
      int lu = lst[2 * u + 1], lv = lst[2 * v + 1];
      int iu = lu % n, ju = (lu / n) % n, ku = lu / (n * n);
      int iv = lv % n, jv = (lv / n) % n, kv = lv / (n * n);
      double val = mu[0] * sBf[ku * n + kv] * sBf[ju * n + jv] * sAf[iu * n + iv] +
                   mu[1] * sBf[ku * n + kv] * sAf[ju * n + jv] * sBf[iu * n + iv] +
                   mu[2] * sAf[ku * n + kv] * sBf[ju * n + jv] * sBf[iu * n + iv];
      if (val != 0.0) S[(int64_t)lst[2 * u] * nG + lst[2 * v]] += val;
    }
    __syncthreads();
    // Schur complement of the cell interior (diagonal A_II): cross terms ...
    const int m = p - 1;
    for (int q = threadIdx.x; q < m * m * m; q += blockDim.x) {
      int l[3] = {1 + q % m, 1 + (q / m) % m, 1 + q / (m * m)};
      double D = mu[0] * sAf[l[0] * n + l[0]] * sBf[l[1] * n + l[1]] * sBf[l[2] * n + l[2]] +
                 mu[1] * sBf[l[0] * n + l[0]] * sAf[l[1] * n + l[1]] * sBf[l[2] * n + l[2]] +
                 mu[2] * sBf[l[0] * n + l[0]] * sBf[l[1] * n + l[1]] * sAf[l[2] * n + l[2]];
      int f[3], nf = 0;
      double cf[3];
      int t[3];
      for (int ax = 0; ax < 3; ++ax) t[ax] = star_from_local(C.full[ax], p, side[ax], l[ax]);
      for (int ax = 0; ax < 3; ++ax) {
        if (!C.full[ax]) continue;
        int tt[3] = {t[0], t[1], t[2]};
        tt[ax] = c;
        int lf = side[ax] ? 0 : p;
        int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
        f[nf] = C.ginv[tt[0] + dim0 * (tt[1] + dim1 * tt[2])];
        cf[nf++] = mu[ax] * sAf[lf * n + l[ax]] * sBf[l[b1] * n + l[b1]] * sBf[l[b2] * n + l[b2]];
      }
      for (int u = 0; u < nf; ++u)
        for (int v = 0; v < nf; ++v)
          if (u != v) S[(int64_t)f[u] * nG + f[v]] -= cf[u] * cf[v] / D;
    }
    // ... and diagonal terms, one face dof at a time along its normal line
    for (int ax = 0; ax < 3; ++ax) {
      if (!C.full[ax]) continue;
      int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
      int lf = side[ax] ? 0 : p;
      for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
        int l[3];
        l[b1] = 1 + q % m;
        l[b2] = 1 + q / m;
        int tt[3];
        tt[ax] = c;
        tt[b1] = star_from_local(C.full[b1], p, side[b1], l[b1]);
        tt[b2] = star_from_local(C.full[b2], p, side[b2], l[b2]);
        int fk = C.ginv[tt[0] + dim0 * (tt[1] + dim1 * tt[2])];
        double tang = sBf[l[b1] * n + l[b1]] * sBf[l[b2] * n + l[b2]];
        double s = 0.0;
        for (int ii = 1; ii < p; ++ii) {
          l[ax] = ii;
          double cf = mu[ax] * sAf[lf * n + ii] * tang;
          double D = mu[0] * sAf[l[0] * n + l[0]] * sBf[l[1] * n + l[1]] * sBf[l[2] * n + l[2]] +
                     mu[1] * sBf[l[0] * n + l[0]] * sAf[l[1] * n + l[1]] * sBf[l[2] * n + l[2]] +
                     mu[2] * sBf[l[0] * n + l[0]] * sBf[l[1] * n + l[1]] * sAf[l[2] * n + l[2]];
          s += cf * cf / D;
        }
        S[(int64_t)fk * nG + fk] -= s;
      }
    }
    __syncthreads();
  }
}

// Cholesky of S in place (lower triangle holds L on exit).
__global__ void __launch_bounds__(256) k_factor(FactorArgs a) {
  __shared__ double Dk[PANEL][PANEL + 1];
  __shared__ double Ta[PANEL][PANEL + 1], Tb[PANEL][PANEL + 1];
  __shared__ int bad;
  const int slot = blockIdx.x;
  const PatchDev P = a.patches[a.plist[slot]];
  const ClassDev &C = a.cls[P.cls];
  const int nG = C.nG, n0 = C.n0;
  double *S = a.S + (int64_t)slot * a.ldS;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  // ---- level 0: diagonal pivots, sparse rank-1 updates of the trailing rows
  for (int j = 0; j < n0; ++j) {
    const int rb = C.r0_ptr[j], re = C.r0_ptr[j + 1], cnt = re - rb;
    double piv = S[(int64_t)j * nG + j];
    if (!(piv > 0.0)) {
      if (threadIdx.x == 0) bad = 1;
      piv = 1.0;
    }
    const double d = sqrt(piv);
    __syncthreads();
    for (int q = threadIdx.x; q < cnt; q += blockDim.x) S[(int64_t)C.r0_idx[rb + q] * nG + j] /= d;
    if (threadIdx.x == 0) S[(int64_t)j * nG + j] = d;
    __syncthreads();
    for (int q = threadIdx.x; q < cnt * cnt; q += blockDim.x) {
      int u = q / cnt, v = q % cnt;
      int r = C.r0_idx[rb + u], s = C.r0_idx[rb + v];
      if (s > r) continue;
      S[(int64_t)r * nG + s] -= S[(int64_t)r * nG + j] * S[(int64_t)s * nG + j];
    }
    __syncthreads();
  }
  // ---- dense blocked right-looking Cholesky of the trailing block
  for (int kb = n0; kb < nG; kb += PANEL) {
    const int w = min(PANEL, nG - kb);
    for (int q = threadIdx.x; q < PANEL * PANEL; q += blockDim.x) {
      int i = q / PANEL, jj = q % PANEL;
      Dk[i][jj] = (i < w && jj <= i) ? S[(int64_t)(kb + i) * nG + kb + jj] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      const int i = threadIdx.x;
      for (int j = 0; j < w; ++j) {
        double djj = Dk[j][j];
        if (!(djj > 0.0)) {
          if (i == 0) bad = 1;
          djj = 1.0;
        }
        double dj = sqrt(djj);
        __syncwarp();
        if (i == j) Dk[j][j] = dj;
        if (i > j && i < w) Dk[i][j] /= dj;
        __syncwarp();
        if (i > j && i < w)
          for (int k = j + 1; k <= i; ++k) Dk[i][k] -= Dk[i][j] * Dk[k][j];
        __syncwarp();
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < PANEL * PANEL; q += blockDim.x) {
      int i = q / PANEL, jj = q % PANEL;
      if (i < w && jj <= i) S[(int64_t)(kb + i) * nG + kb + jj] = Dk[i][jj];
    }
    // panel rows below: x L_kk^T = s
    for (int r = kb + w + threadIdx.x; r < nG; r += blockDim.x) {
      double *row = S + (int64_t)r * nG + kb;
      double x[PANEL];
#pragma unroll
      for (int jj = 0; jj < PANEL; ++jj) {
        if (jj < w) {
          double s = row[jj];
          for (int k = 0; k < jj; ++k) s -= x[k] * Dk[jj][k];
          x[jj] = s / Dk[jj][jj];
          row[jj] = x[jj];
        }
      }
    }
    __syncthreads();
    // trailing update S[r][s] -= L[r][panel] . L[s][panel], s <= r, by 32x32 tiles
    const int t0 = kb + w, nt = (nG - t0 + PANEL - 1) / PANEL;
    for (int tile = 0; tile < nt * (nt + 1) / 2; ++tile) {
      int ti = 0;
      while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
      int tj = tile - ti * (ti + 1) / 2;
      const int r0 = t0 + ti * PANEL, s0 = t0 + tj * PANEL;
      for (int q = threadIdx.x; q < PANEL * PANEL; q += blockDim.x) {
        int i = q / PANEL, k = q % PANEL;
        Ta[i][k] = (r0 + i < nG && k < w) ? S[(int64_t)(r0 + i) * nG + kb + k] : 0.0;
        Tb[i][k] = (s0 + i < nG && k < w) ? S[(int64_t)(s0 + i) * nG + kb + k] : 0.0;
      }
      __syncthreads();
      for (int q = threadIdx.x; q < PANEL * PANEL; q += blockDim.x) {
        int i = q / PANEL, jj = q % PANEL;
        int r = r0 + i, s = s0 + jj;
        if (r < nG && s < nG && s <= r) {
          double acc = 0.0;
#pragma unroll 8
          for (int k = 0; k < PANEL; ++k) acc += Ta[i][k] * Tb[jj][k];
          S[(int64_t)r * nG + s] -= acc;
        }
      }
      __syncthreads();
    }
  }
  if (threadIdx.x == 0 && bad) atomicExch(a.status, 1);
}

// Inverse of a w x w lower-triangular block (row stride lds) into out
// (row stride ldo): thread per column.
__device__ void tri_inverse(const double *L, int lds, int w, double *out, int ldo, bool to32, float *out32) {
  for (int cc = threadIdx.x; cc < w; cc += blockDim.x) {
    double x[PANEL];
    for (int i = 0; i < w; ++i) {
      if (i < cc) { x[i] = 0.0; continue; }
      double s = i == cc ? 1.0 : 0.0;
      for (int k = cc; k < i; ++k) s -= L[(int64_t)i * lds + k] * x[k];
      x[i] = s / L[(int64_t)i * lds + i];
    }
    for (int i = 0; i < w; ++i) {
      if (out) out[(int64_t)i * ldo + cc] = x[i];
      if (to32) out32[(int64_t)i * ldo + cc] = (float)x[i];
    }
  }
}

__global__ void __launch_bounds__(256) k_pack(FactorArgs a) {
  const int slot = blockIdx.x;
  const PatchDev P = a.patches[a.plist[slot]];
  const ClassDev &C = a.cls[P.cls];
  const int nG = C.nG, n0 = C.n0, n1 = C.n1, n2 = C.n2;
  const double *S = a.S + (int64_t)slot * a.ldS;
  double *V = a.L64 + P.voff;
  float *W = a.L32 ? a.L32 + P.voff : nullptr;
  auto put = [&](int64_t off, double v) {
    V[off] = v;
    if (W) W[off] = (float)v;
  };
  for (int j = threadIdx.x; j < n0; j += blockDim.x) put(C.off_dinv0 + j, 1.0 / S[(int64_t)j * nG + j]);
  for (int q = threadIdx.x; q < C.K0 * C.ldr0; q += blockDim.x) {
    int col = C.ell_col[q], r = q % C.ldr0;
    put(C.off_ell + q, col >= 0 ? S[(int64_t)(n0 + r) * nG + col] : 0.0);
  }
  for (int b = 0; b < C.nlines; ++b) {
    int s0 = n0 + C.line_start[b], w = C.line_len[b];
    int64_t off = C.off_lines + C.line_off[b];
    tri_inverse(S + (int64_t)s0 * nG + s0, nG, w, V + off, w, W != nullptr, W ? W + off : nullptr);
  }
  if (C.sc) {
    // Schur-coupling form: both line solves at once, (L_b L_b^T)^{-1} = L_b^{-T} L_b^{-1}
    // (symmetric, w x w) per line; formed in the line's block of the workspace, whose
    // factor values are no longer needed, then written over the line inverse
    __syncthreads();
    double *Sw0 = a.S + (int64_t)slot * a.ldS;
    for (int b = 0; b < C.nlines; ++b) {
      const int s0 = n0 + C.line_start[b], w = C.line_len[b];
      const int64_t off = C.off_lines + C.line_off[b];
      for (int q = threadIdx.x; q < w * w; q += blockDim.x) {
        const int i = q / w, j = q % w, k0 = i > j ? i : j;
        double m = 0.0;
        for (int k = k0; k < w; ++k) m += V[off + (int64_t)k * w + i] * V[off + (int64_t)k * w + j];
        Sw0[(int64_t)(s0 + i) * nG + s0 + j] = m;
      }
    }
    __syncthreads();
    for (int b = 0; b < C.nlines; ++b) {
      const int s0 = n0 + C.line_start[b], w = C.line_len[b];
      const int64_t off = C.off_lines + C.line_off[b];
      for (int q = threadIdx.x; q < w * w; q += blockDim.x) put(off + q, Sw0[(int64_t)(s0 + q / w) * nG + s0 + q % w]);
    }
  }
  if (!C.sc)
    for (int64_t q = threadIdx.x; q < (int64_t)n2 * C.ld21; q += blockDim.x) {
      int r = (int)(q / C.ld21), cc = (int)(q % C.ld21);
      put(C.off_l21 + q, cc < n1 ? S[(int64_t)(n0 + n1 + r) * nG + n0 + cc] : 0.0);
    }
  // top level: Z = L_top^{-1} by forward substitution, one column per thread;
  // column c of Z (below the diagonal) is kept in row c of the strict upper
  // triangle of the workspace, which the factorisation no longer uses.
  const int base = n0 + n1;
  double *Sw = a.S + (int64_t)slot * a.ldS;
  for (int cc = threadIdx.x; cc < n2; cc += blockDim.x) {
    double *zc = Sw + (int64_t)(base + cc) * nG + base;  // zc[i] = Z[i][cc], i > cc
    const double zdiag = 1.0 / S[(int64_t)(base + cc) * nG + base + cc];
    for (int i = cc + 1; i < n2; ++i) {
      const double *Li = S + (int64_t)(base + i) * nG + base;
      double s = Li[cc] * zdiag;
      for (int k = cc + 1; k < i; ++k) s += Li[k] * zc[k];
      zc[i] = -s / Li[i];
    }
  }
  __syncthreads();
  if (!C.sc) {
    for (int r = 0; r < n2; ++r) {
      const int len = C.zoff[r + 1] - C.zoff[r];
      const int64_t off = C.off_z + C.zoff[r];
      for (int cc = threadIdx.x; cc < len; cc += blockDim.x) {
        double v = 0.0;
        if (cc == r) v = 1.0 / S[(int64_t)(base + r) * nG + base + r];
        else if (cc < r) v = S[(int64_t)(base + cc) * nG + base + r];
        put(off + cc, v);
      }
    }
    return;
  }
  // Schur-coupling form: W = Z^T Z = (L_top L_top^T)^{-1}, its lower triangle by
  // rows.  With Zt[x][k] = Z[k][x] (row x of Zt is column x of Z, stored in row
  // base + x of the workspace above the diagonal, 1 / L_xx on it, zero before
  // it), W[r][c] = sum_k Zt[r][k] Zt[c][k]: a symmetric rank-n2 product by
  // 32 x 32 tiles, each thread owning four entries of a tile.
  __shared__ double Ta[PANEL][PANEL + 1], Tb[PANEL][PANEL + 1];
  auto zt = [&](int x, int k) -> double {
    if (x >= n2 || k >= n2 || k < x) return 0.0;
    if (k == x) return 1.0 / S[(int64_t)(base + x) * nG + base + x];
    return Sw[(int64_t)(base + x) * nG + base + k];
  };
  const int nt = (n2 + PANEL - 1) / PANEL;
  for (int tile = 0; tile < nt * (nt + 1) / 2; ++tile) {
    int ti = 0;
    while ((ti + 1) * (ti + 2) / 2 <= tile) ++ti;
    const int tj = tile - ti * (ti + 1) / 2;
    const int r0 = ti * PANEL, c0 = tj * PANEL;
    double acc[PANEL * PANEL / 256];
#pragma unroll
    for (int m = 0; m < PANEL * PANEL / 256; ++m) acc[m] = 0.0;
    for (int k0 = r0; k0 < n2; k0 += PANEL) {  // Zt[r][k] = 0 for k < r0 <= r
      for (int q = threadIdx.x; q < PANEL * PANEL; q += blockDim.x) {
        const int i = q / PANEL, k = q % PANEL;
        Ta[i][k] = zt(r0 + i, k0 + k);
        Tb[i][k] = zt(c0 + i, k0 + k);
      }
      __syncthreads();
#pragma unroll
      for (int m = 0; m < PANEL * PANEL / 256; ++m) {
        const int q = threadIdx.x + 256 * m, i = q / PANEL, j = q % PANEL;
        double s = 0.0;
#pragma unroll 8
        for (int k = 0; k < PANEL; ++k) s += Ta[i][k] * Tb[j][k];
        acc[m] += s;
      }
      __syncthreads();
    }
#pragma unroll
    for (int m = 0; m < PANEL * PANEL / 256; ++m) {
      const int q = threadIdx.x + 256 * m, r = r0 + q / PANEL, cc = c0 + q % PANEL;
      if (r < n2 && cc <= r) put(C.off_z + C.zoff[r] + cc, acc[m]);
    }
  }
  for (int r = threadIdx.x; r < n2; r += blockDim.x)  // zero padding of each row
    for (int cc = r + 1; cc < C.zoff[r + 1] - C.zoff[r]; ++cc) put(C.off_z + C.zoff[r] + cc, 0.0);
}

// Schur-coupling form: the values of S_TB (top rows of S_G in the lower
// columns, S's own pattern) before the factorisation overwrites S
__global__ void __launch_bounds__(256) k_extract_st(FactorArgs a) {
  const int slot = blockIdx.x;
  const PatchDev P = a.patches[a.plist[slot]];
  const ClassDev &C = a.cls[P.cls];
  if (!C.sc || C.KT == 0) return;
  const int nG = C.nG, base = C.n0 + C.n1;
  const double *S = a.S + (int64_t)slot * a.ldS;
  double *V = a.L64 + P.voff;
  float *W = a.L32 ? a.L32 + P.voff : nullptr;
  for (int q = threadIdx.x; q < C.KT * C.ldT; q += blockDim.x) {
    const int col = C.st_col[q], t = q % C.ldT;
    const double v = (col >= 0 && t < C.n2) ? S[(int64_t)(base + t) * nG + col] : 0.0;
    V[C.off_st + q] = v;
    if (W) W[C.off_st + q] = (float)v;
  }
}

size_t assemble_smem_bytes(int n) {
  int maxc = n * n * n;  // upper bound of the closure list
  return sizeof(double) * (2 * n * n + 24) + sizeof(int) * (8 + 32 + 2 * maxc) + 64;
}

void launch_factor_batch(const FactorArgs &a, int count, cudaStream_t st) {
  if (count <= 0) return;
  size_t sm = assemble_smem_bytes(a.g.n);
  cudaFuncSetAttribute(k_assemble_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  k_assemble_schur<<<count, 256, sm, st>>>(a);
  k_extract_st<<<count, 256, 0, st>>>(a);
  k_factor<<<count, 256, 0, st>>>(a);
  k_pack<<<count, 256, 0, st>>>(a);
}

void launch_assemble_factor_only(const FactorArgs &a, int count, cudaStream_t st) {
  if (count <= 0) return;
  size_t sm = assemble_smem_bytes(a.g.n);
  cudaFuncSetAttribute(k_assemble_schur, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  k_assemble_schur<<<count, 256, sm, st>>>(a);
  k_factor<<<count, 256, 0, st>>>(a);
}

// ---- coarse operator inverse from its banded Cholesky factor: one thread
// per column c solves L L^T x = e_c in place in row c of the output (the
// inverse is symmetric).
__global__ void k_banded_inverse(int m, int bw, const double *__restrict__ Lb, double *__restrict__ out) {
  int cidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (cidx >= m) return;
  double *x = out + (int64_t)cidx * m;
  for (int i = 0; i < m; ++i) x[i] = 0.0;
  // forward: L y = e_c (y_i = 0 for i < c)
  for (int i = cidx; i < m; ++i) {
    double s = i == cidx ? 1.0 : 0.0;
    int k0 = max(cidx, i - bw);
    for (int k = k0; k < i; ++k) s -= Lb[(int64_t)i * (bw + 1) + (i - k)] * x[k];
    x[i] = s / Lb[(int64_t)i * (bw + 1)];
  }
  // backward: L^T x = y
  for (int i = m - 1; i >= 0; --i) {
    double s = x[i];
    int k1 = min(m - 1, i + bw);
    for (int k = i + 1; k <= k1; ++k) s -= Lb[(int64_t)k * (bw + 1) + (k - i)] * x[k];
    x[i] = s / Lb[(int64_t)i * (bw + 1)];
  }
}

void launch_banded_inverse(int m, int bw, const double *Lb, double *out, cudaStream_t st) {
  if (m <= 0) return;
  k_banded_inverse<<<(m + 127) / 128, 128, 0, st>>>(m, bw, Lb, out);
}

}  // namespace fdm
