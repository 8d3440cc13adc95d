// Additive vertex-star relaxation kernels (Sections 2.4-2.6 of the paper).
//
// One sweep z = omega sum_j R_j^T A_j^{-1} R_j r runs as three kernels:
//   restrict: per cell, E_K = (T^T (x) T^T (x) T^T)(W_K r_K) (the FDM-basis
//             residual, W = 1/multiplicity), then the cell's share of the
//             Schur condensation g_G = r_G - A_GI A_II^{-1} r_I (eq:LDLT): every
//             face node f of K gets E_K(f) - sum_i A_fi E_K(i) / A_ii over the
//             interior line through f.  A_II is diagonal in the FDM basis and the
//             coupling of f to that line is mu_a Af[f][i] Bf Bf, so this is a
//             cell-local, patch-independent quantity.
//   patch:    per vertex star, gather of the condensed interface residual (sum
//             over the star's cells), forward and backward solves with the
//             sparse Cholesky factor of the interface Schur complement; writes
//             the interface solution x_G only.
//   interp:   per cell, the additive sum over the 8 stars of the cell's
//             vertices: interface nodes directly from the stars' x_G; interior
//             nodes by the back-substitution x_I = A_II^{-1}(r_I - A_IG x_G)
//             summed over the stars, which needs only the summed face values
//             (the 4 stars containing a face node are exactly the stars whose
//             back-substitution uses that face):
//               z(m) = (8 r(m) - sum_faces A_mf z(f)) / A_mm;
//             then z_K = (T (x) T (x) T) z_fdm, omega, owner write.
#include <algorithm>

#include "bulk.cuh"
#include "device.cuh"
#include "kernels.h"

namespace fdm {

template <typename T>
__device__ __forceinline__ T interior_diag(const T *sAf, const T *sBf, const T *mu, int n, int i, int j, int k) {
  T ai = sAf[i * n + i], aj = sAf[j * n + j], ak = sAf[k * n + k];
  T bi = sBf[i * n + i], bj = sBf[j * n + j], bk = sBf[k * n + k];
  return mu[0] * ai * bj * bk + mu[1] * bi * aj * bk + mu[2] * bi * bj * ak;
}

// face coupling A(f, m) of a face node f (local lf along axis ax) to the
// interior node m = l (same tangential coordinates) of one cell
template <typename T>
__device__ __forceinline__ T face_coupling(const T *sAf, const T *sBf, const T *mu, int n, int ax, int lf,
                                           const int l[3]) {
  const int b1 = ax == 0 ? 1 : 0, b2 = ax == 2 ? 1 : 2;
  return mu[ax] * sAf[lf * n + l[ax]] * sBf[l[b1] * n + l[b1]] * sBf[l[b2] * n + l[b2]];
}

// ------------------------------------------------------------------ restrict
template <typename T, typename Tin>
__global__ void __launch_bounds__(256) k_restrict_fdm(Grid g, const Tin *__restrict__ r, const T *__restrict__ tab,
                                                      const double *__restrict__ mug, T *__restrict__ E) {
  extern __shared__ unsigned char smem_[];
  T *sT = reinterpret_cast<T *>(smem_);
  const int n = g.n, p = g.p, n3 = n * n * n;
  T *sAf = sT + n * n, *sBf = sAf + n * n;
  T *b0 = sBf + n * n, *b1 = b0 + n3;
  __shared__ T mu[3];
  const int cell = blockIdx.x;
  const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    sT[i] = tab[tab_off(TAB_T, n) + i];
    sAf[i] = tab[tab_off(TAB_AF, n) + i];
    sBf[i] = tab[tab_off(TAB_BF, n) + i];
  }
  if (threadIdx.x < 3) mu[threadIdx.x] = T(mug[3 * cell + threadIdx.x]);
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
    int gx = cx * p + i, gy = cy * p + j, gz = cz * p + k;
    bool dir = node_dirichlet(g, gx, gy, gz);
    int mult = ((i == 0 && cx > 0) || (i == p && cx < g.nx - 1) ? 2 : 1) *
               ((j == 0 && cy > 0) || (j == p && cy < g.ny - 1) ? 2 : 1) *
               ((k == 0 && cz > 0) || (k == p && cz < g.nz - 1) ? 2 : 1);
    b0[idx] = dir ? T(0) : T(r[gidx(g, gx, gy, gz)]) / T(mult);
  }
  __syncthreads();
  contract(b0, b1, sT, true, 0, n, T(1), false);
  __syncthreads();
  contract(b1, b0, sT, true, 1, n, T(1), false);
  __syncthreads();
  contract(b0, b1, sT, true, 2, n, T(1), false);
  __syncthreads();
  // 1/A_ii of the interior nodes, once per node (b0 is free now)
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int l[3] = {idx % n, (idx / n) % n, idx / (n * n)};
    bool in = l[0] > 0 && l[0] < p && l[1] > 0 && l[1] < p && l[2] > 0 && l[2] < p;
    b0[idx] = in ? T(1) / interior_diag(sAf, sBf, mu, n, l[0], l[1], l[2]) : T(0);
  }
  __syncthreads();
  T *out = E + (int64_t)cell * n3;
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int l[3] = {idx % n, (idx / n) % n, idx / (n * n)};
    int nb = 0, ax = -1;
    for (int a = 0; a < 3; ++a)
      if (l[a] == 0 || l[a] == p) { ++nb; ax = a; }
    T v = b1[idx];
    if (nb == 1) {  // face node: subtract A_fI A_II^{-1} E_I along the interior line
      const int lf = l[ax], stride = ax == 0 ? 1 : (ax == 1 ? n : n * n);
      const int b1x = ax == 0 ? 1 : 0, b2x = ax == 2 ? 1 : 2;
      const T tang = mu[ax] * sBf[l[b1x] * n + l[b1x]] * sBf[l[b2x] * n + l[b2x]];
      T s = 0;
      for (int ii = 1; ii < p; ++ii) {
        const int m = idx + (ii - lf) * stride;
        s += sAf[lf * n + ii] * b1[m] * b0[m];
      }
      v -= tang * s;
    }
    out[idx] = v;
  }
}

// ------------------------------------------------------------------ patch solve
// four consecutive elements with 128-bit loads (16-byte aligned address)
template <typename T> struct V4 { T x, y, z, w; };
__device__ __forceinline__ V4<float> load4(const float *p) {
  float4 v = *reinterpret_cast<const float4 *>(p);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> load4(const double *p) {
  double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
  return {a.x, a.y, b.x, b.y};
}
// read-once streams (the W block of the patch solve): 128-bit global loads
// that do not allocate in L1, so that the class index tables stay there
// (volatile: never speculated, since a caller may hold a shared-memory W and
// take the generic path instead)
__device__ __forceinline__ V4<float> load4_stream(const float *p) {
  V4<float> v;
  asm volatile("ld.global.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(p));
  return v;
}
__device__ __forceinline__ V4<double> load4_stream(const double *p) {
  V4<double> v;
  asm volatile("ld.global.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
  asm volatile("ld.global.L1::no_allocate.v2.f64 {%0, %1}, [%2];" : "=d"(v.z), "=d"(v.w) : "l"(p + 2));
  return v;
}
__device__ __forceinline__ float load_na(const float *p) {
  float v;
  asm volatile("ld.global.L1::no_allocate.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ double load_na(const double *p) {
  double v;
  asm volatile("ld.global.L1::no_allocate.f64 %0, [%1];" : "=d"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void store4(float *p, const V4<float> &v) {
  *reinterpret_cast<float4 *>(p) = make_float4(v.x, v.y, v.z, v.w);
}
__device__ __forceinline__ void store4(double *p, const V4<double> &v) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(v.x, v.y);
  reinterpret_cast<double2 *>(p)[1] = make_double2(v.z, v.w);
}

// L2 eviction-priority policies: the forward solve reads the factor's large
// sections (L21, Z) as evict-last so that they survive until the backward
// solve, which reads them as evict-first (their last use in this sweep)
__device__ __forceinline__ uint64_t policy_keep() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t policy_normal() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t policy_drop() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ V4<float> load4h(const float *p, uint64_t pol) {
  if (!__isGlobal(p)) return load4(p);
  float4 v;
  asm("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p), "l"(pol));
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4<double> load4h(const double *p, uint64_t pol) {
  if (!__isGlobal(p)) return load4(p);
  double2 a, b;
  asm("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(a.x), "=d"(a.y) : "l"(p), "l"(pol));
  asm("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;" : "=d"(b.x), "=d"(b.y) : "l"(p + 2), "l"(pol));
  return {a.x, a.y, b.x, b.y};
}

// zero g, y, x and tmp (zero-padded factor columns then multiply finite values
// only), find the star's cells and gather the condensed FDM residual on the
// interface (fixed cell order)
template <typename T, int NT, int NV = 3>
__device__ __forceinline__ void patch_gather(const PatchSolveArgs<T> &a, const PatchDev &P, const ClassDev &C, T *gv,
                                             int *sCell) {
  const int tid = threadIdx.x;
  const Grid &g = a.g;
  const int n = g.n, n3 = n * n * n;
  const int nG = C.nG;
  for (int i = tid; i < NV * nG + a.tmpcap; i += NT) gv[i] = T(0);
  if (tid < 8) {
    int s[3] = {tid & 1, (tid >> 1) & 1, tid >> 2};
    int ncl[3] = {g.nx, g.ny, g.nz};
    int cc[3];
    bool ok = true;
    for (int ax = 0; ax < 3; ++ax) {
      if (!C.full[ax] && s[ax]) ok = false;
      cc[ax] = star_cell_along(C.full[ax], P.v[ax], ncl[ax], s[ax]);
    }
    sCell[tid] = ok ? cc[0] + g.nx * (cc[1] + g.ny * cc[2]) : -1;
  }
  __syncthreads();

  // ---- gather the condensed FDM residual on the interface (fixed cell order)
  const T *E = a.E;
  for (int k = tid; k < nG; k += NT) {
    const int *src = C.gsrc + 8 * k;
    T r = 0;
    for (int e = 0; e < 8; ++e) {
      int code = src[e];
      if (code < 0) break;
      r += E[(int64_t)sCell[code >> 16] * n3 + (code & 0xffff)];
    }
    gv[k] = r;
  }
  __syncthreads();

}

// forward and backward solves with the factor values Lv of this patch (global
// or shared memory), then the interface solution in factor order

// Sums over the 32 lanes of RB values per lane (RB = 2, 4 or 8) with a butterfly
// that halves the number of values per lane at each of the first log2(RB)
// stages: 2 + 1 + 3 shuffles for RB = 4 (4 + 2 + 1 + 2 for RB = 8) instead of
// 5 per value.  On return lane l holds the total of value index
// rb_slot<RB>(l) in acc[0]; the lanes l with (l & (32 / RB - 1)) == 0 hold the
// RB totals.
template <int RB>
__device__ __forceinline__ int rb_slot(int lane) {
  return lane / (32 / RB);  // RB = 2, 4 or 8
}
template <typename T, int RB>
__device__ __forceinline__ void multi_warp_sum(T (&acc)[RB], int lane) {
#pragma unroll
  for (int half = RB / 2, o = 16; half >= 1; half >>= 1, o >>= 1) {
    const bool up = (lane & o) != 0;  // the upper lane keeps the upper half of the values
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const T send = up ? acc[j] : acc[j + half];
      const T keep = up ? acc[j + half] : acc[j];
      acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
#pragma unroll
  for (int o = 32 / RB / 2; o > 0; o >>= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], o);
}

// RB: rows per warp in the forward row-oriented products (their loads in flight together)
template <typename T, int NT, int RB>
__device__ __forceinline__ void patch_solve_body(const PatchSolveArgs<T> &a, const PatchDev &P, const ClassDev &C,
                                                 const T *Lv, T *gv) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nG = C.nG, n0 = C.n0, n1 = C.n1, n2 = C.n2;
  T *yv = gv + nG, *xv = yv + nG, *tmp = xv + nG;  // tmp: a.tmpcap elements
  // L2 policies of the large factor sections (evict_normal both ways when hints are off)
  const uint64_t keep = a.l2hint ? policy_keep() : policy_normal(), drop = a.l2hint ? policy_drop() : policy_normal();
  // ---- forward solve L y = g (level 0 diagonal, level-1 lines, dense top block)
  const T *dinv0 = Lv + C.off_dinv0;
  const T *ell = Lv + C.off_ell;
  for (int j = tid; j < n0; j += NT) yv[j] = gv[j] * dinv0[j];
  __syncthreads();
  for (int r = tid; r < C.nrow0; r += NT) {  // g_{>0} -= L_{>0,0} y_0
    T acc = 0;
#pragma unroll 4
    for (int e = 0; e < C.K0; ++e) {
      int col = C.ell_col[e * C.ldr0 + r];
      if (col >= 0) acc += ell[e * C.ldr0 + r] * yv[col];
    }
    gv[n0 + r] -= acc;
  }
  __syncthreads();
  for (int i = tid; i < n1; i += NT) {  // y_1 = L_11^{-1} g_1, line by line
    int b = C.line_of[i], s0 = C.line_start[b], w = C.line_len[b];
    const T *Li = Lv + C.off_lines + C.line_off[b] + (int64_t)(i - s0) * w;
    T acc = 0;
    for (int cc = 0; cc <= i - s0; ++cc) acc += Li[cc] * gv[n0 + s0 + cc];
    yv[n0 + i] = acc;
  }
  __syncthreads();
  if (n2 > 0) {
    const T *L21 = Lv + C.off_l21;
    const T *Z = Lv + C.off_z;
    const int base = n0 + n1;
    if (n1 > 0) {  // g_2 -= L21 y_1: a warp takes RB rows at a time (their loads in flight together)
      const int ng = C.ld21 / 4;
      for (int r0 = warp * RB; r0 < n2; r0 += NW * RB) {
        T acc[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) acc[u] = 0;
        for (int q4 = lane; q4 < ng; q4 += 32) {
          V4<T> v[RB];
#pragma unroll
          for (int u = 0; u < RB; ++u)
            v[u] = r0 + u < n2 ? load4h(L21 + (int64_t)(r0 + u) * C.ld21 + 4 * q4, keep) : V4<T>{0, 0, 0, 0};
          const T *yy = yv + n0 + 4 * q4;  // padding columns of L21 are zero, yv is finite there
#pragma unroll
          for (int u = 0; u < RB; ++u) acc[u] += v[u].x * yy[0] + v[u].y * yy[1] + v[u].z * yy[2] + v[u].w * yy[3];
        }
        if (RB == 4) {  // butterfly (measured faster for four rows, slower for eight)
          multi_warp_sum<T, RB>(acc, lane);
          if ((lane & (32 / RB - 1)) == 0) {
            const int u = rb_slot<RB>(lane);
            if (r0 + u < n2) gv[base + r0 + u] -= acc[0];
          }
        } else {
#pragma unroll
          for (int u = 0; u < RB; ++u) acc[u] = warp_sum(acc[u]);
          if (lane == 0)
#pragma unroll
            for (int u = 0; u < RB; ++u)
              if (r0 + u < n2) gv[base + r0 + u] -= acc[u];
        }
      }
      __syncthreads();
    }
    // y_2 = Z g_2 with Z = L_top^{-1} (rows zero-padded to 4), RB rows per warp at a time
    for (int r0 = warp * RB; r0 < n2; r0 += NW * RB) {
      T acc[RB];
      int ngu[RB];
      const T *row[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        acc[u] = 0;
        const int r = r0 + u < n2 ? r0 + u : n2 - 1;
        row[u] = Z + C.zoff[r];
        ngu[u] = r0 + u < n2 ? (C.zoff[r + 1] - C.zoff[r]) / 4 : 0;
      }
      int ngmax = 0;
#pragma unroll
      for (int u = 0; u < RB; ++u) ngmax = ngu[u] > ngmax ? ngu[u] : ngmax;
      for (int q4 = lane; q4 < ngmax; q4 += 32) {
        V4<T> v[RB];
#pragma unroll
        for (int u = 0; u < RB; ++u) v[u] = q4 < ngu[u] ? load4h(row[u] + 4 * q4, keep) : V4<T>{0, 0, 0, 0};
        const T *gg = gv + base + 4 * q4;
#pragma unroll
        for (int u = 0; u < RB; ++u) acc[u] += v[u].x * gg[0] + v[u].y * gg[1] + v[u].z * gg[2] + v[u].w * gg[3];
      }
      if (RB == 4) {
        multi_warp_sum<T, RB>(acc, lane);
        if ((lane & (32 / RB - 1)) == 0) {
          const int u = rb_slot<RB>(lane);
          if (r0 + u < n2) yv[base + r0 + u] = acc[0];
        }
      } else {
#pragma unroll
        for (int u = 0; u < RB; ++u) acc[u] = warp_sum(acc[u]);
        if (lane == 0)
#pragma unroll
          for (int u = 0; u < RB; ++u)
            if (r0 + u < n2) yv[base + r0 + u] = acc[u];
      }
    }
    __syncthreads();
    // ---- backward solve L^T x = y
    // x_2 = Z^T y_2: threads own 4-column groups, rows split into slices
    {
      const int ngz = (n2 + 3) / 4, ldz = 4 * ngz;
      const int slices = max(1, min(NT / ngz, a.tmpcap / ldz));
      const int gq = tid % ngz, sl = tid / ngz;
      if (sl < slices) {
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
        // rows r = sl (mod slices) with r >= 4 gq (Z[r][c] = 0 for c > r): the threads of
        // a slice walk the same rows, so a warp reads contiguous groups of one row
        const int lo = 4 * gq > sl ? sl + (4 * gq - sl + slices - 1) / slices * slices : sl;
#pragma unroll 4
        for (int r = lo; r < n2; r += slices) {
          V4<T> v = load4h(Z + C.zoff[r] + 4 * gq, drop);
          T yr = yv[base + r];
          a0 += v.x * yr; a1 += v.y * yr; a2 += v.z * yr; a3 += v.w * yr;
        }
        T *dst = tmp + (int64_t)sl * ldz + 4 * gq;
        dst[0] = a0; dst[1] = a1; dst[2] = a2; dst[3] = a3;
      }
      __syncthreads();
      for (int cc = tid; cc < n2; cc += NT) {
        T s = 0;
        for (int q = 0; q < slices; ++q) s += tmp[q * ldz + cc];
        xv[base + cc] = s;
      }
      __syncthreads();
    }
    // t1 = L21^T x2: threads own 4-column groups, rows split into slices
    // (no level-1 rows, e.g. p = 1: nothing to do)
    if (n1 > 0) {
      const int ng = C.ld21 / 4;
      const int slices = max(1, min(NT / ng, a.tmpcap / C.ld21));
      const int gq = tid % ng, sl = tid / ng;
      if (sl < slices) {
        T a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll 4
        for (int r = sl; r < n2; r += slices) {
          V4<T> v = load4h(L21 + (int64_t)r * C.ld21 + 4 * gq, drop);
          T xr = xv[base + r];
          a0 += v.x * xr; a1 += v.y * xr; a2 += v.z * xr; a3 += v.w * xr;
        }
        T *dst = tmp + (int64_t)sl * C.ld21 + 4 * gq;
        dst[0] = a0; dst[1] = a1; dst[2] = a2; dst[3] = a3;
      }
      __syncthreads();
      for (int cc = tid; cc < n1; cc += NT) {
        T s = 0;
        for (int q = 0; q < slices; ++q) s += tmp[q * C.ld21 + cc];
        tmp[cc] = s;  // only this thread reads column cc of the slices
      }
      __syncthreads();
    }
  } else {
    for (int cc = tid; cc < n1; cc += NT) tmp[cc] = 0;
    __syncthreads();
  }
  for (int i = tid; i < n1; i += NT) {  // x_1 = L_11^{-T} (y_1 - L21^T x_2)
    int b = C.line_of[i], s0 = C.line_start[b], w = C.line_len[b];
    const T *Lb = Lv + C.off_lines + C.line_off[b];
    T s = 0;
    for (int cc = i - s0; cc < w; ++cc) s += Lb[cc * w + (i - s0)] * (yv[n0 + s0 + cc] - tmp[s0 + cc]);
    xv[n0 + i] = s;
  }
  __syncthreads();
  for (int j = tid; j < n0; j += NT) {  // x_0 = D_0^{-1} (y_0 - L_{>0,0}^T x_{>0})
    T s = yv[j];
    const int q1 = C.c0_ptr[j + 1];
#pragma unroll 4
    for (int q = C.c0_ptr[j]; q < q1; ++q) {
      const int pos = C.c0_pos[q];
      s -= ell[pos] * xv[n0 + pos % C.ldr0];
    }
    xv[j] = s * dinv0[j];
  }
  __syncthreads();

  // ---- the interface solution, in factor order
  T *X = a.X + P.xoff;
  for (int k = tid; k < nG; k += NT) X[k] = xv[k];
}

// 256 threads: at most 42 registers with four rows per warp (six CTAs per SM),
// 51 with eight (five CTAs per SM)
template <typename T, int NT, int RB>
__global__ void __launch_bounds__(NT, NT == 256 ? (RB == 4 ? 6 : 5) : 1) k_patch_solve(PatchSolveArgs<T> a) {
  extern __shared__ unsigned char smem_[];
  const int tid = threadIdx.x;
  const PatchDev P = a.patches[a.order[blockIdx.x]];
  const ClassDev &C = a.cls[P.cls];
  __shared__ int sCell[8];
  T *gv = reinterpret_cast<T *>(smem_);
  const T *Lv = a.L + P.voff;
  // bring the factor into L2 a section ahead of its use (not all at once, so
  // that the sections are still resident when the backward solve re-reads them)
  auto prefetch_l2 = [&](int64_t e0, int64_t e1) {
    if (tid != 0 || a.prefetch == 0) return;
    const char *src = reinterpret_cast<const char *>(Lv + e0);
    const int64_t bytes = (e1 - e0) * (int64_t)sizeof(T);
    for (int64_t off = 0; off < bytes; off += 32768)
      bulk::prefetch_l2(src + off, (uint32_t)(bytes - off < 32768 ? bytes - off : 32768));
  };
  if (a.prefetch == 1) prefetch_l2(0, C.nval);  // whole factor at the start
  else if (a.prefetch == 2) prefetch_l2(0, C.off_l21);  // level 0 and lines; L21 and Z follow later
  patch_gather<T, NT>(a, P, C, gv, sCell);
  if (a.prefetch == 2) prefetch_l2(C.off_l21, C.nval);  // L21 and Z, needed after level 0 and the lines
  patch_solve_body<T, NT, RB>(a, P, C, Lv, gv);
}

// Persistent variant with the whole factor of the current patch resident in
// shared memory: one thread starts a bulk copy (cp.async.bulk) of the patch's
// factor values into shared memory and an L2 prefetch of the next patch's,
// the CTA gathers the interface residual meanwhile, waits on the mbarrier
// (bounded by timeout_ns) and runs both solves from shared memory, so every
// factor value leaves DRAM once per sweep.  Used where the largest class
// factor fits in shared memory.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, 1) k_patch_resident(PatchSolveArgs<T> a, int npatch, int fcap) {
  extern __shared__ __align__(128) unsigned char smem_[];
  const int tid = threadIdx.x;
  T *F = reinterpret_cast<T *>(smem_);  // fcap elements (a multiple of 4)
  T *gv = F + fcap;
  __shared__ __align__(8) uint64_t bar[2];  // [0] factor arrived, [1] test hook: never completed
  __shared__ int sCell[8];
  __shared__ int sFail;
  if (tid == 0) {
    bulk::mbar_init(&bar[0], 1);
    bulk::mbar_init(&bar[1], 1);
    bulk::fence_mbar_init();
    sFail = 0;
  }
  __syncthreads();
  uint32_t parity = 0;
  for (int it = blockIdx.x; it < npatch; it += gridDim.x) {
    const PatchDev P = a.patches[a.order[it]];
    const ClassDev &C = a.cls[P.cls];
    if (tid == 0) {
      // every thread finished reading F for the previous patch (barrier at the loop end)
      bulk::fence_proxy_async();
      const uint32_t bytes = (uint32_t)(C.nval * (int64_t)sizeof(T));
      bulk::mbar_arrive_expect_tx(&bar[0], bytes);
      const char *src = reinterpret_cast<const char *>(a.L + P.voff);
      char *dst = reinterpret_cast<char *>(F);
      for (uint32_t off = 0; off < bytes; off += 32768)
        bulk::bulk_g2s(dst + off, src + off, bytes - off < 32768 ? bytes - off : 32768, &bar[0]);
      const int nx = it + gridDim.x;
      if (nx < npatch) {
        const PatchDev Q = a.patches[a.order[nx]];
        const uint32_t qb = (uint32_t)(a.cls[Q.cls].nval * (int64_t)sizeof(T));
        const char *qs = reinterpret_cast<const char *>(a.L + Q.voff);
        for (uint32_t off = 0; off < qb; off += 32768) bulk::prefetch_l2(qs + off, qb - off < 32768 ? qb - off : 32768);
      }
    }
    patch_gather<T, NT>(a, P, C, gv, sCell);
    bool ok = true;
    if (a.inject_stall) ok = bulk::mbar_wait_bounded(&bar[1], 0, a.timeout_ns);  // never completes
    ok = ok && bulk::mbar_wait_bounded(&bar[0], parity, a.timeout_ns);
    if (!ok) sFail = 1;
    __syncthreads();
    if (sFail) {
      // give the copy in flight a second bounded wait before leaving
      bulk::mbar_wait_bounded(&bar[0], parity, a.timeout_ns);
      if (tid == 0) atomicExch(a.status, 1);
      return;
    }
    parity ^= 1u;
    patch_solve_body<T, NT, 4>(a, P, C, F, gv);
    __syncthreads();
  }
}

// ------------------------------------------------------------------ interpolate
template <typename T, typename Tout>
__global__ void __launch_bounds__(256) k_interp_fdm(InterpArgs<T> a, double omega, Tout *__restrict__ z) {
  extern __shared__ unsigned char smem_[];
  const Grid &g = a.g;
  const int n = g.n, p = g.p, n3 = n * n * n, c = p - 1;
  T *sT = reinterpret_cast<T *>(smem_);
  T *sAf = sT + n * n, *sBf = sAf + n * n;
  T *b0 = sBf + n * n, *b1 = b0 + n3;
  __shared__ T mu[3];
  const int cell = blockIdx.x;
  const int ce[3] = {cell % g.nx, (cell / g.nx) % g.ny, cell / (g.nx * g.ny)};
  const int ncl[3] = {g.nx, g.ny, g.nz};
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    sT[i] = a.tab[tab_off(TAB_T, n) + i];
    sAf[i] = a.tab[tab_off(TAB_AF, n) + i];
    sBf[i] = a.tab[tab_off(TAB_BF, n) + i];
  }
  if (threadIdx.x < 3) mu[threadIdx.x] = T(a.mu[3 * cell + threadIdx.x]);
  // interface-type nodes of the cell: sum of the stars' interface solutions
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int li[3] = {idx % n, (idx / n) % n, idx / (n * n)};
    bool onb = false;
    for (int ax = 0; ax < 3; ++ax) onb |= (li[ax] == 0 || li[ax] == p);
    if (!onb) continue;
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
      const PatchDev P = a.patches[v[0] + (g.nx + 1) * (v[1] + (g.ny + 1) * v[2])];
      const ClassDev &C = a.cls[P.cls];
      int k = C.ginv[t[0] + C.dim[0] * (t[1] + C.dim[1] * t[2])];
      if (k >= 0) acc += a.X[P.xoff + k];
    }
    b0[idx] = acc;
  }
  __syncthreads();
  // interior nodes: (8 r(m) - sum over the 6 face nodes of A_mf z(f)) / A_mm
  const T *Ek = a.E + (int64_t)cell * n3;
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int l[3] = {idx % n, (idx / n) % n, idx / (n * n)};
    bool onb = false;
    for (int ax = 0; ax < 3; ++ax) onb |= (l[ax] == 0 || l[ax] == p);
    if (onb) continue;
    T s = T(8) * Ek[idx];
    for (int ax = 0; ax < 3; ++ax) {
      const int stride = ax == 0 ? 1 : (ax == 1 ? n : n * n);
      s -= face_coupling(sAf, sBf, mu, n, ax, 0, l) * b0[idx - l[ax] * stride];
      s -= face_coupling(sAf, sBf, mu, n, ax, p, l) * b0[idx + (p - l[ax]) * stride];
    }
    b0[idx] = s / interior_diag(sAf, sBf, mu, n, l[0], l[1], l[2]);
  }
  __syncthreads();
  contract(b0, b1, sT, false, 0, n, T(1), false);
  __syncthreads();
  contract(b1, b0, sT, false, 1, n, T(1), false);
  __syncthreads();
  contract(b0, b1, sT, false, 2, n, T(1), false);
  __syncthreads();
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int i = idx % n, j = (idx / n) % n, k = idx / (n * n);
    if ((i == 0 && ce[0] > 0) || (j == 0 && ce[1] > 0) || (k == 0 && ce[2] > 0)) continue;  // not owner
    int gx = ce[0] * p + i, gy = ce[1] * p + j, gz = ce[2] * p + k;
    bool dir = node_dirichlet(g, gx, gy, gz);
    z[gidx(g, gx, gy, gz)] = dir ? Tout(0) : Tout(omega * b1[idx]);
  }
}

// ------------------------------------------------------------------ launchers
template <typename T, typename Tin>
void launch_restrict_fdm(const Grid &g, const Tin *r, const T *tab, const double *mu, T *E, cudaStream_t st) {
  if (launch_restrict_fast<T, Tin>(g, r, tab, mu, E, st)) return;
  size_t sm = sizeof(T) * (3 * g.n * g.n + 2 * g.n * g.n * g.n);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_restrict_fdm<T, Tin>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_restrict_fdm<T, Tin><<<g.ncell, 256, sm, st>>>(g, r, tab, mu, E);
}

template <typename T, typename Tout>
void launch_interp_fdm(const InterpArgs<T> &a, double omega, Tout *z, cudaStream_t st) {
  if (launch_interp_fast<T, Tout>(a, omega, z, st)) return;
  if (a.addv) fail(FDM_EINVAL, "interpolation with an added vector needs the specialised kernel");
  size_t sm = sizeof(T) * (3 * a.g.n * a.g.n + 2 * a.g.n * a.g.n * a.g.n);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_interp_fdm<T, Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  k_interp_fdm<T, Tout><<<a.g.ncell, 256, sm, st>>>(a, omega, z);
}

// ------------------------------------------------------------------ Schur-coupling form
// The same exact patch solve, organised around the 2 x 2 block form of the
// interface Schur complement with B = levels 0 and 1, T = the top level:
//   y_B = S_BB^{-1} g_B,  x_T = W (g_T - S_TB y_B),  x_B = y_B - S_BB^{-1} S_BT x_T,
// where S_BB = L_BB L_BB^T (diagonal level 0, sparse L10, line blocks of L11:
// the leading block of L_G) and W = (L_TT L_TT^T)^{-1} is the inverse of the
// top block's Schur complement.  S_TB keeps S_G's own sparsity (no fill), so
// the dense L21 block of the factor is not stored, and W is read once where
// Z = L_TT^{-1} is read twice (forward and backward).

// u = S_BB^{-1} in over the lower block (n0 + n1 entries; t1: n1 scratch) in three phases:
//   t_1 = g_1 - L_10 (D_0^{-1} g_0)            (y_0 = L_00^{-1} g_0 formed where used)
//   u_1 = (L_11 L_11^T)^{-1} t_1               (the symmetric inverse of each line block,
//                                               stored in place of the line inverse)
//   u_0 = L_00^{-T} (y_0 - L_10^T u_1)
// out may alias in (each phase reads in only at indices it or an earlier phase
// owns).  fin, when given, also receives y - u (the final lower values).
template <typename T, int NT>
__device__ __forceinline__ void bb_solve(const ClassDev &C, const T *Lv, const T *in, T *out, T *t1,
                                         const T *y = nullptr, T *fin = nullptr) {
  const int tid = threadIdx.x, n0 = C.n0, n1 = C.n1;
  const T *dinv0 = Lv + C.off_dinv0, *ell = Lv + C.off_ell;
  for (int r = tid; r < n1; r += NT) {
    T acc = 0;
#pragma unroll 4
    for (int e = 0; e < C.K0; ++e) {
      const int col = C.ell_col[e * C.ldr0 + r];
      if (col >= 0) acc += ell[e * C.ldr0 + r] * (in[col] * dinv0[col]);
    }
    t1[r] = in[n0 + r] - acc;
  }
  __syncthreads();
  for (int r = tid; r < n1; r += NT) {  // one row of one line's symmetric block per thread
    const int b = C.line_of[r], s0 = C.line_start[b], w = C.line_len[b], i = r - s0;
    const T *Mb = Lv + C.off_lines + C.line_off[b];
    T acc = 0;
    for (int cc = 0; cc < w; ++cc) acc += Mb[cc * w + i] * t1[s0 + cc];
    out[n0 + r] = acc;
    if (fin) fin[n0 + r] = y[n0 + r] - acc;
  }
  __syncthreads();
  for (int j = tid; j < n0; j += NT) {
    T s = in[j] * dinv0[j];
    const int q1 = C.cB_ptr[j + 1];
    for (int q = C.cB_ptr[j]; q < q1; ++q) {
      const int pos = C.cB_pos[q];
      s -= ell[pos] * out[n0 + pos % C.ldr0];
    }
    s *= dinv0[j];
    out[j] = s;
    if (fin) fin[j] = y[j] - s;
  }
  __syncthreads();
}

// x = W v for the symmetric W given by its lower triangle in rows (row r holds
// W[r][0..r], zero-padded to a multiple of 4).  A warp takes four rows at a
// time; each lane reads the same column groups of the four rows, adds the row
// dots (the lower triangle with the diagonal, butterfly-reduced) and
// accumulates the strictly lower entries times v_r into its warp's column
// accumulator (acc, NW rows of ld, zero on entry): the lower triangle is read
// once and every entry used twice.  The warp accumulators are summed in fixed
// order, so the result does not depend on timing.
template <typename T, int NT, int RB>
__device__ __forceinline__ void sym_apply(const ClassDev &C, const T *Wv, const T *v, T *x, T *acc, int ld) {
  constexpr int NW = NT / 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, n2 = C.n2;
  T *aw = acc + warp * ld;
  // 128-bit shared accesses where v and the accumulators are 16-byte aligned
  // (acc always is; v = g_T is when the lower block has a multiple of 4 rows)
  const bool vec = ((reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(acc)) & 15) == 0;
  const bool wglob = __isGlobal(Wv);  // W streams from global memory (else staged in shared memory)
  for (int r0 = warp * RB; r0 < n2; r0 += NW * RB) {
    T rs[RB], vr[RB];
    int ngu[RB];
    const T *row[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int r = r0 + u < n2 ? r0 + u : n2 - 1;
      row[u] = Wv + C.zoff[r];
      ngu[u] = r0 + u < n2 ? (C.zoff[r + 1] - C.zoff[r]) / 4 : 0;
      rs[u] = 0;
      vr[u] = r0 + u < n2 ? v[r0 + u] : T(0);
    }
    int ngmax = 0;
#pragma unroll
    for (int u = 0; u < RB; ++u) ngmax = ngu[u] > ngmax ? ngu[u] : ngmax;
    for (int q4 = lane; q4 < ngmax; q4 += 32) {
      V4<T> w[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u)
        w[u] = q4 < ngu[u] ? (wglob ? load4_stream(row[u] + 4 * q4) : load4(row[u] + 4 * q4)) : V4<T>{0, 0, 0, 0};
      const int cb = 4 * q4;
      const V4<T> vv = vec ? load4(v + cb) : V4<T>{v[cb], v[cb + 1], v[cb + 2], v[cb + 3]};  // padding of W is zero
      T c0 = 0, c1 = 0, c2 = 0, c3 = 0;
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        rs[u] += w[u].x * vv.x + w[u].y * vv.y + w[u].z * vv.z + w[u].w * vv.w;
        const int r = r0 + u;
        c0 += (cb < r ? w[u].x : T(0)) * vr[u];
        c1 += (cb + 1 < r ? w[u].y : T(0)) * vr[u];
        c2 += (cb + 2 < r ? w[u].z : T(0)) * vr[u];
        c3 += (cb + 3 < r ? w[u].w : T(0)) * vr[u];
      }
      if (vec) {
        V4<T> a4 = load4(aw + cb);
        a4.x += c0;
        a4.y += c1;
        a4.z += c2;
        a4.w += c3;
        store4(aw + cb, a4);
      } else {
        aw[cb] += c0;
        aw[cb + 1] += c1;
        aw[cb + 2] += c2;
        aw[cb + 3] += c3;
      }
    }
    multi_warp_sum<T, RB>(rs, lane);
    if ((lane & (32 / RB - 1)) == 0) {
      const int u = rb_slot<RB>(lane);
      if (r0 + u < n2) x[r0 + u] = rs[0];
    }
  }
  __syncthreads();
  for (int cc = tid; cc < n2; cc += NT) {
    T s = x[cc];
    for (int q = 0; q < NW; ++q) s += acc[q * ld + cc];
    x[cc] = s;
  }
  __syncthreads();
}

// The values before W (level-0 pivots, L10, the line blocks, S_TB: the small,
// latency-bound phases) are staged in shared memory by one bulk copy
// (cp.async.bulk) issued before the gather when they fit in a.headcap
// elements; the mbarrier wait is bounded by a.timeout_ns (status word on
// expiry).  W streams from global memory.
// The gather of the Schur-coupling kernels: the star's cells in closed form
// (slot s = x side + 2 y side + 4 z side: the lowest cell of the star plus
// the sides' strides), so no shared table and no barrier; zeroes y and the
// scratch (the range after g, which the gather fills completely).  The caller
// ends the phase with a barrier.
template <typename T, int NT>
__device__ __forceinline__ void sc_gather(const PatchSolveArgs<T> &a, const PatchDev &P, const ClassDev &C, T *gv) {
  const int tid = threadIdx.x;
  const Grid &g = a.g;
  const int n3 = g.n * g.n * g.n, nG = C.nG;
  for (int i = nG + tid; i < 2 * nG + a.tmpcap; i += NT) gv[i] = T(0);
  const int lo = star_cell_along(C.full[0], P.v[0], g.nx, 0) +
                 g.nx * (star_cell_along(C.full[1], P.v[1], g.ny, 0) + g.ny * star_cell_along(C.full[2], P.v[2], g.nz, 0));
  const int sy = g.nx, sz = g.nx * g.ny;
  const T *E = a.E;
  // the eight codes of a dof in two 16-byte loads, then all its cell values in
  // flight at once; summed in code order up to the first -1
  for (int k = tid; k < nG; k += NT) {
    const int4 c0 = reinterpret_cast<const int4 *>(C.gsrc + 8 * k)[0];
    const int4 c1 = reinterpret_cast<const int4 *>(C.gsrc + 8 * k)[1];
    const int code[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    T e[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int cd = code[q];
      const int slot = cd >> 16;
      const int cell = lo + (slot & 1) + ((slot >> 1) & 1) * sy + (slot >> 2) * sz;
      const T *ep = cd >= 0 ? E + (int64_t)cell * n3 + (cd & 0xffff) : E;  // a valid address either way
      e[q] = cd >= 0 ? load_na(ep) : T(0);
    }
    T r = 0;
    bool live = true;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      live = live && code[q] >= 0;
      r += live ? e[q] : T(0);
    }
    gv[k] = r;
  }
}

// everything after the gather: Lh holds the values before S_TB (staged or
// global), S_TB from Lh when stage_st else from global, W from global
template <typename T, int NT, int SRB>
__device__ __forceinline__ void sc_patch_compute(const PatchSolveArgs<T> &a, const PatchDev &P, const ClassDev &C,
                                                 const T *Lh, const T *Lv, T *gv, bool stage_st) {
  const int tid = threadIdx.x;
  const int nG = C.nG, nb = C.n0 + C.n1, n2 = C.n2, ld = C.ldT;
  // gv: g, later r_B and u_B; yv: y_B, then x_T in its top part
  T *yv = gv + nG, *tmp = yv + nG;
  const int l1 = (C.n1 + 3) & ~3;
  // acc at a 16-byte aligned offset from gv (gv itself is aligned): tmp has 4 elements of slack
  T *t1 = tmp, *acc = gv + ((2 * nG + 2 * l1 + 3) & ~3);
  T *X = a.X + P.xoff;
  bb_solve<T, NT>(C, Lh, gv, yv, t1);  // y_B = S_BB^{-1} g_B
  const T *st = (stage_st ? Lh : Lv) + C.off_st;
  for (int t = tid; t < n2; t += NT) {  // v_T = g_T - S_TB y_B, in place
    T s = 0;
    for (int e = 0; e < C.KT; ++e) {
      const int col = C.st_col[e * ld + t];
      if (col >= 0) s += st[e * ld + t] * yv[col];
    }
    gv[nb + t] -= s;
  }
  __syncthreads();
  sym_apply<T, NT, SRB>(C, Lv + C.off_z, gv + nb, yv + nb, acc, ld);  // x_T = W v_T
  for (int k = tid; k < n2; k += NT) X[nb + k] = yv[nb + k];
  for (int cc = tid; cc < nb; cc += NT) {  // r_B = S_BT x_T (g_B is no longer needed)
    T s = 0;
    const int q1 = C.ct_ptr[cc + 1];
    for (int q = C.ct_ptr[cc]; q < q1; ++q) {
      const int pos = C.ct_pos[q];
      s += st[pos] * yv[nb + pos % ld];
    }
    gv[cc] = s;
  }
  __syncthreads();
  bb_solve<T, NT>(C, Lh, gv, gv, t1, yv, X);  // u_B = S_BB^{-1} r_B in place, X_B = y_B - u_B
}

// the solve of the patch at position slot of a.order by the whole CTA
template <typename T, int NT, int SRB>
__device__ __forceinline__ void sc_patch_one(const PatchSolveArgs<T> &a, int slot) {
  extern __shared__ __align__(128) unsigned char smem_[];
  const int tid = threadIdx.x;
  const PatchDev P = a.patches[a.order[slot]];
  const ClassDev &C = a.cls[P.cls];
  __shared__ __align__(8) uint64_t bar, stall;  // stall: test hook, never completed
  __shared__ int sFail;
  T *H = reinterpret_cast<T *>(smem_);  // a.headcap elements (a multiple of 4)
  T *gv = H + a.headcap;
  const T *Lv = a.L + P.voff;
  const int64_t hend = a.stage_st ? C.off_z : C.off_st;  // staged prefix (a multiple of 4 elements)
  const bool stage = hend > 0 && hend <= a.headcap;
  if (tid == 0) {
    if (stage) {
      sFail = 0;
      bulk::mbar_init(&bar, 1);
      bulk::mbar_init(&stall, 1);
      bulk::fence_mbar_init();
      const uint32_t bytes = (uint32_t)(hend * (int64_t)sizeof(T));  // a multiple of 16
      bulk::mbar_arrive_expect_tx(&bar, bytes);
      for (uint32_t off = 0; off < bytes; off += 32768)
        bulk::bulk_g2s(reinterpret_cast<char *>(H) + off, reinterpret_cast<const char *>(Lv) + off,
                       bytes - off < 32768 ? bytes - off : 32768, &bar);
    }
    // W (a.prefetch: the whole value block) into L2 while the gather and the lower solve run
    const int64_t pf0 = a.prefetch ? 0 : C.off_z;
    const uint32_t wb = (uint32_t)((C.nval - pf0) * (int64_t)sizeof(T));
    const char *ws = reinterpret_cast<const char *>(Lv + pf0);
    for (uint32_t off = 0; off < wb; off += 32768) bulk::prefetch_l2(ws + off, wb - off < 32768 ? wb - off : 32768);
  }
  __syncthreads();  // the barriers' initialisation and sFail are visible
  sc_gather<T, NT>(a, P, C, gv);  // also zeroes y and tmp
  const T *Lh = Lv;
  if (stage) {  // the staging wait shares the gather's barrier
    bool ok = !a.inject_stall || bulk::mbar_wait_bounded(&stall, 0, a.timeout_ns);  // never completes
    ok = ok && bulk::mbar_wait_bounded(&bar, 0, a.timeout_ns);
    if (!ok) sFail = 1;
  }
  __syncthreads();
  if (stage) {
    if (sFail) {
      bulk::mbar_wait_bounded(&bar, 0, a.timeout_ns);  // a second bounded wait for the copy in flight
      if (tid == 0) atomicExch(a.status, 1);
      return;
    }
    Lh = H;
  }
  sc_patch_compute<T, NT, SRB>(a, P, C, Lh, Lv, gv, a.stage_st != 0);
}

template <typename T, int NT, int SRB, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_patch_solve_sc(PatchSolveArgs<T> a) {
  sc_patch_one<T, NT, SRB>(a, blockIdx.x);
}

// The patches of many problems in one launch: work[b] = (problem, position in
// that problem's patch order), the list sorted by the patches' value counts,
// largest first; a CTA whose problem is no longer active (converged) returns
// at once.
template <typename T, int NT, int SRB, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_patch_solve_sc_multi(const PatchSolveArgs<T> *__restrict__ args,
                                                                   const int2 *__restrict__ work,
                                                                   const int *__restrict__ active) {
  const int2 w = work[blockIdx.x];
  if (active[w.x] == 0) return;  // uniform over the CTA
  sc_patch_one<T, NT, SRB>(args[w.x], w.y);
}

// Persistent variant: each CTA walks the patch order with a stride of the
// grid.  While it solves one patch, the next one's lower-block values (before
// S_TB) are bulk-copied into the other of two shared-memory buffers and its
// S_TB and W are prefetched into L2, so that every phase of the next solve
// reads on-chip memory or L2.  Each buffer has its own mbarrier (one phase per
// copy); every wait is bounded by a.timeout_ns, after which the CTA waits once
// more (bounded) for its copies in flight, sets the status word and returns.
template <typename T, int NT, int SRB, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_patch_solve_scp(PatchSolveArgs<T> a, int npatch) {
  extern __shared__ __align__(128) unsigned char smem_[];
  const int tid = threadIdx.x;
  __shared__ int sCell[8];
  __shared__ __align__(8) uint64_t bar[3];  // [2]: test hook, never completed
  __shared__ int sFail, sPend[2];
  T *const H0 = reinterpret_cast<T *>(smem_);  // two buffers of a.headcap elements (multiples of 4)
  T *const H1 = H0 + a.headcap;
  T *gv = H1 + a.headcap;
  auto issue = [&](int it, int b) {  // thread 0: stage patch `it` into buffer b, S_TB and W into L2
    const PatchDev Q = a.patches[a.order[it]];
    const ClassDev &D = a.cls[Q.cls];
    const T *Lq = a.L + Q.voff;
    sPend[b] = 0;
    if (D.off_st > 0 && D.off_st <= a.headcap) {
      bulk::fence_proxy_async();  // the buffer's previous contents were read by every thread
      const uint32_t bytes = (uint32_t)(D.off_st * (int64_t)sizeof(T));  // a multiple of 16
      char *dst = reinterpret_cast<char *>(b ? H1 : H0);
      bulk::mbar_arrive_expect_tx(&bar[b], bytes);
      for (uint32_t off = 0; off < bytes; off += 32768)
        bulk::bulk_g2s(dst + off, reinterpret_cast<const char *>(Lq) + off, bytes - off < 32768 ? bytes - off : 32768,
                       &bar[b]);
      sPend[b] = 1;
    }
    const uint32_t wb = (uint32_t)((D.nval - D.off_st) * (int64_t)sizeof(T));
    const char *ws = reinterpret_cast<const char *>(Lq + D.off_st);
    for (uint32_t off = 0; off < wb; off += 32768) bulk::prefetch_l2(ws + off, wb - off < 32768 ? wb - off : 32768);
  };
  if (tid == 0) {
    bulk::mbar_init(&bar[0], 1);
    bulk::mbar_init(&bar[1], 1);
    bulk::mbar_init(&bar[2], 1);  // the test hook's barrier is a valid one that nothing completes
    bulk::fence_mbar_init();
    sFail = 0;
    sPend[0] = sPend[1] = 0;
    if ((int)blockIdx.x < npatch) issue(blockIdx.x, 0);
  }
  __syncthreads();
  uint32_t par[2] = {0, 0};
  int b = 0;
  for (int it = blockIdx.x; it < npatch; it += gridDim.x, b ^= 1) {
    const PatchDev P = a.patches[a.order[it]];
    const ClassDev &C = a.cls[P.cls];
    if (tid == 0 && it + (int)gridDim.x < npatch) issue(it + gridDim.x, b ^ 1);
    patch_gather<T, NT, 2>(a, P, C, gv, sCell);  // also zeroes y and tmp (barriers inside)
    const T *Lv = a.L + P.voff;
    const T *Lh = Lv;
    if (sPend[b]) {
      bool ok = !a.inject_stall || bulk::mbar_wait_bounded(&bar[2], 0, a.timeout_ns);  // never completes
      ok = ok && bulk::mbar_wait_bounded(&bar[b], par[b], a.timeout_ns);
      if (!ok) sFail = 1;
      __syncthreads();
      if (sFail) {
        for (int q = 0; q < 2; ++q)  // a second bounded wait for every copy in flight
          if (sPend[q]) bulk::mbar_wait_bounded(&bar[q], par[q], a.timeout_ns);
        if (tid == 0) atomicExch(a.status, 1);
        return;
      }
      par[b] ^= 1u;
      Lh = b ? H1 : H0;
    }
    sc_patch_compute<T, NT, SRB>(a, P, C, Lh, Lv, gv, false);
    __syncthreads();  // buffer b and gv are free for the next patch
  }
}

// Persistent variant with each patch's whole solve operator staged in shared
// memory (level-0 pivots, L10, the line blocks, S_TB and W): two buffers of
// a.headcap elements; while the CTA solves one patch from one buffer, the next
// patch's values are bulk-copied into the other, so the copies overlap the
// solves and every phase after the gather (which reads the L2-resident cell
// residual) runs on chip.  Each stored value leaves DRAM once per sweep.  The
// launcher guarantees a.headcap >= the largest class's value count.  Each
// buffer has its own mbarrier (one phase per copy); every wait is bounded by
// a.timeout_ns, after which the CTA waits once more (bounded) for its copies
// in flight, sets the status word and returns.
template <typename T, int NT, int SRB>
__global__ void __launch_bounds__(NT, 1) k_patch_solve_scf(PatchSolveArgs<T> a, int npatch) {
  extern __shared__ __align__(128) unsigned char smem_[];
  const int tid = threadIdx.x;
  __shared__ __align__(8) uint64_t bar[3];  // [2]: test hook, never completed
  __shared__ int sFail, sPend[2];
  T *const H0 = reinterpret_cast<T *>(smem_);
  T *const H1 = H0 + a.headcap;
  T *gv = H1 + a.headcap;
  auto issue = [&](int it, int b) {  // thread 0: copy patch `it`'s values into buffer b
    const PatchDev Q = a.patches[a.order[it]];
    const ClassDev &D = a.cls[Q.cls];
    sPend[b] = 0;
    if (D.nval > 0) {
      bulk::fence_proxy_async();  // the buffer's previous contents were read by every thread
      const uint32_t bytes = (uint32_t)(D.nval * (int64_t)sizeof(T));  // a multiple of 16
      char *dst = reinterpret_cast<char *>(b ? H1 : H0);
      const char *src = reinterpret_cast<const char *>(a.L + Q.voff);
      bulk::mbar_arrive_expect_tx(&bar[b], bytes);
      for (uint32_t off = 0; off < bytes; off += 32768)
        bulk::bulk_g2s(dst + off, src + off, bytes - off < 32768 ? bytes - off : 32768, &bar[b]);
      sPend[b] = 1;
    }
  };
  if (tid == 0) {
    bulk::mbar_init(&bar[0], 1);
    bulk::mbar_init(&bar[1], 1);
    bulk::mbar_init(&bar[2], 1);
    bulk::fence_mbar_init();
    sFail = 0;
    sPend[0] = sPend[1] = 0;
    if ((int)blockIdx.x < npatch) issue(blockIdx.x, 0);
  }
  __syncthreads();
  uint32_t par[2] = {0, 0};
  int b = 0;
  for (int it = blockIdx.x; it < npatch; it += gridDim.x, b ^= 1) {
    const PatchDev P = a.patches[a.order[it]];
    const ClassDev &C = a.cls[P.cls];
    if (tid == 0 && it + (int)gridDim.x < npatch) issue(it + gridDim.x, b ^ 1);
    sc_gather<T, NT>(a, P, C, gv);  // also zeroes y and the scratch
    if (sPend[b]) {
      bool ok = !a.inject_stall || bulk::mbar_wait_bounded(&bar[2], 0, a.timeout_ns);  // never completes
      ok = ok && bulk::mbar_wait_bounded(&bar[b], par[b], a.timeout_ns);
      if (!ok) sFail = 1;
    }
    __syncthreads();  // the gather is complete and every thread has seen its wait end
    if (sFail) {
      for (int q = 0; q < 2; ++q)  // a second bounded wait for every copy in flight
        if (sPend[q]) bulk::mbar_wait_bounded(&bar[q], par[q], a.timeout_ns);
      if (tid == 0) atomicExch(a.status, 1);
      return;
    }
    if (sPend[b]) par[b] ^= 1u;
    const T *Hb = b ? H1 : H0;
    sc_patch_compute<T, NT, SRB>(a, P, C, Hb, Hb, gv, true);
    __syncthreads();  // buffer b and gv are free for the next patch
  }
}

int patch_sc_tmp(int maxN1, int maxN2, int threads) {
  const int l1 = (maxN1 + 3) & ~3, l2 = (maxN2 + 3) & ~3;
  return 2 * l1 + (threads / 32) * l2 + 4;  // + 4: the accumulators' 16-byte alignment
}

template <typename T>
size_t patch_sc_smem(int maxG, int maxN1, int maxN2, int threads, int headcap) {
  return sizeof(T) * ((size_t)headcap + 2 * (size_t)maxG + patch_sc_tmp(maxN1, maxN2, threads));
}

template <typename T>
void launch_patch_scp(const PatchSolveArgs<T> &a, int npatch, size_t smem, cudaStream_t st) {
  if (npatch <= 0) return;
  static size_t attr = 0;
  static int per_sm = 0, nsm = 0;
  if (attr < smem) {
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_scp<T, 256, 2, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    FDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_patch_solve_scp<T, 256, 2, 5>, 256, smem));
    int dev = 0;
    FDM_CUDA(cudaGetDevice(&dev));
    FDM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    attr = smem;
  }
  const int grid = std::max(1, std::min(npatch, std::max(per_sm, 1) * nsm));
  k_patch_solve_scp<T, 256, 2, 5><<<grid, 256, smem, st>>>(a, npatch);
}

// the fully staged persistent kernel: one CTA per SM (the two buffers take
// most of its shared memory), threads 256, 512 or 1024
template <typename T, int NT, int SRB>
void launch_scf_nt(const PatchSolveArgs<T> &a, int npatch, size_t smem, cudaStream_t st) {
  static size_t attr = 0;
  static int per_sm = 0, nsm = 0;
  if (attr < smem) {
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_scf<T, NT, SRB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    FDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_patch_solve_scf<T, NT, SRB>, NT, smem));
    int dev = 0;
    FDM_CUDA(cudaGetDevice(&dev));
    FDM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    attr = smem;
  }
  if (per_sm < 1) fail(FDM_EINVAL, "fully staged patch solve: launch configuration does not fit an SM");
  const int grid = std::max(1, std::min(npatch, per_sm * nsm));
  k_patch_solve_scf<T, NT, SRB><<<grid, NT, smem, st>>>(a, npatch);
}

template <typename T>
void launch_patch_scf(const PatchSolveArgs<T> &a, int npatch, size_t smem, int threads, cudaStream_t st) {
  if (npatch <= 0) return;
  if (threads >= 1024) launch_scf_nt<T, 1024, 2>(a, npatch, smem, st);
  else if (threads >= 512) launch_scf_nt<T, 512, 2>(a, npatch, smem, st);
  else launch_scf_nt<T, 256, 4>(a, npatch, smem, st);
}

template <typename T>
void launch_patch_sc(const PatchSolveArgs<T> &a, int npatch, size_t smem, int threads, cudaStream_t st) {
  if (npatch <= 0) return;
  static bool attr = false;
  if (!attr) {
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_sc<T, 256, 2, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024));
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_sc<T, 256, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024));
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_sc<T, 512, 4, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024));
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_sc<T, 128, 2, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024));
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_sc<T, 256, 2, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, 224 * 1024));
    attr = true;
  }
  if (threads <= 128) k_patch_solve_sc<T, 128, 2, 8><<<npatch, 128, smem, st>>>(a);
  else if (threads == 256 && !a.stage_st) k_patch_solve_sc<T, 256, 2, 6><<<npatch, 256, smem, st>>>(a);
  else if (threads >= 512) k_patch_solve_sc<T, 512, 4, 2><<<npatch, 512, smem, st>>>(a);
  else if (a.rows8) k_patch_solve_sc<T, 256, 4, 4><<<npatch, 256, smem, st>>>(a);
  else k_patch_solve_sc<T, 256, 2, 5><<<npatch, 256, smem, st>>>(a);
}

template <typename T>
void launch_patch_sc_multi(const PatchSolveArgs<T> *args, const int2 *work, int nwork, const int *active, size_t smem,
                           cudaStream_t st) {
  if (nwork <= 0) return;
  static bool attr = false;
  if (!attr) {
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_sc_multi<T, 256, 4, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  224 * 1024));
    attr = true;
  }
  k_patch_solve_sc_multi<T, 256, 4, 4><<<nwork, 256, smem, st>>>(args, work, active);
}

int patch_tmp_elems(int maxN1, int maxN2) {
  // tmp holds a level-1 vector (n1) or the sliced partial sums of L21^T x_2
  // and Z^T y_2 (slices * row length, slices clamped to fit)
  int tmpn = 4 * PATCH_THREADS_MAX;
  int l1 = (maxN1 + 3) & ~3, l2 = (maxN2 + 3) & ~3;
  if (l1 > tmpn) tmpn = l1;
  if (l2 > tmpn) tmpn = l2;
  return tmpn;
}

template <typename T>
size_t patch_smem_bytes(int n, int maxG, int maxN1, int maxN2) {
  (void)n;
  return sizeof(T) * (3 * maxG + patch_tmp_elems(maxN1, maxN2));
}

// ctas_per_sm > 0 pads the dynamic shared memory so that at most that many
// patch CTAs are resident per SM (bounds the factors in flight in L2)
template <typename T>
size_t patch_smem_for_occupancy(size_t need, int ctas_per_sm) {
  if (ctas_per_sm <= 0) return need;
  size_t cap = (size_t)(227 * 1024) / ctas_per_sm;
  if (cap > 200 * 1024) cap = 200 * 1024;
  cap = cap > 1024 ? cap - 1024 : cap;  // room for static shared memory and the per-CTA reserve
  return need > cap ? need : cap;
}

template <typename T, int NT>
void launch_patch_nt(const PatchSolveArgs<T> &a, int npatch, size_t smem, cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_patch_solve<T, NT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(k_patch_solve<T, NT, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr = true;
  }
  if (a.rows8) k_patch_solve<T, NT, 8><<<npatch, NT, smem, st>>>(a);
  else k_patch_solve<T, NT, 4><<<npatch, NT, smem, st>>>(a);
}

int patch_resident_tmp(int maxN1, int maxN2, int threads) {
  int tmpn = 4 * threads;
  int l1 = (maxN1 + 3) & ~3, l2 = (maxN2 + 3) & ~3;
  return std::max(tmpn, std::max(l1, l2));
}

template <typename T>
size_t patch_resident_smem(int fcap, int maxG, int tmpcap) {
  return sizeof(T) * ((size_t)fcap + 3 * (size_t)maxG + tmpcap);
}

template <typename T, int NT>
void launch_resident_nt(const PatchSolveArgs<T> &a, int npatch, int fcap, size_t smem, cudaStream_t st) {
  static size_t attr = 0;
  static int per_sm = 0, nsm = 0;
  if (attr < smem) {
    FDM_CUDA(cudaFuncSetAttribute(k_patch_resident<T, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    FDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_patch_resident<T, NT>, NT, smem));
    int dev = 0;
    FDM_CUDA(cudaGetDevice(&dev));
    FDM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    attr = smem;
  }
  const int grid = std::max(1, std::min(npatch, std::max(per_sm, 1) * nsm));
  k_patch_resident<T, NT><<<grid, NT, smem, st>>>(a, npatch, fcap);
  FDM_CUDA(cudaGetLastError());
}

template <typename T>
void launch_patch_resident(const PatchSolveArgs<T> &a, int npatch, int fcap, size_t smem, int threads,
                           cudaStream_t st) {
  if (npatch <= 0) return;
  if (threads >= 1024) launch_resident_nt<T, 1024>(a, npatch, fcap, smem, st);
  else if (threads >= 512) launch_resident_nt<T, 512>(a, npatch, fcap, smem, st);
  else launch_resident_nt<T, 256>(a, npatch, fcap, smem, st);
}

template <typename T>
void launch_patch_solve(const PatchSolveArgs<T> &a, int npatch, size_t smem, int threads, cudaStream_t st) {
  if (npatch <= 0) return;
  if (threads >= 1024) launch_patch_nt<T, 1024>(a, npatch, smem, st);
  else if (threads >= 512) launch_patch_nt<T, 512>(a, npatch, smem, st);
  else launch_patch_nt<T, 256>(a, npatch, smem, st);
}

#define INST(T)                                                                                          \
  template void launch_restrict_fdm<T, double>(const Grid &, const double *, const T *, const double *, T *, \
                                               cudaStream_t);                                                \
  template void launch_restrict_fdm<T, float>(const Grid &, const float *, const T *, const double *, T *,   \
                                              cudaStream_t);                                                 \
  template void launch_interp_fdm<T, double>(const InterpArgs<T> &, double, double *, cudaStream_t);        \
  template void launch_interp_fdm<T, float>(const InterpArgs<T> &, double, float *, cudaStream_t);          \
  template size_t patch_smem_bytes<T>(int, int, int, int);                                                       \
  template void launch_patch_solve<T>(const PatchSolveArgs<T> &, int, size_t, int, cudaStream_t);        \
  template size_t patch_resident_smem<T>(int, int, int);                                                    \
  template void launch_patch_resident<T>(const PatchSolveArgs<T> &, int, int, size_t, int, cudaStream_t);  \
  template size_t patch_smem_for_occupancy<T>(size_t, int);                                                 \
  template size_t patch_sc_smem<T>(int, int, int, int, int);                                                \
  template void launch_patch_sc<T>(const PatchSolveArgs<T> &, int, size_t, int, cudaStream_t);             \
  template void launch_patch_sc_multi<T>(const PatchSolveArgs<T> *, const int2 *, int, const int *, size_t,    \
                                         cudaStream_t);                                                        \
  template void launch_patch_scp<T>(const PatchSolveArgs<T> &, int, size_t, cudaStream_t);                  \
  template void launch_patch_scf<T>(const PatchSolveArgs<T> &, int, size_t, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace fdm
