// Warp-per-patch form of the Schur-coupling patch solve (Sections 2.4-2.6).
//
// The same exact star solve as the CTA kernels of k_asm.cu, for the same
// factor layout:
//   y_B = S_BB^{-1} g_B,  x_T = W (g_T - S_TB y_B),  x_B = y_B - S_BB^{-1} S_BT x_T,
// with S_BB = L_BB L_BB^T (diagonal level 0, sparse L10, symmetric inverses of
// the level-1 line blocks) and W = (L_TT L_TT^T)^{-1} stored as its lower
// triangle.  Here one warp solves one patch: every phase is separated by a
// warp barrier only, each lane walks its share of the rows with all loads of
// a row issued together, and the column half of the symmetric W product
// accumulates in registers of the lane that owns the column.  A CTA holds
// WPB independent patches, so an SM keeps tens of patch solves in flight and
// the latency of one phase of one patch is covered by the others; the class
// tables (the same for every patch of a class) are shared through L1.
#include "bulk.cuh"
#include "kernels.h"

namespace fdm {
namespace {

template <typename T> struct W4 { T x, y, z, w; };
__device__ __forceinline__ W4<float> ldg4(const float *p) {
  const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ W4<double> ldg4(const double *p) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p)), b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  return {a.x, a.y, b.x, b.y};
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// per-warp shared memory: g [maxG] | y [maxG] | t1 [l1] | q0 [l0], each
// section padded to 4 elements
__host__ __device__ __forceinline__ int up4(int n) { return (n + 3) & ~3; }

// S_BB^{-1} over the lower block for one warp (in and out may alias):
//   q0 = D_0^{-1} in_0,  t_1 = in_1 - L_10 q0,  out_1 = (L_11 L_11^T)^{-1} t_1 (line blocks),
//   out_0 = D_0^{-1} (q0 - L_10^T out_1);
// fin, when given, receives y - out (the final lower values).
template <typename T>
__device__ __forceinline__ void warp_bb_solve(const ClassDev &C, const T *__restrict__ Lv, const T *in, T *out, T *t1,
                                              T *q0, int lane, const T *y = nullptr, T *fin = nullptr) {
  const int n0 = C.n0, n1 = C.n1, ldr0 = C.ldr0;
  const T *dinv0 = Lv + C.off_dinv0, *ell = Lv + C.off_ell;
  for (int j = lane; j < n0; j += 32) q0[j] = in[j] * __ldg(dinv0 + j);
  __syncwarp();
  for (int r = lane; r < n1; r += 32) {
    T acc = 0;
#pragma unroll 4
    for (int e = 0; e < C.K0; ++e) {
      const int col = __ldg(C.ell_col + e * ldr0 + r);
      const T v = __ldg(ell + e * ldr0 + r);
      acc += col >= 0 ? v * q0[col] : T(0);
    }
    t1[r] = in[n0 + r] - acc;
  }
  __syncwarp();
  for (int r = lane; r < n1; r += 32) {
    const int b = __ldg(C.line_of + r);
    const int s0 = __ldg(C.line_start + b), w = __ldg(C.line_len + b), i = r - s0;
    const T *Mb = Lv + C.off_lines + __ldg(C.line_off + b);
    T acc = 0;
    for (int cc = 0; cc < w; ++cc) acc += __ldg(Mb + cc * w + i) * t1[s0 + cc];
    out[n0 + r] = acc;
    if (fin) fin[n0 + r] = y[n0 + r] - acc;
  }
  __syncwarp();
  for (int j = lane; j < n0; j += 32) {
    T s = q0[j];
    const int q1 = __ldg(C.cB_ptr + j + 1);
#pragma unroll 4
    for (int q = __ldg(C.cB_ptr + j); q < q1; ++q) {
      const int pos = __ldg(C.cB_pos + q);
      s -= __ldg(ell + pos) * out[n0 + pos % ldr0];
    }
    s *= __ldg(dinv0 + j);
    out[j] = s;
    if (fin) fin[j] = y[j] - s;
  }
  __syncwarp();
}

// x = W v for one warp, W symmetric with its lower triangle stored by rows
// (row r holds W[r][0..r], zero-padded to a multiple of 4 at zoff[r]).  Lane l
// owns the column groups q4 = l + 32 q (q < NQ): it reads those groups of RB
// rows at a time, adds their row dots (butterfly over the warp) and keeps the
// strictly lower entries times v_r as column sums in registers.  x must not
// alias v; the row dots are written to x, the column sums added at the end.
template <typename T, int NQ, int RB>
__device__ __forceinline__ void warp_sym_apply(const ClassDev &C, const T *__restrict__ Wv, const T *v, T *x,
                                               int lane) {
  const int n2 = C.n2;
  T cacc[NQ][4];
  T vv[NQ][4];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int cb = 4 * (lane + 32 * q);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      cacc[q][i] = 0;
      vv[q][i] = cb + i < n2 ? v[cb + i] : T(0);
    }
  }
  for (int r0 = 0; r0 < n2; r0 += RB) {
    W4<T> wr[RB][NQ];
    T vr[RB];
#pragma unroll
    for (int u = 0; u < RB; ++u) {
      const int r = r0 + u < n2 ? r0 + u : n2 - 1;
      const int z0 = __ldg(C.zoff + r), ng = r0 + u < n2 ? (__ldg(C.zoff + r + 1) - z0) / 4 : 0;
      vr[u] = r0 + u < n2 ? v[r] : T(0);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int q4 = lane + 32 * q;
        wr[u][q] = q4 < ng ? ldg4(Wv + z0 + 4 * q4) : W4<T>{0, 0, 0, 0};
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
        const W4<T> &w = wr[u][q];
        s += w.x * vv[q][0] + w.y * vv[q][1] + w.z * vv[q][2] + w.w * vv[q][3];
        cacc[q][0] += (cb < r ? w.x : T(0)) * vr[u];
        cacc[q][1] += (cb + 1 < r ? w.y : T(0)) * vr[u];
        cacc[q][2] += (cb + 2 < r ? w.z : T(0)) * vr[u];
        cacc[q][3] += (cb + 3 < r ? w.w : T(0)) * vr[u];
      }
      rs[u] = s;
    }
#pragma unroll
    for (int u = 0; u < RB; ++u) rs[u] = warp_sum(rs[u]);
    if (lane < RB && r0 + lane < n2) {
      T s = rs[0];
#pragma unroll
      for (int u = 1; u < RB; ++u) s = lane == u ? rs[u] : s;
      x[r0 + lane] = s;
    }
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int cb = 4 * (lane + 32 * q);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (cb + i < n2) x[cb + i] += cacc[q][i];
  }
  __syncwarp();
}

}  // namespace

// One warp per patch (patch index = blockIdx.x * WPB + warp in the solve
// order); ws = per-warp shared-memory elements.  No CTA barrier: a warp whose
// index is past the last patch returns at once.
template <typename T, int WPB, int NQ, int RB, int MINB>
__global__ void __launch_bounds__(WPB * 32, MINB) k_patch_solve_scw(PatchSolveArgs<T> a, int npatch, int ws) {
  extern __shared__ __align__(16) unsigned char smem_[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int it = blockIdx.x * WPB + warp;
  if (it >= npatch) return;
  const PatchDev P = a.patches[a.order[it]];
  const ClassDev &C = a.cls[P.cls];
  const int nG = C.nG, n0 = C.n0, n1 = C.n1, n2 = C.n2, nb = n0 + n1, ldT = C.ldT;
  T *g = reinterpret_cast<T *>(smem_) + (size_t)warp * ws;
  T *y = g + up4(nG);
  T *t1 = y + up4(nG);
  T *q0 = t1 + up4(n1);
  const T *__restrict__ Lv = a.L + P.voff;
  T *X = a.X + P.xoff;
  // the star's cells in closed form: slot s = x side + 2 y side + 4 z side
  const Grid &gr = a.g;
  const int lo = star_cell_along(C.full[0], P.v[0], gr.nx, 0) +
                 gr.nx * (star_cell_along(C.full[1], P.v[1], gr.ny, 0) + gr.ny * star_cell_along(C.full[2], P.v[2], gr.nz, 0));
  const int sy = gr.nx, sz = gr.nx * gr.ny, n3 = gr.n * gr.n * gr.n;
  // gather: the condensed cell residuals of each interface dof summed over the
  // star's cells in the fixed order of its code list (-1 terminated)
  for (int k = lane; k < nG; k += 32) {
    const int4 c0 = __ldg(reinterpret_cast<const int4 *>(C.gsrc + 8 * k));
    const int4 c1 = __ldg(reinterpret_cast<const int4 *>(C.gsrc + 8 * k) + 1);
    const int code[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
    T e[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int cd = code[q];
      const int slot = cd >> 16;
      const int cell = lo + (slot & 1) + ((slot >> 1) & 1) * sy + (slot >> 2) * sz;
      e[q] = cd >= 0 ? a.E[(int64_t)cell * n3 + (cd & 0xffff)] : T(0);
    }
    T r = 0;
    bool live = true;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      live = live && code[q] >= 0;
      r += live ? e[q] : T(0);
    }
    g[k] = r;
  }
  __syncwarp();
  // y_B = S_BB^{-1} g_B
  warp_bb_solve<T>(C, Lv, g, y, t1, q0, lane);
  // v_T = g_T - S_TB y_B, in place
  const T *st = Lv + C.off_st;
  for (int t = lane; t < n2; t += 32) {
    T s = 0;
#pragma unroll 8
    for (int e = 0; e < C.KT; ++e) {
      const int col = __ldg(C.st_col + e * ldT + t);
      const T v = __ldg(st + e * ldT + t);
      s += col >= 0 ? v * y[col] : T(0);
    }
    g[nb + t] -= s;
  }
  __syncwarp();
  // x_T = W v_T (into y_T), written out
  if (n2 > 0) warp_sym_apply<T, NQ, RB>(C, Lv + C.off_z, g + nb, y + nb, lane);
  for (int k = lane; k < n2; k += 32) X[nb + k] = y[nb + k];
  // r_B = S_BT x_T (g_B is no longer needed)
  for (int cc = lane; cc < nb; cc += 32) {
    T s = 0;
    const int q1 = __ldg(C.ct_ptr + cc + 1);
#pragma unroll 4
    for (int q = __ldg(C.ct_ptr + cc); q < q1; ++q) {
      const int pos = __ldg(C.ct_pos + q);
      s += __ldg(st + pos) * y[nb + pos % ldT];
    }
    g[cc] = s;
  }
  __syncwarp();
  // u_B = S_BB^{-1} r_B in place, X_B = y_B - u_B
  warp_bb_solve<T>(C, Lv, g, g, t1, q0, lane, y, X);
}

// per-warp shared-memory elements for the largest class
int patch_scw_ws(int maxG, int maxN0, int maxN1) { return 2 * up4(maxG) + up4(maxN1) + up4(maxN0); }

// largest top block (n2) the register column sums of the W product cover: 4 x 32 x NQ
int patch_scw_max_n2(int nq) { return 128 * nq; }

template <typename T, int WPB, int NQ, int RB, int MINB>
void launch_scw_cfg(const PatchSolveArgs<T> &a, int npatch, int ws, cudaStream_t st) {
  const size_t smem = sizeof(T) * (size_t)WPB * ws;
  static size_t attr = 0;
  if (attr < smem) {
    FDM_CUDA(cudaFuncSetAttribute(k_patch_solve_scw<T, WPB, NQ, RB, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr = smem;
  }
  k_patch_solve_scw<T, WPB, NQ, RB, MINB><<<(npatch + WPB - 1) / WPB, WPB * 32, smem, st>>>(a, npatch, ws);
}

// warps: patches per CTA (4 or 8); maxN2 selects the register width of the W
// product's column sums (the caller checks maxN2 <= patch_scw_max_n2(4))
template <typename T>
void launch_patch_scw(const PatchSolveArgs<T> &a, int npatch, int ws, int warps, int maxN2, cudaStream_t st) {
  if (npatch <= 0) return;
  // FP32: 64 registers (32 warps per SM); FP64 values take twice the registers
  constexpr int M = sizeof(T) == 4 ? 1 : 2;
  if (maxN2 <= patch_scw_max_n2(2)) {
    if (warps <= 4) launch_scw_cfg<T, 4, 2, 2, 8 / M>(a, npatch, ws, st);
    else launch_scw_cfg<T, 8, 2, 2, 4 / M>(a, npatch, ws, st);
  } else {
    if (warps <= 4) launch_scw_cfg<T, 4, 4, 1, 8 / M>(a, npatch, ws, st);
    else launch_scw_cfg<T, 8, 4, 1, 4 / M>(a, npatch, ws, st);
  }
}

template void launch_patch_scw<float>(const PatchSolveArgs<float> &, int, int, int, int, cudaStream_t);
template void launch_patch_scw<double>(const PatchSolveArgs<double> &, int, int, int, int, cudaStream_t);

}  // namespace fdm
