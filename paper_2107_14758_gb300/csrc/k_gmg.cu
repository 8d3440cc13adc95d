// Geometric multigrid on the Q1 coarse problem (Section 3: the p-coarse
// problem is itself solved by multigrid).  Every level is a tensor grid of
// free vertices m = cells - 1 per axis, numbered lexicographically (x fastest),
// whose operator is a 27-point stencil stored coefficient-major, A[k][i] with
// k = (dx+1) + 3 (dy+1) + 9 (dz+1), so that consecutive threads (consecutive
// vertices) read consecutive words.  The level's damped-Jacobi weights
// dw = omega / A[13] are a separate array.
//
// One thread per vertex everywhere: the levels are HBM/L2-bound streams of the
// stencil (27 words per vertex) and launch-bound once they are small; the
// kernels are kept separate so that each is a plain gather without
// recomputation.
#include "kernels.h"

namespace fdm {

namespace {

constexpr int GMG_THREADS = 256;

template <typename T>
__device__ __forceinline__ void vertex_of(const GmgDev<T> &L, int i, int &ix, int &iy, int &iz) {
  ix = i % L.m[0];
  const int q = i / L.m[0];
  iy = q % L.m[1];
  iz = q / L.m[1];
}

// sum_k A[k][i] * val(j_k) over the stencil neighbours j_k that are free vertices
template <typename T, typename F>
__device__ __forceinline__ T stencil_sum(const GmgDev<T> &L, int i, F val) {
  int ix, iy, iz;
  vertex_of(L, i, ix, iy, iz);
  T s = T(0);
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz) {
    const int jz = iz + dz;
    if (jz < 0 || jz >= L.m[2]) continue;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int jy = iy + dy;
      if (jy < 0 || jy >= L.m[1]) continue;
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int jx = ix + dx;
        if (jx < 0 || jx >= L.m[0]) continue;
        const int k = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        s = fma(__ldg(L.A + (size_t)k * L.nf + i), val(jx + L.m[0] * (jy + L.m[1] * jz)), s);
      }
    }
  }
  return s;
}

// two Jacobi sweeps from x = 0: x1 = dw b, x2 = x1 + dw (b - A x1), with x1
// formed on the fly at every neighbour (no x1 array)
template <typename T>
__global__ void __launch_bounds__(GMG_THREADS) k_gmg_pre2(GmgDev<T> L, const T *__restrict__ b, T *__restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nf) return;
  const T ax = stencil_sum(L, i, [&](int j) { return __ldg(L.dw + j) * __ldg(b + j); });
  const T dwi = L.dw[i], bi = b[i];
  x[i] = dwi * bi + dwi * (bi - ax);
}

// one Jacobi sweep from x = 0: x = dw b
template <typename T>
__global__ void __launch_bounds__(GMG_THREADS) k_gmg_scale(GmgDev<T> L, const T *__restrict__ b, T *__restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nf) return;
  x[i] = L.dw[i] * b[i];
}

// out = x + dw (b - A x)
template <typename T>
__global__ void __launch_bounds__(GMG_THREADS) k_gmg_sweep(GmgDev<T> L, const T *__restrict__ b,
                                                           const T *__restrict__ x, T *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nf) return;
  const T ax = stencil_sum(L, i, [&](int j) { return __ldg(x + j); });
  out[i] = x[i] + L.dw[i] * (b[i] - ax);
}

// r = b - A x
template <typename T>
__global__ void __launch_bounds__(GMG_THREADS) k_gmg_resid(GmgDev<T> L, const T *__restrict__ b,
                                                           const T *__restrict__ x, T *__restrict__ r) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= L.nf) return;
  const T ax = stencil_sum(L, i, [&](int j) { return __ldg(x + j); });
  r[i] = b[i] - ax;
}

// weights of coarse vertex V at the fine vertices 2V-1, 2V, 2V+1 of one axis
template <typename T>
__device__ __forceinline__ void child_weights(const T *t, int V, T w[3]) {
  w[0] = t[2 * V - 1];
  w[1] = T(1);
  w[2] = T(1) - t[2 * V + 1];
}

// bc[I] = sum_i P[i][I] r[i]: coarse vertex I gathers its 27 fine children
// (all free: 2V +- 1 lies in [1, 2 mc + 1] = [1, mf])
template <typename T>
__global__ void __launch_bounds__(GMG_THREADS) k_gmg_restrict(GmgDev<T> F, GmgDev<T> C, const T *__restrict__ r,
                                                              T *__restrict__ bc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  if (I >= C.nf) return;
  int IX, IY, IZ;
  vertex_of(C, I, IX, IY, IZ);
  T wx[3], wy[3], wz[3];
  child_weights(F.t[0], IX + 1, wx);
  child_weights(F.t[1], IY + 1, wy);
  child_weights(F.t[2], IZ + 1, wz);
  const int fx = 2 * IX + 1, fy = 2 * IY + 1, fz = 2 * IZ + 1;  // free index of the centre child
  T s = T(0);
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int j = (fx + dx - 1) + F.m[0] * ((fy + dy - 1) + F.m[1] * (fz + dz - 1));
        s = fma(wx[dx] * wy[dy] * wz[dz], __ldg(r + j), s);
      }
  bc[I] = s;
}

// parents of fine vertex v (1..mf) along one axis: coarse free indices and weights
template <typename T>
__device__ __forceinline__ int parents(const T *t, int v, int mc, int idx[2], T w[2]) {
  if ((v & 1) == 0) {
    idx[0] = v / 2 - 1;
    w[0] = T(1);
    return 1;
  }
  int k = 0;
  const T tv = t[v];
  if ((v - 1) / 2 >= 1) { idx[k] = (v - 1) / 2 - 1; w[k] = T(1) - tv; ++k; }
  if ((v + 1) / 2 <= mc) { idx[k] = (v + 1) / 2 - 1; w[k] = tv; ++k; }
  return k;
}

// x[i] += sum_I P[i][I] xc[I]
template <typename T>
__global__ void __launch_bounds__(GMG_THREADS) k_gmg_prolong(GmgDev<T> F, GmgDev<T> C, const T *__restrict__ xc,
                                                             T *__restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F.nf) return;
  int ix, iy, iz;
  vertex_of(F, i, ix, iy, iz);
  int px[2], py[2], pz[2];
  T wx[2], wy[2], wz[2];
  const int nx = parents(F.t[0], ix + 1, C.m[0], px, wx);
  const int ny = parents(F.t[1], iy + 1, C.m[1], py, wy);
  const int nz = parents(F.t[2], iz + 1, C.m[2], pz, wz);
  T s = T(0);
  for (int c = 0; c < nz; ++c)
    for (int b = 0; b < ny; ++b)
      for (int a = 0; a < nx; ++a)
        s = fma(wx[a] * wy[b] * wz[c], __ldg(xc + px[a] + C.m[0] * (py[b] + C.m[1] * pz[c])), s);
  x[i] += s;
}

inline int blocks(int n) { return (n + GMG_THREADS - 1) / GMG_THREADS; }

}  // namespace

template <typename T>
void launch_gmg_pre(const GmgDev<T> &L, int nu, const T *b, T *x, cudaStream_t st) {
  if (L.nf == 0) return;
  if (nu >= 2) k_gmg_pre2<T><<<blocks(L.nf), GMG_THREADS, 0, st>>>(L, b, x);
  else k_gmg_scale<T><<<blocks(L.nf), GMG_THREADS, 0, st>>>(L, b, x);
}
template <typename T>
void launch_gmg_sweep(const GmgDev<T> &L, const T *b, const T *x, T *out, cudaStream_t st) {
  if (L.nf == 0) return;
  k_gmg_sweep<T><<<blocks(L.nf), GMG_THREADS, 0, st>>>(L, b, x, out);
}
template <typename T>
void launch_gmg_resid(const GmgDev<T> &L, const T *b, const T *x, T *r, cudaStream_t st) {
  if (L.nf == 0) return;
  k_gmg_resid<T><<<blocks(L.nf), GMG_THREADS, 0, st>>>(L, b, x, r);
}
template <typename T>
void launch_gmg_restrict(const GmgDev<T> &F, const GmgDev<T> &C, const T *r, T *bc, cudaStream_t st) {
  if (C.nf == 0) return;
  k_gmg_restrict<T><<<blocks(C.nf), GMG_THREADS, 0, st>>>(F, C, r, bc);
}
template <typename T>
void launch_gmg_prolong(const GmgDev<T> &F, const GmgDev<T> &C, const T *xc, T *x, cudaStream_t st) {
  if (F.nf == 0) return;
  k_gmg_prolong<T><<<blocks(F.nf), GMG_THREADS, 0, st>>>(F, C, xc, x);
}

#define FDM_GMG_INST(T)                                                                                   \
  template void launch_gmg_pre<T>(const GmgDev<T> &, int, const T *, T *, cudaStream_t);                 \
  template void launch_gmg_sweep<T>(const GmgDev<T> &, const T *, const T *, T *, cudaStream_t);         \
  template void launch_gmg_resid<T>(const GmgDev<T> &, const T *, const T *, T *, cudaStream_t);         \
  template void launch_gmg_restrict<T>(const GmgDev<T> &, const GmgDev<T> &, const T *, T *, cudaStream_t); \
  template void launch_gmg_prolong<T>(const GmgDev<T> &, const GmgDev<T> &, const T *, T *, cudaStream_t);
FDM_GMG_INST(double)
FDM_GMG_INST(float)
#undef FDM_GMG_INST

}  // namespace fdm
