// Cell-local kernels specialised on the number of GLL points n = p + 1 (a
// template parameter), so that index arithmetic folds into constants and the
// one-dimensional contractions unroll completely.
//
// Layout: one thread per line of a cell ("pencil").  The n x n x n values of a
// cell sit in shared memory with padded pitches, node (i, j, k) at
// i + (n+1) j + (n+1)^2 k, so that lines along x, y and z are read without
// bank conflicts; a line's n values go to registers and each of its n outputs
// is one dot product with a row of a 1D matrix (read as a shared-memory
// broadcast).  Several cells share a CTA when n is small.
//
//   box stiffness (eq. (kron), Section 2.2): y_K = mu1 (B (x) B (x) A) u_K
//     + mu2 (B (x) A (x) B) u_K + mu3 (A (x) B (x) B) u_K in 7 line passes;
//     cell-local results, summed over cells by a node gather.
//   restrict (Section 2.4): E_K = (T^T)^{(x)3} (W_K r_K), then the cell's share
//     of the Schur condensation on its face nodes.
//   interp (Sections 2.4-2.6): interface values summed over the 8 stars,
//     interior values by the summed back-substitution, then T^{(x)3}, omega
//     and an owner write.
#include <type_traits>

#include "device.cuh"
#include "kernels.h"

namespace fdm {
namespace {

template <int N>
__device__ __forceinline__ int pid(int i, int j, int k) {
  return i + (N + 1) * (j + (N + 1) * k);
}
template <int N>
constexpr int psize() {
  return (N + 1) * (N + 1) * N;
}
template <int N>
constexpr int cells_per_cta() {
  return N * N >= 128 ? 1 : 128 / (N * N);
}

__device__ __forceinline__ float mad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double mad(double a, double b, double c) { return ::fma(a, b, c); }

// sum_m M[r][m] x[m] (TR: sum_m M[m][r] x[m]), M row-major N x N
template <typename T, int N, bool TR>
__device__ __forceinline__ T row_dot(const T *M, int r, const T (&x)[N]) {
  T s = 0;
#pragma unroll
  for (int m = 0; m < N; ++m) s = mad(TR ? M[m * N + r] : M[r * N + m], x[m], s);
  return s;
}

// one pass along `axis` for the line `l` of a cell: dst = M' src (M' = M or M^T)
template <typename T, int N, bool TR>
__device__ __forceinline__ void line_pass(const T *src, T *dst, const T *M, int axis, int l) {
  const int a = l % N, b = l / N;
  T x[N];
#pragma unroll
  for (int m = 0; m < N; ++m)
    x[m] = src[axis == 0 ? pid<N>(m, a, b) : (axis == 1 ? pid<N>(a, m, b) : pid<N>(a, b, m))];
#pragma unroll
  for (int r = 0; r < N; ++r)
    dst[axis == 0 ? pid<N>(r, a, b) : (axis == 1 ? pid<N>(a, r, b) : pid<N>(a, b, r))] = row_dot<T, N, TR>(M, r, x);
}

// ------------------------------------------------------------------ box stiffness
template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_box_op(Grid g, const double *__restrict__ mub,
                                                                       const T *__restrict__ tab,
                                                                       const Tin *__restrict__ u, T *__restrict__ E) {
  extern __shared__ __align__(16) unsigned char smem_[];
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>(), PS = psize<N>(), N3 = N * N * N;
  T *sA = reinterpret_cast<T *>(smem_), *sB = sA + N * N;
  const int c = threadIdx.x / L, l = threadIdx.x % L;
  T *U = sB + N * N + c * 4 * PS, *B1 = U + PS, *B2 = B1 + PS, *B3 = B2 + PS;
  const int cell = blockIdx.x * CPB + c;
  const bool valid = cell < g.ncell;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    sA[i] = tab[tab_off(TAB_A, N) + i];
    sB[i] = tab[tab_off(TAB_B, N) + i];
  }
  T mu0 = 0, mu1 = 0, mu2 = 0;
  if (valid) {
    const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
    mu0 = T(mub[3 * cell]);
    mu1 = T(mub[3 * cell + 1]);
    mu2 = T(mub[3 * cell + 2]);
    for (int idx = l; idx < N3; idx += L) {
      const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
      const int gx = cx * P + i, gy = cy * P + j, gz = cz * P + k;
      const bool dir = gx == 0 || gy == 0 || gz == 0 || gx == g.N[0] - 1 || gy == g.N[1] - 1 || gz == g.N[2] - 1;
      U[pid<N>(i, j, k)] = dir ? T(0) : T(u[gidx(g, gx, gy, gz)]);
    }
  }
  __syncthreads();
  {  // x: B1 = Bx u, B2 = Ax u
    const int a = l % N, b = l / N;
    T x[N];
#pragma unroll
    for (int m = 0; m < N; ++m) x[m] = U[pid<N>(m, a, b)];
#pragma unroll
    for (int r = 0; r < N; ++r) {
      B1[pid<N>(r, a, b)] = row_dot<T, N, false>(sB, r, x);
      B2[pid<N>(r, a, b)] = row_dot<T, N, false>(sA, r, x);
    }
  }
  __syncthreads();
  {  // y: U = By Bx u, B3 = mu2 Ay Bx u + mu1 By Ax u
    const int a = l % N, b = l / N;
    T x1[N], x2[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      x1[m] = B1[pid<N>(a, m, b)];
      x2[m] = B2[pid<N>(a, m, b)];
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
      U[pid<N>(a, r, b)] = row_dot<T, N, false>(sB, r, x1);
      B3[pid<N>(a, r, b)] = mu1 * row_dot<T, N, false>(sA, r, x1) + mu0 * row_dot<T, N, false>(sB, r, x2);
    }
  }
  __syncthreads();
  if (valid) {  // z: y = Bz B3 + mu3 Az U, cell-local, natural layout
    const int a = l % N, b = l / N;
    T x3[N], x0[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      x3[m] = B3[pid<N>(a, b, m)];
      x0[m] = U[pid<N>(a, b, m)];
    }
    T *out = E + (int64_t)cell * N3;
#pragma unroll
    for (int r = 0; r < N; ++r)
      out[a + N * (b + N * r)] = row_dot<T, N, false>(sB, r, x3) + mu2 * row_dot<T, N, false>(sA, r, x0);
  }
}

// direct stiffness summation over the cells containing each node (fixed order)
template <typename T, typename Tout, int N>
__global__ void __launch_bounds__(256) k_gather_t(Grid g, const T *__restrict__ E, Tout *__restrict__ y) {
  constexpr int P = N - 1, N3 = N * N * N;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ndof;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int gc[3] = {int(id % g.N[0]), int((id / g.N[0]) % g.N[1]), int(id / ((int64_t)g.N[0] * g.N[1]))};
    const int ncl[3] = {g.nx, g.ny, g.nz};
    bool dir = false;
    int cA[3][2], lA[3][2], cnt[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) {
      const int v = gc[ax];
      dir |= v == 0 || v == g.N[ax] - 1;
      const int q = v / P, rm = v - q * P;
      if (rm == 0) {
        cnt[ax] = 0;
        if (q > 0) { cA[ax][cnt[ax]] = q - 1; lA[ax][cnt[ax]++] = P; }
        if (q < ncl[ax]) { cA[ax][cnt[ax]] = q; lA[ax][cnt[ax]++] = 0; }
      } else {
        cA[ax][0] = q;
        lA[ax][0] = rm;
        cnt[ax] = 1;
      }
    }
    if (dir) {
      y[id] = Tout(0);
      continue;
    }
    T s = 0;
    for (int a2 = 0; a2 < cnt[2]; ++a2)
      for (int a1 = 0; a1 < cnt[1]; ++a1)
        for (int a0 = 0; a0 < cnt[0]; ++a0) {
          const int cell = cA[0][a0] + g.nx * (cA[1][a1] + g.ny * cA[2][a2]);
          s += E[(int64_t)cell * N3 + lA[0][a0] + N * (lA[1][a1] + N * lA[2][a2])];
        }
    y[id] = Tout(s);
  }
}

// A_mm of an interior node (FDM basis: diagonal) and the coupling of face node
// (local lf along axis ax) to the interior node with the same tangential indices
template <typename T, int N>
__device__ __forceinline__ T diag_ii(const T *Af, const T *Bf, T m0, T m1, T m2, int i, int j, int k) {
  const T ai = Af[i * N + i], aj = Af[j * N + j], ak = Af[k * N + k];
  const T bi = Bf[i * N + i], bj = Bf[j * N + j], bk = Bf[k * N + k];
  return m0 * ai * bj * bk + m1 * bi * aj * bk + m2 * bi * bj * ak;
}

// ------------------------------------------------------------------ restrict
template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_restrict_t(Grid g, const Tin *__restrict__ r,
                                                                           const T *__restrict__ tab,
                                                                           const double *__restrict__ mug,
                                                                           T *__restrict__ E) {
  extern __shared__ __align__(16) unsigned char smem_[];
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>(), PS = psize<N>(), N3 = N * N * N;
  T *sT = reinterpret_cast<T *>(smem_), *sAf = sT + N * N, *sBf = sAf + N * N;
  const int c = threadIdx.x / L, l = threadIdx.x % L;
  T *U = sBf + N * N + c * 2 * PS, *V = U + PS;
  const int cell = blockIdx.x * CPB + c;
  const bool valid = cell < g.ncell;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    sT[i] = tab[tab_off(TAB_T, N) + i];
    sAf[i] = tab[tab_off(TAB_AF, N) + i];
    sBf[i] = tab[tab_off(TAB_BF, N) + i];
  }
  int cx = 0, cy = 0, cz = 0;
  T m0 = 0, m1 = 0, m2 = 0;
  if (valid) {
    cx = cell % g.nx;
    cy = (cell / g.nx) % g.ny;
    cz = cell / (g.nx * g.ny);
    m0 = T(mug[3 * cell]);
    m1 = T(mug[3 * cell + 1]);
    m2 = T(mug[3 * cell + 2]);
    for (int idx = l; idx < N3; idx += L) {  // W_K r_K, W = 1 / multiplicity, Dirichlet entries 0
      const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
      const int gx = cx * P + i, gy = cy * P + j, gz = cz * P + k;
      const bool dir = gx == 0 || gy == 0 || gz == 0 || gx == g.N[0] - 1 || gy == g.N[1] - 1 || gz == g.N[2] - 1;
      const int mult = ((i == 0 && cx > 0) || (i == P && cx < g.nx - 1) ? 2 : 1) *
                       ((j == 0 && cy > 0) || (j == P && cy < g.ny - 1) ? 2 : 1) *
                       ((k == 0 && cz > 0) || (k == P && cz < g.nz - 1) ? 2 : 1);
      U[pid<N>(i, j, k)] = dir ? T(0) : T(r[gidx(g, gx, gy, gz)]) / T(mult);
    }
  }
  __syncthreads();
  line_pass<T, N, true>(U, V, sT, 0, l);
  __syncthreads();
  line_pass<T, N, true>(V, U, sT, 1, l);
  __syncthreads();
  line_pass<T, N, true>(U, V, sT, 2, l);
  __syncthreads();
  // V holds the FDM-basis residual; U <- t(m) / A_mm on interior nodes
  for (int idx = l; idx < N3; idx += L) {
    const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
    const bool in = i > 0 && i < P && j > 0 && j < P && k > 0 && k < P;
    U[pid<N>(i, j, k)] = in ? V[pid<N>(i, j, k)] / diag_ii<T, N>(sAf, sBf, m0, m1, m2, i, j, k) : T(0);
  }
  __syncthreads();
  if (!valid) return;
  T *out = E + (int64_t)cell * N3;
  for (int idx = l; idx < N3; idx += L) {
    const int li[3] = {idx % N, (idx / N) % N, idx / (N * N)};
    int nb = 0, ax = -1;
#pragma unroll
    for (int a = 0; a < 3; ++a)
      if (li[a] == 0 || li[a] == P) { ++nb; ax = a; }
    T v = V[pid<N>(li[0], li[1], li[2])];
    if (nb == 1) {  // face node: subtract A_fI A_II^{-1} t_I along the interior line through it
      const int lf = li[ax];
      const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
      const T mu_ax = ax == 0 ? m0 : (ax == 1 ? m1 : m2);
      const T tang = mu_ax * sBf[li[t1] * N + li[t1]] * sBf[li[t2] * N + li[t2]];
      T s = 0;
#pragma unroll
      for (int ii = 1; ii < P; ++ii) {
        int q[3] = {li[0], li[1], li[2]};
        q[ax] = ii;
        s += sAf[lf * N + ii] * U[pid<N>(q[0], q[1], q[2])];
      }
      v -= tang * s;
    }
    out[idx] = v;
  }
}

// ------------------------------------------------------------------ interp
template <typename T, typename Tout, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_interp_t(InterpArgs<T> a, double omega,
                                                                         Tout *__restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_[];
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>(), PS = psize<N>(), N3 = N * N * N, CI = P - 1;
  const Grid &g = a.g;
  T *sT = reinterpret_cast<T *>(smem_), *sAf = sT + N * N, *sBf = sAf + N * N;
  const int c = threadIdx.x / L, l = threadIdx.x % L;
  T *U = sBf + N * N + c * 2 * PS, *V = U + PS;
  const int cell = blockIdx.x * CPB + c;
  const bool valid = cell < g.ncell;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    sT[i] = a.tab[tab_off(TAB_T, N) + i];
    sAf[i] = a.tab[tab_off(TAB_AF, N) + i];
    sBf[i] = a.tab[tab_off(TAB_BF, N) + i];
  }
  int ce[3] = {0, 0, 0};
  T m0 = 0, m1 = 0, m2 = 0;
  const int ncl[3] = {g.nx, g.ny, g.nz};
  if (valid) {
    ce[0] = cell % g.nx;
    ce[1] = (cell / g.nx) % g.ny;
    ce[2] = cell / (g.nx * g.ny);
    m0 = T(a.mu[3 * cell]);
    m1 = T(a.mu[3 * cell + 1]);
    m2 = T(a.mu[3 * cell + 2]);
    // interface-type nodes: the sum of the stars' interface solutions
    for (int idx = l; idx < N3; idx += L) {
      const int li[3] = {idx % N, (idx / N) % N, idx / (N * N)};
      const bool onb = li[0] == 0 || li[0] == P || li[1] == 0 || li[1] == P || li[2] == 0 || li[2] == P;
      if (!onb) continue;
      T acc = 0;
      for (int o = 0; o < 8; ++o) {
        const int oo[3] = {o & 1, (o >> 1) & 1, o >> 2};
        int v[3], t[3];
        bool ok = true;
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
          v[ax] = ce[ax] + oo[ax];
          const bool full = v[ax] >= 1 && v[ax] <= ncl[ax] - 1;
          const int i = li[ax];
          if (full) {
            if (oo[ax] == 0) { ok = ok && i <= P - 1; t[ax] = i + CI; }
            else { ok = ok && i >= 1; t[ax] = i - 1; }
          } else {
            ok = ok && i >= 1 && i <= P - 1;
            t[ax] = i - 1;
          }
        }
        if (!ok) continue;
        const PatchDev Pd = a.patches[v[0] + (g.nx + 1) * (v[1] + (g.ny + 1) * v[2])];
        const ClassDev &C = a.cls[Pd.cls];
        const int k = C.ginv[t[0] + C.dim[0] * (t[1] + C.dim[1] * t[2])];
        if (k >= 0) acc += a.X[Pd.xoff + k];
      }
      U[pid<N>(li[0], li[1], li[2])] = acc;
    }
  }
  __syncthreads();
  if (valid) {  // interior nodes: (8 r(m) - sum over the 6 face nodes of A_mf z(f)) / A_mm
    const T *Ek = a.E + (int64_t)cell * N3;
    for (int idx = l; idx < N3; idx += L) {
      const int li[3] = {idx % N, (idx / N) % N, idx / (N * N)};
      const bool onb = li[0] == 0 || li[0] == P || li[1] == 0 || li[1] == P || li[2] == 0 || li[2] == P;
      if (onb) continue;
      T s = T(8) * Ek[idx];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const int t1 = ax == 0 ? 1 : 0, t2 = ax == 2 ? 1 : 2;
        const T mu_ax = ax == 0 ? m0 : (ax == 1 ? m1 : m2);
        const T tang = mu_ax * sBf[li[t1] * N + li[t1]] * sBf[li[t2] * N + li[t2]];
        int q0[3] = {li[0], li[1], li[2]}, qp[3] = {li[0], li[1], li[2]};
        q0[ax] = 0;
        qp[ax] = P;
        s -= tang * sAf[0 * N + li[ax]] * U[pid<N>(q0[0], q0[1], q0[2])];
        s -= tang * sAf[P * N + li[ax]] * U[pid<N>(qp[0], qp[1], qp[2])];
      }
      U[pid<N>(li[0], li[1], li[2])] = s / diag_ii<T, N>(sAf, sBf, m0, m1, m2, li[0], li[1], li[2]);
    }
  }
  __syncthreads();
  line_pass<T, N, false>(U, V, sT, 0, l);
  __syncthreads();
  line_pass<T, N, false>(V, U, sT, 1, l);
  __syncthreads();
  line_pass<T, N, false>(U, V, sT, 2, l);
  __syncthreads();
  if (!valid) return;
  for (int idx = l; idx < N3; idx += L) {
    const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
    if ((i == 0 && ce[0] > 0) || (j == 0 && ce[1] > 0) || (k == 0 && ce[2] > 0)) continue;  // not owner
    const int gx = ce[0] * P + i, gy = ce[1] * P + j, gz = ce[2] * P + k;
    const bool dir = gx == 0 || gy == 0 || gz == 0 || gx == g.N[0] - 1 || gy == g.N[1] - 1 || gz == g.N[2] - 1;
    z[gidx(g, gx, gy, gz)] = dir ? Tout(0) : Tout(omega * V[pid<N>(i, j, k)]);
  }
}

// ------------------------------------------------------------------ launchers
template <typename F>
bool dispatch_n(int n, F &&f) {
  switch (n) {
    case 2: f(std::integral_constant<int, 2>{}); return true;
    case 3: f(std::integral_constant<int, 3>{}); return true;
    case 4: f(std::integral_constant<int, 4>{}); return true;
    case 5: f(std::integral_constant<int, 5>{}); return true;
    case 6: f(std::integral_constant<int, 6>{}); return true;
    case 7: f(std::integral_constant<int, 7>{}); return true;
    case 8: f(std::integral_constant<int, 8>{}); return true;
    case 9: f(std::integral_constant<int, 9>{}); return true;
    case 10: f(std::integral_constant<int, 10>{}); return true;
    case 11: f(std::integral_constant<int, 11>{}); return true;
    case 12: f(std::integral_constant<int, 12>{}); return true;
    case 13: f(std::integral_constant<int, 13>{}); return true;
    case 14: f(std::integral_constant<int, 14>{}); return true;
    case 15: f(std::integral_constant<int, 15>{}); return true;
    case 16: f(std::integral_constant<int, 16>{}); return true;
    default: return false;
  }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) FDM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

inline int gather_blocks(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)(b < 4 * 152 * 8 ? (b > 0 ? b : 1) : 4 * 152 * 8);
}

}  // namespace

template <typename T, typename Tin, typename Tout>
bool launch_box_op_fast(const OpArgs &a, const Tin *u, Tout *y, T *E, cudaStream_t st) {
  if constexpr (!std::is_same<T, Tin>::value) {
    return false;
  } else {
    if (a.general) return false;
    const T *tab = reinterpret_cast<const T *>(a.tab);
    return dispatch_n(a.g.n, [&](auto nc) {
      constexpr int N = decltype(nc)::value;
      constexpr int CPB = cells_per_cta<N>();
      const size_t sm = sizeof(T) * (2 * N * N + (size_t)CPB * 4 * psize<N>());
      set_smem(k_box_op<T, Tin, N>, sm);
      k_box_op<T, Tin, N><<<(a.g.ncell + CPB - 1) / CPB, CPB * N * N, sm, st>>>(a.g, a.mu_box, tab, u, E);
      k_gather_t<T, Tout, N><<<gather_blocks(a.g.ndof), 256, 0, st>>>(a.g, E, y);
    });
  }
}

template <typename T, typename Tin>
bool launch_restrict_fast(const Grid &g, const Tin *r, const T *tab, const double *mu, T *E, cudaStream_t st) {
  if constexpr (!std::is_same<T, Tin>::value) {
    return false;
  } else {
    return dispatch_n(g.n, [&](auto nc) {
      constexpr int N = decltype(nc)::value;
      constexpr int CPB = cells_per_cta<N>();
      const size_t sm = sizeof(T) * (3 * N * N + (size_t)CPB * 2 * psize<N>());
      set_smem(k_restrict_t<T, Tin, N>, sm);
      k_restrict_t<T, Tin, N><<<(g.ncell + CPB - 1) / CPB, CPB * N * N, sm, st>>>(g, r, tab, mu, E);
    });
  }
}

template <typename T, typename Tout>
bool launch_interp_fast(const InterpArgs<T> &a, double omega, Tout *z, cudaStream_t st) {
  if constexpr (!std::is_same<T, Tout>::value) {
    return false;
  } else {
    return dispatch_n(a.g.n, [&](auto nc) {
      constexpr int N = decltype(nc)::value;
      constexpr int CPB = cells_per_cta<N>();
      const size_t sm = sizeof(T) * (3 * N * N + (size_t)CPB * 2 * psize<N>());
      set_smem(k_interp_t<T, Tout, N>, sm);
      k_interp_t<T, Tout, N><<<(a.g.ncell + CPB - 1) / CPB, CPB * N * N, sm, st>>>(a, omega, z);
    });
  }
}

template bool launch_box_op_fast<double, double, double>(const OpArgs &, const double *, double *, double *,
                                                         cudaStream_t);
template bool launch_box_op_fast<float, float, float>(const OpArgs &, const float *, float *, float *, cudaStream_t);
template bool launch_box_op_fast<double, double, float>(const OpArgs &, const double *, float *, double *,
                                                        cudaStream_t);
template bool launch_restrict_fast<float, float>(const Grid &, const float *, const float *, const double *, float *,
                                                 cudaStream_t);
template bool launch_restrict_fast<double, double>(const Grid &, const double *, const double *, const double *,
                                                   double *, cudaStream_t);
template bool launch_restrict_fast<float, double>(const Grid &, const double *, const float *, const double *,
                                                  float *, cudaStream_t);
template bool launch_restrict_fast<double, float>(const Grid &, const float *, const double *, const double *,
                                                  double *, cudaStream_t);
template bool launch_interp_fast<float, float>(const InterpArgs<float> &, double, float *, cudaStream_t);
template bool launch_interp_fast<double, double>(const InterpArgs<double> &, double, double *, cudaStream_t);
template bool launch_interp_fast<float, double>(const InterpArgs<float> &, double, double *, cudaStream_t);
template bool launch_interp_fast<double, float>(const InterpArgs<double> &, double, float *, cudaStream_t);

}  // namespace fdm
