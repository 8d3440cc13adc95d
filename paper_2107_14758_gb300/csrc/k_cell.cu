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
// Even-odd form of a centrosymmetric 1D matrix (M[i][j] = M[n-1-i][n-1-j],
// true of the GLL stiffness and mass matrices by the symmetry of the nodes):
// with h = n/2, x_e = x_m + x_{n-1-m}, x_o = x_m - x_{n-1-m} (m < h),
//   y_i       = sum_m Me[i][m] x_e + Mo[i][m] x_o (+ M[i][h] x_h for odd n),
//   y_{n-1-i} = sum_m Me[i][m] x_e - Mo[i][m] x_o (+ M[i][h] x_h),
//   y_h       = sum_m M[h][m] x_e + M[h][h] x_h     (odd n),
// Me = (M[i][m] + M[i][n-1-m]) / 2, Mo = (M[i][m] - M[i][n-1-m]) / 2:
// about n^2 / 2 multiply-adds per line instead of n^2.
template <typename T, int N>
struct EO {
  static constexpr int H = N / 2, S = 2 * H * H + 2 * (H + 1);
  // layout in shared memory: e[H][H], o[H][H], c[H+1] (M[i][h], i < H; M[h][h] at H), r[H+1] (M[h][m])
  static __device__ __forceinline__ void build(const T *M, T *t, int tid, int nthreads) {
    for (int q = tid; q < H * H; q += nthreads) {
      const int i = q / H, m = q % H;
      t[q] = T(0.5) * (M[i * N + m] + M[i * N + (N - 1 - m)]);
      t[H * H + q] = T(0.5) * (M[i * N + m] - M[i * N + (N - 1 - m)]);
    }
    if (N % 2 == 1)
      for (int q = tid; q <= H; q += nthreads) {
        t[2 * H * H + q] = M[q * N + H];
        t[2 * H * H + H + 1 + q] = M[H * N + q];
      }
  }
};

template <typename T, int N>
struct Line {  // a line split into even and odd parts
  static constexpr int H = N / 2;
  T e[H > 0 ? H : 1], o[H > 0 ? H : 1], mid;
  __device__ __forceinline__ void split(const T (&x)[N]) {
#pragma unroll
    for (int m = 0; m < H; ++m) {
      e[m] = x[m] + x[N - 1 - m];
      o[m] = x[m] - x[N - 1 - m];
    }
    mid = N % 2 == 1 ? x[H] : T(0);
  }
};

// rows i and n-1-i of y = M x (i < h), and the middle row for odd n
template <typename T, int N>
__device__ __forceinline__ void eo_pair(const T *t, int i, const Line<T, N> &x, T &yi, T &yj) {
  constexpr int H = N / 2;
  T se = 0, so = 0;
#pragma unroll
  for (int m = 0; m < H; ++m) {
    se = mad(t[i * H + m], x.e[m], se);
    so = mad(t[H * H + i * H + m], x.o[m], so);
  }
  if (N % 2 == 1) se = mad(t[2 * H * H + i], x.mid, se);
  yi = se + so;
  yj = se - so;
}
template <typename T, int N>
__device__ __forceinline__ T eo_mid(const T *t, const Line<T, N> &x) {
  constexpr int H = N / 2;
  T s = t[2 * H * H + H] * x.mid;
#pragma unroll
  for (int m = 0; m < H; ++m) s = mad(t[2 * H * H + H + 1 + m], x.e[m], s);
  return s;
}

template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_box_op(Grid g, const double *__restrict__ mub,
                                                                       const T *__restrict__ tab,
                                                                       const Tin *__restrict__ u, T *__restrict__ E) {
  extern __shared__ __align__(16) unsigned char smem_[];
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>(), PS = psize<N>(), N3 = N * N * N, H = N / 2;
  constexpr int ES = EO<T, N>::S;
  T *tA = reinterpret_cast<T *>(smem_), *tB = tA + ES;
  const int c = threadIdx.x / L, l = threadIdx.x % L;
  T *U = tB + ES + c * 4 * PS, *B1 = U + PS, *B2 = B1 + PS, *B3 = B2 + PS;
  const int cell = blockIdx.x * CPB + c;
  const bool valid = cell < g.ncell;
  EO<T, N>::build(tab + tab_off(TAB_A, N), tA, threadIdx.x, blockDim.x);
  EO<T, N>::build(tab + tab_off(TAB_B, N), tB, threadIdx.x, blockDim.x);
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
  const int a = l % N, b = l / N;
  {  // x: B1 = Bx u, B2 = Ax u
    T x[N];
#pragma unroll
    for (int m = 0; m < N; ++m) x[m] = U[pid<N>(m, a, b)];
    Line<T, N> xs;
    xs.split(x);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      T y0, y1;
      eo_pair<T, N>(tB, i, xs, y0, y1);
      B1[pid<N>(i, a, b)] = y0;
      B1[pid<N>(N - 1 - i, a, b)] = y1;
      eo_pair<T, N>(tA, i, xs, y0, y1);
      B2[pid<N>(i, a, b)] = y0;
      B2[pid<N>(N - 1 - i, a, b)] = y1;
    }
    if (N % 2 == 1) {
      B1[pid<N>(H, a, b)] = eo_mid<T, N>(tB, xs);
      B2[pid<N>(H, a, b)] = eo_mid<T, N>(tA, xs);
    }
  }
  __syncthreads();
  {  // y: U = By Bx u, B3 = mu2 Ay Bx u + mu1 By Ax u
    T x1[N], x2[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      x1[m] = B1[pid<N>(a, m, b)];
      x2[m] = B2[pid<N>(a, m, b)];
    }
    Line<T, N> s1, s2;
    s1.split(x1);
    s2.split(x2);
#pragma unroll
    for (int i = 0; i < H; ++i) {
      T p0, p1, q0, q1, r0, r1;
      eo_pair<T, N>(tB, i, s1, p0, p1);
      eo_pair<T, N>(tA, i, s1, q0, q1);
      eo_pair<T, N>(tB, i, s2, r0, r1);
      U[pid<N>(a, i, b)] = p0;
      U[pid<N>(a, N - 1 - i, b)] = p1;
      B3[pid<N>(a, i, b)] = mu1 * q0 + mu0 * r0;
      B3[pid<N>(a, N - 1 - i, b)] = mu1 * q1 + mu0 * r1;
    }
    if (N % 2 == 1) {
      U[pid<N>(a, H, b)] = eo_mid<T, N>(tB, s1);
      B3[pid<N>(a, H, b)] = mu1 * eo_mid<T, N>(tA, s1) + mu0 * eo_mid<T, N>(tB, s2);
    }
  }
  __syncthreads();
  if (valid) {  // z: y = Bz B3 + mu3 Az U, cell-local, natural layout
    T x3[N], x0[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      x3[m] = B3[pid<N>(a, b, m)];
      x0[m] = U[pid<N>(a, b, m)];
    }
    Line<T, N> s3, s0;
    s3.split(x3);
    s0.split(x0);
    T *out = E + (int64_t)cell * N3;
#pragma unroll
    for (int i = 0; i < H; ++i) {
      T p0, p1, q0, q1;
      eo_pair<T, N>(tB, i, s3, p0, p1);
      eo_pair<T, N>(tA, i, s0, q0, q1);
      out[a + N * (b + N * i)] = p0 + mu2 * q0;
      out[a + N * (b + N * (N - 1 - i))] = p1 + mu2 * q1;
    }
    if (N % 2 == 1) out[a + N * (b + N * H)] = eo_mid<T, N>(tB, s3) + mu2 * eo_mid<T, N>(tA, s0);
  }
}

// direct stiffness summation over the cells containing each node (fixed
// order); grid = (x blocks, y, z): no index divisions beyond constants
template <typename T, typename Tout, int N>
__global__ void __launch_bounds__(128) k_gather_t(Grid g, const T *__restrict__ E, const double *__restrict__ rsub,
                                                  Tout *__restrict__ y) {
  constexpr int P = N - 1, N3 = N * N * N;
  const int gx = blockIdx.x * blockDim.x + threadIdx.x, gy = blockIdx.y, gz = blockIdx.z;
  if (gx >= g.N[0]) return;
  const int64_t id = gx + (int64_t)g.N[0] * (gy + (int64_t)g.N[1] * gz);
  if (gx == 0 || gy == 0 || gz == 0 || gx == g.N[0] - 1 || gy == g.N[1] - 1 || gz == g.N[2] - 1) {
    y[id] = Tout(0);
    return;
  }
  const int gc[3] = {gx, gy, gz};
  int cA[3][2], lA[3][2], cnt[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int q = gc[ax] / P, rm = gc[ax] - q * P;
    if (rm == 0) {  // on a cell face along this axis (interior node: both neighbours exist)
      cA[ax][0] = q - 1; lA[ax][0] = P;
      cA[ax][1] = q;     lA[ax][1] = 0;
      cnt[ax] = 2;
    } else {
      cA[ax][0] = q; lA[ax][0] = rm;
      cnt[ax] = 1;
    }
  }
  T s = 0;
  for (int a2 = 0; a2 < cnt[2]; ++a2)
    for (int a1 = 0; a1 < cnt[1]; ++a1)
      for (int a0 = 0; a0 < cnt[0]; ++a0) {
        const int cell = cA[0][a0] + g.nx * (cA[1][a1] + g.ny * cA[2][a2]);
        s += E[(int64_t)cell * N3 + lA[0][a0] + N * (lA[1][a1] + N * lA[2][a2])];
      }
  y[id] = rsub ? Tout(T(rsub[id]) - s) : Tout(s);  // rsub: the residual r - A u
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
  // V holds the FDM-basis residual t; U <- t(m) / A_mm on interior nodes
  for (int idx = l; idx < N3; idx += L) {
    const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
    const bool in = i > 0 && i < P && j > 0 && j < P && k > 0 && k < P;
    if (in) U[pid<N>(i, j, k)] = V[pid<N>(i, j, k)] / diag_ii<T, N>(sAf, sBf, m0, m1, m2, i, j, k);
  }
  __syncthreads();
  // face nodes: t(f) -= A_fI A_II^{-1} t_I along the interior line through f;
  // thread l owns, for each axis, the line with tangential indices (a, b)
  {
    const int a = l % N, b = l / N;
    if (a > 0 && a < P && b > 0 && b < P) {
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) {
        const T mu_ax = ax == 0 ? m0 : (ax == 1 ? m1 : m2);
        const T tang = mu_ax * sBf[a * N + a] * sBf[b * N + b];
        T s0 = 0, sp = 0;
#pragma unroll
        for (int ii = 1; ii < P; ++ii) {
          const T w = U[ax == 0 ? pid<N>(ii, a, b) : (ax == 1 ? pid<N>(a, ii, b) : pid<N>(a, b, ii))];
          s0 += sAf[0 * N + ii] * w;
          sp += sAf[P * N + ii] * w;
        }
        const int f0 = ax == 0 ? pid<N>(0, a, b) : (ax == 1 ? pid<N>(a, 0, b) : pid<N>(a, b, 0));
        const int fp = ax == 0 ? pid<N>(P, a, b) : (ax == 1 ? pid<N>(a, P, b) : pid<N>(a, b, P));
        V[f0] -= tang * s0;
        V[fp] -= tang * sp;
      }
    }
  }
  __syncthreads();
  if (!valid) return;
  T *out = E + (int64_t)cell * N3;
  for (int idx = l; idx < N3; idx += L) {
    const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
    out[idx] = V[pid<N>(i, j, k)];
  }
}

// ------------------------------------------------------------------ interp
template <typename T, typename Tout, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_interp_t(InterpArgs<T> a, double omega,
                                                                         Tout *__restrict__ z) {
  extern __shared__ __align__(16) unsigned char smem_[];
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>(), PS = psize<N>(), N3 = N * N * N;
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
  if (valid) {
    ce[0] = cell % g.nx;
    ce[1] = (cell / g.nx) % g.ny;
    ce[2] = cell / (g.nx * g.ny);
    m0 = T(a.mu[3 * cell]);
    m1 = T(a.mu[3 * cell + 1]);
    m2 = T(a.mu[3 * cell + 2]);
  }
  // the stars of the cell's 8 corners: class and offset of their solutions
  __shared__ int sCls[cells_per_cta<N>()][8];
  __shared__ int64_t sOff[cells_per_cta<N>()][8];
  for (int o = l; o < 8; o += L) {  // L = n^2 >= 4: one or two corners per thread
    sCls[c][o] = 0;
    sOff[c][o] = 0;
    if (valid) {
      const int v0 = ce[0] + (o & 1), v1 = ce[1] + ((o >> 1) & 1), v2 = ce[2] + (o >> 2);
      const PatchDev Pd = a.patches[v0 + (g.nx + 1) * (v1 + (g.ny + 1) * v2)];
      sCls[c][o] = Pd.cls;
      sOff[c][o] = Pd.xoff;
    }
  }
  __syncthreads();
  if (valid) {  // interface-type nodes: the sum of the stars' interface solutions
    for (int idx = l; idx < N3; idx += L) {
      const int li[3] = {idx % N, (idx / N) % N, idx / (N * N)};
      const bool onb = li[0] == 0 || li[0] == P || li[1] == 0 || li[1] == P || li[2] == 0 || li[2] == P;
      if (!onb) continue;
      T acc = 0;
#pragma unroll
      for (int o = 0; o < 8; ++o) {
        const int k = a.cmap[(sCls[c][o] * 8 + o) * N3 + idx];
        if (k >= 0) acc += a.X[sOff[c][o] + k];
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
    const int64_t id = gidx(g, gx, gy, gz);
    // z = omega * relaxation, plus a.addv where given (the V-cycle's pre-smoothed x1)
    z[id] = dir ? Tout(0) : (a.addv ? Tout(a.addv[id] + T(omega) * V[pid<N>(i, j, k)]) : Tout(omega * V[pid<N>(i, j, k)]));
  }
}

// ------------------------------------------------------------------ coarse space
// trilinear hat functions of the Q1 coarse space at the GLL nodes: h0 = (1 - xi)/2, h1 = (1 + xi)/2
// Restriction, per cell: the 8 corner sums of h_a(x_i) h_b(y_j) h_c(z_k) (W r)_ijk,
// W = 1 / multiplicity; thread l sums one y-line of its cell.
template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_coarse_restrict_t(Grid g, const Tin *__restrict__ r,
                                                                                  const T *__restrict__ tab,
                                                                                  T *__restrict__ cellbuf) {
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>();
  const int c = threadIdx.x / L, l = threadIdx.x % L;
  const int cell = blockIdx.x * CPB + c;
  const bool valid = cell < g.ncell;
  const T *xi = tab + tab_off(TAB_XI, N);
  T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  if (valid) {  // thread l sums the y-line (i, k): consecutive threads read consecutive x
    const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
    const int i = l % N, k = l / N;
    const int gx = cx * P + i, gz = cz * P + k;
    const bool dxz = gx == 0 || gz == 0 || gx == g.N[0] - 1 || gz == g.N[2] - 1;
    if (!dxz) {
      const int mxz = ((i == 0 && cx > 0) || (i == P && cx < g.nx - 1) ? 2 : 1) *
                      ((k == 0 && cz > 0) || (k == P && cz < g.nz - 1) ? 2 : 1);
      T s0 = 0, s1 = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        const int gy = cy * P + j;
        if (gy == 0 || gy == g.N[1] - 1) continue;
        const int m = mxz * ((j == 0 && cy > 0) || (j == P && cy < g.ny - 1) ? 2 : 1);
        const T v = T(r[gidx(g, gx, gy, gz)]) / T(m);
        s0 += T(0.5) * (T(1) - xi[j]) * v;
        s1 += T(0.5) * (T(1) + xi[j]) * v;
      }
      const T hx[2] = {T(0.5) * (T(1) - xi[i]), T(0.5) * (T(1) + xi[i])};
      const T hz[2] = {T(0.5) * (T(1) - xi[k]), T(0.5) * (T(1) + xi[k])};
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[q] = hx[q & 1] * (((q >> 1) & 1) ? s1 : s0) * hz[q >> 2];
    }
  }
  // sum over the cell's lines in line order (deterministic)
  __shared__ T red[CPB * L][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) red[threadIdx.x][q] = acc[q];
  __syncthreads();
  if (valid)
    for (int q = l; q < 8; q += L) {  // L = n^2 >= 4
      T v = 0;
      for (int t = 0; t < L; ++t) v += red[c * L + t][q];
      cellbuf[(int64_t)cell * 8 + q] = v;
    }
}

// Prolongation z (+)= P x_c: thread l evaluates one y-line of its cell from the
// 8 corner values, written by the owning cell.
template <typename T, typename Tout, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_coarse_prolong_t(Grid g, const T *__restrict__ xc,
                                                                                 const T *__restrict__ tab,
                                                                                 const int *__restrict__ cfree,
                                                                                 Tout *__restrict__ z, int accumulate) {
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>();
  const int c = threadIdx.x / L, l = threadIdx.x % L;
  const int cell = blockIdx.x * CPB + c;
  if (cell >= g.ncell) return;
  const int ce[3] = {cell % g.nx, (cell / g.nx) % g.ny, cell / (g.nx * g.ny)};
  const T *xi = tab + tab_off(TAB_XI, N);
  T cv[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int v = (ce[0] + (q & 1)) + (g.nx + 1) * ((ce[1] + ((q >> 1) & 1)) + (g.ny + 1) * (ce[2] + (q >> 2)));
    const int f = cfree[v];
    cv[q] = f >= 0 ? xc[f] : T(0);
  }
  const int i = l % N, k = l / N;  // the y-line (i, k): consecutive threads write consecutive x
  if ((i == 0 && ce[0] > 0) || (k == 0 && ce[2] > 0)) return;  // not the owner of this line
  const int gx = ce[0] * P + i, gz = ce[2] * P + k;
  const bool dxz = gx == 0 || gz == 0 || gx == g.N[0] - 1 || gz == g.N[2] - 1;
  const T hx[2] = {T(0.5) * (T(1) - xi[i]), T(0.5) * (T(1) + xi[i])};
  const T hz[2] = {T(0.5) * (T(1) - xi[k]), T(0.5) * (T(1) + xi[k])};
  T e[2];  // the corner values combined along x and z, for the y = 0 and y = 1 corners
#pragma unroll
  for (int b = 0; b < 2; ++b)
    e[b] = cv[2 * b] * hx[0] * hz[0] + cv[2 * b + 1] * hx[1] * hz[0] + cv[2 * b + 4] * hx[0] * hz[1] +
           cv[2 * b + 5] * hx[1] * hz[1];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j == 0 && ce[1] > 0) continue;
    const int gy = ce[1] * P + j;
    const T s = (dxz || gy == 0 || gy == g.N[1] - 1) ? T(0)
                                                      : T(0.5) * (T(1) - xi[j]) * e[0] + T(0.5) * (T(1) + xi[j]) * e[1];
    const int64_t id = gidx(g, gx, gy, gz);
    z[id] = accumulate ? Tout(z[id] + s) : Tout(s);
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

}  // namespace

template <typename T, typename Tin, typename Tout>
bool launch_box_op_fast(const OpArgs &a, const Tin *u, Tout *y, T *E, cudaStream_t st, const double *rsub) {
  if constexpr (!std::is_same<T, Tin>::value) {
    return false;
  } else {
    if (a.general) return false;
    const T *tab = reinterpret_cast<const T *>(a.tab);
    return dispatch_n(a.g.n, [&](auto nc) {
      constexpr int N = decltype(nc)::value;
      constexpr int CPB = cells_per_cta<N>();
      const size_t sm = sizeof(T) * (2 * EO<T, N>::S + (size_t)CPB * 4 * psize<N>());
      set_smem(k_box_op<T, Tin, N>, sm);
      k_box_op<T, Tin, N><<<(a.g.ncell + CPB - 1) / CPB, CPB * N * N, sm, st>>>(a.g, a.mu_box, tab, u, E);
      k_gather_t<T, Tout, N><<<dim3((a.g.N[0] + 127) / 128, a.g.N[1], a.g.N[2]), 128, 0, st>>>(a.g, E, rsub, y);
    });
  }
}

template <typename T, typename Tin>
bool launch_restrict_fast(const Grid &g, const Tin *r, const T *tab, const double *mu, T *E, cudaStream_t st) {
  if constexpr (!std::is_same<T, Tin>::value && !std::is_same<Tin, double>::value) {
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
  if constexpr (!std::is_same<T, Tout>::value && !std::is_same<Tout, double>::value) {
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

template <typename T, typename Tin>
bool launch_coarse_restrict_fast(const Grid &g, const Tin *r, const T *tab, T *cellbuf, cudaStream_t st) {
  if constexpr (!std::is_same<T, Tin>::value) {
    return false;
  } else {
    return dispatch_n(g.n, [&](auto nc) {
      constexpr int N = decltype(nc)::value;
      constexpr int CPB = cells_per_cta<N>();
      k_coarse_restrict_t<T, Tin, N><<<(g.ncell + CPB - 1) / CPB, CPB * N * N, 0, st>>>(g, r, tab, cellbuf);
    });
  }
}

template <typename T, typename Tout>
bool launch_coarse_prolong_fast(const Grid &g, const T *xc, const T *tab, const int *cfree, Tout *z, bool accumulate,
                                cudaStream_t st) {
  if constexpr (!std::is_same<T, Tout>::value) {
    return false;
  } else {
    return dispatch_n(g.n, [&](auto nc) {
      constexpr int N = decltype(nc)::value;
      constexpr int CPB = cells_per_cta<N>();
      k_coarse_prolong_t<T, Tout, N><<<(g.ncell + CPB - 1) / CPB, CPB * N * N, 0, st>>>(g, xc, tab, cfree, z,
                                                                                        accumulate ? 1 : 0);
    });
  }
}

template bool launch_coarse_restrict_fast<float, float>(const Grid &, const float *, const float *, float *,
                                                        cudaStream_t);
template bool launch_coarse_restrict_fast<double, double>(const Grid &, const double *, const double *, double *,
                                                          cudaStream_t);
template bool launch_coarse_prolong_fast<float, float>(const Grid &, const float *, const float *, const int *,
                                                       float *, bool, cudaStream_t);
template bool launch_coarse_prolong_fast<double, double>(const Grid &, const double *, const double *, const int *,
                                                         double *, bool, cudaStream_t);
template bool launch_box_op_fast<double, double, double>(const OpArgs &, const double *, double *, double *,
                                                         cudaStream_t, const double *);
template bool launch_box_op_fast<float, float, float>(const OpArgs &, const float *, float *, float *, cudaStream_t,
                                                      const double *);
template bool launch_box_op_fast<double, double, float>(const OpArgs &, const double *, float *, double *,
                                                        cudaStream_t, const double *);
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
