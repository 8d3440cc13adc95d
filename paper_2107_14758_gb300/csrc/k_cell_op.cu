// Cell operators specialised on n: box-cell stiffness (even-odd form), curved-cell
// stiffness (Gauss quadrature) and the node gather; helpers in k_cell.cuh.
#include <algorithm>

#include "k_cell.cuh"

namespace fdm {
namespace {

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
  // two buffers per cell: every pass reads a thread's whole line into registers
  // before writing the same line's positions, so results overwrite their inputs
  T *U = tB + ES + c * 2 * PS, *V = U + PS;
  T *B1 = U, *B2 = V, *B3 = V;
  const int cell = blockIdx.x * CPB + c;
  const bool valid = cell < g.ncell;
  EO<T, N>::build(tab + tab_off(TAB_A, N), tA, threadIdx.x, blockDim.x);
  EO<T, N>::build(tab + tab_off(TAB_B, N), tB, threadIdx.x, blockDim.x);
  // the cell's three coefficients, converted once per cell (read after the first barrier)
  __shared__ T sMu[CPB][3];
  if (l < 3) sMu[c][l] = valid ? T(mub[3 * cell + l]) : T(0);
  if (valid) {
    const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
    for (int idx = l; idx < N3; idx += L) {
      const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
      const int gx = cx * P + i, gy = cy * P + j, gz = cz * P + k;
      const bool dir = node_dirichlet(g, gx, gy, gz);
      U[pid<N>(i, j, k)] = dir ? T(0) : T(u[gidx(g, gx, gy, gz)]);
    }
  }
  __syncthreads();
  const T mu0 = sMu[c][0], mu1 = sMu[c][1], mu2 = sMu[c][2];
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

// ------------------------------------------------------------------ box cells, element modes
// The same box-cell stiffness in the 1D generalised eigenbasis of (A, B)
// (Section 2.3's fast diagonalisation, applied as an operator): with the
// modes V = S^T B by rows, A = V^T diag(lam) V and B = V^T V, so
//   y_K = (V^T)^{(x)3} D V^{(x)3} u_K,  D_ijk = mu1 lam_i + mu2 lam_j + mu3 lam_k
// (i along x): three forward passes, the diagonal, three backward passes, six
// line passes against seven, with no coefficient products inside them.  Modes
// are even or odd about the element centre and stored even first, so a
// forward pass contracts the half sums of a line with the even modes and the
// half differences with the odd ones, and a backward pass forms each node
// pair from its even and odd mode sums: n^2 / 2 multiply-adds per line.
// Passes run in place (each thread reads its whole line before writing it):
// forward along z and y, then along x the forward pass, the diagonal and the
// backward pass in registers, then backward along y and z, the last one
// writing the cell-local result in natural layout.
template <typename T, int N>
__device__ __forceinline__ int line_at(int axis, int m, int a, int b) {
  return axis == 0 ? pid<N>(m, a, b) : (axis == 1 ? pid<N>(a, m, b) : pid<N>(a, b, m));
}
// nodes -> modes along one line
template <typename T, int N>
__device__ __forceinline__ void modes_fwd(const T *V, const T (&x)[N], T (&w)[N]) {
  constexpr int H = N / 2, NE = (N + 1) / 2;
  T sp[NE], dm[H > 0 ? H : 1];
#pragma unroll
  for (int j = 0; j < H; ++j) {
    sp[j] = x[j] + x[N - 1 - j];
    dm[j] = x[j] - x[N - 1 - j];
  }
  if (N % 2 == 1) sp[H] = x[H];
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    T acc = 0;
#pragma unroll
    for (int j = 0; j < NE; ++j) acc = mad(V[k * N + j], sp[j], acc);
    w[k] = acc;
  }
#pragma unroll
  for (int k = NE; k < N; ++k) {
    T acc = 0;
#pragma unroll
    for (int j = 0; j < H; ++j) acc = mad(V[k * N + j], dm[j], acc);
    w[k] = acc;
  }
}
// modes -> nodes along one line
template <typename T, int N>
__device__ __forceinline__ void modes_bwd(const T *V, const T (&w)[N], T (&x)[N]) {
  constexpr int H = N / 2, NE = (N + 1) / 2;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    T e = 0, o = 0;
#pragma unroll
    for (int k = 0; k < NE; ++k) e = mad(V[k * N + i], w[k], e);
#pragma unroll
    for (int k = NE; k < N; ++k) o = mad(V[k * N + i], w[k], o);
    x[i] = e + o;
    x[N - 1 - i] = e - o;
  }
  if (N % 2 == 1) {
    T e = 0;
#pragma unroll
    for (int k = 0; k < NE; ++k) e = mad(V[k * N + H], w[k], e);
    x[H] = e;
  }
}

template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_box_op_modes(Grid g, const double *__restrict__ mub,
                                                                             const T *__restrict__ tab,
                                                                             const Tin *__restrict__ u,
                                                                             T *__restrict__ E) {
  extern __shared__ __align__(16) unsigned char smem_[];
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>(), PS = psize<N>(), N3 = N * N * N;
  T *sV = reinterpret_cast<T *>(smem_), *sLam = sV + N * N;
  const int c = threadIdx.x / L, l = threadIdx.x % L;
  T *U = sLam + N + c * PS;
  const int cell = blockIdx.x * CPB + c;
  const bool valid = cell < g.ncell;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) sV[i] = tab[tab_off(TAB_VE, N) + i];
  for (int i = threadIdx.x; i < N; i += blockDim.x) sLam[i] = tab[tab_off(TAB_LE, N) + i];
  __shared__ T sMu[CPB][3];
  if (l < 3) sMu[c][l] = valid ? T(mub[3 * cell + l]) : T(0);
  if (valid) {
    const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
    for (int idx = l; idx < N3; idx += L) {
      const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
      const int gx = cx * P + i, gy = cy * P + j, gz = cz * P + k;
      const bool dir = node_dirichlet(g, gx, gy, gz);
      U[pid<N>(i, j, k)] = dir ? T(0) : T(u[gidx(g, gx, gy, gz)]);
    }
  }
  __syncthreads();
  const int a = l % N, b = l / N;
  T x[N], w[N];
#pragma unroll
  for (int axis = 2; axis >= 1; --axis) {  // forward along z, then y
#pragma unroll
    for (int m = 0; m < N; ++m) x[m] = U[line_at<T, N>(axis, m, a, b)];
    modes_fwd<T, N>(sV, x, w);
#pragma unroll
    for (int m = 0; m < N; ++m) U[line_at<T, N>(axis, m, a, b)] = w[m];
    __syncthreads();
  }
  {  // along x: forward, D (y mode a, z mode b), backward
#pragma unroll
    for (int m = 0; m < N; ++m) x[m] = U[pid<N>(m, a, b)];
    modes_fwd<T, N>(sV, x, w);
    const T mu0 = sMu[c][0], cl = sMu[c][1] * sLam[a] + sMu[c][2] * sLam[b];
#pragma unroll
    for (int m = 0; m < N; ++m) w[m] *= mad(mu0, sLam[m], cl);
    modes_bwd<T, N>(sV, w, x);
#pragma unroll
    for (int m = 0; m < N; ++m) U[pid<N>(m, a, b)] = x[m];
  }
  __syncthreads();
  {  // backward along y
#pragma unroll
    for (int m = 0; m < N; ++m) w[m] = U[pid<N>(a, m, b)];
    modes_bwd<T, N>(sV, w, x);
#pragma unroll
    for (int m = 0; m < N; ++m) U[pid<N>(a, m, b)] = x[m];
  }
  __syncthreads();
  if (valid) {  // backward along z, cell-local result in natural layout
#pragma unroll
    for (int m = 0; m < N; ++m) w[m] = U[pid<N>(a, b, m)];
    modes_bwd<T, N>(sV, w, x);
    T *out = E + (int64_t)cell * N3;
#pragma unroll
    for (int m = 0; m < N; ++m) out[a + N * (b + N * m)] = x[m];
  }
}

// ------------------------------------------------------------------ curved cells
// Gauss quadrature with n points per direction (Section 2.7):
// y = sum_q grad_hat phi . (w_q kappa Ghat_q) grad_hat u, with V[q][m] = l_m(x_q) and
// D[q][m] = l_m'(x_q): gradients at the points by three line passes, the 3x3
// coefficient per point, three transposed passes back.  Gw: [cell][q][6].
template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(cells_per_cta<N>() * N * N) k_gen_op(Grid g, const T *__restrict__ tab,
                                                                       const T *__restrict__ Gw,
                                                                       const Tin *__restrict__ u, T *__restrict__ E) {
  extern __shared__ __align__(16) unsigned char smem_[];
  constexpr int P = N - 1, L = N * N, CPB = cells_per_cta<N>(), PS = psize<N>(), N3 = N * N * N;
  T *sV = reinterpret_cast<T *>(smem_), *sD = sV + N * N;
  const int c = threadIdx.x / L, l = threadIdx.x % L;
  T *U = sD + N * N + c * 5 * PS, *B1 = U + PS, *B2 = B1 + PS, *B3 = B2 + PS, *B4 = B3 + PS;
  const int cell = blockIdx.x * CPB + c;
  const bool valid = cell < g.ncell;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    sV[i] = tab[tab_off(TAB_VQ, N) + i];
    sD[i] = tab[tab_off(TAB_DQ, N) + i];
  }
  if (valid) {
    const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
    for (int idx = l; idx < N3; idx += L) {
      const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
      const int gx = cx * P + i, gy = cy * P + j, gz = cz * P + k;
      const bool dir = node_dirichlet(g, gx, gy, gz);
      U[pid<N>(i, j, k)] = dir ? T(0) : T(u[gidx(g, gx, gy, gz)]);
    }
  }
  __syncthreads();
  const int a = l % N, b = l / N;
  {  // x: B1 = Dx u, B2 = Vx u
    T x[N];
#pragma unroll
    for (int m = 0; m < N; ++m) x[m] = U[pid<N>(m, a, b)];
#pragma unroll
    for (int r = 0; r < N; ++r) {
      B1[pid<N>(r, a, b)] = row_dot<T, N, false>(sD, r, x);
      B2[pid<N>(r, a, b)] = row_dot<T, N, false>(sV, r, x);
    }
  }
  __syncthreads();
  {  // y: B3 = Vy Dx u, B4 = Dy Vx u, U = Vy Vx u
    T x1[N], x2[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      x1[m] = B1[pid<N>(a, m, b)];
      x2[m] = B2[pid<N>(a, m, b)];
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
      B3[pid<N>(a, r, b)] = row_dot<T, N, false>(sV, r, x1);
      B4[pid<N>(a, r, b)] = row_dot<T, N, false>(sD, r, x2);
      U[pid<N>(a, r, b)] = row_dot<T, N, false>(sV, r, x2);
    }
  }
  __syncthreads();
  {  // z: gradients at the points and the coefficient, written over the thread's own z-line
    T x3[N], x4[N], x0[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      x3[m] = B3[pid<N>(a, b, m)];
      x4[m] = B4[pid<N>(a, b, m)];
      x0[m] = U[pid<N>(a, b, m)];
    }
    const T *G = Gw + ((int64_t)(valid ? cell : 0) * N3 + a + N * b) * 6;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      const T gx = row_dot<T, N, false>(sV, k, x3), gy = row_dot<T, N, false>(sV, k, x4),
              gz = row_dot<T, N, false>(sD, k, x0);
      const T *Gq = G + (int64_t)k * N * N * 6;
      B3[pid<N>(a, b, k)] = Gq[0] * gx + Gq[3] * gy + Gq[4] * gz;
      B4[pid<N>(a, b, k)] = Gq[3] * gx + Gq[1] * gy + Gq[5] * gz;
      U[pid<N>(a, b, k)] = Gq[4] * gx + Gq[5] * gy + Gq[2] * gz;
    }
  }
  {  // z back, one flux at a time (the same thread's line): Vz^T fx, Vz^T fy, Dz^T fz
    T f[N], t[N];
#pragma unroll
    for (int w = 0; w < 3; ++w) {
      T *buf = w == 0 ? B3 : (w == 1 ? B4 : U);
      const T *M = w == 2 ? sD : sV;
#pragma unroll
      for (int m = 0; m < N; ++m) f[m] = buf[pid<N>(a, b, m)];
#pragma unroll
      for (int r = 0; r < N; ++r) t[r] = row_dot<T, N, true>(M, r, f);
#pragma unroll
      for (int r = 0; r < N; ++r) buf[pid<N>(a, b, r)] = t[r];
    }
  }
  __syncthreads();
  {  // y back: B1 = Vy^T (Vz^T fx), B2 = Dy^T (Vz^T fy) + Vy^T (Dz^T fz)
    T x3[N], x4[N], x0[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      x3[m] = B3[pid<N>(a, m, b)];
      x4[m] = B4[pid<N>(a, m, b)];
      x0[m] = U[pid<N>(a, m, b)];
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
      B1[pid<N>(a, r, b)] = row_dot<T, N, true>(sV, r, x3);
      B2[pid<N>(a, r, b)] = row_dot<T, N, true>(sD, r, x4) + row_dot<T, N, true>(sV, r, x0);
    }
  }
  __syncthreads();
  if (valid) {  // x back: y = Dx^T B1 + Vx^T B2, cell-local, natural layout
    T x1[N], x2[N];
#pragma unroll
    for (int m = 0; m < N; ++m) {
      x1[m] = B1[pid<N>(m, a, b)];
      x2[m] = B2[pid<N>(m, a, b)];
    }
    T *out = E + (int64_t)cell * N3;
#pragma unroll
    for (int r = 0; r < N; ++r)
      out[r + N * (a + N * b)] = row_dot<T, N, true>(sD, r, x1) + row_dot<T, N, true>(sV, r, x2);
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
  if (node_dirichlet(g, gx, gy, gz)) {
    y[id] = Tout(0);
    return;
  }
  const int gc[3] = {gx, gy, gz};
  const int ncl[3] = {g.nx, g.ny, g.nz};
  int cA[3][2], lA[3][2], cnt[3];
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    const int q = gc[ax] / P, rm = gc[ax] - q * P;
    if (rm == 0) {  // on a cell face along this axis: the cells on either side that exist
      cnt[ax] = 0;  // (one at a traction-free boundary face)
      if (q > 0) { cA[ax][cnt[ax]] = q - 1; lA[ax][cnt[ax]++] = P; }
      if (q < ncl[ax]) { cA[ax][cnt[ax]] = q; lA[ax][cnt[ax]++] = 0; }
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

}  // namespace


// The same direct stiffness summation by cell rows: a thread takes the n - 1
// nodes of one cell along one x node row (the last cell also the row's end
// node), works out the row's y and z cells once, loads each cell row's n
// values together, and sums exactly as k_gather_t does (the (z, y) cell pairs
// in the same nested order, along x the left cell before its own), so the
// results are identical; the rows of a block go through shared memory and are
// written back in node order.
template <typename T, typename Tout, int N>
__global__ void __launch_bounds__(256) k_gather_rows(Grid g, const T *__restrict__ E, const double *__restrict__ rsub,
                                                     Tout *__restrict__ y, int rows_per_block) {
  extern __shared__ __align__(16) unsigned char smem_[];
  constexpr int P = N - 1, N3 = N * N * N;
  T *rowbuf = reinterpret_cast<T *>(smem_);  // rows_per_block x N0
  const int N0 = g.N[0], nrow = g.N[1] * g.N[2], nx = g.nx;
  const int r0 = blockIdx.x * rows_per_block;
  const int nr = min(rows_per_block, nrow - r0);
  for (int t = threadIdx.x; t < nr * nx; t += blockDim.x) {
    const int rl = t / nx, cx = t - rl * nx, row = r0 + rl;
    const int gy = row % g.N[1], gz = row / g.N[1];
    int cy[2], ly[2], cz[2], lz[2], ny_ = 0, nz_ = 0;
    {
      const int q = gy / P, rm = gy - q * P;
      if (rm == 0) {
        if (q > 0) { cy[ny_] = q - 1; ly[ny_++] = P; }
        if (q < g.ny) { cy[ny_] = q; ly[ny_++] = 0; }
      } else { cy[0] = q; ly[0] = rm; ny_ = 1; }
    }
    {
      const int q = gz / P, rm = gz - q * P;
      if (rm == 0) {
        if (q > 0) { cz[nz_] = q - 1; lz[nz_++] = P; }
        if (q < g.nz) { cz[nz_] = q; lz[nz_++] = 0; }
      } else { cz[0] = q; lz[0] = rm; nz_ = 1; }
    }
    T s[N];
#pragma unroll
    for (int i = 0; i < N; ++i) s[i] = 0;
    for (int a2 = 0; a2 < nz_; ++a2)
      for (int a1 = 0; a1 < ny_; ++a1) {
        const int64_t cyz = (int64_t)g.nx * (cy[a1] + g.ny * cz[a2]);
        const int lyz = N * (ly[a1] + N * lz[a2]);
        const T *own = E + (cyz + cx) * N3 + lyz;
        T v[N];
#pragma unroll
        for (int i = 0; i < N; ++i) v[i] = own[i];
        if (cx > 0) s[0] += E[(cyz + cx - 1) * N3 + lyz + P];
#pragma unroll
        for (int i = 0; i < N; ++i) s[i] += v[i];
      }
    T *rb = rowbuf + (size_t)rl * N0 + cx * P;
#pragma unroll
    for (int i = 0; i < P; ++i) rb[i] = s[i];
    if (cx == nx - 1) rb[P] = s[P];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nr * N0; t += blockDim.x) {
    const int rl = t / N0, gx = t - rl * N0, row = r0 + rl;
    const int gy = row % g.N[1], gz = row / g.N[1];
    const int64_t id = gx + (int64_t)N0 * row;
    const T sv = rowbuf[t];
    y[id] = node_dirichlet(g, gx, gy, gz) ? Tout(0) : (rsub ? Tout(T(rsub[id]) - sv) : Tout(sv));
  }
}

// rows per block of the row gather (0: the node gather instead)
inline int gather_rows_per_block(const Grid &g, size_t elem) {
  const int rpb = std::max(1, std::min(64, 256 / std::max(g.nx, 1)));
  return (size_t)rpb * g.N[0] * elem <= 48 * 1024 ? rpb : 0;
}
template <typename T, typename Tout, int N>
void launch_gather_node_sums(const Grid &g, const T *E, const double *rsub, Tout *y, cudaStream_t st) {
  const int rpb = gather_rows_per_block(g, sizeof(T));
  if (rpb > 0) {
    const int nrow = g.N[1] * g.N[2];
    k_gather_rows<T, Tout, N><<<(nrow + rpb - 1) / rpb, 256, (size_t)rpb * g.N[0] * sizeof(T), st>>>(g, E, rsub, y, rpb);
  } else {
    k_gather_t<T, Tout, N><<<dim3((g.N[0] + 127) / 128, g.N[1], g.N[2]), 128, 0, st>>>(g, E, rsub, y);
  }
}

template <typename T, typename Tin, typename Tout>
bool launch_box_op_fast(const OpArgs &a, const Tin *u, Tout *y, T *E, cudaStream_t st, const double *rsub) {
  if constexpr (!std::is_same<T, Tin>::value) {
    return false;
  } else {
    const T *tab = reinterpret_cast<const T *>(a.tab);
    return dispatch_n(a.g.n, [&](auto nc) {
      constexpr int N = decltype(nc)::value;
      constexpr int CPB = cells_per_cta<N>();
      if (a.general) {  // curved cells: Gauss quadrature with the per-point coefficient
        const size_t sm = sizeof(T) * (2 * N * N + (size_t)CPB * 5 * psize<N>());
        set_smem(k_gen_op<T, Tin, N>, sm);
        k_gen_op<T, Tin, N><<<(a.g.ncell + CPB - 1) / CPB, CPB * N * N, sm, st>>>(
            a.g, tab, reinterpret_cast<const T *>(a.Gw), u, E);
      } else if (std::is_same<T, double>::value) {  // FP64: bound by the FP64 pipe, six passes
        const size_t sm = sizeof(T) * (N * N + N + (size_t)CPB * psize<N>());
        set_smem(k_box_op_modes<T, Tin, N>, sm);
        k_box_op_modes<T, Tin, N><<<(a.g.ncell + CPB - 1) / CPB, CPB * N * N, sm, st>>>(a.g, a.mu_box, tab, u, E);
      } else {
        const size_t sm = sizeof(T) * (2 * EO<T, N>::S + (size_t)CPB * 2 * psize<N>());
        set_smem(k_box_op<T, Tin, N>, sm);
        k_box_op<T, Tin, N><<<(a.g.ncell + CPB - 1) / CPB, CPB * N * N, sm, st>>>(a.g, a.mu_box, tab, u, E);
      }
      launch_gather_node_sums<T, Tout, N>(a.g, E, rsub, y, st);
    });
  }
}

template <typename T, typename Tout>
void launch_gather_cells(const Grid &g, const T *E, const double *rsub, Tout *y, cudaStream_t st) {
  if (!dispatch_n(g.n, [&](auto NC) {
        constexpr int N = decltype(NC)::value;
        launch_gather_node_sums<T, Tout, N>(g, E, rsub, y, st);
      }))
    fail(FDM_EINVAL, "node gather: unsupported degree");
}
template void launch_gather_cells<double, double>(const Grid &, const double *, const double *, double *,
                                                  cudaStream_t);
template void launch_gather_cells<float, float>(const Grid &, const float *, const double *, float *, cudaStream_t);

template bool launch_box_op_fast<double, double, double>(const OpArgs &, const double *, double *, double *,
                                                         cudaStream_t, const double *);
template bool launch_box_op_fast<float, float, float>(const OpArgs &, const float *, float *, float *, cudaStream_t,
                                                      const double *);
template bool launch_box_op_fast<double, double, float>(const OpArgs &, const double *, float *, double *,
                                                        cudaStream_t, const double *);

}  // namespace fdm
