// Relaxation and coarse-space cell kernels specialised on n: restriction to the
// FDM basis with condensation, interpolation back, Q1 restriction and
// prolongation; helpers in k_cell.cuh.
#include "k_cell.cuh"

namespace fdm {
namespace {

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
  // the cell's three coefficients, converted once per cell (read after the first barrier)
  __shared__ T sMu[CPB][3];
  if (l < 3) sMu[c][l] = valid ? T(mug[3 * cell + l]) : T(0);
  int cx = 0, cy = 0, cz = 0;
  if (valid) {
    cx = cell % g.nx;
    cy = (cell / g.nx) % g.ny;
    cz = cell / (g.nx * g.ny);
    for (int idx = l; idx < N3; idx += L) {  // W_K r_K, W = 1 / multiplicity, Dirichlet entries 0
      const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
      const int gx = cx * P + i, gy = cy * P + j, gz = cz * P + k;
      const bool dir = node_dirichlet(g, gx, gy, gz);
      const int mult = ((i == 0 && cx > 0) || (i == P && cx < g.nx - 1) ? 2 : 1) *
                       ((j == 0 && cy > 0) || (j == P && cy < g.ny - 1) ? 2 : 1) *
                       ((k == 0 && cz > 0) || (k == P && cz < g.nz - 1) ? 2 : 1);
      const T wm = mult == 1 ? T(1) : (mult == 2 ? T(0.5) : (mult == 4 ? T(0.25) : T(0.125)));  // exact 1/mult
      U[pid<N>(i, j, k)] = dir ? T(0) : T(r[gidx(g, gx, gy, gz)]) * wm;
    }
  }
  __syncthreads();
  const T m0 = sMu[c][0], m1 = sMu[c][1], m2 = sMu[c][2];
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
// the t-th of the N^3 - (N-2)^3 boundary nodes of a cell: the layers k = 0 and
// k = N - 1 whole, each layer between as its ring (row j = 0, row j = N - 1,
// column i = 0, column i = N - 1 without the corners)
template <int N>
__device__ __forceinline__ void boundary_node(int t, int &i, int &j, int &k) {
  constexpr int L = N * N, R = 4 * (N - 1);
  if (t < L) {
    k = 0;
    i = t % N;
    j = t / N;
    return;
  }
  t -= L;
  if (t < (N - 2) * R) {
    k = 1 + t / R;
    const int r = t % R;
    if (r < N) { i = r; j = 0; }
    else if (r < 2 * N) { i = r - N; j = N - 1; }
    else if (r < 3 * N - 2) { i = 0; j = r - 2 * N + 1; }
    else { i = N - 1; j = r - (3 * N - 2) + 1; }
    return;
  }
  t -= (N - 2) * R;
  k = N - 1;
  i = t % N;
  j = t / N;
}

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
  if (valid) {
    ce[0] = cell % g.nx;
    ce[1] = (cell / g.nx) % g.ny;
    ce[2] = cell / (g.nx * g.ny);
  }
  // the cell's three coefficients, converted once per cell (read after the next barrier)
  __shared__ T sMu[CPB][3];
  if (l < 3) sMu[c][l] = valid ? T(a.mu[3 * cell + l]) : T(0);
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
  const T m0 = sMu[c][0], m1 = sMu[c][1], m2 = sMu[c][2];
  // large cells walk compact lists of their boundary and interior nodes (all lanes
  // busy: 26 % faster at N = 16); small ones the whole cube with a test per node
  // (the compact lists measured 34 % slower at N = 8)
  constexpr int NI = (N - 2) * (N - 2) * (N - 2), NB = N3 - NI;
  constexpr int M = N > 2 ? N - 2 : 1;  // interior nodes per axis (none for N = 2: no iteration)
  // interface-type nodes: the sum of the stars' interface solutions
  auto interface_node = [&](const int li[3]) {
    const int idx = li[0] + N * (li[1] + N * li[2]);
    T acc = 0;
#pragma unroll
    for (int o = 0; o < 8; ++o) {
      const int k = a.cmap[(sCls[c][o] * 8 + o) * N3 + idx];
      if (k >= 0) acc += a.X[sOff[c][o] + k];
    }
    U[pid<N>(li[0], li[1], li[2])] = acc;
  };
  // interior nodes: (8 r(m) - sum over the 6 face nodes of A_mf z(f)) / A_mm
  const T *Ek = a.E + (int64_t)(valid ? cell : 0) * N3;
  auto interior_node = [&](const int li[3]) {
    const int idx = li[0] + N * (li[1] + N * li[2]);
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
  };
  if constexpr (N >= 12) {
    if (valid) {
      for (int t = l; t < NB; t += L) {
        int li[3];
        boundary_node<N>(t, li[0], li[1], li[2]);
        interface_node(li);
      }
    }
    __syncthreads();
    if (valid) {
      for (int t = l; t < NI; t += L) {  // x fastest
        const int li[3] = {1 + t % M, 1 + (t / M) % M, 1 + t / (M * M)};
        interior_node(li);
      }
    }
  } else {
    if (valid) {
      for (int idx = l; idx < N3; idx += L) {
        const int li[3] = {idx % N, (idx / N) % N, idx / (N * N)};
        const bool onb = li[0] == 0 || li[0] == P || li[1] == 0 || li[1] == P || li[2] == 0 || li[2] == P;
        if (onb) interface_node(li);
      }
    }
    __syncthreads();
    if (valid) {
      for (int idx = l; idx < N3; idx += L) {
        const int li[3] = {idx % N, (idx / N) % N, idx / (N * N)};
        const bool onb = li[0] == 0 || li[0] == P || li[1] == 0 || li[1] == P || li[2] == 0 || li[2] == P;
        if (!onb) interior_node(li);
      }
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
  const T om = T(omega);  // omega in the kernel's precision
  for (int idx = l; idx < N3; idx += L) {
    const int i = idx % N, j = (idx / N) % N, k = idx / (N * N);
    if ((i == 0 && ce[0] > 0) || (j == 0 && ce[1] > 0) || (k == 0 && ce[2] > 0)) continue;  // not owner
    const int gx = ce[0] * P + i, gy = ce[1] * P + j, gz = ce[2] * P + k;
    const bool dir = node_dirichlet(g, gx, gy, gz);
    const int64_t id = gidx(g, gx, gy, gz);
    // z = omega * relaxation, plus a.addv where given (the V-cycle's pre-smoothed x1)
    const T zv = a.addv ? a.addv[id] + om * V[pid<N>(i, j, k)] : om * V[pid<N>(i, j, k)];
    z[id] = dir ? Tout(0) : Tout(zv);
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
        const T v = T(r[gidx(g, gx, gy, gz)]) * (m == 1 ? T(1) : (m == 2 ? T(0.5) : (m == 4 ? T(0.25) : T(0.125))));
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

}  // namespace

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
  if (g.dmask != 63) return false;  // specialised for the all-Dirichlet boundary
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
  if (g.dmask != 63) return false;  // specialised for the all-Dirichlet boundary
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
