// Primal linear elasticity on box cells (Section 4.1): the operator
//   a(v, u) = int 2 mu eps(v):eps(u) + lam div v div u = int sum_{a,d} d_d v_a sigma_ad(u),
//   sigma_ad = mu (d_d u_a + d_a u_d) + lam delta_ad div u,
// by sum factorisation on the (p+1)^3 Gauss points of each cell (exact: the
// integrands have degree <= 2p per axis).  Vectors are component-major
// [3][ndof].  Two cell kernels and a node gather per component:
//   k_elast_grad:  per (cell, component b), the three reference derivatives of
//                  u_b at the Gauss points (8 line passes) -> G[b][d][cell][q^3];
//   k_elast_flux:  per (cell, component a), the weighted fluxes
//                  F_ad = w vol sigma_ad / L_d formed from the 9 derivatives,
//                  then the transposed passes (8) -> cell-local output E[a];
//   the node gather of the scalar operator sums E[a] over the cells of each node.
// The cell kernels keep four n^3 arrays in shared memory (128 KB at n = 16 in
// FP64) and run one CTA per (cell, component), 256 threads looping over the
// outputs of each pass.
#include "k_cell.cuh"
#include "kernels.h"

namespace fdm {

namespace {

constexpr int EL_THREADS = 256;

// out[z][y][r] = sum_c M[r][c] in[z][y][c]  (trans: M[c][r]); n = N at compile time
template <typename T, int N, bool TR>
__device__ __forceinline__ void pass_x(const T *M, const T *in, T *out, bool acc) {
  constexpr int N3 = N * N * N;
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int r = o % N, zy = o / N;
    const T *src = in + zy * N;
    T s = 0;
#pragma unroll
    for (int c = 0; c < N; ++c) s = fma(TR ? M[c * N + r] : M[r * N + c], src[c], s);
    out[o] = acc ? out[o] + s : s;
  }
}
template <typename T, int N, bool TR>
__device__ __forceinline__ void pass_y(const T *M, const T *in, T *out, bool acc) {
  constexpr int N3 = N * N * N;
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int x = o % N, r = (o / N) % N, z = o / (N * N);
    const T *src = in + z * N * N + x;
    T s = 0;
#pragma unroll
    for (int c = 0; c < N; ++c) s = fma(TR ? M[c * N + r] : M[r * N + c], src[c * N], s);
    out[o] = acc ? out[o] + s : s;
  }
}
template <typename T, int N, bool TR>
__device__ __forceinline__ void pass_z(const T *M, const T *in, T *out, bool acc) {
  constexpr int N2 = N * N, N3 = N2 * N;
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int xy = o % N2, r = o / N2;
    const T *src = in + xy;
    T s = 0;
#pragma unroll
    for (int c = 0; c < N; ++c) s = fma(TR ? M[c * N + r] : M[r * N + c], src[c * N2], s);
    out[o] = acc ? out[o] + s : s;
  }
}

template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(EL_THREADS) k_elast_grad(Grid g, const Tin *__restrict__ u,
                                                           const T *__restrict__ tab, T *__restrict__ G) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n = N, n3 = N * N * N;
  const int p = g.p;
  T *M = reinterpret_cast<T *>(smem_raw);  // V, D (2 n^2)
  T *U = M + 2 * n * n, *S1 = U + n3, *S2 = S1 + n3, *S3 = S2 + n3;
  const int cell = blockIdx.x, b = blockIdx.y;
  const int cx = cell % g.nx, cy = (cell / g.nx) % g.ny, cz = cell / (g.nx * g.ny);
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    M[i] = tab[tab_off(TAB_VQ, n) + i];
    M[n * n + i] = tab[tab_off(TAB_DQ, n) + i];
  }
  const Tin *ub = u + (int64_t)b * g.ndof;
  for (int o = threadIdx.x; o < n3; o += blockDim.x) {
    const int i = o % n, j = (o / n) % n, k = o / (n * n);
    const int gx = cx * p + i, gy = cy * p + j, gz = cz * p + k;
    const bool dir = node_dirichlet(g, gx, gy, gz);
    U[o] = dir ? T(0) : T(ub[gidx(g, gx, gy, gz)]);  // Dirichlet entries of the input are ignored
  }
  __syncthreads();
  const T *V = M, *D = M + n * n;
  T *Gb = G + (int64_t)(3 * b) * g.ncell * n3 + (int64_t)cell * n3;  // G[b][d][cell][q^3]
  const int64_t dstride = (int64_t)g.ncell * n3;
  pass_z<T, N, false>(V, U, S1, false);   // V_z u
  __syncthreads();
  pass_y<T, N, false>(V, S1, S2, false);  // V_y V_z u
  pass_y<T, N, false>(D, S1, S3, false);  // D_y V_z u
  __syncthreads();
  pass_x<T, N, false>(D, S2, Gb, false);               // d/dxi_x
  pass_x<T, N, false>(V, S3, Gb + dstride, false);     // d/dxi_y
  pass_z<T, N, false>(D, U, S1, false);                // D_z u
  __syncthreads();
  pass_y<T, N, false>(V, S1, S2, false);
  __syncthreads();
  pass_x<T, N, false>(V, S2, Gb + 2 * dstride, false);  // d/dxi_z
}

template <typename T, int N>
__global__ void __launch_bounds__(EL_THREADS) k_elast_flux(Grid g, const T *__restrict__ G, const T *__restrict__ tab,
                                                           const T *__restrict__ wq, const double *__restrict__ Lc,
                                                           double mu, double lam, T *__restrict__ E) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int n = N, n3 = N * N * N;
  T *M = reinterpret_cast<T *>(smem_raw);
  T *S0 = M + 2 * n * n, *S1 = S0 + n3, *S2 = S1 + n3, *S3 = S2 + n3;
  const int cell = blockIdx.x, a = blockIdx.y;
  for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
    M[i] = tab[tab_off(TAB_VQ, n) + i];
    M[n * n + i] = tab[tab_off(TAB_DQ, n) + i];
  }
  // the pointwise stress in the kernel's precision (FP32 inside the FP32 preconditioner)
  const T L[3] = {T(Lc[3 * cell]), T(Lc[3 * cell + 1]), T(Lc[3 * cell + 2])};
  const T vol = L[0] * L[1] * L[2];
  const T iL[3] = {T(1) / L[0], T(1) / L[1], T(1) / L[2]};  // no divisions per point
  const T tmu = T(mu), tlam = T(lam);
  const int64_t dstride = (int64_t)g.ncell * n3;
  const T *Gc = G + (int64_t)cell * n3;
  // physical derivative d_d u_b at point o
  auto grad = [&](int b, int d, int o) { return Gc[(3 * b + d) * dstride + o] * iL[d]; };
  T *F[3] = {S0, S1, S2};
  for (int o = threadIdx.x; o < n3; o += blockDim.x) {
    const int i = o % n, j = (o / n) % n, k = o / (n * n);
    const T w = wq[i] * wq[j] * wq[k] * vol;
    const T div = grad(0, 0, o) + grad(1, 1, o) + grad(2, 2, o);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      T s = tmu * (grad(a, d, o) + grad(d, a, o));
      if (d == a) s += tlam * div;
      F[d][o] = w * s * iL[d];
    }
  }
  __syncthreads();
  const T *V = M, *D = M + n * n;
  // y = V_z^T [V_y^T D_x^T F_x + D_y^T V_x^T F_y] + D_z^T V_y^T V_x^T F_z, four buffers
  pass_x<T, N, true>(D, S0, S3, false);  // S3 = D_x^T F_x
  __syncthreads();
  pass_x<T, N, true>(V, S1, S0, false);  // S0 = V_x^T F_y
  __syncthreads();
  pass_y<T, N, true>(V, S3, S1, false);  // S1 = V_y^T S3
  __syncthreads();
  pass_y<T, N, true>(D, S0, S1, true);   // S1 += D_y^T S0
  pass_x<T, N, true>(V, S2, S3, false);  // S3 = V_x^T F_z
  __syncthreads();
  pass_y<T, N, true>(V, S3, S0, false);  // S0 = V_y^T S3
  __syncthreads();
  pass_z<T, N, true>(V, S1, S2, false);  // S2 = V_z^T S1
  __syncthreads();
  pass_z<T, N, true>(D, S0, S2, true);   // S2 += D_z^T S0
  __syncthreads();
  T *Ea = E + (int64_t)a * g.ncell * n3 + (int64_t)cell * n3;
  for (int o = threadIdx.x; o < n3; o += blockDim.x) Ea[o] = S2[o];
}

}  // namespace

template <typename T>
size_t elast_smem(int n) {
  return sizeof(T) * (2 * (size_t)n * n + 4 * (size_t)n * n * n);
}

template <typename T, typename Tin>
void launch_elast_cells(const Grid &g, const Tin *u, const T *tab, const T *wq, const double *Lc, double mu, double lam,
                        T *G, T *E, cudaStream_t st) {
  const size_t sm = elast_smem<T>(g.n);
  if (!dispatch_n(g.n, [&](auto NC) {
        constexpr int N = decltype(NC)::value;
        set_smem(k_elast_grad<T, Tin, N>, sm);
        set_smem(k_elast_flux<T, N>, sm);
        k_elast_grad<T, Tin, N><<<dim3(g.ncell, 3), EL_THREADS, sm, st>>>(g, u, tab, G);
        k_elast_flux<T, N><<<dim3(g.ncell, 3), EL_THREADS, sm, st>>>(g, G, tab, wq, Lc, mu, lam, E);
      }))
    fail(FDM_EINVAL, "elasticity operator: unsupported degree");
}

template size_t elast_smem<double>(int);
template size_t elast_smem<float>(int);
template void launch_elast_cells<double, double>(const Grid &, const double *, const double *, const double *,
                                                 const double *, double, double, double *, double *, cudaStream_t);
template void launch_elast_cells<float, float>(const Grid &, const float *, const float *, const float *,
                                               const double *, double, double, float *, float *, cudaStream_t);
template void launch_elast_cells<float, double>(const Grid &, const double *, const float *, const float *,
                                                const double *, double, double, float *, float *, cudaStream_t);

}  // namespace fdm
