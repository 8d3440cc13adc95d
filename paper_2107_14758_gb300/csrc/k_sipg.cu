// Symmetric interior penalty DG (SIPG) for the Poisson equation on DQ_p box
// cells (Section 5, Eqs. sipg_lhs, dirichlet_stiffness, interior_stiffness):
// the operator, the vertex-star patch solve and the transfers to the Q1
// coarse space.  Vectors are cell-major [cell][z][y][x] (cells x fastest),
// (p+1)^3 GLL nodal values per cell.
//
//   k_sipg_faces:  per cell and face, the trace and the normal derivative
//                  d/dx_a of u (F[cell][2 a + side][value, derivative][N^2]);
//   k_sipg_cell:   per cell, the cell term sum_d (vol/h_d^2) A_hat (x) B_hat
//                  (x) B_hat by sum factorisation, plus the six facet terms
//                  from its own and its neighbours' face data: penalty
//                  sigma [u] on the face layer, -{d_n u} on the face layer,
//                  -w [u] d_n phi_i along the normal lines, with the
//                  tangential mass h_t1 h_t2 B_hat (x) B_hat;
//   k_sipg_patch:  the exact solve with a star's matrix.  On a star of 8 box
//                  cells that matrix is the Kronecker sum Ax (x) My (x) Mz +
//                  Mx (x) Ay (x) Mz + Mx (x) My (x) Az of 2(p+1)-square 1D
//                  two-cell operators (cell and facet terms) and masses, so
//                  with S^T A S = Lambda, S^T M S = I per axis its inverse is
//                  (S (x) S (x) S) (Lambda_x + Lambda_y + Lambda_z)^{-1}
//                  (S (x) S (x) S)^T: six line passes over the star tensor
//                  in shared memory, one line per thread.  The stars of the
//                  vertices of one parity class (vx, vy, vz mod 2) share no
//                  cell, so each of the 8 classes is one launch that adds its
//                  stars' results into the output without conflicts, in a
//                  fixed order.
#include "k_cell.cuh"
#include "kernels.h"

namespace fdm {

namespace {

constexpr int SIPG_THREADS = 256;

template <typename T>
__device__ __forceinline__ T dcast(double v) { return T(v); }

// element index of the node with normal index m and tangential (r, s) on a
// face normal to axis a (r along the lower remaining axis)
template <int N>
__device__ __forceinline__ int face_node(int a, int m, int r, int s) {
  return a == 0 ? m + N * (r + N * s) : (a == 1 ? r + N * (m + N * s) : r + N * (s + N * m));
}

template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(128) k_sipg_faces(SipgDev<T> d, const Tin *__restrict__ u, T *__restrict__ F) {
  constexpr int N2 = N * N, N3 = N2 * N;
  __shared__ T U[N3];
  __shared__ T dd[2 * N];
  const int cell = blockIdx.x;
  const int cx = cell % d.nx, cy = (cell / d.nx) % d.ny, cz = cell / (d.nx * d.ny);
  const Tin *uc = u + (int64_t)cell * N3;
  for (int o = threadIdx.x; o < N3; o += blockDim.x) U[o] = T(uc[o]);
  if (threadIdx.x < 2 * N) dd[threadIdx.x] = d.tab[2 * N2 + threadIdx.x];  // dm, dp
  __syncthreads();
  const T ih[3] = {T(1) / dcast<T>(d.hx[cx]), T(1) / dcast<T>(d.hy[cy]), T(1) / dcast<T>(d.hz[cz])};
  T *Fc = F + (int64_t)cell * 12 * N2;
  for (int t = threadIdx.x; t < 6 * N2; t += blockDim.x) {
    const int f = t / N2, q = t % N2, a = f >> 1, side = f & 1;
    const int r = q % N, s = q / N;
    const T *dv = dd + side * N;
    T der = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) der = fma(dv[m], U[face_node<N>(a, m, r, s)], der);
    Fc[(2 * f) * N2 + q] = U[face_node<N>(a, side ? N - 1 : 0, r, s)];
    Fc[(2 * f + 1) * N2 + q] = der * ih[a];
  }
}

// y = A u (rsub == nullptr) or y = rsub - A u, per cell
template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(SIPG_THREADS) k_sipg_cell(SipgDev<T> d, const Tin *__restrict__ u,
                                                            const T *__restrict__ F, const double *__restrict__ rsub,
                                                            T *__restrict__ y) {
  constexpr int N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *A = reinterpret_cast<T *>(smem_raw), *B = A + N2;
  T *dm = B + N2, *dp = dm + N;
  T *U = dp + N, *P1 = U + N3, *P2 = P1 + N3, *P3 = P2 + N3;
  T *J = P3 + N3, *G = J + 6 * N2, *Jt = G + 6 * N2, *Gt = Jt + 6 * N2;  // face buffers [6][N^2]
  __shared__ T fsig[6], fwgt[6];
  __shared__ int fin[6];
  const int cell = blockIdx.x;
  const int c[3] = {cell % d.nx, (cell / d.nx) % d.ny, cell / (d.nx * d.ny)};
  const int nc[3] = {d.nx, d.ny, d.nz};
  const int stride[3] = {1, d.nx, d.nx * d.ny};
  const double *hax[3] = {d.hx, d.hy, d.hz};
  for (int i = threadIdx.x; i < 2 * N2 + 2 * N; i += blockDim.x) A[i] = d.tab[i];
  const Tin *uc = u + (int64_t)cell * N3;
  for (int o = threadIdx.x; o < N3; o += blockDim.x) U[o] = T(uc[o]);
  if (threadIdx.x < 6) {
    const int f = threadIdx.x, a = f >> 1, side = f & 1;
    const double h = hax[a][c[a]];
    const bool inner = side ? c[a] < nc[a] - 1 : c[a] > 0;
    fin[f] = inner;
    if (inner) {
      const double hn = hax[a][c[a] + (side ? 1 : -1)];
      fsig[f] = T(d.eta * 0.25 * (1.0 / h + 1.0 / hn));
      fwgt[f] = T(0.5);
    } else {
      fsig[f] = T(d.eta / (2.0 * h));
      fwgt[f] = T(1);
    }
  }
  const T h[3] = {dcast<T>(d.hx[c[0]]), dcast<T>(d.hy[c[1]]), dcast<T>(d.hz[c[2]])};
  const T cxv = h[1] * h[2] / h[0], cyv = h[0] * h[2] / h[1], czv = h[0] * h[1] / h[2];
  __syncthreads();
  // face quantities in the outward-normal frame: Jn = u_own - u_nb, Gn = n . {grad u}
  for (int t = threadIdx.x; t < 6 * N2; t += blockDim.x) {
    const int f = t / N2, q = t % N2, a = f >> 1, side = f & 1;
    const T *Fo = F + ((int64_t)cell * 12 + 2 * f) * N2;
    T jn = Fo[q], gn = Fo[N2 + q];
    if (fin[f]) {
      const int nb = cell + (side ? stride[a] : -stride[a]);
      const T *Fn = F + ((int64_t)nb * 12 + 2 * (2 * a + 1 - side)) * N2;
      jn -= Fn[q];
      gn = T(0.5) * (gn + Fn[N2 + q]);
    }
    J[t] = jn;
    G[t] = side ? gn : -gn;
  }
  // cell term: P1 = A_x U, P2 = B_x U
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int i = o % N, jk = o - i;
    T s1 = 0, s2 = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const T v = U[jk + m];
      s1 = fma(A[i * N + m], v, s1);
      s2 = fma(B[i * N + m], v, s2);
    }
    P1[o] = s1;
    P2[o] = s2;
  }
  __syncthreads();
  // tangential mass, first factor (along r): Jt = B_r J, Gt = B_r G
  for (int t = threadIdx.x; t < 6 * N2; t += blockDim.x) {
    const int q = t % N2, r = q % N, base = t - r;
    T sj = 0, sg = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      sj = fma(B[r * N + m], J[base + m], sj);
      sg = fma(B[r * N + m], G[base + m], sg);
    }
    Jt[t] = sj;
    Gt[t] = sg;
  }
  // U = cx B_y P1 + cy A_y P2 (terms that end with B_z), P3 = B_y P2 (ends with cz A_z)
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int i = o % N, j = (o / N) % N, k = o / N2;
    const int base = i + N2 * k;
    T s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const T v1 = P1[base + N * m], v2 = P2[base + N * m];
      s1 = fma(B[j * N + m], v1, s1);
      s2 = fma(A[j * N + m], v2, s2);
      s3 = fma(B[j * N + m], v2, s3);
    }
    U[o] = cxv * s1 + cyv * s2;
    P3[o] = s3;
  }
  __syncthreads();
  // second tangential factor (along s) with h_t1 h_t2: J = h h B_s Jt, G = h h B_s Gt
  for (int t = threadIdx.x; t < 6 * N2; t += blockDim.x) {
    const int f = t / N2, q = t % N2, r = q % N, s = q / N, a = f >> 1;
    const T *jt = Jt + f * N2 + r, *gt = Gt + f * N2 + r;
    T sj = 0, sg = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      sj = fma(B[s * N + m], jt[N * m], sj);
      sg = fma(B[s * N + m], gt[N * m], sg);
    }
    const T ht = a == 0 ? h[1] * h[2] : (a == 1 ? h[0] * h[2] : h[0] * h[1]);
    J[t] = ht * sj;
    G[t] = ht * sg;
  }
  // P1 = B_z U + cz A_z P3
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int xy = o % N2, k = o / N2;
    T s = 0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      s = fma(B[k * N + m], U[xy + N2 * m], s);
      s = fma(czv * A[k * N + m], P3[xy + N2 * m], s);
    }
    P1[o] = s;
  }
  __syncthreads();
  // facet terms: face layer += sigma Jn - Gn; normal lines -= w (n . grad phi_m) Jn
  T *yc = y + (int64_t)cell * N3;
  const double *rs = rsub ? rsub + (int64_t)cell * N3 : nullptr;
  const T ih[3] = {T(1) / h[0], T(1) / h[1], T(1) / h[2]};
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int idx[3] = {o % N, (o / N) % N, o / N2};
    T acc = P1[o];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int m = idx[a];
      const int r = a == 0 ? idx[1] : idx[0], s = a == 2 ? idx[1] : idx[2];
      const int q = r + N * s;
#pragma unroll
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * a + side;
        const T jn = J[f * N2 + q];
        const T dn = side ? dp[m] : -dm[m];  // n . grad phi_m, times h_a
        acc = fma(-fwgt[f] * dn * ih[a], jn, acc);
        if (m == (side ? N - 1 : 0)) acc += fsig[f] * jn - G[f * N2 + q];
      }
    }
    yc[o] = rs ? T(rs[o]) - acc : acc;
  }
}

// one line of the star tensor (index X + MP (Y + M Z)) along `axis`
template <int M, int MP, int AXIS>
__device__ __forceinline__ int line_index(int l, int m) {
  const int a = l % M, b = l / M;
  return AXIS == 0 ? m + MP * (a + M * b) : (AXIS == 1 ? a + MP * (m + M * b) : a + MP * (b + M * m));
}

// sum over m = 0..M-1 of row[m] x[m], accumulated in that order, the row (in
// shared memory, 16-byte aligned where M allows) read by vector loads: with the
// row shared by the whole warp each load is a broadcast, and one vector load
// replaces two or four scalar ones
template <typename T, int M>
__device__ __forceinline__ T row_dot(const T *row, const T (&x)[M]) {
  T s = 0;
  if constexpr (sizeof(T) == 4 && M % 4 == 0) {
    const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
    for (int q = 0; q < M / 4; ++q) {
      const float4 v = r4[q];
      s = fma(v.x, x[4 * q], s);
      s = fma(v.y, x[4 * q + 1], s);
      s = fma(v.z, x[4 * q + 2], s);
      s = fma(v.w, x[4 * q + 3], s);
    }
  } else if constexpr (sizeof(T) == 4) {
    const float2 *r2 = reinterpret_cast<const float2 *>(row);
#pragma unroll
    for (int q = 0; q < M / 2; ++q) {
      const float2 v = r2[q];
      s = fma(v.x, x[2 * q], s);
      s = fma(v.y, x[2 * q + 1], s);
    }
  } else {
    const double2 *r2 = reinterpret_cast<const double2 *>(row);
#pragma unroll
    for (int q = 0; q < M / 2; ++q) {
      const double2 v = r2[q];
      s = fma(v.x, x[2 * q], s);
      s = fma(v.y, x[2 * q + 1], s);
    }
  }
  return s;
}

// in place: line <- R line, R row-major [i][m] (R = S^T for the transform to
// the eigenbasis, S for the way back).  The thread holds its input line in
// registers and writes each output as soon as it is formed.
template <typename T, int M, int MP, int AXIS>
__device__ __forceinline__ void star_pass(T *U, const T *R, int nthr) {
  for (int l = threadIdx.x; l < M * M; l += nthr) {
    T x[M];
#pragma unroll
    for (int m = 0; m < M; ++m) x[m] = U[line_index<M, MP, AXIS>(l, m)];
#pragma unroll 2
    for (int i = 0; i < M; ++i) U[line_index<M, MP, AXIS>(l, i)] = row_dot<T, M>(R + i * M, x);
  }
}

template <typename T, typename Tin, typename Tout, int N>
__global__ void __launch_bounds__(SIPG_THREADS) k_sipg_patch(SipgDev<T> d, int color, const int *__restrict__ vlist,
                                                             const Tin *__restrict__ r, Tout *__restrict__ z,
                                                             T *__restrict__ zpatch, double omega) {
  constexpr int M = 2 * N, MP = M + 1, M2 = M * M, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *S = reinterpret_cast<T *>(smem_raw);  // [3][M][M]: S per axis, row-major
  T *ST = S + 3 * M2;                      // [3][M][M]: S^T per axis, row-major
  T *lam = ST + 3 * M2;                    // [3][M]
  T *U = lam + 3 * M;                      // [M][M][MP]
  const int nvx = d.nx + 1, nvy = d.ny + 1;
  int v[3];
  if (vlist) {
    const int vv = vlist[blockIdx.x];
    v[0] = vv % nvx;
    v[1] = (vv / nvx) % nvy;
    v[2] = vv / (nvx * nvy);
  } else {
    // vertices 1..nc-1 of parity (color >> axis) & 1 along each axis
    const int nc[3] = {d.nx, d.ny, d.nz};
    int cnt[3], first[3];
    for (int a = 0; a < 3; ++a) {
      first[a] = ((color >> a) & 1) ? 1 : 2;
      cnt[a] = first[a] <= nc[a] - 1 ? (nc[a] - 1 - first[a]) / 2 + 1 : 0;
    }
    const int b = blockIdx.x;
    v[0] = first[0] + 2 * (b % cnt[0]);
    v[1] = first[1] + 2 * ((b / cnt[0]) % cnt[1]);
    v[2] = first[2] + 2 * (b / (cnt[0] * cnt[1]));
  }
  const int nthr = blockDim.x;
  for (int a = 0; a < 3; ++a) {
    const T *Sa = d.S + d.soff[a] + (int64_t)(v[a] - 1) * M2;
    const T *la = d.lam + d.loff[a] + (int64_t)(v[a] - 1) * M;
    for (int t = threadIdx.x; t < M2; t += nthr) {
      const T v = Sa[t];
      S[a * M2 + t] = v;
      ST[a * M2 + (t % M) * M + t / M] = v;
    }
    for (int t = threadIdx.x; t < M; t += nthr) lam[a * M + t] = la[t];
  }
  __syncthreads();
  const T *Sx = S, *Sy = S + M2, *Sz = S + 2 * M2;
  const T *STx = ST, *STy = ST + M2, *STz = ST + 2 * M2;
  // gather fused with the x pass: the thread of line (Y, Z) reads two cell rows
  for (int l = threadIdx.x; l < M2; l += nthr) {
    const int Y = l % M, Z = l / M;
    const int cb = Y / N, j = Y % N, cc = Z / N, k = Z % N;
    T x[M];
#pragma unroll
    for (int ca = 0; ca < 2; ++ca) {
      const int cell = (v[0] - 1 + ca) + d.nx * ((v[1] - 1 + cb) + d.ny * (v[2] - 1 + cc));
      const Tin *row = r + (int64_t)cell * N3 + N * (j + N * k);
#pragma unroll
      for (int i = 0; i < N; ++i) x[ca * N + i] = T(row[i]);
    }
#pragma unroll 2
    for (int i = 0; i < M; ++i) U[i + MP * (Y + M * Z)] = row_dot<T, M>(STx + i * M, x);
  }
  __syncthreads();
  star_pass<T, M, MP, 1>(U, STy, nthr);
  __syncthreads();
  // z pass forward with the division by the eigenvalue sums, then back; the
  // line stays with its thread, so no barrier between the two
  for (int l = threadIdx.x; l < M2; l += nthr) {
    const int X = l % M, Y = l / M;
    T *line = U + X + MP * Y;
    T x[M];
#pragma unroll
    for (int m = 0; m < M; ++m) x[m] = line[MP * M * m];
    const T lxy = lam[X] + lam[M + Y];
#pragma unroll 2
    for (int i = 0; i < M; ++i) line[MP * M * i] = row_dot<T, M>(STz + i * M, x) / (lxy + lam[2 * M + i]);
#pragma unroll
    for (int m = 0; m < M; ++m) x[m] = line[MP * M * m];
#pragma unroll 2
    for (int m = 0; m < M; ++m) line[MP * M * m] = row_dot<T, M>(Sz + m * M, x);
  }
  __syncthreads();
  star_pass<T, M, MP, 1>(U, Sy, nthr);
  __syncthreads();
  // x pass back fused with the scatter (z += omega result) or the patch output
  const T w = T(omega);
  for (int l = threadIdx.x; l < M2; l += nthr) {
    const int Y = l % M, Z = l / M;
    const int cb = Y / N, j = Y % N, cc = Z / N, k = Z % N;
    T x[M];
#pragma unroll
    for (int m = 0; m < M; ++m) x[m] = U[m + MP * (Y + M * Z)];
    T *zp = zpatch ? zpatch + (int64_t)blockIdx.x * M * M2 + M * (Y + M * Z) : nullptr;
    Tout *row[2];
#pragma unroll
    for (int ca = 0; ca < 2; ++ca)
      row[ca] = z + (int64_t)((v[0] - 1 + ca) + d.nx * ((v[1] - 1 + cb) + d.ny * (v[2] - 1 + cc))) * N3 +
                N * (j + N * k);
#pragma unroll 2
    for (int m = 0; m < M; ++m) {
      const T s = row_dot<T, M>(Sx + m * M, x);
      if (zp) zp[m] = s;
      else {
        Tout *o = row[m / N] + m % N;
        *o = Tout(*o + Tout(w * s));
      }
    }
  }
}

// per cell, the 8 corner sums of the Q1 restriction: sum_nodes hat_s r
template <typename T, typename Tin, int N>
__global__ void __launch_bounds__(128) k_sipg_restrict_cells(SipgDev<T> d, const Tin *__restrict__ r,
                                                             T *__restrict__ cellbuf) {
  constexpr int N3 = N * N * N;
  __shared__ T red[8][4];
  const int cell = blockIdx.x;
  const T *xi = d.tab + 2 * N * N + 2 * N;
  const Tin *rc = r + (int64_t)cell * N3;
  T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int i = o % N, j = (o / N) % N, k = o / (N * N);
    const T v = T(rc[o]);
    const T hx[2] = {T(0.5) * (T(1) - xi[i]), T(0.5) * (T(1) + xi[i])};
    const T hy[2] = {T(0.5) * (T(1) - xi[j]), T(0.5) * (T(1) + xi[j])};
    const T hz[2] = {T(0.5) * (T(1) - xi[k]), T(0.5) * (T(1) + xi[k])};
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[s] = fma(hx[s & 1] * hy[(s >> 1) & 1] * hz[s >> 2], v, acc[s]);
  }
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const T w = warp_sum(acc[s]);
    if ((threadIdx.x & 31) == 0) red[s][threadIdx.x >> 5] = w;
  }
  __syncthreads();
  if (threadIdx.x < 8) {
    T w = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) w += red[threadIdx.x][k];
    cellbuf[(int64_t)cell * 8 + threadIdx.x] = w;
  }
}

// rc[free vertex] = sum over its cells of their corner sums (fixed order)
template <typename T>
__global__ void k_sipg_restrict_vertices(SipgDev<T> d, const int *__restrict__ cfree, const T *__restrict__ cellbuf,
                                         T *__restrict__ rc) {
  const int nvx = d.nx + 1, nvy = d.ny + 1, nv = nvx * nvy * (d.nz + 1);
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += gridDim.x * blockDim.x) {
    const int f = cfree[v];
    if (f < 0) continue;
    const int vx = v % nvx, vy = (v / nvx) % nvy, vz = v / (nvx * nvy);
    T s = 0;
    for (int o = 0; o < 8; ++o) {  // the cell at offset (-1 + ox, ...) sees v as its corner (1 - ox, ...)
      const int ox = o & 1, oy = (o >> 1) & 1, oz = o >> 2;
      const int cx = vx - 1 + ox, cy = vy - 1 + oy, cz = vz - 1 + oz;
      if (cx < 0 || cy < 0 || cz < 0 || cx >= d.nx || cy >= d.ny || cz >= d.nz) continue;
      const int corner = (1 - ox) | ((1 - oy) << 1) | ((1 - oz) << 2);
      s += cellbuf[(int64_t)(cx + d.nx * (cy + d.ny * cz)) * 8 + corner];
    }
    rc[f] = s;
  }
}

// x += P xc: each node takes the trilinear interpolant of its cell's vertex values
template <typename T, int N>
__global__ void k_sipg_prolong(SipgDev<T> d, const int *__restrict__ cfree, const T *__restrict__ xc,
                               T *__restrict__ x) {
  constexpr int N3 = N * N * N;
  const int cell = blockIdx.x;
  const int cx = cell % d.nx, cy = (cell / d.nx) % d.ny, cz = cell / (d.nx * d.ny);
  const int nvx = d.nx + 1, nvy = d.ny + 1;
  const T *xi = d.tab + 2 * N * N + 2 * N;
  T cv[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int f = cfree[(cx + (s & 1)) + nvx * ((cy + ((s >> 1) & 1)) + nvy * (cz + (s >> 2)))];
    cv[s] = f >= 0 ? xc[f] : T(0);
  }
  T *xcell = x + (int64_t)cell * N3;
  for (int o = threadIdx.x; o < N3; o += blockDim.x) {
    const int i = o % N, j = (o / N) % N, k = o / (N * N);
    const T hx[2] = {T(0.5) * (T(1) - xi[i]), T(0.5) * (T(1) + xi[i])};
    const T hy[2] = {T(0.5) * (T(1) - xi[j]), T(0.5) * (T(1) + xi[j])};
    const T hz[2] = {T(0.5) * (T(1) - xi[k]), T(0.5) * (T(1) + xi[k])};
    T s = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) s = fma(hx[c & 1] * hy[(c >> 1) & 1] * hz[c >> 2], cv[c], s);
    xcell[o] += s;
  }
}

// n = p + 1 at compile time, 2..SIPG_MAX_N
template <typename F>
bool dispatch_sipg(int n, F &&f) {
  static_assert(SIPG_MAX_N == 11, "dispatch_sipg lists n = 2..11");
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
    default: return false;
  }
}

}  // namespace

template <typename T>
size_t sipg_cell_smem(int n) {
  return sizeof(T) * (2 * (size_t)n * n + 2 * (size_t)n + 4 * (size_t)n * n * n + 24 * (size_t)n * n);
}

template <typename T>
size_t sipg_patch_smem(int n) {
  const size_t m = 2 * (size_t)n;
  return sizeof(T) * (6 * m * m + 3 * m + m * m * (m + 1));
}

template <typename T, typename Tin>
void launch_sipg_op(const SipgDev<T> &d, const Tin *u, T *F, const double *rsub, T *y, cudaStream_t st) {
  const size_t sm = sipg_cell_smem<T>(d.n);
  if (!dispatch_sipg(d.n, [&](auto NC) {
        constexpr int N = decltype(NC)::value;
        k_sipg_faces<T, Tin, N><<<d.ncell, 128, 0, st>>>(d, u, F);
        set_smem(k_sipg_cell<T, Tin, N>, sm);
        k_sipg_cell<T, Tin, N><<<d.ncell, SIPG_THREADS, sm, st>>>(d, u, F, rsub, y);
      }))
    fail(FDM_EINVAL, "SIPG operator: unsupported degree");
}

template <typename T, typename Tin, typename Tout>
void launch_sipg_patch(const SipgDev<T> &d, int color, int nblocks, const int *vlist, const Tin *r, Tout *z,
                       T *zpatch, double omega, cudaStream_t st) {
  if (nblocks <= 0) return;
  const size_t sm = sipg_patch_smem<T>(d.n);
  if (!dispatch_sipg(d.n, [&](auto NC) {
        constexpr int N = decltype(NC)::value;
        set_smem(k_sipg_patch<T, Tin, Tout, N>, sm);
        k_sipg_patch<T, Tin, Tout, N><<<nblocks, SIPG_THREADS, sm, st>>>(d, color, vlist, r, z, zpatch, omega);
      }))
    fail(FDM_EINVAL, "SIPG patch solve: unsupported degree");
}

// z = (addv or 0) + omega * (sum of the star solutions holding each value),
// the stars of all interior vertices solved in one launch into zp[star][(2n)^3]
// (stars lexicographic over the interior vertices, star values x fastest):
// per value the up to 8 stars of its cell's corners in a fixed order
template <typename T, typename Tout>
__global__ void k_sipg_star_gather(SipgDev<T> d, const T *__restrict__ zp, T omega, const T *__restrict__ addv,
                                   Tout *__restrict__ z) {
  const int n = d.n, n3 = n * n * n, m = 2 * n;
  const int64_t total = (int64_t)d.ncell * n3;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int cell = (int)(idx / n3), l = (int)(idx % n3);
    const int cx = cell % d.nx, cy = (cell / d.nx) % d.ny, cz = cell / (d.nx * d.ny);
    const int i = l % n, j = (l / n) % n, k = l / (n * n);
    T acc = 0;
    for (int c = 0; c < 2; ++c)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const int vx = cx + a, vy = cy + b, vz = cz + c;
          if (vx < 1 || vy < 1 || vz < 1 || vx > d.nx - 1 || vy > d.ny - 1 || vz > d.nz - 1) continue;
          const int64_t star = (vx - 1) + (int64_t)(d.nx - 1) * ((vy - 1) + (int64_t)(d.ny - 1) * (vz - 1));
          const int X = (1 - a) * n + i, Y = (1 - b) * n + j, Z = (1 - c) * n + k;
          acc += zp[star * m * m * m + X + m * (Y + m * Z)];
        }
    z[idx] = Tout((addv ? addv[idx] : T(0)) + omega * acc);
  }
}

template <typename T, typename Tout>
void launch_sipg_star_gather(const SipgDev<T> &d, const T *zp, double omega, const T *addv, Tout *z,
                             cudaStream_t st) {
  const int64_t total = (int64_t)d.ncell * d.n * d.n * d.n;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 152 * 16));
  k_sipg_star_gather<T, Tout><<<blocks, 256, 0, st>>>(d, zp, T(omega), addv, z);
}

template <typename T, typename Tin>
void launch_sipg_restrict(const SipgDev<T> &d, const Tin *r, const int *cfree, T *cellbuf, T *rc, cudaStream_t st) {
  if (!dispatch_sipg(d.n, [&](auto NC) {
        constexpr int N = decltype(NC)::value;
        k_sipg_restrict_cells<T, Tin, N><<<d.ncell, 128, 0, st>>>(d, r, cellbuf);
      }))
    fail(FDM_EINVAL, "SIPG restriction: unsupported degree");
  const int nv = (d.nx + 1) * (d.ny + 1) * (d.nz + 1);
  k_sipg_restrict_vertices<T><<<(nv + 255) / 256, 256, 0, st>>>(d, cfree, cellbuf, rc);
}

template <typename T>
void launch_sipg_prolong(const SipgDev<T> &d, const int *cfree, const T *xc, T *x, cudaStream_t st) {
  if (!dispatch_sipg(d.n, [&](auto NC) {
        constexpr int N = decltype(NC)::value;
        k_sipg_prolong<T, N><<<d.ncell, 128, 0, st>>>(d, cfree, xc, x);
      }))
    fail(FDM_EINVAL, "SIPG prolongation: unsupported degree");
}

template size_t sipg_cell_smem<double>(int);
template size_t sipg_cell_smem<float>(int);
template size_t sipg_patch_smem<double>(int);
template size_t sipg_patch_smem<float>(int);
template void launch_sipg_op<double, double>(const SipgDev<double> &, const double *, double *, const double *,
                                             double *, cudaStream_t);
template void launch_sipg_op<float, float>(const SipgDev<float> &, const float *, float *, const double *, float *,
                                           cudaStream_t);
template void launch_sipg_patch<double, double, double>(const SipgDev<double> &, int, int, const int *,
                                                        const double *, double *, double *, double, cudaStream_t);
template void launch_sipg_patch<float, double, float>(const SipgDev<float> &, int, int, const int *, const double *,
                                                      float *, float *, double, cudaStream_t);
template void launch_sipg_patch<float, float, double>(const SipgDev<float> &, int, int, const int *, const float *,
                                                      double *, float *, double, cudaStream_t);
template void launch_sipg_patch<float, double, double>(const SipgDev<float> &, int, int, const int *,
                                                       const double *, double *, float *, double, cudaStream_t);
template void launch_sipg_patch<float, float, float>(const SipgDev<float> &, int, int, const int *, const float *,
                                                     float *, float *, double, cudaStream_t);
template void launch_sipg_star_gather<double, double>(const SipgDev<double> &, const double *, double,
                                                     const double *, double *, cudaStream_t);
template void launch_sipg_star_gather<float, float>(const SipgDev<float> &, const float *, double, const float *,
                                                   float *, cudaStream_t);
template void launch_sipg_star_gather<float, double>(const SipgDev<float> &, const float *, double, const float *,
                                                    double *, cudaStream_t);
template void launch_sipg_restrict<double, double>(const SipgDev<double> &, const double *, const int *, double *,
                                                   double *, cudaStream_t);
template void launch_sipg_restrict<float, float>(const SipgDev<float> &, const float *, const int *, float *, float *,
                                                 cudaStream_t);
template void launch_sipg_prolong<double>(const SipgDev<double> &, const int *, const double *, double *,
                                          cudaStream_t);
template void launch_sipg_prolong<float>(const SipgDev<float> &, const int *, const float *, float *, cudaStream_t);

}  // namespace fdm
