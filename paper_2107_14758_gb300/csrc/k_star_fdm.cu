// Star-local fast diagonalisation of the SDC blocks on box cells (Section 4.1
// with traction-free faces): one CTA per (star, block) solves the Kronecker-sum
// star system exactly, A_v^{-1} = (S (x) S (x) S) D^{-1} (S (x) S (x) S)^T, by
// six passes of 1D products over the star's node box in shared memory; a second
// kernel sums the star solutions per node in a fixed order.
#include <algorithm>

#include "device.cuh"
#include "kernels.h"

namespace fdm {

namespace {

constexpr size_t kStarSmemCap = 227 * 1024;  // dynamic shared memory a CTA may use on sm_103

// one pass along an axis: every line of len values (stride `stride`) is
// replaced by S^T line (fwd) or S line, in place (the line is held in registers)
template <typename T, int LB>
__device__ __forceinline__ void star_line_pass(T *buf, const T *S, int len, int nlines, int lb, int sb, int sc,
                                               int stride, bool fwd) {
  for (int l = threadIdx.x; l < nlines; l += blockDim.x) {
    T *q = buf + (l % lb) * sb + (l / lb) * sc;
    T v[LB];
#pragma unroll
    for (int i = 0; i < LB; ++i)
      if (i < len) v[i] = q[i * stride];
    for (int o = 0; o < len; ++o) {
      T acc = T(0);
      if (fwd) {
#pragma unroll
        for (int i = 0; i < LB; ++i)
          if (i < len) acc += S[i * len + o] * v[i];
      } else {
#pragma unroll
        for (int i = 0; i < LB; ++i)
          if (i < len) acc += S[o * len + i] * v[i];
      }
      q[o * stride] = acc;
    }
  }
}

template <typename T, typename Tin, int LB>
__global__ void __launch_bounds__(512) k_star_fdm_solve(StarFdmDev<T> d, const Tin *__restrict__ r,
                                                        T *__restrict__ X) {
  extern __shared__ unsigned char smem_[];
  T *buf = reinterpret_cast<T *>(smem_);
  const Grid &g = d.g;
  const int s = blockIdx.x, j = blockIdx.y;
  const int v = d.svert[s];
  const int nvx = g.nx + 1, nvy = g.ny + 1;
  const int vc[3] = {v % nvx, (v / nvx) % nvy, v / (nvx * nvy)};
  int lo[3], len[3];
  const T *src[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = d.ax[a].lo[vc[a]];
    len[a] = d.ax[a].len[vc[a]];
    src[a] = d.tab + d.ax[a].soff[vc[a]];
  }
  const int lx = len[0], ly = len[1], lz = len[2], nb = lx * ly * lz;
  T *S[3], *lam[3];
  T *ptr = buf + nb;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    S[a] = ptr;
    lam[a] = ptr + len[a] * len[a];
    ptr += len[a] * len[a] + len[a];
    for (int i = threadIdx.x; i < len[a] * len[a] + len[a]; i += blockDim.x) S[a][i] = src[a][i];
  }
  const Tin *rj = r + (int64_t)j * g.ndof;
  for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
    const int i = idx % lx, jj = (idx / lx) % ly, k = idx / (lx * ly);
    buf[idx] = T(rj[gidx(g, lo[0] + i, lo[1] + jj, lo[2] + k)]);
  }
  __syncthreads();
  star_line_pass<T, LB>(buf, S[0], lx, ly * lz, ly, lx, lx * ly, 1, true);
  __syncthreads();
  star_line_pass<T, LB>(buf, S[1], ly, lx * lz, lx, 1, lx * ly, lx, true);
  __syncthreads();
  star_line_pass<T, LB>(buf, S[2], lz, lx * ly, lx, 1, lx, lx * ly, true);
  __syncthreads();
  const T c0 = T(d.c[j][0]), c1 = T(d.c[j][1]), c2 = T(d.c[j][2]);
  for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) {
    const int i = idx % lx, jj = (idx / lx) % ly, k = idx / (lx * ly);
    buf[idx] = buf[idx] / (c0 * lam[0][i] + c1 * lam[1][jj] + c2 * lam[2][k]);
  }
  __syncthreads();
  star_line_pass<T, LB>(buf, S[2], lz, lx * ly, lx, 1, lx, lx * ly, false);
  __syncthreads();
  star_line_pass<T, LB>(buf, S[1], ly, lx * lz, lx, 1, lx * ly, lx, false);
  __syncthreads();
  star_line_pass<T, LB>(buf, S[0], lx, ly * lz, ly, lx, lx * ly, 1, false);
  __syncthreads();
  T *out = X + (int64_t)j * d.xstride + d.off[s];
  for (int idx = threadIdx.x; idx < nb; idx += blockDim.x) out[idx] = buf[idx];
}

template <typename T, typename Tout>
__global__ void __launch_bounds__(256) k_star_fdm_gather(StarFdmDev<T> d, const T *__restrict__ X, T omega,
                                                         const T *__restrict__ addv, Tout *__restrict__ z) {
  const Grid &g = d.g;
  const int j = blockIdx.y, p = g.p;
  const int nvx = g.nx + 1, nvy = g.ny + 1;
  const T *Xj = X + (int64_t)j * d.xstride;
  for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < g.ndof;
       id += (int64_t)gridDim.x * blockDim.x) {
    const int xyz[3] = {(int)(id % g.N[0]), (int)((id / g.N[0]) % g.N[1]), (int)(id / ((int64_t)g.N[0] * g.N[1]))};
    const int64_t o = (int64_t)j * g.ndof + id;
    if (node_dirichlet(g, xyz[0], xyz[1], xyz[2])) {
      z[o] = Tout(0);
      continue;
    }
    // the stars holding the node along each axis: its vertex's, or those of
    // the two ends of its element
    int c0[3], nc[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      c0[a] = xyz[a] / p;
      nc[a] = xyz[a] % p == 0 ? 1 : 2;
    }
    T sum = T(0);
    for (int cz = 0; cz < nc[2]; ++cz) {
      const int vz = c0[2] + cz, lz = d.ax[2].len[vz];
      if (lz == 0) continue;
      for (int cy = 0; cy < nc[1]; ++cy) {
        const int vy = c0[1] + cy, ly = d.ax[1].len[vy];
        if (ly == 0) continue;
        for (int cx = 0; cx < nc[0]; ++cx) {
          const int vx = c0[0] + cx, lx = d.ax[0].len[vx];
          if (lx == 0) continue;
          const int sidx = d.vstar[vx + nvx * (vy + nvy * vz)];
          if (sidx < 0) continue;
          const int pos = (xyz[0] - d.ax[0].lo[vx]) + lx * ((xyz[1] - d.ax[1].lo[vy]) + ly * (xyz[2] - d.ax[2].lo[vz]));
          sum += Xj[d.off[sidx] + pos];
        }
      }
    }
    z[o] = addv ? Tout(addv[o] + omega * sum) : Tout(omega * sum);
  }
}

int star_threads(int maxlen) {
  const int lines = maxlen * maxlen, rounds = (lines + 511) / 512;
  const int t = (lines + rounds - 1) / rounds;
  return std::max(32, (t + 31) / 32 * 32);
}

template <typename T, typename Tin, int LB>
void star_solve_lb(const StarFdmDev<T> &d, const Tin *r, T *X, int ncomp, cudaStream_t st) {
  const size_t sm = star_fdm_smem(d.maxlen, sizeof(T));
  FDM_CUDA(cudaFuncSetAttribute(k_star_fdm_solve<T, Tin, LB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kStarSmemCap));
  k_star_fdm_solve<T, Tin, LB><<<dim3(d.nstar, ncomp), star_threads(d.maxlen), sm, st>>>(d, r, X);
}

}  // namespace

size_t star_fdm_smem(int maxlen, size_t elem) {
  return elem * ((size_t)maxlen * maxlen * maxlen + 3 * ((size_t)maxlen * maxlen + maxlen));
}

template <typename T, typename Tin>
void launch_star_fdm_solve(const StarFdmDev<T> &d, const Tin *r, T *X, int ncomp, cudaStream_t st) {
  if (d.nstar == 0 || ncomp == 0) return;
  if (d.maxlen > STAR_FDM_MAX_LEN || star_fdm_smem(d.maxlen, sizeof(T)) > kStarSmemCap)
    fail(FDM_EINVAL, "star FDM: star larger than the shared memory of one CTA");
  if (d.maxlen <= 4) star_solve_lb<T, Tin, 4>(d, r, X, ncomp, st);
  else if (d.maxlen <= 8) star_solve_lb<T, Tin, 8>(d, r, X, ncomp, st);
  else if (d.maxlen <= 16) star_solve_lb<T, Tin, 16>(d, r, X, ncomp, st);
  else star_solve_lb<T, Tin, 32>(d, r, X, ncomp, st);
}

template <typename T, typename Tout>
void launch_star_fdm_gather(const StarFdmDev<T> &d, const T *X, double omega, const T *addv, Tout *z, int ncomp,
                            cudaStream_t st) {
  if (ncomp == 0) return;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((d.g.ndof + 255) / 256, 152 * 8));
  k_star_fdm_gather<T, Tout><<<dim3(blocks, ncomp), 256, 0, st>>>(d, X, T(omega), addv, z);
}

template void launch_star_fdm_solve<double, double>(const StarFdmDev<double> &, const double *, double *, int,
                                                    cudaStream_t);
template void launch_star_fdm_solve<float, double>(const StarFdmDev<float> &, const double *, float *, int,
                                                   cudaStream_t);
template void launch_star_fdm_solve<float, float>(const StarFdmDev<float> &, const float *, float *, int,
                                                  cudaStream_t);
template void launch_star_fdm_gather<double, double>(const StarFdmDev<double> &, const double *, double,
                                                     const double *, double *, int, cudaStream_t);
template void launch_star_fdm_gather<float, float>(const StarFdmDev<float> &, const float *, double, const float *,
                                                   float *, int, cudaStream_t);
template void launch_star_fdm_gather<float, double>(const StarFdmDev<float> &, const float *, double, const float *,
                                                    double *, int, cudaStream_t);

}  // namespace fdm
