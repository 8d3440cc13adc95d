// Vertex-star patch solve on a thread-block cluster (interior stars, the
// classes with a dense top level: n1 > 0 and n2 > 0).
//
// A cluster of CS CTAs shares one patch.  CTA k bulk-copies (cp.async.bulk)
// a contiguous block of rows [r0, r1) of the patch's L21 block into its shared
// memory at the start and keeps it for both triangular solves, so L21 leaves
// DRAM once.  Every CTA gathers the condensed residual and runs the small
// level-0 and level-1 forward phases itself (identical work, no exchange).
// Then, with values exchanged through distributed shared memory:
//   g2[r] -= L21[r] y1            own rows, from shared memory
//   g2 gathered from the peers                                  (cluster sync)
//   y2[r] = Z[r] g2               rows r = k (mod CS), Z streamed from global
//   px2 = sum over those rows of Z[r]^T y2[r]   (partial of x2 = Z^T y2)
//   x2[r] = sum over the CTAs of px2[r]  own L21 rows          (cluster sync)
//   pt1 = sum over own rows of L21[r]^T x2[r] (partial of L21^T x2)
//   CTA 0: t1 = sum of the pt1, x2 from the peers, then the level-1 and
//          level-0 backward phases
// Sums over CTAs run in rank order (deterministic).  The wait for the bulk
// copy is bounded by %globaltimer; on time-out the status word is set and the
// CTA still passes every cluster barrier (all CTAs of a cluster run the same
// barriers), after a second bounded wait for its copy.
#include <cooperative_groups.h>

#include "bulk.cuh"
#include "device.cuh"
#include "kernels.h"

namespace cg = cooperative_groups;

namespace fdm {
namespace {

template <typename T>
struct V4c { T x, y, z, w; };
__device__ __forceinline__ V4c<float> ld4c(const float *p) {
  float4 v = *reinterpret_cast<const float4 *>(p);
  return {v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ V4c<double> ld4c(const double *p) {
  double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
  return {a.x, a.y, b.x, b.y};
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT, 1) k_patch_cluster(ClusterArgs<T> a) {
  extern __shared__ __align__(128) unsigned char smem_[];
  constexpr int NW = NT / 32, RB = 4;
  cg::cluster_group cl = cg::this_cluster();
  const int CS = a.cs;
  const int rank = (int)cl.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int pidx = blockIdx.x / CS;
  const PatchDev P = a.patches[a.order[pidx]];
  const ClassDev &C = a.cls[P.cls];
  const Grid &g = a.g;
  const int n = g.n, n3 = n * n * n;
  const int nG = C.nG, n0 = C.n0, n1 = C.n1, n2 = C.n2, base = n0 + n1, ld21 = C.ld21;
  const int rows = (n2 + CS - 1) / CS;
  const int r0 = min(n2, rank * rows), r1 = min(n2, r0 + rows);
  T *Ls = reinterpret_cast<T *>(smem_);           // a.rows_cap * a.ld_cap
  T *gv = Ls + (size_t)a.rows_cap * a.ld_cap;      // nG
  T *yv = gv + a.maxG, *xv = yv + a.maxG;          // nG each
  T *px2 = xv + a.maxG;                            // n2 (rounded up to 4)
  T *pt1 = px2 + a.n2_cap;                         // ld21
  T *tmp = pt1 + a.ld_cap;                         // a.tmpcap
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int sCell[8];
  __shared__ int sFail;
  const T *Lv = a.L + P.voff;

  if (tid == 0) {
    bulk::mbar_init(&bar[0], 1);
    bulk::mbar_init(&bar[1], 1);
    bulk::fence_mbar_init();
    sFail = 0;
    const uint32_t bytes = (uint32_t)((int64_t)(r1 - r0) * ld21 * (int64_t)sizeof(T));
    bulk::mbar_arrive_expect_tx(&bar[0], bytes);
    const char *src = reinterpret_cast<const char *>(Lv + C.off_l21 + (int64_t)r0 * ld21);
    char *dst = reinterpret_cast<char *>(Ls);
    for (uint32_t off = 0; off < bytes; off += 32768)
      bulk::bulk_g2s(dst + off, src + off, bytes - off < 32768 ? bytes - off : 32768, &bar[0]);
  }
  for (int i = tid; i < 3 * a.maxG + a.n2_cap + a.ld_cap + a.tmpcap; i += NT) gv[i] = T(0);
  if (tid < 8) {
    const int s[3] = {tid & 1, (tid >> 1) & 1, tid >> 2};
    const int ncl[3] = {g.nx, g.ny, g.nz};
    int cc[3];
    bool ok = true;
    for (int ax = 0; ax < 3; ++ax) {
      if (!C.full[ax] && s[ax]) ok = false;
      cc[ax] = star_cell_along(C.full[ax], P.v[ax], ncl[ax], s[ax]);
    }
    sCell[tid] = ok ? cc[0] + g.nx * (cc[1] + g.ny * cc[2]) : -1;
  }
  __syncthreads();
  // ---- gather the condensed residual on the interface (fixed cell order)
  for (int k = tid; k < nG; k += NT) {
    const int *src = C.gsrc + 8 * k;
    T r = 0;
    for (int e = 0; e < 8; ++e) {
      const int code = src[e];
      if (code < 0) break;
      r += a.E[(int64_t)sCell[code >> 16] * n3 + (code & 0xffff)];
    }
    gv[k] = r;
  }
  __syncthreads();
  // ---- level 0 and level 1 forward (every CTA)
  const T *dinv0 = Lv + C.off_dinv0;
  const T *ell = Lv + C.off_ell;
  for (int j = tid; j < n0; j += NT) yv[j] = gv[j] * dinv0[j];
  __syncthreads();
  for (int r = tid; r < C.nrow0; r += NT) {
    T acc = 0;
#pragma unroll 4
    for (int e = 0; e < C.K0; ++e) {
      const int col = C.ell_col[e * C.ldr0 + r];
      if (col >= 0) acc += ell[e * C.ldr0 + r] * yv[col];
    }
    gv[n0 + r] -= acc;
  }
  __syncthreads();
  for (int i = tid; i < n1; i += NT) {
    const int b = C.line_of[i], s0 = C.line_start[b], w = C.line_len[b];
    const T *Li = Lv + C.off_lines + C.line_off[b] + (int64_t)(i - s0) * w;
    T acc = 0;
    for (int cc = 0; cc <= i - s0; ++cc) acc += Li[cc] * gv[n0 + s0 + cc];
    yv[n0 + i] = acc;
  }
  // ---- own L21 rows have arrived?
  bool ok = true;
  if (a.inject_stall) ok = bulk::mbar_wait_bounded(&bar[1], 0, a.timeout_ns);  // test hook: never completes
  ok = ok && bulk::mbar_wait_bounded(&bar[0], 0, a.timeout_ns);
  if (!ok) sFail = 1;
  __syncthreads();
  if (sFail) {
    bulk::mbar_wait_bounded(&bar[0], 0, a.timeout_ns);  // let the copy finish before shared memory is reused
    if (tid == 0) atomicExch(a.status, 1);
  }
  // ---- g2[r] -= L21[r] y1 for the own rows (shared memory), RB rows per warp
  {
    const int ng = ld21 / 4;
    for (int q0 = r0 + warp * RB; q0 < r1; q0 += NW * RB) {
      T acc[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) acc[u] = 0;
      for (int q4 = lane; q4 < ng; q4 += 32) {
        const T *yy = yv + n0 + 4 * q4;  // padding columns of L21 are zero, yv is finite there
#pragma unroll
        for (int u = 0; u < RB; ++u)
          if (q0 + u < r1) {
            const V4c<T> v = ld4c(Ls + (int64_t)(q0 + u - r0) * ld21 + 4 * q4);
            acc[u] += v.x * yy[0] + v.y * yy[1] + v.z * yy[2] + v.w * yy[3];
          }
      }
#pragma unroll
      for (int u = 0; u < RB; ++u) acc[u] = warp_sum(acc[u]);
      if (lane == 0)
        for (int u = 0; u < RB; ++u)
          if (q0 + u < r1) gv[base + q0 + u] -= acc[u];
    }
  }
  cl.sync();
  // ---- the other CTAs' rows of g2
  for (int r = tid; r < n2; r += NT) {
    const int owner = r / rows;
    if (owner != rank) gv[base + r] = cl.map_shared_rank(gv, owner)[base + r];
  }
  __syncthreads();
  // ---- y2 = Z g2 for the rows r = rank (mod CS); Z streamed from global memory
  const T *Z = Lv + C.off_z;
  {
    const int nmine = (n2 - rank + CS - 1) / CS;  // rows rank, rank + CS, ...
    for (int m0 = warp * RB; m0 < nmine; m0 += NW * RB) {
      T acc[RB];
      int ngu[RB];
      const T *row[RB];
#pragma unroll
      for (int u = 0; u < RB; ++u) {
        acc[u] = 0;
        const int r = m0 + u < nmine ? rank + (m0 + u) * CS : rank;
        row[u] = Z + C.zoff[r];
        ngu[u] = m0 + u < nmine ? (C.zoff[r + 1] - C.zoff[r]) / 4 : 0;
      }
      int ngmax = 0;
#pragma unroll
      for (int u = 0; u < RB; ++u) ngmax = ngu[u] > ngmax ? ngu[u] : ngmax;
      for (int q4 = lane; q4 < ngmax; q4 += 32) {
        const T *gg = gv + base + 4 * q4;
#pragma unroll
        for (int u = 0; u < RB; ++u)
          if (q4 < ngu[u]) {
            const V4c<T> v = ld4c(row[u] + 4 * q4);
            acc[u] += v.x * gg[0] + v.y * gg[1] + v.z * gg[2] + v.w * gg[3];
          }
      }
#pragma unroll
      for (int u = 0; u < RB; ++u) acc[u] = warp_sum(acc[u]);
      if (lane == 0)
        for (int u = 0; u < RB; ++u)
          if (m0 + u < nmine) yv[base + rank + (m0 + u) * CS] = acc[u];
    }
  }
  __syncthreads();
  // ---- px2 = sum over the own Z rows of Z[r]^T y2[r]: threads own 4-column groups,
  //      rows split into slices, partial sums in tmp, then summed in slice order
  {
    const int nmine = (n2 - rank + CS - 1) / CS;
    const int ngz = (n2 + 3) / 4, ldz = 4 * ngz;
    const int slices = max(1, min(NT / ngz, a.tmpcap / ldz));
    const int gq = tid % ngz, sl = tid / ngz;
    if (sl < slices && tid < slices * ngz) {
      T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (int m = sl; m < nmine; m += slices) {
        const int r = rank + m * CS;
        if (4 * gq > r) continue;  // Z[r][c] = 0 for c > r
        const V4c<T> v = ld4c(Z + C.zoff[r] + 4 * gq);
        const T yr = yv[base + r];
        s0 += v.x * yr; s1 += v.y * yr; s2 += v.z * yr; s3 += v.w * yr;
      }
      T *dst = tmp + (int64_t)sl * ldz + 4 * gq;
      dst[0] = s0; dst[1] = s1; dst[2] = s2; dst[3] = s3;
    }
    __syncthreads();
    for (int c = tid; c < n2; c += NT) {
      T s = 0;
      for (int q = 0; q < slices; ++q) s += tmp[q * ldz + c];
      px2[c] = s;
    }
  }
  cl.sync();
  // ---- x2 on the own L21 rows: the sum of the CTAs' partials, in rank order
  for (int r = r0 + tid; r < r1; r += NT) {
    T s = 0;
    for (int j = 0; j < CS; ++j) s += cl.map_shared_rank(px2, j)[r];
    xv[base + r] = s;
  }
  __syncthreads();
  // ---- pt1 = sum over the own rows of L21[r]^T x2[r] (shared memory)
  {
    const int ng = ld21 / 4;
    const int slices = max(1, min(NT / ng, a.tmpcap / ld21));
    const int gq = tid % ng, sl = tid / ng;
    if (sl < slices && tid < slices * ng) {
      T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      for (int r = r0 + sl; r < r1; r += slices) {
        const V4c<T> v = ld4c(Ls + (int64_t)(r - r0) * ld21 + 4 * gq);
        const T xr = xv[base + r];
        s0 += v.x * xr; s1 += v.y * xr; s2 += v.z * xr; s3 += v.w * xr;
      }
      T *dst = tmp + (int64_t)sl * ld21 + 4 * gq;
      dst[0] = s0; dst[1] = s1; dst[2] = s2; dst[3] = s3;
    }
    __syncthreads();
    for (int c = tid; c < n1; c += NT) {
      T s = 0;
      for (int q = 0; q < slices; ++q) s += tmp[q * ld21 + c];
      pt1[c] = s;
    }
  }
  T *X = a.X + P.xoff;
  for (int r = r0 + tid; r < r1; r += NT) X[base + r] = xv[base + r];
  cl.sync();
  if (rank == 0) {
    // t1 = L21^T x2 (the CTAs' partials in rank order), then the backward level-1 and level-0 phases
    for (int c = tid; c < n1; c += NT) {
      T s = 0;
      for (int j = 0; j < CS; ++j) s += cl.map_shared_rank(pt1, j)[c];
      tmp[c] = s;
    }
    // the level-0 backward phase reads x at every interface row: the other CTAs' x2
    for (int r = tid; r < n2; r += NT) {
      const int owner = r / rows;
      if (owner != 0) xv[base + r] = cl.map_shared_rank(xv, owner)[base + r];
    }
    __syncthreads();
    for (int i = tid; i < n1; i += NT) {
      const int b = C.line_of[i], s0 = C.line_start[b], w = C.line_len[b];
      const T *Lb = Lv + C.off_lines + C.line_off[b];
      T s = 0;
      for (int cc = i - s0; cc < w; ++cc) s += Lb[cc * w + (i - s0)] * (yv[n0 + s0 + cc] - tmp[s0 + cc]);
      xv[n0 + i] = s;
    }
    __syncthreads();
    for (int j = tid; j < n0; j += NT) {
      T s = yv[j];
      for (int q = C.c0_ptr[j]; q < C.c0_ptr[j + 1]; ++q) {
        const int pos = C.c0_pos[q];
        s -= ell[pos] * xv[n0 + pos % C.ldr0];
      }
      xv[j] = s * dinv0[j];
    }
    __syncthreads();
    for (int k = tid; k < base; k += NT) X[k] = xv[k];
  }
  cl.sync();  // the peers keep their shared memory until CTA 0 has read it
}

}  // namespace

template <typename T>
size_t patch_cluster_smem(const ClusterArgs<T> &a) {
  return sizeof(T) * ((size_t)a.rows_cap * a.ld_cap + 3 * (size_t)a.maxG + a.n2_cap + a.ld_cap + a.tmpcap);
}

template <typename T>
int patch_cluster_fits(const ClusterArgs<T> &a, int threads) {
  const size_t sm = patch_cluster_smem(a);
  if (sm > 224 * 1024) return 0;
  auto kern = threads >= 512 ? k_patch_cluster<T, 512> : k_patch_cluster<T, 256>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess ||
      cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.cs * 4);
  cfg.blockDim = dim3(threads >= 512 ? 512 : 256);
  cfg.dynamicSmemBytes = sm;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return nclusters;
}

template <typename T>
void launch_patch_cluster(const ClusterArgs<T> &a, int threads, cudaStream_t st) {
  if (a.npatch <= 0) return;
  const size_t sm = patch_cluster_smem(a);
  auto kern = threads >= 512 ? k_patch_cluster<T, 512> : k_patch_cluster<T, 256>;
  FDM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
  FDM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.npatch * a.cs);
  cfg.blockDim = dim3(threads >= 512 ? 512 : 256);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = a.cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  FDM_CUDA(cudaLaunchKernelEx(&cfg, kern, a));
}

template size_t patch_cluster_smem<float>(const ClusterArgs<float> &);
template size_t patch_cluster_smem<double>(const ClusterArgs<double> &);
template int patch_cluster_fits<float>(const ClusterArgs<float> &, int);
template int patch_cluster_fits<double>(const ClusterArgs<double> &, int);
template void launch_patch_cluster<float>(const ClusterArgs<float> &, int, cudaStream_t);
template void launch_patch_cluster<double>(const ClusterArgs<double> &, int, cudaStream_t);

}  // namespace fdm
