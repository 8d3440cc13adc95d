// Device-side helpers shared by the fdmpc kernels.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"

namespace fdm {

constexpr int NMAX = 16;  // kernels support p <= 15 (n = p + 1 <= 16)

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 1D tables in precision T for one degree, laid out as consecutive n x n
// row-major blocks: A, B, Af, Bf, T, Vq, Dq, then the n GLL nodes (in the
// eighth block), the element modes V (rows, even modes first) and their n
// eigenvalues.
enum { TAB_A = 0, TAB_B = 1, TAB_AF = 2, TAB_BF = 3, TAB_T = 4, TAB_VQ = 5, TAB_DQ = 6, TAB_XI = 7, TAB_VE = 8,
       TAB_LE = 9 };
__host__ __device__ inline int tab_off(int which, int n) { return which * n * n; }
__host__ __device__ inline int tab_size(int n) { return 9 * n * n + n; }

// Per-patch description on the device.
struct PatchDev {
  int cls;          // class id 0..7
  int v[3];         // vertex coordinates
  int64_t voff;     // offset of the patch's factor values
  int64_t xoff;     // offset of the patch's solution in the star buffer
};

// Geometry of the mesh needed by device code.
struct Grid {
  int p, n, nx, ny, nz;
  int N[3];
  int64_t ndof;
  int ncell;
  // Dirichlet faces: bit 2a for the face at the lower end of axis a, bit 2a+1 for
  // the upper end (63 = the whole boundary, the default); the other boundary
  // faces are traction-free / natural (used by the elasticity context)
  int dmask = 63;
};

// whether grid node (x, y, z) lies on a Dirichlet face
__host__ __device__ inline bool node_dirichlet(const Grid &g, int x, int y, int z) {
  return ((g.dmask & 1) && x == 0) || ((g.dmask & 2) && x == g.N[0] - 1) || ((g.dmask & 4) && y == 0) ||
         ((g.dmask & 8) && y == g.N[1] - 1) || ((g.dmask & 16) && z == 0) || ((g.dmask & 32) && z == g.N[2] - 1);
}

__host__ __device__ inline int64_t gidx(const Grid &g, int x, int y, int z) {
  return x + (int64_t)g.N[0] * (y + (int64_t)g.N[1] * z);
}

// star-local coordinate along one axis -> cell side and cell-local index.
// full axis: side 0 covers t in [0, p-1] (local t+1), side 1 covers t in
// [p-1, 2p-2] (local t-p+1); clipped axis: one cell, local t+1.
__device__ __forceinline__ int star_cell_along(int full, int v, int ncell_axis, int side) {
  if (full) return v - 1 + side;
  return v == 0 ? 0 : ncell_axis - 1;
}

// out[.., i, ..] = sum_m M'[i][m] in[.., m, ..] along `axis` (0 = x, fastest),
// M' = M or M^T; M row-major with `rows` x `cols`; in has extent `cols` and
// out extent `rows` along the axis, and n along the other axes.  When acc is
// set the result is added to out.
template <typename T>
__device__ __forceinline__ void contract(const T *__restrict__ in, T *__restrict__ out, const T *__restrict__ M,
                                         bool transpose, int axis, int n, T scale, bool acc) {
  const int n3 = n * n * n;
  const int stride = axis == 0 ? 1 : (axis == 1 ? n : n * n);
  for (int idx = threadIdx.x; idx < n3; idx += blockDim.x) {
    int i = (idx / stride) % n;
    int base = idx - i * stride;
    T s = 0;
    if (transpose) {
#pragma unroll 4
      for (int m = 0; m < n; ++m) s += M[m * n + i] * in[base + m * stride];
    } else {
#pragma unroll 4
      for (int m = 0; m < n; ++m) s += M[i * n + m] * in[base + m * stride];
    }
    out[idx] = acc ? out[idx] + scale * s : scale * s;
  }
}

}  // namespace fdm
