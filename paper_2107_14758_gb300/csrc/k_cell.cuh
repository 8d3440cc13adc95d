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
//     + mu2 (B (x) A (x) B) u_K + mu3 (A (x) B (x) B) u_K in 7 line passes
//     (FP32), or in the element eigenbasis of (A, B) in 6 passes and a
//     diagonal (FP64); cell-local results, summed over cells by a node gather.
//   restrict (Section 2.4): E_K = (T^T)^{(x)3} (W_K r_K), then the cell's share
//     of the Schur condensation on its face nodes.
//   interp (Sections 2.4-2.6): interface values summed over the 8 stars,
//     interior values by the summed back-substitution, then T^{(x)3}, omega
//     and an owner write.
#pragma once
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

// ------------------------------------------------------------------ launch helpers
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
}  // namespace fdm
