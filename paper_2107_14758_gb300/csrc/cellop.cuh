// Sum-factorised cell stiffness on curved cells, shared by the operator
// kernels and the surrogate's patch-condition labels.
#pragma once
#include "device.cuh"

namespace fdm {

// Curved cells (Section 2.7): y = sum_q w_q grad_hat phi . Ghat grad_hat u with
// Gauss points q = n per direction; Gw holds w_q * Ghat (xx, yy, zz, xy, xz, yz).
template <typename T>
__device__ void cell_stiffness_gen(const T *sV, const T *sD, const T *__restrict__ Gw, int n, T *u, T *b1, T *b2,
                                   T *b3, T *b4, T *out) {
  const int n3 = n * n * n;
  contract(u, b1, sD, false, 0, n, T(1), false);  // Dx u
  contract(u, b2, sV, false, 0, n, T(1), false);  // Vx u
  __syncthreads();
  contract(b1, b3, sV, false, 1, n, T(1), false);  // Vy Dx u
  contract(b2, b4, sD, false, 1, n, T(1), false);  // Dy Vx u
  __syncthreads();
  contract(b2, b1, sV, false, 1, n, T(1), false);  // Vy Vx u
  __syncthreads();
  contract(b3, u, sV, false, 2, n, T(1), false);    // gx = Vz Vy Dx u
  contract(b4, b2, sV, false, 2, n, T(1), false);   // gy = Vz Dy Vx u
  contract(b1, out, sD, false, 2, n, T(1), false);  // gz = Dz Vy Vx u
  __syncthreads();
  for (int q = threadIdx.x; q < n3; q += blockDim.x) {
    const T *G = Gw + 6 * q;
    T gx = u[q], gy = b2[q], gz = out[q];
    u[q] = G[0] * gx + G[3] * gy + G[4] * gz;
    b2[q] = G[3] * gx + G[1] * gy + G[5] * gz;
    out[q] = G[4] * gx + G[5] * gy + G[2] * gz;
  }
  __syncthreads();
  contract(u, b1, sV, true, 2, n, T(1), false);    // Vz^T fx
  contract(b2, b3, sV, true, 2, n, T(1), false);   // Vz^T fy
  contract(out, b4, sD, true, 2, n, T(1), false);  // Dz^T fz
  __syncthreads();
  contract(b1, u, sV, true, 1, n, T(1), false);    // Vy^T Vz^T fx
  contract(b3, b2, sD, true, 1, n, T(1), false);   // Dy^T Vz^T fy
  __syncthreads();
  contract(b4, b2, sV, true, 1, n, T(1), true);    // + Vy^T Dz^T fz
  __syncthreads();
  contract(u, out, sD, true, 0, n, T(1), false);   // Dx^T (...)
  __syncthreads();
  contract(b2, out, sV, true, 0, n, T(1), true);   // + Vx^T (...)
  __syncthreads();
}

}  // namespace fdm
