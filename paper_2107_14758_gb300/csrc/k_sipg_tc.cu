// Tensor-core form of the SIPG vertex-star solve (Section 5) at DQ_7: the six
// line passes of the fast-diagonalisation solve
//   u = (S_x (x) S_y (x) S_z) Lambda^{-1} (S_x^T (x) S_y^T (x) S_z^T) g
// over a star's 16^3 values are products of the 256 lines (rows) with one
// 16 x 16 matrix (a 1D eigenvector matrix or its transpose), issued as
// tcgen05.mma kind::tf32 (two 128-row tiles x two K-steps of 8, FP32
// accumulation in tensor memory).  Operands sit in shared memory in the
// K-major canonical layout without swizzle: core matrices of 8 rows x 4 values
// (128 bytes), adjacent along K at 128 bytes, along rows at 512 bytes.  Each
// thread reads one line's 16 accumulators back (tcgen05.ld, its warp's lane
// quarter) and writes them, rounded to TF32, into the next pass's operand in
// that pass's line order; the division by the eigenvalue sums sits between the
// two z passes, the gather from the cells before the first pass and the
// scatter to the cells after the last.  Every wait on the MMA completion is
// bounded; on expiry the CTA records it in the status word, waits once more
// (bounded), frees its tensor memory and returns.
#include <cstdint>

#include "bulk.cuh"
#include "kernels.h"

namespace fdm {
namespace {

constexpr int TC_M = 16;               // values per star line: 2 (p + 1) at p = 7
constexpr int TC_N = 8;                // values per cell line
constexpr int TC_THREADS = 256;        // one line per thread and pass
constexpr int TC_TMEM_COLS = 32;       // two 128 x 16 FP32 accumulator tiles

__device__ __forceinline__ uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// offset (in values) of element (row, k) of a [rows x 16] operand
__device__ __forceinline__ int canon16(int row, int k) {
  return ((row >> 3) * 4 + (k >> 2)) * 32 + (row & 7) * 4 + (k & 3);
}

// shared-memory matrix descriptor: start address, leading (K) byte offset 128,
// stride (row group) byte offset 512, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(512u >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor: D FP32, A and B TF32, both K-major, N = 16, M = 128
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tile] = A[tile] B (K = 16) for both tiles, then one arrive on bar when done
__device__ __forceinline__ void tc_pass_issue(uint32_t tmem, uint32_t a_addr, uint32_t b_addr, uint64_t *bar) {
#pragma unroll
  for (int t = 0; t < 2; ++t)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint64_t ad = smem_desc(a_addr + (uint32_t)(t * 16 * 512 + s * 256));
      const uint64_t bd = smem_desc(b_addr + (uint32_t)(s * 256));
      const uint32_t acc = s;
      asm volatile(
          "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
          " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem + (uint32_t)(t * 16)),
          "l"(ad), "l"(bd), "r"(kIdescTf32), "r"(acc)
          : "memory");
    }
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}

// this thread's line of the last pass: 16 FP32 accumulators of its TMEM lane
__device__ __forceinline__ void tc_load_line(uint32_t tmem, int warp, float (&v)[16]) {
  const uint32_t addr = tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)((warp >> 2) * 16);
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(addr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

}  // namespace

namespace {

// writes line value v (index i of this thread's line of pass `pass`) into the
// operand of the next pass; the line coordinates (a, b) of this thread are
// (tid & 15, tid >> 4) in the pass's line order
__device__ __forceinline__ int next_slot(int pass, int a, int b, int i) {
  switch (pass) {
    case 1: return canon16(i + 16 * b, a);   // x -> y: (X = i, Y = a, Z = b) to row X + 16 Z, k = Y
    case 2: return canon16(a + 16 * i, b);   // y -> z: (X = a, Y = i, Z = b) to row X + 16 Y, k = Z
    case 3: return canon16(a + 16 * b, i);   // z -> z: own row, k = Z
    case 4: return canon16(a + 16 * i, b);   // z -> y: (X = a, Y = b, Z = i) to row X + 16 Z, k = Y
    default: return canon16(i + 16 * b, a);  // y -> x: (X = a, Y = i, Z = b) to row Y + 16 Z, k = X
  }
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(TC_THREADS) k_sipg_patch_tc(SipgDev<float> d, int color, const int *__restrict__ vlist,
                                                              const Tin *__restrict__ r, Tout *__restrict__ z,
                                                              float *__restrict__ zpatch, double omega,
                                                              uint64_t timeout_ns, int *status) {
  constexpr int M = TC_M, M2 = M * M, N = TC_N, N3 = N * N * N;
  __shared__ __align__(128) float A[M * M2];  // the current pass's operand
  __shared__ __align__(128) float B[6][M2];   // S_x^T, S_y^T, S_z^T, S_z, S_y, S_x
  __shared__ float lam[3][M];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tslot;
  __shared__ int sfail;
  const int tid = threadIdx.x, warp = tid >> 5;
  int v[3];
  if (vlist) {
    const int nvx = d.nx + 1, nvy = d.ny + 1, vv = vlist[blockIdx.x];
    v[0] = vv % nvx;
    v[1] = (vv / nvx) % nvy;
    v[2] = vv / (nvx * nvy);
  } else {  // vertices 1..nc-1 of parity (color >> axis) & 1 along each axis
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
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tslot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    bulk::mbar_init(&bar, 1);
    bulk::fence_mbar_init();
    sfail = 0;
  }
  for (int a = 0; a < 3; ++a) {
    const float *Sa = d.S + d.soff[a] + (int64_t)(v[a] - 1) * M2;
    for (int t = tid; t < M2; t += TC_THREADS) {
      const int row = t / M, col = t % M;
      const float s = to_tf32(Sa[t]);
      B[a][canon16(col, row)] = s;      // rows of S_a^T
      B[5 - a][canon16(row, col)] = s;  // rows of S_a
    }
    for (int t = tid; t < M; t += TC_THREADS) lam[a][t] = d.lam[d.loff[a] + (int64_t)(v[a] - 1) * M + t];
  }
  // the first pass's operand: the star's values gathered from its 8 cells, lines along x
  for (int idx = tid; idx < M * M2; idx += TC_THREADS) {
    const int row = idx >> 4, X = idx & 15, Y = row & 15, Z = row >> 4;
    const int cell = (v[0] - 1 + (X >> 3)) + d.nx * ((v[1] - 1 + (Y >> 3)) + d.ny * (v[2] - 1 + (Z >> 3)));
    A[canon16(row, X)] = to_tf32(float(r[(int64_t)cell * N3 + (X & 7) + N * ((Y & 7) + N * (Z & 7))]));
  }
  const int la = tid & 15, lb = tid >> 4;
  float val[16];
  bool failed = false;
  uint32_t fail_par = 0;
  for (int pass = 1; pass <= 6; ++pass) {
    bulk::fence_proxy_async();  // this thread's operand writes, visible to the tensor cores
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    if (tid == 0) tc_pass_issue(tmem, su32(A), su32(B[pass - 1]), &bar);
    if (!bulk::mbar_wait_bounded(&bar, (pass - 1) & 1, timeout_ns)) sfail = 1;
    __syncthreads();
    if (sfail) {
      failed = true;
      fail_par = (uint32_t)((pass - 1) & 1);
      break;
    }
    tc_fence_after();
    tc_load_line(tmem, warp, val);
    if (pass == 3) {  // Lambda^{-1}: lines (X, Y), values along z
#pragma unroll
      for (int i = 0; i < 16; ++i) val[i] /= lam[0][la] + lam[1][lb] + lam[2][i];
    }
    if (pass < 6) {
#pragma unroll
      for (int i = 0; i < 16; ++i) A[next_slot(pass, la, lb, i)] = to_tf32(val[i]);
    }
  }
  if (failed) {
    bulk::mbar_wait_bounded(&bar, fail_par, timeout_ns);  // a second bounded wait for the MMAs in flight
    if (tid == 0) atomicExch(status, 1);
  } else {
    // the last pass: lines (Y, Z), values along x, into the cells (or the patch output)
    const int Y = la, Z = lb;
    if (zpatch) {
      float *zp = zpatch + (int64_t)blockIdx.x * M * M2 + M * (Y + M * Z);
#pragma unroll
      for (int i = 0; i < 16; ++i) zp[i] = val[i];
    } else {
      const float w = float(omega);
#pragma unroll
      for (int ca = 0; ca < 2; ++ca) {
        const int cell = (v[0] - 1 + ca) + d.nx * ((v[1] - 1 + (Y >> 3)) + d.ny * (v[2] - 1 + (Z >> 3)));
        Tout *row = z + (int64_t)cell * N3 + N * ((Y & 7) + N * (Z & 7));
#pragma unroll
        for (int i = 0; i < N; ++i) row[i] = Tout(row[i] + Tout(w * val[ca * N + i]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tslot), "r"(TC_TMEM_COLS) : "memory");
  }
}

}  // namespace

template <typename Tin, typename Tout>
void launch_sipg_patch_tc(const SipgDev<float> &d, int color, int nblocks, const int *vlist, const Tin *r, Tout *z,
                          float *zpatch, double omega, uint64_t timeout_ns, int *status, cudaStream_t st) {
  if (nblocks <= 0) return;
  if (d.n != TC_N) fail(FDM_EINVAL, "SIPG tensor-core star solve: DQ_7 only (16 values per star line)");
  k_sipg_patch_tc<Tin, Tout><<<nblocks, TC_THREADS, 0, st>>>(d, color, vlist, r, z, zpatch, omega, timeout_ns, status);
}

template void launch_sipg_patch_tc<double, float>(const SipgDev<float> &, int, int, const int *, const double *, float *,
                                                  float *, double, uint64_t, int *, cudaStream_t);
template void launch_sipg_patch_tc<float, double>(const SipgDev<float> &, int, int, const int *, const float *, double *,
                                                  float *, double, uint64_t, int *, cudaStream_t);
template void launch_sipg_patch_tc<float, float>(const SipgDev<float> &, int, int, const int *, const float *, float *,
                                                 float *, double, uint64_t, int *, cudaStream_t);
template void launch_sipg_patch_tc<double, double>(const SipgDev<float> &, int, int, const int *, const double *,
                                                   double *, float *, double, uint64_t, int *, cudaStream_t);

}  // namespace fdm
