// Internal declarations of the fdmpc library (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/fdmpc.h"

namespace fdm {

constexpr int PMAX = 31;
constexpr int PANEL = 32;  // tile width of the dense set-up factorisation

// ---------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};
[[noreturn]] void fail(int code, const std::string &msg);
// Device allocation on behalf of a context that has `used` bytes allocated so
// far (updated): fails with FDM_ENOMEM when cudaMalloc fails or when the
// context would exceed the byte limit in the environment variable
// FDM_ALLOC_LIMIT_BYTES (unset, empty or not a number: no limit).  The limit
// caps a context's device memory and lets a caller reach the FDM_ENOMEM
// paths without exhausting a GPU.
void *device_alloc(size_t bytes, size_t &used);
#define FDM_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess)                                                          \
      ::fdm::fail(FDM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
  } while (0)

// ---------------------------------------------------------------- 1D basis
struct Basis1D {
  int p = 0, n = 0;
  std::vector<double> xi, wgll;        // GLL nodes/weights
  std::vector<double> xq, wq;          // Gauss nodes/weights (q = n)
  std::vector<double> A, B;            // reference stiffness/mass, GLL basis (n x n)
  std::vector<double> S, lam;          // interior eigenvectors ((p-1)^2) and eigenvalues
  std::vector<double> T;               // u_gll = T u_fdm (n x n)
  std::vector<double> Af, Bf;          // T^T A T, T^T B T with exact structural zeros
  std::vector<double> Vq, Dq;          // Lagrange values / derivatives at Gauss points (q x n)
  std::vector<double> Ve, lame;        // element modes: V = S^T B by rows (even modes first), eigenvalues
};
void cell_modes(Basis1D &b);  // fills Ve, lame from A, B
Basis1D make_basis(int p);  // throws via fail() on error

// ---------------------------------------------------------------- geometric multigrid (Q1 problem)
// A level on the host: n cells and m = n - 1 free vertices per axis, vertex
// coordinates x[n+1], the 27-point stencil A[27][nf] (offset k = (dx+1) +
// 3 (dy+1) + 9 (dz+1), zero towards Dirichlet vertices) and, once the level has
// been coarsened, the interpolation parameter t[v] of its odd vertices.
struct GmgHostLevel {
  int n[3] = {0, 0, 0}, m[3] = {0, 0, 0}, nf = 0;
  std::vector<double> x[3], t[3], A;
};
// Appends up to max_levels coarser levels to lev (lev[0] given): every other
// vertex per axis while all cell counts are even and >= 4, linear interpolation
// in the vertex coordinates, Galerkin operators P^T A P.
void gmg_coarsen(std::vector<GmgHostLevel> &lev, int max_levels);

// ---------------------------------------------------------------- SIPG star pencils (Section 5)
// l_i'(-1) and l_i'(+1) of the Lagrange basis on the nodes xi (first and last at -1, +1)
void sipg_end_derivatives(const std::vector<double> &xi, std::vector<double> &dm, std::vector<double> &dp);
// the 2n x 2n stiffness A and mass M (row-major, cell c0's values first) of a
// star's 1D two-cell pencil: half-widths h0, h1 of the star's cells and hl, hr
// of the cells beyond (<= 0: the domain boundary), penalty eta
void sipg_star_pencil(int n, const double *A1, const double *B1, const double *dm, const double *dp, double eta,
                      double h0, double h1, double hl, double hr, double *A, double *M);
// A S = M S diag(lam), S^T M S = I (S row-major, column i = eigenvector i);
// fails with FDM_ENOTSPD unless M and A are positive definite
void sym_gen_eig(int m, const double *A, const double *M, double *S, double *lam);

// one bulk copy of the streamed patch solve: kind | first << 8 | last << 9,
// item range [a0, a1) (rows, lines or ELL slices), byte count, element offset
enum { CK_DINV = 0, CK_ELL_F = 1, CK_LINES_F = 2, CK_L21_F = 3, CK_Z_F = 4, CK_Z_B = 5, CK_L21_B = 6,
       CK_LINES_B = 7, CK_ELL_B = 8 };
struct ChunkDev {
  int kind, a0, a1, bytes;
  int64_t off;
};

// ---------------------------------------------------------------- patch classes
// A vertex star spans, per axis, either the full range [p v - (p-1), p v + (p-1)]
// (2p-1 nodes, "full", containing the vertex plane at local p-1) or, at the
// Dirichlet boundary, the interior of one cell (p-1 nodes, "clipped").
// class id = full_x + 2 full_y + 4 full_z.
struct PatchClass {
  int id = 0;
  int full[3] = {0, 0, 0};
  int dim[3] = {0, 0, 0};
  int nd = 0, nI = 0, nG = 0;
  int n0 = 0, n1 = 0, n2 = 0;  // level sizes of the interface ordering
  int nlines = 0;
  std::vector<int> gpos;        // [nG] star-local linear index of interface dof k (factor order)
  std::vector<int> line_start, line_len;  // lines of level 1 (offsets within level 1)
  // level-0 off-diagonal block in ELL form over rows n0..nG-1
  int K0 = 0, nrow0 = 0;        // entries per row, rows = nG - n0
  int ldr0 = 0;                 // ELL slice stride (nrow0 rounded up to 4: 16-byte aligned slices)
  std::vector<int> ell_col;     // [K0 * ldr0] level-0 column or -1
  std::vector<int> c0_ptr, c0_pos;  // per level-0 column: positions e*ldr0 + r in the ELL block
  std::vector<int> r0_ptr, r0_idx;  // per level-0 column: rows (>= n0, ascending) of L
  int ld21 = 0;                 // row stride of L21 (n1 rounded up to 4)
  // Schur-coupling form: S_TB (top rows x levels 0 and 1, S's own pattern) in
  // ELL by top rows, and the positions of each lower column for S_BT x
  bool sc = false;
  int KT = 0, ldT = 0;          // entries per top row, slice stride (n2 rounded up to 4)
  int64_t off_st = 0, nnzST = 0, nnzSC = 0;
  std::vector<int> st_col;      // [KT * ldT] lower column or -1
  std::vector<int> ct_ptr, ct_pos;  // per lower column (n0 + n1): positions e*ldT + t
  std::vector<int> cB_ptr, cB_pos;  // per level-0 column: ELL positions of level-1 rows only
  // value layout of one patch (in elements)
  int64_t off_dinv0 = 0, off_ell = 0, off_lines = 0, off_l21 = 0, off_z = 0, nval = 0;
  std::vector<int> line_off;    // [nlines] offsets of the inverse line blocks
  std::vector<int> zoff;        // [n2+1] row offsets of Z = L_top^{-1} (rows padded to 4)
  int64_t nnzL = 0;             // structurally nonzero entries of L_Gamma
  std::vector<uint8_t> pattern; // [nG*nG] symbolic pattern of L (row-major, lower)
  std::vector<int> ginv;        // [nd] interface index of each star position, -1 if interior
  std::vector<int> line_of;     // [n1] line of each level-1 row
  std::vector<int> gsrc;        // [8*nG] cells containing each interface dof (slot << 16 | local)
};

std::vector<PatchClass> build_classes(int p, bool sc);

// ---------------------------------------------------------------- device views
// Per-class tables on the device (concatenated over classes).
struct ClassDev {
  int nd, nI, nG, n0, n1, n2, nlines, K0, nrow0, ld21;
  int dim[3], full[3];
  int64_t off_dinv0, off_ell, off_lines, off_l21, off_z, nval;
  const int *gpos;       // [nG]
  const int *line_start; // [nlines]
  const int *line_len;   // [nlines]
  const int *line_off;   // [nlines]
  int ldr0;              // ELL slice stride
  const int *ell_col;    // [K0*ldr0]
  const int *c0_ptr;     // [n0+1]
  const int *c0_pos;
  const int *r0_ptr;     // [n0+1]
  const int *r0_idx;
  const int *zoff;       // [n2+1]
  const int *ginv;       // [nd] interface index of a star position, -1 if interior
  const int *line_of;    // [n1] line index of each level-1 row
  const int *gsrc;       // [8*nG] (star cell slot << 16 | cell-local index), -1 terminated
  const ChunkDev *sched32, *sched64;  // streamed-solve schedules (FP32 / FP64 values)
  int nsched32, nsched64;
  // Schur-coupling form
  int sc, KT, ldT;
  int64_t off_st;
  const int *st_col;     // [KT*ldT]
  const int *ct_ptr;     // [n0+n1+1]
  const int *ct_pos;
  const int *cB_ptr;     // [n0+1]
  const int *cB_pos;
};
std::vector<ChunkDev> build_schedule(const struct PatchClass &C, int elem_bytes, int cap_bytes);

}  // namespace fdm
