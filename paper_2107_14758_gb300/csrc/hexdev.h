// Device view of a general hexahedral mesh (fdm_hexmesh after its numeric
// set-up) for the GPU apply of hexgpu.cu: the cell maps, the inverse maps of
// the deterministic sums, the geometry factors, the stars' Schur-coupling
// factors with level schedules of their sparse triangular solves, and the Q1
// coarse space.  Not part of the C-ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fdm {

// per star: class, interior count, interface size, offsets of its node list
// (interiors then interface, in factor order), its values and its solution
struct HexStarDev {
  int cls, ni, nG;
  int64_t nodes_off, voff, xoff;
};

// per class: the Schur-coupling split (B = first nB interface positions,
// T = last t) and int offsets into the concatenated class tables `ct`:
//   lev_f[nlf+1], rows_f[nB]:   forward levels of L_BB (rows by level)
//   lptr[nB+1], lcol, lpos:     the strictly lower entries of each row of L_BB
//                               (column, value position); ldiag[nB] the diagonal's
//   lev_b[nlb+1], rows_b[nB]:   backward levels of L_BB^T
//   tptr[nB+1], trow, tpos:     the entries below the diagonal of each column
//   stptr[t+1], stcol:          S_TB rows (columns in B); values in row order
//   sbtptr[nB+1], sbtrow, sbtpos: per B column its S_TB entries (top row, value position)
// value positions are relative to the star's value block: L_BB (nnzL values in
// row order), S_TB from off_st, the lower triangle of W by rows from off_w.
struct HexClassDev {
  int nB, t, nlf, nlb;
  int lev_f, rows_f, lptr, lcol, lpos, ldiag, lev_b, rows_b, tptr, trow, tpos, stptr, stcol, sbtptr, sbtrow,
      sbtpos;
  int off_st, off_w;
  int zoff;  // dense form: int offset of the row offsets [nG + 1] of the lower triangle of S_G^{-1}
};

template <typename T>
struct HexDev {
  int p = 0, n = 0, nc = 0, nstar = 0, nco = 0;
  int64_t nnode = 0;
  const int *cell_nodes = nullptr;   // [nc][n^3]
  const int *cell_fdm = nullptr;     // [nc][n^3]
  const int8_t *cell_sign = nullptr; // [nc][n^3]
  const uint8_t *dirichlet = nullptr;  // [nnode]
  const T *inv_mult = nullptr;       // [nnode] 1 / number of cells holding the node
  const T *mu = nullptr;             // [nc][3] averaged surrogate
  const T *tab = nullptr;            // T, Af, Bf, Vq, Dq (n x n each), xi (n)
  const T *geom = nullptr;           // [nc][n^3][6] w kappa |det J| J^-1 J^-T at the Gauss points
  const int *cell_m = nullptr;       // [nc] stars holding the cell's interior functions
  const int64_t *slot_cells_ptr = nullptr;
  const int *slot_cells = nullptr;   // e n^3 + c, by cell
  const int64_t *slot_stars_ptr = nullptr;
  const int *slot_stars = nullptr;   // (star, position) pairs, by star
  const int *node_owner = nullptr;   // [nnode] e n^3 + l
  const int64_t *node_cells_ptr = nullptr;
  const int *node_cells = nullptr;   // e n^3 + l, by cell
  const HexStarDev *stars = nullptr;
  const HexClassDev *classes = nullptr;
  const int *ct = nullptr;           // concatenated class tables
  const int *star_nodes = nullptr;
  const T *vals = nullptr;           // Schur-coupling values of every star
  const int *cells8 = nullptr;       // [nc][8] corner vertices
  const int *coarse_of = nullptr;    // [nv] coarse unknown of a vertex or -1
  const int64_t *vcell_ptr = nullptr;  // [nco + 1] cells of each coarse vertex (by cell)
  const int *vcell = nullptr;        // e * 8 + corner
  const int *coarse_vertex = nullptr;  // [nco]
  const T *Acinv = nullptr;          // [nco][nco] dense inverse of the Q1 Galerkin operator
};

enum { HTAB_T = 0, HTAB_AF = 1, HTAB_BF = 2, HTAB_VQ = 3, HTAB_DQ = 4, HTAB_XI = 5 };
__host__ __device__ inline int htab(int which, int n) { return which * n * n; }

// one relaxation sweep's pieces and the operator (hexgpu.cu kernels)
template <typename T, typename Tin>
void launch_hex_restrict(const HexDev<T> &d, const Tin *r, T *CE, cudaStream_t st);
template <typename T>
void launch_hex_assemble(const HexDev<T> &d, const T *CE, T *rc, cudaStream_t st);
template <typename T>
void launch_hex_star_solve(const HexDev<T> &d, const T *rc, T *X, int maxG, cudaStream_t st);
// the dense form: x_G = S_G^{-1} g_G with the lower triangle of S_G^{-1} by rows
// (row r at zoff[r], padded to a multiple of 4 values); list: the star indices
// of three size bins (interfaces up to 256, 512, 1024 values) one after the
// other, count and the largest interface of each bin; bins: mask of the bins
// to launch (bit b = bin b), the largest first
template <typename T>
void launch_hex_star_dense(const HexDev<T> &d, const T *rc, T *X, const int *list, const int count[3],
                           const int maxg[3], unsigned bins, cudaStream_t st);
template <typename T>
void launch_hex_slot_stars(const HexDev<T> &d, const T *X, T *zf, cudaStream_t st);
template <typename T, typename Tout>
void launch_hex_interp(const HexDev<T> &d, const T *CE, const T *zf, double omega, Tout *z, cudaStream_t st);
template <typename T, typename Tin>
void launch_hex_op_cells(const HexDev<T> &d, const Tin *u, T *Y, cudaStream_t st);
template <typename T, typename Tout>
void launch_hex_gather(const HexDev<T> &d, const T *Y, const Tout *rsub, Tout *y, cudaStream_t st);
// rc = P^T r (Cc: [nc][8] per-cell corner sums, scratch)
template <typename T>
void launch_hex_coarse_restrict(const HexDev<T> &d, const T *r, T *Cc, T *rc, cudaStream_t st);
template <typename T>
void launch_hex_coarse_prolong(const HexDev<T> &d, const T *xc, T *x, cudaStream_t st);  // x += P xc

}  // namespace fdm
