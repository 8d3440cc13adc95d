// The host topology and numeric set-up of a general hexahedral mesh
// (fdm_hexmesh_*), shared by the host set-up (hexmesh.cpp) and the GPU
// context built from it (hexgpu.cu); not part of the C-ABI.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

struct fdm_hexmesh {
  int p = 0, n = 0, nv = 0, nc = 0;
  int64_t nnode = 0;
  std::vector<int32_t> cell_nodes;   // [nc][n^3] global node of each cell-local GLL node
  std::vector<int32_t> cell_fdm;     // [nc][n^3] global FDM function of each cell-local FDM function
  std::vector<int8_t> cell_sign;     // [nc][n^3] its sign
  std::vector<uint8_t> dirichlet;    // [nnode]
  std::vector<int32_t> star_vertex;  // [nstar]
  std::vector<int64_t> star_ptr;     // [nstar + 1] into star_nodes
  std::vector<int32_t> star_nodes;   // per star: cell interiors, faces, edges, vertex
  std::vector<int64_t> pat_ptr;      // [nstar + 1] into pat_rowptr (each star: its size + 1 entries)
  std::vector<int64_t> pat_rowptr;   // per star: CSR row pointers (star-local, from 0)
  std::vector<int64_t> pat_colptr;   // [nstar + 1] into pat_cols
  std::vector<int32_t> pat_cols;     // per star: CSR column indices (star-local positions)
  std::vector<int32_t> star_nint;    // [nstar] cell-interior functions (the first positions)
  std::vector<int32_t> star_class;   // [nstar] sparsity class
  // per class: its interface Schur complement S_G = A_GG - A_GI D^{-1} A_IG factored
  // symbolically: elimination tree and the rows of L (lower, diagonal included)
  std::vector<int32_t> class_star;   // [nclass] first star of the class
  std::vector<int64_t> class_nnzl;   // [nclass] nonzeros of L
  std::vector<int64_t> fill_ptr;     // [nclass + 1] into fill_rowptr (interface size + 1 each)
  std::vector<int64_t> fill_rowptr;  // per class: CSR row pointers of L from 0
  std::vector<int64_t> fill_colptr;  // [nclass + 1] into fill_cols
  std::vector<int32_t> fill_cols;    // per class: columns of each row of L (interface positions, sorted)
  std::vector<int64_t> etree_ptr;    // [nclass + 1] into etree
  std::vector<int32_t> etree;        // per class: parent of each interface column (-1: root)
  // Schur-coupling form per class: the top block T = the last t interface
  // positions; the rows of L_BB (fill of S_BB) and of S_TB (S_G's pattern)
  std::vector<int32_t> sc_t;         // [nclass]
  std::vector<int64_t> sc_ptr;       // [nclass + 1] into sc_rowptr (nB + 1 + t + 1 entries each)
  std::vector<int64_t> sc_rowptr;    // per class: L_BB row pointers from 0, then S_TB row pointers from 0
  std::vector<int64_t> sc_colptr;    // [nclass + 1] into sc_cols
  std::vector<int32_t> sc_cols;      // per class: L_BB columns, then S_TB columns (B positions)
  std::vector<int64_t> sc_values_ptr;  // [nstar + 1] into sc_values
  std::vector<double> sc_values;     // per star: L_BB, S_TB, then the lower triangle of W = S_T^{-1} by rows
  // inverse maps for the apply: per FDM slot its (cell, local index) pairs and
  // its (star, position) pairs, per node its owner (lowest cell, local index)
  std::vector<int64_t> slot_cells_ptr;  // [nnode + 1]
  std::vector<int32_t> slot_cells;      // e * (p+1)^3 + c, by cell
  std::vector<int64_t> slot_stars_ptr;  // [nnode + 1]
  std::vector<int32_t> slot_stars;      // (star, position) pairs, by star
  std::vector<int32_t> node_owner;      // [nnode] e * (p+1)^3 + l
  std::vector<int64_t> node_cells_ptr;  // [nnode + 1]
  std::vector<int32_t> node_cells;      // e * (p+1)^3 + l of every cell-local node of each node, by cell
  // kept for the numeric set-up
  std::vector<int> cells;            // [nc][8]
  std::vector<uint8_t> dvert;        // [nv] Dirichlet vertices (empty: every boundary face is Dirichlet);
                                     // a boundary face is Dirichlet when its 4 vertices are marked
  std::vector<double> Af, Bf, xq, wq;
  // numeric set-up (fdm_hexmesh_factor)
  std::vector<double> mu;            // [nc][3] averaged surrogate coefficients
  std::vector<double> geom;          // [nc][q^3][6] w_q kappa |det J| J^{-1} J^{-T}: xx, yy, zz, xy, xz, yz
  std::vector<int32_t> coarse_of;    // [nv] coarse unknown of each vertex (-1: none)
  std::vector<double> coarse;        // [nco][nco] Q1 Galerkin operator P^T A P
  std::vector<int64_t> diag_ptr;     // [nstar + 1] into diag
  std::vector<double> diag;          // per star: the diagonal interior block D
  std::vector<int64_t> factor_ptr;   // [nstar + 1] into factor
  std::vector<double> factor;        // per star: L of S_G in its class's fill pattern (row by row)
  std::string err;
};
