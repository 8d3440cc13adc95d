// Host set-up of the vertex-star relaxation on a conforming hexahedral mesh
// of any structure (Sections 2.4-2.7 applied to general meshes).  Topology
// (fdm_hexmesh_create): the Q_p node numbering shared by neighbouring cells of
// any orientation, the Dirichlet nodes, the signed map from each cell's
// tensor-product FDM functions to the global FDM functions, the vertex stars
// in canonical order (cell interiors first, then the interface entities in
// minimum-degree order), their separable surrogate patterns, sparsity classes
// with the symbolic factorisations of the interface Schur complement (L form
// and Schur-coupling form), and the inverse maps of the apply.  Numeric set-up
// (fdm_hexmesh_factor): the averaged surrogate and stiffness factors from the
// trilinear geometry, the Q1 coarse operator, and every star's interior pivots
// and interface factors.  Host memory only: no CUDA call.
//
// Numbering.  Entities: the mesh vertices used by cells, the edges (vertex
// pairs) and faces (vertex quadruples) of the cells, and the cells.  Nodes
// (and, slot for slot, FDM functions) are numbered vertex nodes first (one per
// used vertex, by vertex id), then edges ((p-1) each, by first appearance),
// faces ((p-1)^2 each) and cell interiors ((p-1)^3 each, cell-local
// lexicographic order).  An edge's nodes run from its lower-id vertex to the
// higher; a face's nodes are indexed (s, t) in its canonical frame: origin at
// its lowest-id corner, s towards the lower-id of the two neighbouring corners,
// t towards the other.  The GLL points are symmetric, so a reversed axis maps
// node index i to p - i.  The 1D interior FDM functions s_m are even or odd
// under reflection (the pencil is centrosymmetric): a reversed axis keeps the
// eigen-index m and multiplies by the parity of s_m.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

#include "hexmesh_host.h"

namespace {

// Symbolic Cholesky of a symmetric pattern given by its rows (diagonal
// included): column j of L holds the later rows of column j of S and of the
// columns of L whose elimination-tree parent is j.  Returns the rows of L
// (lower, diagonal included) and the parents.
void symbolic_cholesky(const std::vector<std::vector<int>> &S, std::vector<std::vector<int>> &Lrows,
                       std::vector<int> &parent) {
  const int m = (int)S.size();
  std::vector<std::vector<int>> cols(m), children(m);
  parent.assign(m, -1);
  Lrows.assign(m, {});
  for (int j = 0; j < m; ++j) {
    std::vector<int> c;
    for (int i : S[j])
      if (i > j) c.push_back(i);
    for (int ch : children[j]) {
      for (int i : cols[ch])
        if (i > j) c.push_back(i);
      std::vector<int>().swap(cols[ch]);  // a column merges into its parent only
    }
    std::sort(c.begin(), c.end());
    c.erase(std::unique(c.begin(), c.end()), c.end());
    if (!c.empty()) {
      parent[j] = c[0];
      children[c[0]].push_back(j);
    }
    Lrows[j].push_back(j);
    for (int i : c) Lrows[i].push_back(j);
    cols[j] = std::move(c);
  }
}

// Minimum-degree order of the groups (entities) of a symmetric pattern S:
// repeatedly eliminates the group whose neighbours hold the fewest functions
// (ties: the lower group), joining its neighbours into a clique.  Returns the
// positions of S in elimination order, each group's positions together.
std::vector<int> entity_minimum_degree(const std::vector<std::vector<int>> &S, const std::vector<int> &group_of,
                                       int ngroup) {
  std::vector<std::vector<int>> members(ngroup);
  for (int i = 0; i < (int)S.size(); ++i) members[group_of[i]].push_back(i);
  std::vector<std::vector<char>> adj(ngroup, std::vector<char>(ngroup, 0));
  for (int i = 0; i < (int)S.size(); ++i)
    for (int j : S[i])
      if (group_of[i] != group_of[j]) adj[group_of[i]][group_of[j]] = adj[group_of[j]][group_of[i]] = 1;
  std::vector<char> alive(ngroup, 1);
  std::vector<int> out;
  for (int step = 0; step < ngroup; ++step) {
    int best = -1;
    int64_t best_deg = 0;
    for (int g = 0; g < ngroup; ++g) {
      if (!alive[g]) continue;
      int64_t deg = 0;
      for (int h = 0; h < ngroup; ++h)
        if (alive[h] && adj[g][h]) deg += (int64_t)members[h].size();
      if (best < 0 || deg < best_deg) {
        best = g;
        best_deg = deg;
      }
    }
    alive[best] = 0;
    std::vector<int> nb;
    for (int h = 0; h < ngroup; ++h)
      if (alive[h] && adj[best][h]) nb.push_back(h);
    for (int a : nb)
      for (int b : nb)
        if (a != b) adj[a][b] = 1;
    out.insert(out.end(), members[best].begin(), members[best].end());
  }
  return out;
}

std::string &hex_last_error() {
  static std::string e;
  return e;
}

int handle_hex(fdm_hexmesh *h, const fdm::Error &e) {
  if (h) h->err = e.msg;
  hex_last_error() = e.msg;
  return e.code;
}

struct Builder {
  int p, n, nv, nc;
  const int *cells;
  std::vector<int> parity;                          // parity of s_m, m = 1..p-1 (index m - 1)
  std::vector<double> Af, Bf;                       // 1D FDM stiffness and mass (n x n)
  std::vector<int64_t> vbase;                       // node of each vertex, -1 unused
  std::map<std::pair<int, int>, int64_t> ebase;     // first node of each edge
  std::map<std::array<int, 4>, int64_t> fbase;      // first node of each face
  std::map<std::array<int, 4>, int> fcount;         // cells per face
  std::vector<int64_t> cbase;
  std::vector<int64_t> entity;                      // first slot of each node's entity
  int64_t nnode = 0;

  int corner(int e, int a, int b, int c) const { return cells[8 * e + a + 2 * b + 4 * c]; }

  static std::array<int, 4> face_key(std::array<int, 4> v) {
    std::sort(v.begin(), v.end());
    return v;
  }

  // the corners of the face of cell e normal to axis d at side s, indexed by
  // the two tangential axes (d1 < d2) as t1 + 2 t2
  std::array<int, 4> face_corners(int e, int d, int s) const {
    std::array<int, 4> out{};
    const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    for (int t2 = 0; t2 < 2; ++t2)
      for (int t1 = 0; t1 < 2; ++t1) {
        int r[3];
        r[d] = s;
        r[d1] = t1;
        r[d2] = t2;
        out[t1 + 2 * t2] = corner(e, r[0], r[1], r[2]);
      }
    return out;
  }

  void number() {
    vbase.assign(nv, -1);
    for (int e = 0; e < nc; ++e)
      for (int k = 0; k < 8; ++k) {
        const int v = cells[8 * e + k];
        if (v < 0 || v >= nv) fdm::fail(FDM_EINVAL, "fdm_hexmesh_create: vertex index out of range");
      }
    std::vector<char> used(nv, 0);
    for (int e = 0; e < nc; ++e)
      for (int k = 0; k < 8; ++k) used[cells[8 * e + k]] = 1;
    for (int v = 0; v < nv; ++v)
      if (used[v]) vbase[v] = nnode++;
    const int64_t m = p - 1;
    for (int e = 0; e < nc; ++e)
      for (int d = 0; d < 3; ++d)
        for (int a = 0; a < 2; ++a)
          for (int b = 0; b < 2; ++b) {
            int r0[3], r1[3];
            const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
            r0[d] = 0; r1[d] = 1;
            r0[d1] = r1[d1] = a;
            r0[d2] = r1[d2] = b;
            int u = corner(e, r0[0], r0[1], r0[2]), w = corner(e, r1[0], r1[1], r1[2]);
            if (u == w) fdm::fail(FDM_EINVAL, "fdm_hexmesh_create: degenerate cell edge");
            auto key = std::make_pair(std::min(u, w), std::max(u, w));
            if (!ebase.count(key)) {
              ebase[key] = nnode;
              nnode += m;
            }
          }
    for (int e = 0; e < nc; ++e)
      for (int d = 0; d < 3; ++d)
        for (int s = 0; s < 2; ++s) {
          auto key = face_key(face_corners(e, d, s));
          if (key[0] == key[1] || key[1] == key[2] || key[2] == key[3])
            fdm::fail(FDM_EINVAL, "fdm_hexmesh_create: degenerate cell face");
          if (!fbase.count(key)) {
            fbase[key] = nnode;
            nnode += m * m;
          }
          ++fcount[key];
        }
    for (auto &kv : fcount)
      if (kv.second > 2) fdm::fail(FDM_EINVAL, "fdm_hexmesh_create: a face belongs to more than two cells");
    cbase.resize(nc);
    for (int e = 0; e < nc; ++e) {
      cbase[e] = nnode;
      nnode += m * m * m;
    }
    if (nnode > INT32_MAX) fdm::fail(FDM_EINVAL, "fdm_hexmesh_create: more than 2^31 - 1 nodes");
    // the first slot of each node's entity
    entity.assign(nnode, -1);
    for (int v = 0; v < nv; ++v)
      if (vbase[v] >= 0) entity[vbase[v]] = vbase[v];
    for (auto &kv : ebase)
      for (int64_t k = 0; k < m; ++k) entity[kv.second + k] = kv.second;
    for (auto &kv : fbase)
      for (int64_t k = 0; k < m * m; ++k) entity[kv.second + k] = kv.second;
    for (int e = 0; e < nc; ++e)
      for (int64_t k = 0; k < m * m * m; ++k) entity[cbase[e] + k] = cbase[e];
  }

  // The star of vertex v in canonical order: its FDM slots, cell interiors
  // first (nint of them), then faces, edges and the vertex.  The cells around
  // v are walked from every start cell and every assignment of labels 0, 1, 2
  // to its three edges at v; a neighbour across the face normal to label a
  // keeps the labels of the two shared edges and gives a to its third.  Each
  // walk encodes, cell by cell, its three faces and three edges at v by
  // first-seen entity number and Dirichlet flag; the smallest encoding fixes
  // the cell order and the labels.  Stars with equal encodings are the same
  // configuration, so their orders (and patterns) coincide.
  std::vector<int64_t> canonical_star(int v, const std::vector<int> &vc, const std::vector<int32_t> &cell_fdm,
                                      const std::vector<uint8_t> &dirichlet, int &nint,
                                      std::vector<int> &encoding) const {
    const int nvc = (int)vc.size(), n3 = n * n * n;
    struct AtV {
      int e, cv;
      int w[3];                     // the vertex at the other end of the edge along each cell axis
      std::array<int, 4> face[3];   // the face normal to each cell axis that contains v
    };
    std::vector<AtV> C(nvc);
    std::map<std::array<int, 4>, std::vector<int>> fcells;
    for (int k = 0; k < nvc; ++k) {
      AtV &a = C[k];
      a.e = vc[k];
      a.cv = 0;
      while (cells[8 * a.e + a.cv] != v) ++a.cv;
      for (int d = 0; d < 3; ++d) {
        const int o = a.cv ^ (1 << d);
        a.w[d] = cells[8 * a.e + o];
        a.face[d] = face_key(face_corners(a.e, d, (a.cv >> d) & 1));
        fcells[a.face[d]].push_back(k);
      }
    }
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    auto free_slot = [&](int e, const int idx[3]) {
      const int64_t g = cell_fdm[(size_t)e * n3 + idx[0] + n * (idx[1] + n * idx[2])];
      return !dirichlet[g];
    };
    // is the entity of cell k with the given end axes free?  (probe one of its functions)
    auto entity_free = [&](int k, int ends_mask) {
      if (p < 2 && ends_mask != 7) return false;
      int idx[3];
      for (int d = 0; d < 3; ++d) idx[d] = (ends_mask >> d & 1) ? ((C[k].cv >> d) & 1) * p : 1;
      return free_slot(C[k].e, idx);
    };
    std::vector<int> best_enc, best_seq;
    std::vector<std::array<int, 3>> best_frame;
    for (int s0 = 0; s0 < nvc; ++s0)
      for (const auto &pm : perms) {
        std::vector<std::array<int, 3>> frame(nvc);
        std::vector<char> seen(nvc, 0);
        std::vector<int> seq;
        frame[s0] = {pm[0], pm[1], pm[2]};
        seen[s0] = 1;
        seq.push_back(s0);
        for (size_t h = 0; h < seq.size(); ++h) {
          const int k = seq[h];
          for (int a = 0; a < 3; ++a) {
            for (int k2 : fcells[C[k].face[frame[k][a]]]) {
              if (seen[k2]) continue;
              std::array<int, 3> f2{-1, -1, -1};
              bool used[3] = {false, false, false};
              bool ok = true;
              for (int b = 0; b < 3 && ok; ++b) {
                if (b == a) continue;
                const int wb = C[k].w[frame[k][b]];
                int d2 = -1;
                for (int d = 0; d < 3; ++d)
                  if (C[k2].w[d] == wb) d2 = d;
                if (d2 < 0 || used[d2]) ok = false;
                else {
                  f2[b] = d2;
                  used[d2] = true;
                }
              }
              if (!ok) continue;
              for (int d = 0; d < 3; ++d)
                if (!used[d]) f2[a] = d;
              frame[k2] = f2;
              seen[k2] = 1;
              seq.push_back(k2);
            }
          }
        }
        for (int k = 0; k < nvc; ++k)  // cells not reached through faces (not expected)
          if (!seen[k]) {
            frame[k] = {0, 1, 2};
            seq.push_back(k);
          }
        std::map<std::vector<int>, int> ids;
        std::vector<int> enc;
        for (int k : seq) {
          for (int a = 0; a < 3; ++a) {
            const std::array<int, 4> &fk = C[k].face[frame[k][a]];
            auto it = ids.emplace(std::vector<int>{0, fk[0], fk[1], fk[2], fk[3]}, (int)ids.size()).first;
            enc.push_back(2 * it->second + (entity_free(k, 1 << frame[k][a]) ? 1 : 0));
          }
          for (int a = 0; a < 3; ++a) {
            const int w = C[k].w[frame[k][a]];
            auto it = ids.emplace(std::vector<int>{1, std::min(v, w), std::max(v, w)}, (int)ids.size()).first;
            enc.push_back(2 * it->second + (entity_free(k, 7 ^ (1 << frame[k][a])) ? 1 : 0));
          }
        }
        if (best_seq.empty() || enc < best_enc) {
          best_enc.swap(enc);
          best_seq = seq;
          best_frame = frame;
        }
      }
    encoding = best_enc;
    // the order: interiors cell by cell, then faces, edges (first seen in the
    // canonical walk, functions in the first cell's labels), the vertex
    std::vector<int64_t> out;
    std::map<int64_t, char> done;
    const int m = p - 1;
    auto emit = [&](int k, const int idx[3]) {
      const int64_t g = cell_fdm[(size_t)C[k].e * n3 + idx[0] + n * (idx[1] + n * idx[2])];
      if (dirichlet[g] || done.count(g)) return;
      done[g] = 1;
      out.push_back(g);
    };
    for (int k : best_seq) {
      const auto &f = best_frame[k];
      for (int m3 = 1; m3 <= m; ++m3)
        for (int m2 = 1; m2 <= m; ++m2)
          for (int m1 = 1; m1 <= m; ++m1) {
            int idx[3];
            idx[f[0]] = m1;
            idx[f[1]] = m2;
            idx[f[2]] = m3;
            emit(k, idx);
          }
    }
    nint = (int)out.size();
    for (int k : best_seq) {
      const auto &f = best_frame[k];
      for (int a = 0; a < 3; ++a) {
        const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
        for (int mc = 1; mc <= m; ++mc)
          for (int mb = 1; mb <= m; ++mb) {
            int idx[3];
            idx[f[a]] = ((C[k].cv >> f[a]) & 1) * p;
            idx[f[b]] = mb;
            idx[f[c]] = mc;
            emit(k, idx);
          }
      }
    }
    for (int k : best_seq) {
      const auto &f = best_frame[k];
      for (int a = 0; a < 3; ++a)
        for (int ma = 1; ma <= m; ++ma) {
          int idx[3];
          for (int d = 0; d < 3; ++d) idx[d] = ((C[k].cv >> d) & 1) * p;
          idx[f[a]] = ma;
          emit(k, idx);
        }
    }
    {
      int idx[3];
      for (int d = 0; d < 3; ++d) idx[d] = ((C[best_seq[0]].cv >> d) & 1) * p;
      emit(best_seq[0], idx);
    }
    return out;
  }

  // global node and FDM function of cell-local index (i, j, k) (node indices
  // for the GLL map, eigen-indices on the interior axes for the FDM map)
  void map_local(int e, const int idx[3], int64_t &node, int64_t &fdm_fn, int &sign) const {
    const int m = p - 1;
    int ends = 0;
    for (int d = 0; d < 3; ++d) ends += (idx[d] == 0 || idx[d] == p);
    sign = 1;
    if (ends == 3) {
      node = fdm_fn = vbase[corner(e, idx[0] / p, idx[1] / p, idx[2] / p)];
      return;
    }
    if (ends == 0) {
      node = fdm_fn = cbase[e] + (idx[0] - 1) + (int64_t)m * ((idx[1] - 1) + (int64_t)m * (idx[2] - 1));
      return;
    }
    if (ends == 2) {
      int d = 0;  // the edge's axis: the one interior index
      for (int a = 0; a < 3; ++a)
        if (idx[a] != 0 && idx[a] != p) d = a;
      int r0[3], r1[3];
      for (int a = 0; a < 3; ++a) r0[a] = r1[a] = idx[a] / p;
      r0[d] = 0;
      r1[d] = 1;
      const int u = corner(e, r0[0], r0[1], r0[2]), w = corner(e, r1[0], r1[1], r1[2]);
      const int64_t base = ebase.at(std::make_pair(std::min(u, w), std::max(u, w)));
      const bool rev = u > w;
      node = base + (rev ? p - idx[d] : idx[d]) - 1;
      fdm_fn = base + idx[d] - 1;
      if (rev) sign = parity[idx[d] - 1];
      return;
    }
    // a face: normal axis d (the end index), tangential d1 < d2
    int d = 0;
    for (int a = 0; a < 3; ++a)
      if (idx[a] == 0 || idx[a] == p) d = a;
    const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    const auto fc = face_corners(e, d, idx[d] / p);
    int o = 0;  // corner (t1 + 2 t2) with the lowest vertex id
    for (int k = 1; k < 4; ++k)
      if (fc[k] < fc[o]) o = k;
    const int a0 = o & 1, b0 = o >> 1;
    const int n1 = fc[(1 - a0) + 2 * b0], n2 = fc[a0 + 2 * (1 - b0)];  // neighbours along d1, d2
    const bool s_along_d1 = n1 < n2;
    const int i1 = idx[d1], i2 = idx[d2];
    const int pos1 = a0 ? p - i1 : i1, pos2 = b0 ? p - i2 : i2;  // node positions from the origin
    const int64_t base = fbase.at(face_key(fc));
    int s_node, t_node, s_fn, t_fn;
    if (s_along_d1) {
      s_node = pos1; t_node = pos2; s_fn = i1; t_fn = i2;
    } else {
      s_node = pos2; t_node = pos1; s_fn = i2; t_fn = i1;
    }
    node = base + (s_node - 1) + (int64_t)m * (t_node - 1);
    fdm_fn = base + (s_fn - 1) + (int64_t)m * (t_fn - 1);
    if (a0) sign *= parity[i1 - 1];
    if (b0) sign *= parity[i2 - 1];
  }
};

// the parity (+1 even, -1 odd under reflection) of each interior 1D FDM
// function s_m, m = 1..p-1, read off the computed eigenvectors
std::vector<int> interior_parities(const fdm::Basis1D &basis, int p) {
  const int m = p - 1;
  std::vector<int> parity(std::max(m, 0));
  for (int j = 0; j < m; ++j) {
    double even = 0.0, odd = 0.0, scale = 0.0;
    for (int i = 0; i < m; ++i) {
      const double a = basis.S[i * m + j], b = basis.S[(m - 1 - i) * m + j];
      even = std::max(even, std::fabs(a - b));
      odd = std::max(odd, std::fabs(a + b));
      scale = std::max(scale, std::fabs(a));
    }
    if (even <= 1e-10 * scale) parity[j] = 1;
    else if (odd <= 1e-10 * scale) parity[j] = -1;
    else fdm::fail(FDM_EINVAL, "fdm_hexmesh_create: an interior FDM function is neither even nor odd");
  }
  return parity;
}

// appends rows as one CSR block: row pointers from 0 to rowptr, columns to cols
template <typename Rows>
int64_t append_csr(const Rows &rows, std::vector<int64_t> &rowptr, std::vector<int32_t> &cols) {
  int64_t cnt = 0;
  rowptr.push_back(0);
  for (auto &r : rows) {
    cols.insert(cols.end(), r.begin(), r.end());
    cnt += (int64_t)r.size();
    rowptr.push_back(cnt);
  }
  return cnt;
}

// per cell and local index: the node, the FDM slot and its sign
void build_cell_maps(fdm_hexmesh *h, const Builder &B) {
  const int n = h->n, n3 = n * n * n;
  h->cell_nodes.resize((size_t)h->nc * n3);
  h->cell_fdm.resize((size_t)h->nc * n3);
  h->cell_sign.resize((size_t)h->nc * n3);
  for (int e = 0; e < h->nc; ++e)
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const int idx[3] = {i, j, k};
          int64_t node, fn;
          int sign;
          B.map_local(e, idx, node, fn, sign);
          const size_t l = (size_t)e * n3 + i + n * (j + n * k);
          h->cell_nodes[l] = (int32_t)node;
          h->cell_fdm[l] = (int32_t)fn;
          h->cell_sign[l] = (int8_t)sign;
        }
}

// Dirichlet nodes: the closure of every face that belongs to one cell
// whether the 4 corner vertices of a boundary face make it a Dirichlet face
template <typename F>
bool dirichlet_face(const fdm_hexmesh *h, const F &corners) {
  if (h->dvert.empty()) return true;
  for (int v : corners)
    if (!h->dvert[v]) return false;
  return true;
}

void mark_dirichlet(fdm_hexmesh *h, const Builder &B) {
  const int n = h->n, n3 = n * n * n, p = h->p;
  h->dirichlet.assign(B.nnode, 0);
  for (int e = 0; e < h->nc; ++e)
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        if (B.fcount.at(Builder::face_key(B.face_corners(e, d, s))) != 1) continue;
        if (!dirichlet_face(h, B.face_corners(e, d, s))) continue;
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              const int idx[3] = {i, j, k};
              if (idx[d] == (s ? p : 0)) h->dirichlet[h->cell_nodes[(size_t)e * n3 + i + n * (j + n * k)]] = 1;
            }
      }
}

// pattern of S_G = A_GG - A_GI D^{-1} A_IG over interface positions: A_GG plus,
// through every interior function, the interface functions it couples to
// (the interior block is diagonal)
std::vector<std::vector<int>> schur_pattern(const std::vector<std::vector<int>> &rows, int nint) {
  const int ns = (int)rows.size();
  std::vector<std::vector<int>> Sg(ns - nint);
  for (int r = nint; r < ns; ++r) {
    std::vector<int> &o = Sg[r - nint];
    for (int c : rows[r]) {
      if (c >= nint) o.push_back(c - nint);
      else
        for (int c2 : rows[c])
          if (c2 >= nint) o.push_back(c2 - nint);
    }
    std::sort(o.begin(), o.end());
    o.erase(std::unique(o.begin(), o.end()), o.end());
  }
  return Sg;
}

// The vertex stars: their canonical order, surrogate patterns, interface
// order, sparsity classes and each class's symbolic factorisations.
struct StarBuilder {
  fdm_hexmesh *h;
  const Builder &B;
  std::vector<std::vector<int>> vcells;  // cells of each vertex
  std::map<std::vector<int>, int> classes;  // pattern -> class
  // per canonical configuration: the interface permutation, the interior count and the class
  struct StarShape {
    std::vector<int> newpos;
    int nint = 0, cls = -1;
  };
  std::map<std::vector<int>, StarShape> cache;

  StarBuilder(fdm_hexmesh *h_, const Builder &B_) : h(h_), B(B_), vcells(h_->nv) {
    for (int e = 0; e < h->nc; ++e)
      for (int k = 0; k < 8; ++k) vcells[h->cells[8 * (size_t)e + k]].push_back(e);
    h->star_ptr.push_back(0);
    h->pat_ptr.push_back(0);
    h->pat_colptr.push_back(0);
  }

  void push_star(int v, const std::vector<int64_t> &order, int nint) {
    h->star_vertex.push_back(v);
    for (int64_t g : order) h->star_nodes.push_back((int32_t)g);
    h->star_ptr.push_back((int64_t)h->star_nodes.size());
    h->star_nint.push_back(nint);
  }

  // the surrogate pattern of the star in the given order: FDM functions c1, c2
  // of a star cell couple iff for some axis a, Af couples them along a and Bf
  // along the other two axes.  An entity's FDM functions use the slots of its
  // nodes, so the star's functions are those whose slot is a star node.
  std::vector<std::vector<int>> surrogate_pattern(int v, const std::vector<int64_t> &order) const {
    const int n = h->n, n3 = n * n * n;
    std::map<int64_t, int> in_star;
    for (size_t k = 0; k < order.size(); ++k) in_star[order[k]] = (int)k;
    std::vector<std::vector<int>> rows(order.size());
    for (int e : vcells[v]) {
      std::vector<std::pair<int, int>> loc;  // (cell-local FDM index, star position)
      for (int c = 0; c < n3; ++c) {
        auto it = in_star.find(h->cell_fdm[(size_t)e * n3 + c]);
        if (it != in_star.end()) loc.push_back({c, it->second});
      }
      for (auto &x : loc)
        for (auto &y : loc) {
          const int a[3] = {x.first % n, (x.first / n) % n, x.first / (n * n)};
          const int b[3] = {y.first % n, (y.first / n) % n, y.first / (n * n)};
          bool nz = false;
          for (int d = 0; d < 3 && !nz; ++d) {
            bool term = B.Af[a[d] * n + b[d]] != 0.0;
            for (int o = 0; o < 3 && term; ++o)
              if (o != d) term = B.Bf[a[o] * n + b[o]] != 0.0;
            nz = term;
          }
          if (nz) rows[x.second].push_back(y.second);
        }
    }
    for (auto &r : rows) {
      std::sort(r.begin(), r.end());
      r.erase(std::unique(r.begin(), r.end()), r.end());
    }
    return rows;
  }

  // reorders the interface by minimum degree over the star's entities in the
  // pattern of S_G; returns the new position of every old position
  std::vector<int> interface_order(const std::vector<int64_t> &order, const std::vector<std::vector<int>> &rows,
                                   int nint) const {
    const int ns = (int)order.size();
    std::map<int64_t, int> gid_of;
    std::vector<int> group_of(ns - nint);
    for (int r = nint; r < ns; ++r) {
      const int64_t ent = B.entity[order[r]];
      auto it = gid_of.find(ent);
      if (it == gid_of.end()) it = gid_of.emplace(ent, (int)gid_of.size()).first;
      group_of[r - nint] = it->second;  // groups numbered in the canonical order
    }
    const std::vector<int> elim = entity_minimum_degree(schur_pattern(rows, nint), group_of, (int)gid_of.size());
    std::vector<int> newpos(ns);
    for (int r = 0; r < nint; ++r) newpos[r] = r;
    for (int k = 0; k < (int)elim.size(); ++k) newpos[nint + elim[k]] = nint + k;
    return newpos;
  }

  // a new class: the symbolic factorisation of S_G (L form) and the
  // Schur-coupling split (the top block T a suffix of whole entities of the
  // interface order, chosen to minimise nnz(L_BB) + nnz(S_TB) + t (t + 1) / 2)
  void add_class(const std::vector<int64_t> &order, const std::vector<std::vector<int>> &rows, int nint) {
    const int ns = (int)order.size(), nG = ns - nint;
    h->class_star.push_back((int32_t)h->star_vertex.size() - 1);
    const std::vector<std::vector<int>> Sg = schur_pattern(rows, nint);
    std::vector<std::vector<int>> Lrows;
    std::vector<int> parent;
    symbolic_cholesky(Sg, Lrows, parent);
    if (h->fill_ptr.empty()) {
      h->fill_ptr.push_back(0);
      h->fill_colptr.push_back(0);
      h->etree_ptr.push_back(0);
      h->sc_ptr.push_back(0);
      h->sc_colptr.push_back(0);
    }
    h->class_nnzl.push_back(append_csr(Lrows, h->fill_rowptr, h->fill_cols));
    h->fill_ptr.push_back((int64_t)h->fill_rowptr.size());
    h->fill_colptr.push_back((int64_t)h->fill_cols.size());
    h->etree.insert(h->etree.end(), parent.begin(), parent.end());
    h->etree_ptr.push_back((int64_t)h->etree.size());
    std::vector<int> cand{0};
    for (int i = nG - 1; i >= 1; --i)
      if (B.entity[order[nint + i]] != B.entity[order[nint + i - 1]]) cand.push_back(nG - i);
    if (nG > 0) cand.push_back(nG);
    int64_t best = -1;
    int best_t = 0;
    std::vector<std::vector<int>> best_L, best_TB;
    for (int t : cand) {
      const int nB = nG - t;
      std::vector<std::vector<int>> SB(nB), TB(t);
      int64_t ntb = 0;
      for (int r = 0; r < nG; ++r)
        for (int c : Sg[r]) {
          if (c >= nB) continue;
          if (r < nB) SB[r].push_back(c);
          else {
            TB[r - nB].push_back(c);
            ++ntb;
          }
        }
      std::vector<std::vector<int>> Lb;
      std::vector<int> pb;
      symbolic_cholesky(SB, Lb, pb);
      int64_t nl = 0;
      for (auto &x : Lb) nl += (int64_t)x.size();
      const int64_t cost = nl + ntb + (int64_t)t * (t + 1) / 2;
      if (best < 0 || cost < best) {
        best = cost;
        best_t = t;
        best_L.swap(Lb);
        best_TB.swap(TB);
      }
    }
    h->sc_t.push_back(best_t);
    append_csr(best_L, h->sc_rowptr, h->sc_cols);
    append_csr(best_TB, h->sc_rowptr, h->sc_cols);
    h->sc_ptr.push_back((int64_t)h->sc_rowptr.size());
    h->sc_colptr.push_back((int64_t)h->sc_cols.size());
  }

  void add_star(int v) {
    if (vcells[v].empty()) return;
    int nint = 0;
    std::vector<int> enc;
    std::vector<int64_t> order = B.canonical_star(v, vcells[v], h->cell_fdm, h->dirichlet, nint, enc);
    if (order.empty()) return;
    const int ns = (int)order.size();
    auto hit = cache.find(enc);
    if (hit != cache.end()) {  // a configuration seen before: its pattern, interface order and class
      const StarShape &sh = hit->second;
      if ((int)sh.newpos.size() != ns || sh.nint != nint)
        fdm::fail(FDM_EINVAL, "fdm_hexmesh_create: inconsistent star configuration");
      std::vector<int64_t> order2(ns);
      for (int r = 0; r < ns; ++r) order2[sh.newpos[r]] = order[r];
      push_star(v, order2, nint);
      // the pattern of the class's first star (copied out first: the vectors grow)
      const int k0 = h->class_star[sh.cls];
      const std::vector<int64_t> rp0(h->pat_rowptr.begin() + h->pat_ptr[k0],
                                     h->pat_rowptr.begin() + h->pat_ptr[k0] + ns + 1);
      const std::vector<int32_t> c0(h->pat_cols.begin() + h->pat_colptr[k0],
                                    h->pat_cols.begin() + h->pat_colptr[k0] + rp0[ns]);
      h->pat_rowptr.insert(h->pat_rowptr.end(), rp0.begin(), rp0.end());
      h->pat_cols.insert(h->pat_cols.end(), c0.begin(), c0.end());
      h->pat_ptr.push_back((int64_t)h->pat_rowptr.size());
      h->pat_colptr.push_back((int64_t)h->pat_cols.size());
      h->star_class.push_back(sh.cls);
      return;
    }
    const std::vector<std::vector<int>> rows0 = surrogate_pattern(v, order);
    for (int r = 0; r < nint; ++r)
      for (int c : rows0[r])
        if (c < nint && c != r) fdm::fail(FDM_EINVAL, "fdm_hexmesh_create: interior block of a star is not diagonal");
    StarShape shape;
    shape.nint = nint;
    shape.newpos = interface_order(order, rows0, nint);
    std::vector<int64_t> order2(ns);
    std::vector<std::vector<int>> rows(ns);
    for (int r = 0; r < ns; ++r) {
      order2[shape.newpos[r]] = order[r];
      for (int c : rows0[r]) rows[shape.newpos[r]].push_back(shape.newpos[c]);
    }
    for (auto &r : rows) std::sort(r.begin(), r.end());
    push_star(v, order2, nint);
    append_csr(rows, h->pat_rowptr, h->pat_cols);
    h->pat_ptr.push_back((int64_t)h->pat_rowptr.size());
    h->pat_colptr.push_back((int64_t)h->pat_cols.size());
    // the class: stars with equal patterns and interior counts share the
    // symbolic factorisation of their interface Schur complement
    std::vector<int> key{ns, nint};
    for (auto &r : rows) {
      key.push_back((int)r.size());
      key.insert(key.end(), r.begin(), r.end());
    }
    auto found = classes.find(key);
    if (found != classes.end()) shape.cls = found->second;
    else {
      shape.cls = (int)h->class_star.size();
      classes.emplace(std::move(key), shape.cls);
    }
    h->star_class.push_back(shape.cls);
    if (found == classes.end()) add_class(order2, rows, nint);
    cache.emplace(std::move(enc), std::move(shape));
  }
};

// CSR of the inverse of a map l -> target[l] (targets in [0, N)), sources by l
void invert_map(const std::vector<int32_t> &target, int64_t N, std::vector<int64_t> &ptr, std::vector<int32_t> &src) {
  ptr.assign(N + 1, 0);
  for (int32_t g : target) ++ptr[g + 1];
  for (int64_t g = 0; g < N; ++g) ptr[g + 1] += ptr[g];
  src.resize(target.size());
  std::vector<int64_t> at(ptr.begin(), ptr.end() - 1);
  for (size_t l = 0; l < target.size(); ++l) src[at[target[l]]++] = (int32_t)l;
}

// the inverse maps of the apply: FDM slot -> cell copies, FDM slot -> (star,
// position), node -> cell copies and its owner (the lowest cell)
void build_inverse_maps(fdm_hexmesh *h) {
  const int64_t N = h->nnode;
  invert_map(h->cell_fdm, N, h->slot_cells_ptr, h->slot_cells);
  invert_map(h->cell_nodes, N, h->node_cells_ptr, h->node_cells);
  h->node_owner.assign(N, -1);
  for (int64_t g = 0; g < N; ++g)
    if (h->node_cells_ptr[g + 1] > h->node_cells_ptr[g]) h->node_owner[g] = h->node_cells[h->node_cells_ptr[g]];
  const int nstar = (int)h->star_vertex.size();
  h->slot_stars_ptr.assign(N + 1, 0);
  for (int k = 0; k < nstar; ++k)
    for (int64_t t = h->star_ptr[k]; t < h->star_ptr[k + 1]; ++t) ++h->slot_stars_ptr[h->star_nodes[t] + 1];
  for (int64_t g = 0; g < N; ++g) h->slot_stars_ptr[g + 1] += h->slot_stars_ptr[g];
  h->slot_stars.resize(2 * (size_t)h->slot_stars_ptr[N]);
  std::vector<int64_t> sp(h->slot_stars_ptr.begin(), h->slot_stars_ptr.end() - 1);
  for (int k = 0; k < nstar; ++k)
    for (int64_t t = h->star_ptr[k]; t < h->star_ptr[k + 1]; ++t) {
      const int64_t at = sp[h->star_nodes[t]]++;
      h->slot_stars[2 * at] = k;
      h->slot_stars[2 * at + 1] = (int32_t)(t - h->star_ptr[k]);
    }
}

}  // namespace

extern "C" int fdm_hexmesh_create(int nv, int nc, const int *cells, int p, fdm_hexmesh **out) {
  return fdm_hexmesh_create_bc(nv, nc, cells, p, nullptr, out);
}

extern "C" int fdm_hexmesh_create_bc(int nv, int nc, const int *cells, int p, const unsigned char *dirichlet_vertex,
                                     fdm_hexmesh **out) {
  if (!out) return FDM_EINVAL;
  *out = nullptr;
  if (nv < 8 || nc < 1 || !cells || p < 1 || p > 15) {
    hex_last_error() = "fdm_hexmesh_create: need at least 8 vertices, 1 cell and 1 <= p <= 15";
    return FDM_EINVAL;
  }
  fdm_hexmesh *h = new fdm_hexmesh();
  try {
    h->p = p;
    h->n = p + 1;
    h->nv = nv;
    h->nc = nc;
    h->cells.assign(cells, cells + 8 * (size_t)nc);
    if (dirichlet_vertex) h->dvert.assign(dirichlet_vertex, dirichlet_vertex + nv);
    const fdm::Basis1D basis = fdm::make_basis(p);
    h->Af = basis.Af;
    h->Bf = basis.Bf;
    h->xq = basis.xq;
    h->wq = basis.wq;
    Builder B{p, p + 1, nv, nc, cells, interior_parities(basis, p), basis.Af, basis.Bf, {}, {}, {}, {}, {}, {}, 0};
    B.number();
    h->nnode = B.nnode;
    build_cell_maps(h, B);
    mark_dirichlet(h, B);
    StarBuilder stars(h, B);
    for (int v = 0; v < nv; ++v) stars.add_star(v);
    build_inverse_maps(h);
  } catch (const fdm::Error &e) {
    int rc = handle_hex(h, e);
    delete h;
    return rc;
  } catch (const std::exception &e) {
    hex_last_error() = std::string("fdm_hexmesh_create: ") + e.what();
    delete h;
    return FDM_EINVAL;
  }
  *out = h;
  return FDM_OK;
}

namespace {

// value and reference gradient of the 8 trilinear corner functions at t
void trilinear_gradients(const double t[3], double gN[8][3]) {
  for (int c = 0; c < 8; ++c) {
    const int a[3] = {c & 1, (c >> 1) & 1, c >> 2};
    double N[3], dN[3];
    for (int d = 0; d < 3; ++d) {
      N[d] = a[d] ? 0.5 * (1.0 + t[d]) : 0.5 * (1.0 - t[d]);
      dN[d] = a[d] ? 0.5 : -0.5;
    }
    gN[c][0] = dN[0] * N[1] * N[2];
    gN[c][1] = N[0] * dN[1] * N[2];
    gN[c][2] = N[0] * N[1] * dN[2];
  }
}

// in place, the lower triangle of the m x m row-major matrix M becomes its
// Cholesky factor (right-looking); FDM_ENOTSPD naming `what` for a pivot <= 0
void dense_cholesky(std::vector<double> &M, int m, const char *what) {
  for (int j = 0; j < m; ++j) {
    double &djj = M[(size_t)j * m + j];
    if (!(djj > 0.0)) fdm::fail(FDM_ENOTSPD, std::string("fdm_hexmesh_factor: ") + what + " pivot <= 0");
    djj = std::sqrt(djj);
    for (int i = j + 1; i < m; ++i) M[(size_t)i * m + j] /= djj;
    for (int c = j + 1; c < m; ++c) {
      const double lcj = M[(size_t)c * m + j];
      if (lcj == 0.0) continue;
      for (int i = c; i < m; ++i) M[(size_t)i * m + c] -= M[(size_t)i * m + j] * lcj;
    }
  }
}

// appends the entries of the factor L (m x m, row-major) in the rows of its
// symbolic fill; an entry outside the fill above `tol` is an error
void extract_fill(const std::vector<double> &L, int m, const int64_t *rp, const int32_t *cols, double tol,
                  std::vector<double> &out, const char *what) {
  std::vector<char> in_fill((size_t)m * m, 0);
  for (int r = 0; r < m; ++r)
    for (int64_t t = rp[r]; t < rp[r + 1]; ++t) {
      in_fill[(size_t)r * m + cols[t]] = 1;
      out.push_back(L[(size_t)r * m + cols[t]]);
    }
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < r; ++c)
      if (!in_fill[(size_t)r * m + c] && std::fabs(L[(size_t)r * m + c]) > tol)
        fdm::fail(FDM_EINVAL, std::string("fdm_hexmesh_factor: ") + what + " entry outside its symbolic fill");
}

// the coarse unknowns: the vertices not on a boundary face
void coarse_vertices(fdm_hexmesh *h) {
  std::vector<char> bnd(h->nv, 0), used(h->nv, 0);
  std::map<std::array<int, 4>, int> fc;
  for (int e = 0; e < h->nc; ++e)
    for (int d = 0; d < 3; ++d)
      for (int sd = 0; sd < 2; ++sd) {
        std::array<int, 4> f{};
        int t = 0;
        for (int c = 0; c < 8; ++c)
          if (((c >> d) & 1) == sd) f[t++] = h->cells[8 * (size_t)e + c];
        std::sort(f.begin(), f.end());
        ++fc[f];
      }
  for (auto &kv : fc)
    if (kv.second == 1 && dirichlet_face(h, kv.first))
      for (int v : kv.first) bnd[v] = 1;
  for (int c : h->cells) used[c] = 1;
  h->coarse_of.assign(h->nv, -1);
  int nco = 0;
  for (int v = 0; v < h->nv; ++v)
    if (used[v] && !bnd[v]) h->coarse_of[v] = nco++;
  h->coarse.assign((size_t)nco * nco, 0.0);
}

// per cell and Gauss point G = kappa |det J| J^{-1} J^{-T} of the trilinear map:
// the averaged surrogate mu_d = (1/8) sum_q w_q G_dd (Section 2.7), the
// stiffness factors w_q G, and the Q1 Galerkin operator (P^T A P cell by cell
// is the Q1 stiffness of the same quadrature: the trilinear functions lie in Q_p)
void cell_geometry(fdm_hexmesh *h, const double *X, const double *kappa_q, const double *kaxes) {
  const double ka[3] = {kaxes ? kaxes[0] : 1.0, kaxes ? kaxes[1] : 1.0, kaxes ? kaxes[2] : 1.0};
  const int q = h->n, q3 = q * q * q, nc = h->nc;
  const int nco = (int)std::lround(std::sqrt((double)h->coarse.size()));
  h->mu.assign((size_t)nc * 3, 0.0);
  h->geom.assign((size_t)nc * q3 * 6, 0.0);
  for (int e = 0; e < nc; ++e)
    for (int qz = 0; qz < q; ++qz)
      for (int qy = 0; qy < q; ++qy)
        for (int qx = 0; qx < q; ++qx) {
          const double t[3] = {h->xq[qx], h->xq[qy], h->xq[qz]};
          double gN[8][3];
          trilinear_gradients(t, gN);
          double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
          for (int c = 0; c < 8; ++c) {
            const double *xv = X + 3 * (size_t)h->cells[8 * (size_t)e + c];
            for (int i = 0; i < 3; ++i)
              for (int d = 0; d < 3; ++d) J[i][d] += xv[i] * gN[c][d];
          }
          const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                             J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                             J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
          if (!(std::fabs(det) > 0.0)) fdm::fail(FDM_EINVAL, "fdm_hexmesh_factor: degenerate cell geometry");
          // cofactors: (J^{-1})[d][i] = C[i][d] / det
          double C[3][3];
          for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
              const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
              C[i][j] = J[i1][j1] * J[i2][j2] - J[i1][j2] * J[i2][j1];
            }
          const int qi = qx + q * (qy + q * qz);
          const double kap = kappa_q ? kappa_q[(size_t)e * q3 + qi] : 1.0;
          const double w = h->wq[qx] * h->wq[qy] * h->wq[qz];
          double G[3][3];
          for (int d = 0; d < 3; ++d)
            for (int f = 0; f < 3; ++f) {
              double s = 0.0;
              for (int i = 0; i < 3; ++i) s += C[i][d] * ka[i] * C[i][f];
              G[d][f] = kap * s / std::fabs(det);
            }
          for (int d = 0; d < 3; ++d) h->mu[3 * (size_t)e + d] += w * G[d][d] / 8.0;
          double *gq = &h->geom[((size_t)e * q3 + qi) * 6];
          gq[0] = w * G[0][0];
          gq[1] = w * G[1][1];
          gq[2] = w * G[2][2];
          gq[3] = w * G[0][1];
          gq[4] = w * G[0][2];
          gq[5] = w * G[1][2];
          for (int c1 = 0; c1 < 8; ++c1) {
            const int i1 = h->coarse_of[h->cells[8 * (size_t)e + c1]];
            if (i1 < 0) continue;
            for (int c2 = 0; c2 < 8; ++c2) {
              const int i2 = h->coarse_of[h->cells[8 * (size_t)e + c2]];
              if (i2 < 0) continue;
              double s = 0.0;
              for (int d = 0; d < 3; ++d)
                for (int f = 0; f < 3; ++f) s += gN[c1][d] * G[d][f] * gN[c2][f];
              h->coarse[(size_t)i1 * nco + i2] += w * s;
            }
          }
        }
}

// the surrogate matrix of star k in the FDM basis on the star's pattern (the
// sum over its cells of sum_d mu_d (A_f along axis d, B_f along the others),
// with the map's signs): values aligned with the pattern's columns
std::vector<double> star_matrix(const fdm_hexmesh *h, int k, const std::vector<int> &star_cells) {
  const int n = h->n, n3 = n * n * n;
  const int64_t s0 = h->star_ptr[k], ns = h->star_ptr[k + 1] - s0;
  std::map<int32_t, int> pos;
  for (int64_t i = 0; i < ns; ++i) pos[h->star_nodes[s0 + i]] = (int)i;
  const int64_t *rp = h->pat_rowptr.data() + h->pat_ptr[k];
  const int32_t *cols = h->pat_cols.data() + h->pat_colptr[k];
  std::vector<double> A(rp[ns], 0.0);
  for (int e : star_cells) {
    std::vector<std::array<int, 3>> loc;  // (local FDM index, star position, sign)
    for (int c = 0; c < n3; ++c) {
      auto it = pos.find(h->cell_fdm[(size_t)e * n3 + c]);
      if (it != pos.end()) loc.push_back({c, it->second, h->cell_sign[(size_t)e * n3 + c]});
    }
    const double *me = &h->mu[3 * (size_t)e];
    for (auto &x : loc)
      for (auto &y : loc) {
        const int a[3] = {x[0] % n, (x[0] / n) % n, x[0] / (n * n)};
        const int b[3] = {y[0] % n, (y[0] / n) % n, y[0] / (n * n)};
        double v = 0.0;
        for (int d = 0; d < 3; ++d) {
          double t = me[d] * h->Af[a[d] * n + b[d]];
          for (int o = 0; o < 3; ++o)
            if (o != d) t *= h->Bf[a[o] * n + b[o]];
          v += t;
        }
        if (v == 0.0) continue;
        const int32_t *r0 = cols + rp[x[1]], *r1 = cols + rp[x[1] + 1];
        const int32_t *f = std::lower_bound(r0, r1, y[1]);
        if (f == r1 || *f != y[1]) fdm::fail(FDM_EINVAL, "fdm_hexmesh_factor: entry outside the star pattern");
        A[f - cols] += x[2] * y[2] * v;
      }
  }
  return A;
}

// star k: interior pivots D, the Cholesky factor of S_G = A_GG - A_GI D^{-1}
// A_IG in its class's fill (L form), and the Schur-coupling form L_BB, S_TB,
// W = (S_TT - S_TB S_BB^{-1} S_BT)^{-1}
struct StarOut {
  std::vector<double> diag, factor, sc;
  int code = 0;
  std::string msg;
};
void factor_star(const fdm_hexmesh *h, int k, const std::vector<int> &star_cells, StarOut &o) {
  const int64_t ns = h->star_ptr[k + 1] - h->star_ptr[k];
  const int nint = h->star_nint[k], nG = (int)ns - nint;
  const int64_t *rp = h->pat_rowptr.data() + h->pat_ptr[k];
  const int32_t *cols = h->pat_cols.data() + h->pat_colptr[k];
  const std::vector<double> A = star_matrix(h, k, star_cells);
  for (int i = 0; i < nint; ++i) {
    const int32_t *f = std::lower_bound(cols + rp[i], cols + rp[i + 1], i);
    const double d = (f != cols + rp[i + 1] && *f == i) ? A[f - cols] : 0.0;
    if (!(d > 0.0)) fdm::fail(FDM_ENOTSPD, "fdm_hexmesh_factor: interior pivot <= 0");
    o.diag.push_back(d);
  }
  // S_G, dense and symmetric
  std::vector<double> S((size_t)nG * nG, 0.0);
  for (int r = nint; r < ns; ++r)
    for (int64_t t = rp[r]; t < rp[r + 1]; ++t)
      if (cols[t] >= nint) S[(size_t)(r - nint) * nG + (cols[t] - nint)] = A[t];
  for (int i = 0; i < nint; ++i) {
    std::vector<std::pair<int, double>> nb;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
      if (cols[t] >= nint) nb.push_back({cols[t] - nint, A[t]});
    const double d = o.diag[i];
    for (auto &a : nb)
      for (auto &b : nb) S[(size_t)a.first * nG + b.first] -= a.second * b.second / d;
  }
  double smax = 0.0;
  for (double v : S) smax = std::max(smax, std::fabs(v));
  const double tol = 1e-10 * std::sqrt(smax);
  const int cls = h->star_class[k];
  // the L form
  std::vector<double> L = S;
  dense_cholesky(L, nG, "interface");
  extract_fill(L, nG, h->fill_rowptr.data() + h->fill_ptr[cls], h->fill_cols.data() + h->fill_colptr[cls], tol,
               o.factor, "factor");
  // the Schur-coupling form
  const int t = h->sc_t[cls], nB = nG - t;
  const int64_t *rpb = h->sc_rowptr.data() + h->sc_ptr[cls];
  const int64_t *rpt = rpb + nB + 1;
  const int32_t *cb = h->sc_cols.data() + h->sc_colptr[cls];
  const int32_t *ct = cb + rpb[nB];
  std::vector<double> LB((size_t)nB * nB, 0.0);
  for (int r = 0; r < nB; ++r)
    for (int c = 0; c <= r; ++c) LB[(size_t)r * nB + c] = S[(size_t)r * nG + c];
  dense_cholesky(LB, nB, "lower-block");
  extract_fill(LB, nB, rpb, cb, tol, o.sc, "lower-block");
  for (int r = 0; r < t; ++r)
    for (int64_t q2 = rpt[r]; q2 < rpt[r + 1]; ++q2) o.sc.push_back(S[(size_t)(nB + r) * nG + ct[q2]]);
  // Y = L_BB^{-1} S_BT (nB x t), C = S_TT - Y^T Y, W = C^{-1}
  std::vector<double> Y((size_t)nB * t);
  for (int j = 0; j < t; ++j)
    for (int i = 0; i < nB; ++i) {
      double v = S[(size_t)i * nG + nB + j];
      for (int l = 0; l < i; ++l) v -= LB[(size_t)i * nB + l] * Y[(size_t)l * t + j];
      Y[(size_t)i * t + j] = v / LB[(size_t)i * nB + i];
    }
  std::vector<double> Cm((size_t)t * t);
  for (int a = 0; a < t; ++a)
    for (int b = 0; b < t; ++b) {
      double v = S[(size_t)(nB + a) * nG + nB + b];
      for (int i = 0; i < nB; ++i) v -= Y[(size_t)i * t + a] * Y[(size_t)i * t + b];
      Cm[(size_t)a * t + b] = v;
    }
  dense_cholesky(Cm, t, "top-block");
  std::vector<double> Wm((size_t)t * t), col(t);
  for (int j = 0; j < t; ++j) {  // W e_j: forward L y = e_j, backward L^T x = y
    for (int i = 0; i < t; ++i) {
      double v = (i == j) ? 1.0 : 0.0;
      for (int l = 0; l < i; ++l) v -= Cm[(size_t)i * t + l] * col[l];
      col[i] = v / Cm[(size_t)i * t + i];
    }
    for (int i = t - 1; i >= 0; --i) {
      double v = col[i];
      for (int l = i + 1; l < t; ++l) v -= Cm[(size_t)l * t + i] * Wm[(size_t)l * t + j];
      Wm[(size_t)i * t + j] = v / Cm[(size_t)i * t + i];
    }
  }
  for (int r = 0; r < t; ++r)
    for (int c = 0; c <= r; ++c) o.sc.push_back(0.5 * (Wm[(size_t)r * t + c] + Wm[(size_t)c * t + r]));
}

// factor_star over all stars on host threads (FDM_HOST_THREADS, default the
// hardware's), each into its own buffers, concatenated in star order: the
// result does not depend on the thread count; the first failing star in star
// order reports its error
void factor_stars(fdm_hexmesh *h, const std::vector<std::vector<int>> &vcells) {
  const int nstar = (int)h->star_vertex.size();
  std::vector<StarOut> out(nstar);
  int nt = (int)std::thread::hardware_concurrency();
  if (const char *s = std::getenv("FDM_HOST_THREADS")) nt = std::atoi(s);
  nt = std::max(1, std::min({nt, 64, std::max(nstar, 1)}));
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int k = next++; k < nstar; k = next++) {
      try {
        factor_star(h, k, vcells[h->star_vertex[k]], out[k]);
      } catch (const fdm::Error &e) {
        out[k].code = e.code;
        out[k].msg = e.msg;
      } catch (const std::exception &e) {
        out[k].code = FDM_ENOMEM;
        out[k].msg = std::string("fdm_hexmesh_factor: ") + e.what();
      }
    }
  };
  std::vector<std::thread> pool;
  for (int i = 1; i < nt; ++i) pool.emplace_back(work);
  work();
  for (std::thread &t : pool) t.join();
  for (int k = 0; k < nstar; ++k)
    if (out[k].code) fdm::fail(out[k].code, out[k].msg);
  for (int k = 0; k < nstar; ++k) {
    h->diag.insert(h->diag.end(), out[k].diag.begin(), out[k].diag.end());
    h->diag_ptr.push_back((int64_t)h->diag.size());
    h->factor.insert(h->factor.end(), out[k].factor.begin(), out[k].factor.end());
    h->factor_ptr.push_back((int64_t)h->factor.size());
    h->sc_values.insert(h->sc_values.end(), out[k].sc.begin(), out[k].sc.end());
    h->sc_values_ptr.push_back((int64_t)h->sc_values.size());
  }
}

}  // namespace

extern "C" int fdm_hexmesh_factor(fdm_hexmesh *h, int nv, const double *X, const double *kappa_q) {
  return fdm_hexmesh_factor_axes(h, nv, X, kappa_q, nullptr);
}

extern "C" int fdm_hexmesh_factor_axes(fdm_hexmesh *h, int nv, const double *X, const double *kappa_q,
                                       const double *kaxes) {
  if (!h || !X || nv != h->nv) {
    if (h) h->err = "fdm_hexmesh_factor: need the mesh's nv vertex coordinates";
    return FDM_EINVAL;
  }
  try {
    coarse_vertices(h);
    if (kaxes && !(kaxes[0] > 0.0 && kaxes[1] > 0.0 && kaxes[2] > 0.0))
      fdm::fail(FDM_EINVAL, "fdm_hexmesh_factor_axes: the axis coefficients must be positive");
    cell_geometry(h, X, kappa_q, kaxes);
    std::vector<std::vector<int>> vcells(h->nv);
    for (int e = 0; e < h->nc; ++e)
      for (int k = 0; k < 8; ++k) vcells[h->cells[8 * (size_t)e + k]].push_back(e);
    h->diag_ptr.assign(1, 0);
    h->factor_ptr.assign(1, 0);
    h->sc_values_ptr.assign(1, 0);
    h->diag.clear();
    h->factor.clear();
    h->sc_values.clear();
    factor_stars(h, vcells);
  } catch (const fdm::Error &e) {
    return handle_hex(h, e);
  }
  return FDM_OK;
}

extern "C" int fdm_hexmesh_query(fdm_hexmesh *h, int what, void *out, size_t *len) {
  if (!h || !len) return FDM_EINVAL;
  auto put = [&](const void *src, size_t bytes) {
    if (out) {
      if (*len < bytes) {
        h->err = "fdm_hexmesh_query: buffer too small";
        return FDM_EINVAL;
      }
      if (bytes) std::copy((const char *)src, (const char *)src + bytes, (char *)out);
    }
    *len = bytes;
    return FDM_OK;
  };
  const int32_t nstar = (int32_t)h->star_vertex.size();
  switch (what) {
    case FDM_HQ_NNODE: return put(&h->nnode, sizeof(int64_t));
    case FDM_HQ_CELL_NODES: return put(h->cell_nodes.data(), h->cell_nodes.size() * sizeof(int32_t));
    case FDM_HQ_CELL_FDM: return put(h->cell_fdm.data(), h->cell_fdm.size() * sizeof(int32_t));
    case FDM_HQ_CELL_SIGN: return put(h->cell_sign.data(), h->cell_sign.size() * sizeof(int8_t));
    case FDM_HQ_DIRICHLET: return put(h->dirichlet.data(), h->dirichlet.size());
    case FDM_HQ_NSTAR: return put(&nstar, sizeof(int32_t));
    case FDM_HQ_STAR_VERTEX: return put(h->star_vertex.data(), h->star_vertex.size() * sizeof(int32_t));
    case FDM_HQ_STAR_PTR: return put(h->star_ptr.data(), h->star_ptr.size() * sizeof(int64_t));
    case FDM_HQ_STAR_NODES: return put(h->star_nodes.data(), h->star_nodes.size() * sizeof(int32_t));
    case FDM_HQ_PATTERN_PTR: return put(h->pat_ptr.data(), h->pat_ptr.size() * sizeof(int64_t));
    case FDM_HQ_PATTERN_ROWPTR: return put(h->pat_rowptr.data(), h->pat_rowptr.size() * sizeof(int64_t));
    case FDM_HQ_PATTERN_COLPTR: return put(h->pat_colptr.data(), h->pat_colptr.size() * sizeof(int64_t));
    case FDM_HQ_PATTERN_COLS: return put(h->pat_cols.data(), h->pat_cols.size() * sizeof(int32_t));
    case FDM_HQ_STAR_NINT: return put(h->star_nint.data(), h->star_nint.size() * sizeof(int32_t));
    case FDM_HQ_STAR_CLASS: return put(h->star_class.data(), h->star_class.size() * sizeof(int32_t));
    case FDM_HQ_NCLASS: {
      const int32_t nclass = (int32_t)h->class_star.size();
      return put(&nclass, sizeof(int32_t));
    }
    case FDM_HQ_CLASS_STAR: return put(h->class_star.data(), h->class_star.size() * sizeof(int32_t));
    case FDM_HQ_CLASS_NNZL: return put(h->class_nnzl.data(), h->class_nnzl.size() * sizeof(int64_t));
    case FDM_HQ_FILL_PTR: return put(h->fill_ptr.data(), h->fill_ptr.size() * sizeof(int64_t));
    case FDM_HQ_FILL_ROWPTR: return put(h->fill_rowptr.data(), h->fill_rowptr.size() * sizeof(int64_t));
    case FDM_HQ_FILL_COLPTR: return put(h->fill_colptr.data(), h->fill_colptr.size() * sizeof(int64_t));
    case FDM_HQ_FILL_COLS: return put(h->fill_cols.data(), h->fill_cols.size() * sizeof(int32_t));
    case FDM_HQ_ETREE_PTR: return put(h->etree_ptr.data(), h->etree_ptr.size() * sizeof(int64_t));
    case FDM_HQ_ETREE: return put(h->etree.data(), h->etree.size() * sizeof(int32_t));
    case FDM_HQ_MU: return put(h->mu.data(), h->mu.size() * sizeof(double));
    case FDM_HQ_SLOT_CELLS_PTR: return put(h->slot_cells_ptr.data(), h->slot_cells_ptr.size() * sizeof(int64_t));
    case FDM_HQ_SLOT_CELLS: return put(h->slot_cells.data(), h->slot_cells.size() * sizeof(int32_t));
    case FDM_HQ_SLOT_STARS_PTR: return put(h->slot_stars_ptr.data(), h->slot_stars_ptr.size() * sizeof(int64_t));
    case FDM_HQ_SLOT_STARS: return put(h->slot_stars.data(), h->slot_stars.size() * sizeof(int32_t));
    case FDM_HQ_NODE_OWNER: return put(h->node_owner.data(), h->node_owner.size() * sizeof(int32_t));
    case FDM_HQ_NODE_CELLS_PTR: return put(h->node_cells_ptr.data(), h->node_cells_ptr.size() * sizeof(int64_t));
    case FDM_HQ_NODE_CELLS: return put(h->node_cells.data(), h->node_cells.size() * sizeof(int32_t));
    case FDM_HQ_GEOM: return put(h->geom.data(), h->geom.size() * sizeof(double));
    case FDM_HQ_COARSE_OF: return put(h->coarse_of.data(), h->coarse_of.size() * sizeof(int32_t));
    case FDM_HQ_COARSE: return put(h->coarse.data(), h->coarse.size() * sizeof(double));
    case FDM_HQ_DIAG_PTR: return put(h->diag_ptr.data(), h->diag_ptr.size() * sizeof(int64_t));
    case FDM_HQ_DIAG: return put(h->diag.data(), h->diag.size() * sizeof(double));
    case FDM_HQ_FACTOR_PTR: return put(h->factor_ptr.data(), h->factor_ptr.size() * sizeof(int64_t));
    case FDM_HQ_FACTOR: return put(h->factor.data(), h->factor.size() * sizeof(double));
    case FDM_HQ_SC_SPLIT: return put(h->sc_t.data(), h->sc_t.size() * sizeof(int32_t));
    case FDM_HQ_SC_PTR: return put(h->sc_ptr.data(), h->sc_ptr.size() * sizeof(int64_t));
    case FDM_HQ_SC_ROWPTR: return put(h->sc_rowptr.data(), h->sc_rowptr.size() * sizeof(int64_t));
    case FDM_HQ_SC_COLPTR: return put(h->sc_colptr.data(), h->sc_colptr.size() * sizeof(int64_t));
    case FDM_HQ_SC_COLS: return put(h->sc_cols.data(), h->sc_cols.size() * sizeof(int32_t));
    case FDM_HQ_SC_VALUES_PTR: return put(h->sc_values_ptr.data(), h->sc_values_ptr.size() * sizeof(int64_t));
    case FDM_HQ_SC_VALUES: return put(h->sc_values.data(), h->sc_values.size() * sizeof(double));
    default:
      h->err = "fdm_hexmesh_query: unknown query";
      return FDM_EINVAL;
  }
}

extern "C" const char *fdm_hexmesh_last_error(const fdm_hexmesh *h) {
  return h ? h->err.c_str() : hex_last_error().c_str();
}

extern "C" void fdm_hexmesh_destroy(fdm_hexmesh *h) { delete h; }
