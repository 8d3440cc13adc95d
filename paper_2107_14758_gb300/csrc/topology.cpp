// Vertex-star patch classes and their symbolic factorisation (Sections 2.5,
// 2.6 of the paper).
//
// In the FDM basis every patch matrix A_j has interior-first block form with
// A_II diagonal (Section 2.6), so only the interface Schur complement S_G is
// factorised.  The interface is ordered by nested dissection on the vertex
// planes of the star (the entity-graph nested dissection of Section 2.6 on a
// structured star): with F the full axes of the star in x, y, z order,
//   level 2: dofs on the plane of F[0]                        (dense block)
//   level 1: dofs on the plane of F[1] but not of F[0]        (independent
//            lines along F[2], one per coordinate of the remaining axis)
//   level 0: dofs only on the plane of F[2]                   (diagonal)
// (for stars with fewer full axes the top levels drop out).  One symbolic
// factorisation serves all patches of a class; the numeric values differ per
// patch.
#include <algorithm>
#include <cstring>
#include <map>

#include "internal.h"

namespace fdm {

namespace {

struct Bits {
  int nw = 0;
  std::vector<uint64_t> w;
  explicit Bits(int n = 0) : nw((n + 63) / 64), w(nw, 0) {}
  void set(int i) { w[i >> 6] |= (1ull << (i & 63)); }
  bool get(int i) const { return (w[i >> 6] >> (i & 63)) & 1ull; }
  void clear(int i) { w[i >> 6] &= ~(1ull << (i & 63)); }
  void merge(const Bits &o) {
    for (int k = 0; k < nw; ++k) w[k] |= o.w[k];
  }
  int first_from(int i) const {  // first set bit >= i, or -1
    for (int k = i >> 6; k < nw; ++k) {
      uint64_t m = w[k];
      if (k == (i >> 6)) m &= (~0ull) << (i & 63);
      if (m) return (k << 6) + __builtin_ctzll(m);
    }
    return -1;
  }
};

inline bool isv(int i, int p) { return i == 0 || i == p; }
inline bool bf_nz(int i, int j, int p) { return i == j || (isv(i, p) && isv(j, p)); }
inline bool af_nz(int i, int j, int p) { return i == j || isv(i, p) || isv(j, p); }

}  // namespace

std::vector<PatchClass> build_classes(int p) {
  std::vector<PatchClass> out(8);
  for (int id = 0; id < 8; ++id) {
    PatchClass &C = out[id];
    C.id = id;
    for (int a = 0; a < 3; ++a) {
      C.full[a] = (id >> a) & 1;
      C.dim[a] = C.full[a] ? 2 * p - 1 : p - 1;
    }
    C.nd = C.dim[0] * C.dim[1] * C.dim[2];
    if (C.nd == 0) continue;
    const int c = p - 1;  // local coordinate of the vertex plane on full axes
    std::vector<int> F;
    for (int a = 0; a < 3; ++a)
      if (C.full[a]) F.push_back(a);
    const int k = (int)F.size();
    // --- classify and order the interface ---
    struct Key {
      int lev, a, b, c;
      int pos;
    };
    std::vector<Key> keys;
    for (int tz = 0; tz < C.dim[2]; ++tz)
      for (int ty = 0; ty < C.dim[1]; ++ty)
        for (int tx = 0; tx < C.dim[0]; ++tx) {
          int t[3] = {tx, ty, tz};
          int lev = -1;
          for (int i = 0; i < k; ++i)
            if (t[F[i]] == c) { lev = k - 1 - i; break; }
          int pos = tx + C.dim[0] * (ty + C.dim[1] * tz);
          if (lev < 0) { ++C.nI; continue; }
          Key K{lev, 0, 0, 0, pos};
          if (lev == 0) { K.a = tz; K.b = ty; K.c = tx; }
          else if (lev == 1) {
            int plane = F[k - 2], line = F[k - 1], other = 3 - plane - line;
            K.a = t[other]; K.b = t[line]; K.c = 0;
          } else { K.a = tz; K.b = ty; K.c = tx; }
          keys.push_back(K);
        }
    std::sort(keys.begin(), keys.end(), [](const Key &x, const Key &y) {
      if (x.lev != y.lev) return x.lev < y.lev;
      if (x.a != y.a) return x.a < y.a;
      if (x.b != y.b) return x.b < y.b;
      return x.c < y.c;
    });
    C.nG = (int)keys.size();
    const int m = C.nG;
    C.gpos.resize(m);
    std::vector<int> gindex(C.nd, -1);  // star position -> interface index
    for (int i = 0; i < m; ++i) {
      C.gpos[i] = keys[i].pos;
      gindex[keys[i].pos] = i;
      if (keys[i].lev == 0) C.n0++;
      else if (keys[i].lev == 1) C.n1++;
      else C.n2++;
    }
    for (int i = C.n0; i < C.n0 + C.n1; ++i) {  // lines of level 1
      if (i == C.n0 || keys[i].a != keys[i - 1].a) {
        C.line_start.push_back(i - C.n0);
        C.line_len.push_back(0);
      }
      C.line_len.back()++;
    }
    C.nlines = (int)C.line_start.size();
    C.ginv = gindex;
    C.line_of.assign(C.n1, 0);
    for (int b = 0; b < C.nlines; ++b)
      for (int i = 0; i < C.line_len[b]; ++i) C.line_of[C.line_start[b] + i] = b;
    if (m == 0) continue;
    // --- structural pattern of S_G ---
    std::vector<Bits> col(m, Bits(m));  // lower part: col[j] has rows > j
    auto add = [&](int a, int b) {
      if (a == b) return;
      if (a < b) std::swap(a, b);
      col[b].set(a);
    };
    int ncell[3], cell_lo[3][2];
    for (int a = 0; a < 3; ++a) ncell[a] = C.full[a] ? 2 : 1;
    // star cells: along a full axis, side 0 covers t in [0, p-1] (cell-local t+1),
    // side 1 covers t in [p-1, 2p-2] (local t-(p-1)); clipped: t in [0, p-2] (local t+1)
    auto local = [&](int a, int side, int t) {
      return (C.full[a] && side == 1) ? t - (p - 1) : t + 1;
    };
    (void)cell_lo;
    for (int sz = 0; sz < ncell[2]; ++sz)
      for (int sy = 0; sy < ncell[1]; ++sy)
        for (int sx = 0; sx < ncell[0]; ++sx) {
          int side[3] = {sx, sy, sz};
          // star dofs in the closure of this cell
          std::vector<int> rng[3];
          for (int a = 0; a < 3; ++a)
            for (int t = 0; t < C.dim[a]; ++t) {
              int l = local(a, side[a], t);
              if (l >= 0 && l <= p) rng[a].push_back(t);
            }
          std::vector<int> gam;  // (pos) of interface dofs in this cell
          std::vector<int> loc3;
          for (int tz : rng[2])
            for (int ty : rng[1])
              for (int tx : rng[0]) {
                int pos = tx + C.dim[0] * (ty + C.dim[1] * tz);
                if (gindex[pos] >= 0) {
                  gam.push_back(pos);
                  loc3.push_back(local(0, sx, tx) | (local(1, sy, ty) << 8) | (local(2, sz, tz) << 16));
                }
              }
          // A_GG couplings inside the cell
          for (size_t u = 0; u < gam.size(); ++u)
            for (size_t v = 0; v < u; ++v) {
              int iu = loc3[u] & 255, ju = (loc3[u] >> 8) & 255, ku = loc3[u] >> 16;
              int iv = loc3[v] & 255, jv = (loc3[v] >> 8) & 255, kv = loc3[v] >> 16;
              bool nz = (bf_nz(ku, kv, p) && bf_nz(ju, jv, p) && af_nz(iu, iv, p)) ||
                        (bf_nz(ku, kv, p) && af_nz(ju, jv, p) && bf_nz(iu, iv, p)) ||
                        (af_nz(ku, kv, p) && bf_nz(ju, jv, p) && bf_nz(iu, iv, p));
              if (nz) add(gindex[gam[u]], gindex[gam[v]]);
            }
          // Schur fill: interior dof (i,j,k) couples to the star-facing face dofs
          // of this cell with the same tangential coordinates
          for (int tz : rng[2])
            for (int ty : rng[1])
              for (int tx : rng[0]) {
                int t[3] = {tx, ty, tz};
                bool interior = true;
                for (int a = 0; a < 3; ++a)
                  if (C.full[a] && t[a] == c) interior = false;
                int li[3] = {local(0, sx, tx), local(1, sy, ty), local(2, sz, tz)};
                for (int a = 0; a < 3; ++a)
                  if (li[a] == 0 || li[a] == p) interior = false;
                if (!interior) continue;
                int fc[3], nf = 0;
                for (int a = 0; a < 3; ++a) {
                  if (!C.full[a]) continue;
                  int tt[3] = {tx, ty, tz};
                  tt[a] = c;
                  fc[nf++] = gindex[tt[0] + C.dim[0] * (tt[1] + C.dim[1] * tt[2])];
                }
                for (int u = 0; u < nf; ++u)
                  for (int v = 0; v < u; ++v) add(fc[u], fc[v]);
              }
        }
    // --- symbolic Cholesky via the elimination tree ---
    for (int j = 0; j < m; ++j) {
      int par = col[j].first_from(j + 1);
      if (par >= 0) {
        Bits t = col[j];
        t.clear(par);
        col[par].merge(t);
      }
    }
    C.pattern.assign((size_t)m * m, 0);
    C.nnzL = m;
    for (int j = 0; j < m; ++j) {
      C.pattern[(size_t)j * m + j] = 1;
      for (int r = col[j].first_from(j + 1); r >= 0; r = col[j].first_from(r + 1)) {
        C.pattern[(size_t)r * m + j] = 1;
        C.nnzL++;
      }
    }
    // --- checks of the level structure ---
    for (int j = 0; j < C.n0; ++j) {
      int r = col[j].first_from(j + 1);
      if (r >= 0 && r < C.n0) fail(FDM_EINVAL, "symbolic: level 0 block is not diagonal");
    }
    for (int b = 0; b < C.nlines; ++b) {
      int s = C.n0 + C.line_start[b], e = s + C.line_len[b];
      for (int j = s; j < e; ++j)
        for (int r = col[j].first_from(j + 1); r >= 0 && r < C.n0 + C.n1; r = col[j].first_from(r + 1))
          if (r >= e) fail(FDM_EINVAL, "symbolic: level 1 lines are coupled");
    }
    // --- level-0 off-diagonal block: ELL by rows, CSC positions per column ---
    C.nrow0 = m - C.n0;
    std::vector<std::vector<int>> rowcols(C.nrow0);
    C.r0_ptr.assign(C.n0 + 1, 0);
    for (int j = 0; j < C.n0; ++j) {
      for (int r = col[j].first_from(j + 1); r >= 0; r = col[j].first_from(r + 1)) {
        rowcols[r - C.n0].push_back(j);
        C.r0_idx.push_back(r);
      }
      C.r0_ptr[j + 1] = (int)C.r0_idx.size();
    }
    C.K0 = 0;
    for (auto &v : rowcols) C.K0 = std::max(C.K0, (int)v.size());
    C.ell_col.assign((size_t)C.K0 * C.nrow0, -1);
    std::vector<std::vector<int>> colpos(C.n0);
    for (int r = 0; r < C.nrow0; ++r)
      for (size_t e = 0; e < rowcols[r].size(); ++e) {
        C.ell_col[e * C.nrow0 + r] = rowcols[r][e];
        colpos[rowcols[r][e]].push_back((int)(e * C.nrow0 + r));
      }
    C.c0_ptr.assign(C.n0 + 1, 0);
    for (int j = 0; j < C.n0; ++j) {
      for (int q : colpos[j]) C.c0_pos.push_back(q);
      C.c0_ptr[j + 1] = (int)C.c0_pos.size();
    }
    // --- value layout of one patch (elements), 16-byte aligned sections ---
    auto up4 = [](int64_t x) { return (x + 3) & ~int64_t(3); };
    C.ld21 = (int)up4(C.n1);
    C.npanel = (C.n2 + PANEL - 1) / PANEL;
    int64_t off = 0;
    C.off_dinv0 = off;
    off = up4(off + C.n0);
    C.off_ell = off;
    off = up4(off + (int64_t)C.K0 * C.nrow0);
    C.off_lines = off;
    for (int b = 0; b < C.nlines; ++b) {
      C.line_off.push_back((int)(off - C.off_lines));
      off = up4(off + (int64_t)C.line_len[b] * C.line_len[b]);
    }
    C.off_l21 = off;
    off = up4(off + (int64_t)C.n2 * C.ld21);
    C.off_pan = off;
    for (int q = 0; q < C.npanel; ++q) {
      C.pan_off.push_back((int)(off - C.off_pan));
      off += (int64_t)(C.n2 - q * PANEL) * PANEL;
    }
    C.nval = up4(off);
  }
  return out;
}

}  // namespace fdm
