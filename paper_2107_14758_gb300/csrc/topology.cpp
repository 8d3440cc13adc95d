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
#include <functional>
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

std::vector<PatchClass> build_classes(int p, bool sc) {
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
    // gather sources of every interface dof: the star cells whose closure holds it
    // (slot = side_x + 2 side_y + 4 side_z), in slot order
    C.gsrc.assign((size_t)8 * C.nG, -1);
    for (int i = 0; i < C.nG; ++i) {
      int pos = C.gpos[i];
      int tt[3] = {pos % C.dim[0], (pos / C.dim[0]) % C.dim[1], pos / (C.dim[0] * C.dim[1])};
      int cnt = 0;
      for (int slot = 0; slot < 8; ++slot) {
        int l[3];
        bool ok = true;
        for (int a = 0; a < 3 && ok; ++a) {
          int side = (slot >> a) & 1;
          if (!C.full[a]) { ok = side == 0; l[a] = tt[a] + 1; }
          else if (side == 0) { ok = tt[a] <= c; l[a] = tt[a] + 1; }
          else { ok = tt[a] >= c; l[a] = tt[a] - c; }
        }
        if (ok) C.gsrc[(size_t)8 * i + cnt++] = (slot << 16) | (l[0] + (p + 1) * (l[1] + (p + 1) * l[2]));
      }
    }
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
    const std::vector<Bits> col0 = col;  // the pattern of S_G itself (before fill)
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
    // the Schur-coupling form keeps only the level-1 rows (L10); the top rows'
    // level-0 couplings live in S_TB there
    if (sc) {
      C.nrow0 = C.n1;
      rowcols.resize(C.n1);
    }
    C.K0 = 0;
    for (auto &v : rowcols) C.K0 = std::max(C.K0, (int)v.size());
    C.ldr0 = (C.nrow0 + 3) & ~3;
    C.ell_col.assign((size_t)C.K0 * C.ldr0, -1);
    std::vector<std::vector<int>> colpos(C.n0);
    for (int r = 0; r < C.nrow0; ++r)
      for (size_t e = 0; e < rowcols[r].size(); ++e) {
        C.ell_col[e * C.ldr0 + r] = rowcols[r][e];
        colpos[rowcols[r][e]].push_back((int)(e * C.ldr0 + r));
      }
    C.c0_ptr.assign(C.n0 + 1, 0);
    for (int j = 0; j < C.n0; ++j) {
      std::sort(colpos[j].begin(), colpos[j].end());  // ascending slice, then row
      for (int q : colpos[j]) C.c0_pos.push_back(q);
      C.c0_ptr[j + 1] = (int)C.c0_pos.size();
    }
    // level-0 columns restricted to the level-1 rows (the lower block B of
    // the Schur-coupling form)
    C.cB_ptr.assign(C.n0 + 1, 0);
    for (int j = 0; j < C.n0; ++j) {
      for (int q = C.c0_ptr[j]; q < C.c0_ptr[j + 1]; ++q)
        if (C.c0_pos[q] % C.ldr0 < C.n1) C.cB_pos.push_back(C.c0_pos[q]);
      C.cB_ptr[j + 1] = (int)C.cB_pos.size();
    }
    // --- Schur-coupling form: the top rows of S_G in the columns of levels 0
    // and 1, S_TB, with S's own pattern (no fill): ELL by top rows and, for
    // S_BT = S_TB^T, the positions of each lower column in ascending order ---
    auto up4 = [](int64_t x) { return (x + 3) & ~int64_t(3); };
    const int nb = C.n0 + C.n1;
    C.ldT = (int)up4(C.n2);
    std::vector<std::vector<int>> trow(C.n2);
    for (int cc = 0; cc < nb; ++cc)
      for (int r = col0[cc].first_from(nb); r >= 0; r = col0[cc].first_from(r + 1)) trow[r - nb].push_back(cc);
    C.KT = 0;
    for (auto &v : trow) C.KT = std::max(C.KT, (int)v.size());
    C.st_col.assign((size_t)C.KT * C.ldT, -1);
    std::vector<std::vector<int>> tpos(nb);
    for (int t = 0; t < C.n2; ++t)
      for (size_t e = 0; e < trow[t].size(); ++e) {
        C.st_col[e * C.ldT + t] = trow[t][e];
        tpos[trow[t][e]].push_back((int)(e * C.ldT + t));
      }
    C.ct_ptr.assign(nb + 1, 0);
    for (int cc = 0; cc < nb; ++cc) {
      std::sort(tpos[cc].begin(), tpos[cc].end());
      for (int q : tpos[cc]) C.ct_pos.push_back(q);
      C.ct_ptr[cc + 1] = (int)C.ct_pos.size();
    }
    C.nnzST = (int64_t)C.ct_pos.size();
    // stored nonzeros of the Schur-coupling form: level-0 pivots, L10, the line
    // blocks of L11 (lower triangles), S_TB, the lower triangle of W
    C.nnzSC = C.n0 + (int64_t)C.cB_pos.size() + C.nnzST + (int64_t)C.n2 * (C.n2 + 1) / 2;
    for (int b = 0; b < C.nlines; ++b) C.nnzSC += (int64_t)C.line_len[b] * (C.line_len[b] + 1) / 2;
    // --- value layout of one patch (elements), 16-byte aligned sections ---
    C.sc = sc;
    C.ld21 = (int)up4(C.n1);
    int64_t off = 0;
    C.off_dinv0 = off;
    off = up4(off + C.n0);
    C.off_ell = off;
    off = up4(off + (int64_t)C.K0 * C.ldr0);
    C.off_lines = off;
    for (int b = 0; b < C.nlines; ++b) {
      C.line_off.push_back((int)(off - C.off_lines));
      off = up4(off + (int64_t)C.line_len[b] * C.line_len[b]);
    }
    // L form: the dense L21 block; Schur-coupling form: the values of S_TB
    C.off_l21 = off;
    C.off_st = off;
    off = sc ? up4(off + (int64_t)C.KT * C.ldT) : up4(off + (int64_t)C.n2 * C.ld21);
    // top level by rows, each padded to 4: Z = L_top^{-1} (lower triangular; L
    // form) or the lower triangle of W = Z^T Z = (L_top L_top^T)^{-1} (Schur-
    // coupling form)
    C.off_z = off;
    C.zoff.assign(C.n2 + 1, 0);
    for (int r = 0; r < C.n2; ++r) C.zoff[r + 1] = C.zoff[r] + (int)up4(r + 1);
    off += C.zoff[C.n2];
    C.nval = up4(off);
  }
  return out;
}

// Chunk schedule of the streamed patch solve for one class: the factor
// sections in the order the forward solve reads them, then the backward
// solve's sections in reverse, cut into bulk copies of at most cap_bytes
// (whole rows, lines or ELL slices; 16-byte multiples, 16-byte aligned).
std::vector<ChunkDev> build_schedule(const PatchClass &C, int es, int cap) {
  std::vector<ChunkDev> f, out;
  if (C.nG == 0) return out;
  auto up16 = [](int64_t b) { return (int)((b + 15) & ~int64_t(15)); };
  auto need = [&](int64_t b) {
    if (b > cap) fail(FDM_EINVAL, "stream schedule: one row does not fit a chunk buffer");
  };
  // groups [i, j) of consecutive items of sizes sz(i) into chunks
  auto cut = [&](int kind, int nitems, std::function<int64_t(int)> off, std::function<int64_t(int)> sz) {
    std::vector<ChunkDev> v;
    int i = 0;
    while (i < nitems) {
      int64_t b = 0;
      int j = i;
      while (j < nitems && b + sz(j) * es <= cap) b += sz(j++) * es;
      if (j == i) need(sz(i) * es);
      v.push_back({kind, i, j, up16(b), off(i)});
      i = j;
    }
    return v;
  };
  std::vector<ChunkDev> ell, lines, l21, z;
  if (C.n0 > 0) {
    need((int64_t)C.n0 * es);
    f.push_back({CK_DINV, 0, C.n0, up16((int64_t)C.n0 * es), C.off_dinv0});
  }
  if (C.K0 > 0 && C.nrow0 > 0)
    ell = cut(CK_ELL_F, C.K0, [&](int e) { return C.off_ell + (int64_t)e * C.ldr0; },
              [&](int) { return (int64_t)C.ldr0; });
  if (C.nlines > 0)
    lines = cut(CK_LINES_F, C.nlines, [&](int b) { return C.off_lines + C.line_off[b]; },
                [&](int b) { return (int64_t)((C.line_len[b] * C.line_len[b] + 3) & ~3); });
  if (C.n2 > 0 && C.n1 > 0)
    l21 = cut(CK_L21_F, C.n2, [&](int r) { return C.off_l21 + (int64_t)r * C.ld21; },
              [&](int) { return (int64_t)C.ld21; });
  if (C.n2 > 0)
    z = cut(CK_Z_F, C.n2, [&](int r) { return C.off_z + C.zoff[r]; },
            [&](int r) { return (int64_t)(C.zoff[r + 1] - C.zoff[r]); });
  auto flag = [](std::vector<ChunkDev> &v, int kind) {
    for (size_t i = 0; i < v.size(); ++i)
      v[i].kind = kind | ((i == 0) << 8) | ((i + 1 == v.size()) << 9);
  };
  out = f;
  for (auto *sec : {&ell, &lines, &l21, &z}) out.insert(out.end(), sec->begin(), sec->end());
  // backward: Z, L21, lines, ELL, each visited from its last chunk
  const std::pair<std::vector<ChunkDev> *, int> back[4] = {{&z, CK_Z_B}, {&l21, CK_L21_B}, {&lines, CK_LINES_B},
                                                           {&ell, CK_ELL_B}};
  for (auto &bk : back) {
    std::vector<ChunkDev> v(bk.first->rbegin(), bk.first->rend());
    flag(v, bk.second);
    out.insert(out.end(), v.begin(), v.end());
  }
  return out;
}

}  // namespace fdm
