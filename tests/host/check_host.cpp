// Host-logic checks of the library without a GPU: the patch-class tables of
// both factor forms (level sizes, Schur-coupling tables, value layout) and the
// Galerkin coarsening of the multigrid levels against the Q1 stiffness
// assembled directly on the coarsened mesh.  Prints one line per check.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "../../paper_2107_14758_gb300/csrc/internal.h"

namespace fdm {
[[noreturn]] void fail(int code, const std::string &msg) {
  std::printf("FAIL %d %s\n", code, msg.c_str());
  std::exit(1);
}
}  // namespace fdm
using namespace fdm;

static int topology() {
  int bad = 0;
  for (int p = 1; p <= 15; ++p)
    for (int sc = 0; sc < 2; ++sc) {
      const std::vector<PatchClass> cls = build_classes(p, sc != 0);
      for (const PatchClass &C : cls) {
        if (C.nG == 0) continue;
        const int nb = C.n0 + C.n1;
        bool ok = C.n0 + C.n1 + C.n2 == C.nG && C.nval % 4 == 0 && C.off_z % 4 == 0 && C.off_lines % 4 == 0;
        for (int b = 0; b < C.nlines; ++b) ok = ok && C.line_len[b] <= 31;
        if (sc) {
          ok = ok && C.ldT == ((C.n2 + 3) & ~3) && (int)C.st_col.size() == C.KT * C.ldT && C.off_st % 4 == 0 &&
               C.off_st + (int64_t)C.KT * C.ldT <= C.off_z && C.off_z + C.zoff[C.n2] <= C.nval && C.nrow0 == C.n1;
          for (size_t q = 0; q < C.st_col.size(); ++q) {
            const int col = C.st_col[q], t = (int)(q % C.ldT);
            ok = ok && col >= -1 && col < nb && !(col >= 0 && t >= C.n2);
          }
          int cnt = 0;
          for (int cc = 0; cc < nb; ++cc)
            for (int q = C.ct_ptr[cc]; q < C.ct_ptr[cc + 1]; ++q, ++cnt) ok = ok && C.st_col[C.ct_pos[q]] == cc;
          ok = ok && cnt == C.nnzST;
          for (int j = 0; j < C.n0; ++j)
            for (int q = C.cB_ptr[j]; q < C.cB_ptr[j + 1]; ++q)
              ok = ok && C.cB_pos[q] % C.ldr0 < C.n1 && C.ell_col[C.cB_pos[q]] == j;
        } else {
          ok = ok && C.off_l21 + (int64_t)C.n2 * C.ld21 <= C.off_z && C.nrow0 == C.nG - C.n0;
        }
        std::printf("topology p=%d sc=%d cls=%d nG=%d n0=%d n1=%d n2=%d nnzL=%lld nnzSC=%lld nval=%lld ok=%d\n", p, sc,
                    C.id, C.nG, C.n0, C.n1, C.n2, (long long)C.nnzL, (long long)C.nnzSC, (long long)C.nval, ok ? 1 : 0);
        bad += !ok;
      }
    }
  return bad;
}

// Q1 stiffness of a tensor mesh with vertex coordinates x[3] as a 27-point
// stencil over the free vertices (closed-form 1D matrices)
static GmgHostLevel q1_level(const std::vector<double> x[3]) {
  GmgHostLevel L;
  for (int a = 0; a < 3; ++a) {
    L.n[a] = (int)x[a].size() - 1;
    L.m[a] = L.n[a] - 1;
    L.x[a] = x[a];
  }
  L.nf = L.m[0] * L.m[1] * L.m[2];
  L.A.assign((size_t)27 * L.nf, 0.0);
  for (int cz = 0; cz < L.n[2]; ++cz)
    for (int cy = 0; cy < L.n[1]; ++cy)
      for (int cx = 0; cx < L.n[0]; ++cx) {
        const int c[3] = {cx, cy, cz};
        double h[3];
        for (int a = 0; a < 3; ++a) h[a] = x[a][c[a] + 1] - x[a][c[a]];
        for (int t = 0; t < 8; ++t)
          for (int s = 0; s < 8; ++s) {
            const int bt[3] = {t & 1, (t >> 1) & 1, t >> 2}, bs[3] = {s & 1, (s >> 1) & 1, s >> 2};
            double k = 0.0;
            for (int d = 0; d < 3; ++d) {
              double term = 1.0;
              for (int a = 0; a < 3; ++a) {
                const bool same = bt[a] == bs[a];
                term *= a == d ? (same ? 1.0 : -1.0) / h[a] : h[a] / 6.0 * (same ? 2.0 : 1.0);
              }
              k += term;
            }
            int vt[3], vs[3];
            bool free = true;
            for (int a = 0; a < 3; ++a) {
              vt[a] = c[a] + bt[a];
              vs[a] = c[a] + bs[a];
              free = free && vt[a] > 0 && vt[a] < L.n[a] && vs[a] > 0 && vs[a] < L.n[a];
            }
            if (!free) continue;
            const int i = (vt[0] - 1) + L.m[0] * ((vt[1] - 1) + L.m[1] * (vt[2] - 1));
            const int kk = (vs[0] - vt[0] + 1) + 3 * (vs[1] - vt[1] + 1) + 9 * (vs[2] - vt[2] + 1);
            L.A[(size_t)kk * L.nf + i] += k;
          }
      }
  return L;
}

static int gmg() {
  std::vector<double> x[3];
  const int n[3] = {8, 12, 8};
  unsigned s = 12345u;
  for (int a = 0; a < 3; ++a) {  // graded: widths in [0.5, 1.5) from a fixed LCG
    x[a].assign(1, 0.0);
    for (int i = 0; i < n[a]; ++i) {
      s = s * 1664525u + 1013904223u;
      x[a].push_back(x[a].back() + 0.5 + (s >> 8) / 16777216.0);
    }
  }
  std::vector<GmgHostLevel> lev{q1_level(x)};
  gmg_coarsen(lev, 5);
  int bad = 0;
  for (size_t l = 1; l < lev.size(); ++l) {
    std::vector<double> xc[3];
    for (int a = 0; a < 3; ++a)
      for (size_t i = 0; i < lev[l - 1].x[a].size(); i += 2) xc[a].push_back(lev[l - 1].x[a][i]);
    const GmgHostLevel ref = q1_level(xc);
    double err = 0.0, mx = 0.0;
    for (size_t q = 0; q < ref.A.size(); ++q) {
      err = std::max(err, std::fabs(ref.A[q] - lev[l].A[q]));
      mx = std::max(mx, std::fabs(ref.A[q]));
    }
    const bool ok = ref.nf == lev[l].nf && err <= 1e-12 * mx;
    std::printf("gmg level=%zu n=%d,%d,%d nf=%d relerr=%.3e ok=%d\n", l, lev[l].n[0], lev[l].n[1], lev[l].n[2],
                lev[l].nf, err / mx, ok ? 1 : 0);
    bad += !ok;
  }
  std::printf("gmg levels=%zu\n", lev.size() - 1);
  return bad + (lev.size() == 3 ? 0 : 1);  // 8x12x8 -> 4x6x4 -> 2x3x2 (3 is odd: stop)
}

// prints the end derivatives, the 1D star pencil (A, M) and its generalized
// eigendecomposition (S, lam) for p, eta and the half-widths h0 h1 hl hr
static int sipg(int argc, char **argv) {
  if (argc < 8) return 1;
  const int p = std::atoi(argv[2]), n = p + 1, m = 2 * n;
  const double eta = std::atof(argv[3]), h0 = std::atof(argv[4]), h1 = std::atof(argv[5]), hl = std::atof(argv[6]),
               hr = std::atof(argv[7]);
  const Basis1D b = make_basis(p);
  std::vector<double> dm, dp, A(m * m), M(m * m), S(m * m), lam(m);
  sipg_end_derivatives(b.xi, dm, dp);
  sipg_star_pencil(n, b.A.data(), b.B.data(), dm.data(), dp.data(), eta, h0, h1, hl, hr, A.data(), M.data());
  sym_gen_eig(m, A.data(), M.data(), S.data(), lam.data());
  auto put = [](const char *name, const std::vector<double> &v) {
    std::printf("%s", name);
    for (double x : v) std::printf(" %.17g", x);
    std::printf("\n");
  };
  put("dm", dm);
  put("dp", dp);
  put("A", A);
  put("M", M);
  put("S", S);
  put("lam", lam);
  return 0;
}

// prints the library's 1D basis for degree p (Sections 2.1-2.4)
static int basis(int argc, char **argv) {
  if (argc < 3) return 1;
  const Basis1D b = make_basis(std::atoi(argv[2]));
  auto put = [](const char *name, const std::vector<double> &v) {
    std::printf("%s", name);
    for (double x : v) std::printf(" %.17g", x);
    std::printf("\n");
  };
  put("xi", b.xi);
  put("wgll", b.wgll);
  put("A", b.A);
  put("B", b.B);
  put("S", b.S);
  put("lam", b.lam);
  put("T", b.T);
  put("Af", b.Af);
  put("Bf", b.Bf);
  put("Ve", b.Ve);
  put("lame", b.lame);
  return 0;
}

int main(int argc, char **argv) {
  const std::string what = argc > 1 ? argv[1] : "all";
  if (what == "sipg") return sipg(argc, argv);
  if (what == "basis") return basis(argc, argv);
  int bad = 0;
  if (what == "topology" || what == "all") bad += topology();
  if (what == "gmg" || what == "all") bad += gmg();
  std::printf("bad=%d\n", bad);
  return bad != 0;
}
