// Host construction of the 1D operators (Sections 2.1, 2.3, 2.4 of the paper):
// GLL nodes, reference stiffness/mass in the GLL Lagrange basis, the interior
// generalised eigenproblem A_II S = B_II S Lambda with S^T B_II S = I, and the
// FDM basis change T (interior functions = interpolated eigenvectors,
// interface functions B-orthogonal to them).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace fdm {

namespace {

// Legendre P_k and P_{k-1} at x by the Bonnet recursion.
void legendre_pair(int k, double x, double &pk, double &pkm1) {
  pkm1 = 1.0;
  pk = x;
  if (k == 0) { pk = 1.0; pkm1 = 0.0; return; }
  for (int j = 2; j <= k; ++j) {
    double next = ((2 * j - 1) * x * pk - (j - 1) * pkm1) / j;
    pkm1 = pk;
    pk = next;
  }
}

// Gauss-Legendre: roots of P_q by Newton, derivative from
// P_q'(x) = q (x P_q - P_{q-1}) / (x^2 - 1).
void gauss_rule(int q, std::vector<double> &x, std::vector<double> &w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < (q + 1) / 2; ++i) {
    double t = -std::cos(M_PI * (4.0 * i + 3.0) / (4.0 * q + 2.0));
    double d = 0.0;
    for (int it = 0; it < 60; ++it) {
      double pq, pm;
      legendre_pair(q, t, pq, pm);
      d = q * (t * pq - pm) / (t * t - 1.0);
      double step = pq / d;
      t -= step;
      if (std::fabs(step) < 4e-17) break;
    }
    double pq, pm;
    legendre_pair(q, t, pq, pm);
    d = q * (t * pq - pm) / (t * t - 1.0);
    x[i] = t;
    x[q - 1 - i] = -t;
    w[i] = w[q - 1 - i] = 2.0 / ((1.0 - t * t) * d * d);
  }
  if (q % 2 == 1) x[q / 2] = 0.0;
}

// GLL: x = +-1 and the roots of P_p'.  Newton on f = (1-x^2) P_p' = p (P_{p-1} - x P_p),
// f' = -p (p+1) P_p (Legendre's equation).
void gll_rule(int p, std::vector<double> &x, std::vector<double> &w) {
  x.assign(p + 1, 0.0);
  w.assign(p + 1, 0.0);
  x[0] = -1.0;
  x[p] = 1.0;
  for (int i = 1; i <= p / 2; ++i) {
    double t = -std::cos(M_PI * i / p) * (1.0 - 0.0);  // Chebyshev-Lobatto start
    for (int it = 0; it < 60; ++it) {
      double pp, pm;
      legendre_pair(p, t, pp, pm);
      double f = p * (pm - t * pp);
      double fp = -p * (p + 1.0) * pp;
      double step = f / fp;
      t -= step;
      if (std::fabs(step) < 4e-17) break;
    }
    x[i] = t;
    x[p - i] = -t;
  }
  if (p % 2 == 0) x[p / 2] = 0.0;
  for (int i = 0; i <= p; ++i) {
    double pp, pm;
    legendre_pair(p, x[i], pp, pm);
    w[i] = 2.0 / (p * (p + 1.0) * pp * pp);
  }
}

// Values and derivatives of the Lagrange basis on `nodes` at points `pts`
// (row-major m x n), barycentric form.
void lagrange_eval(const std::vector<double> &nodes, const std::vector<double> &pts,
                   std::vector<double> &V, std::vector<double> &D) {
  const int n = (int)nodes.size(), m = (int)pts.size();
  std::vector<double> bw(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) bw[j] /= (nodes[j] - nodes[k]);
  // differentiation matrix at the nodes: Dn[i][j] = (bw_j/bw_i)/(x_i-x_j), Dn[i][i] = -sum
  std::vector<double> Dn(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j)
      if (j != i) {
        Dn[i * n + j] = (bw[j] / bw[i]) / (nodes[i] - nodes[j]);
        s += Dn[i * n + j];
      }
    Dn[i * n + i] = -s;
  }
  V.assign(m * n, 0.0);
  D.assign(m * n, 0.0);
  for (int t = 0; t < m; ++t) {
    int hit = -1;
    for (int k = 0; k < n; ++k)
      if (std::fabs(pts[t] - nodes[k]) < 1e-14) hit = k;
    if (hit >= 0) {
      for (int j = 0; j < n; ++j) {
        V[t * n + j] = (j == hit) ? 1.0 : 0.0;
        D[t * n + j] = Dn[hit * n + j];
      }
      continue;
    }
    double den = 0.0;
    for (int k = 0; k < n; ++k) den += bw[k] / (pts[t] - nodes[k]);
    for (int j = 0; j < n; ++j) {
      double lj = (bw[j] / (pts[t] - nodes[j])) / den;
      double logd = 0.0;
      for (int k = 0; k < n; ++k)
        if (k != j) logd += 1.0 / (pts[t] - nodes[k]);
      V[t * n + j] = lj;
      D[t * n + j] = lj * logd;
    }
  }
}

// Symmetric eigen-decomposition: Householder reduction to tridiagonal form,
// eigenvalues by Sturm-sequence bisection, eigenvectors by inverse iteration
// on the tridiagonal matrix, then back-transformation.  a (m x m, row-major)
// is overwritten by the eigenvectors (columns); d receives the eigenvalues
// in ascending order.  Intended for small matrices with distinct eigenvalues.
void sym_eig(int m, std::vector<double> &a, std::vector<double> &d) {
  std::vector<double> Q(m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[i * m + i] = 1.0;
  std::vector<double> v(m);
  for (int k = 0; k + 2 < m; ++k) {
    double nx = 0.0;
    for (int i = k + 1; i < m; ++i) nx += a[i * m + k] * a[i * m + k];
    nx = std::sqrt(nx);
    if (nx == 0.0) continue;
    double x0 = a[(k + 1) * m + k];
    double alpha = x0 >= 0 ? -nx : nx;
    for (int i = 0; i < m; ++i) v[i] = 0.0;
    for (int i = k + 1; i < m; ++i) v[i] = a[i * m + k];
    v[k + 1] -= alpha;
    double vv = 0.0;
    for (int i = k + 1; i < m; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    // a <- H a H with H = I - 2 v v^T / vv
    for (int j = 0; j < m; ++j) {  // left: rows
      double s = 0.0;
      for (int i = k + 1; i < m; ++i) s += v[i] * a[i * m + j];
      s *= 2.0 / vv;
      for (int i = k + 1; i < m; ++i) a[i * m + j] -= s * v[i];
    }
    for (int i = 0; i < m; ++i) {  // right: columns
      double s = 0.0;
      for (int j = k + 1; j < m; ++j) s += a[i * m + j] * v[j];
      s *= 2.0 / vv;
      for (int j = k + 1; j < m; ++j) a[i * m + j] -= s * v[j];
    }
    for (int i = 0; i < m; ++i) {  // Q <- Q H
      double s = 0.0;
      for (int j = k + 1; j < m; ++j) s += Q[i * m + j] * v[j];
      s *= 2.0 / vv;
      for (int j = k + 1; j < m; ++j) Q[i * m + j] -= s * v[j];
    }
  }
  std::vector<double> diag(m), off(m > 1 ? m - 1 : 1, 0.0);
  for (int i = 0; i < m; ++i) diag[i] = a[i * m + i];
  for (int i = 0; i + 1 < m; ++i) off[i] = 0.5 * (a[(i + 1) * m + i] + a[i * m + i + 1]);
  // Sturm count: number of eigenvalues < x
  auto count_below = [&](double x) {
    int c = 0;
    double q = 1.0;
    for (int i = 0; i < m; ++i) {
      double b2 = i > 0 ? off[i - 1] * off[i - 1] : 0.0;
      q = diag[i] - x - (i > 0 ? b2 / q : 0.0);
      if (q == 0.0) q = -1e-300;
      if (q < 0.0) ++c;
    }
    return c;
  };
  double lo = diag[0], hi = diag[0];
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(off[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(off[i]) : 0.0);
    lo = std::min(lo, diag[i] - r);
    hi = std::max(hi, diag[i] + r);
  }
  d.assign(m, 0.0);
  for (int k = 0; k < m; ++k) {  // k-th smallest eigenvalue
    double l = lo, h = hi;
    for (int it = 0; it < 200 && h - l > 2e-16 * std::max(std::fabs(l), std::fabs(h)); ++it) {
      double mid = 0.5 * (l + h);
      if (count_below(mid) > k) h = mid; else l = mid;
    }
    d[k] = 0.5 * (l + h);
  }
  // inverse iteration on (tri - lambda) with a Thomas solve (tiny shift)
  std::vector<double> Y(m * m, 0.0), y(m), rhs(m), cp(m), dp(m);
  for (int k = 0; k < m; ++k) {
    double shift = d[k] + 1e-13 * std::max(1.0, std::fabs(d[k]));
    for (int i = 0; i < m; ++i) rhs[i] = 1.0 + 0.01 * ((i * 7 + k * 3) % 11);
    for (int it = 0; it < 3; ++it) {
      // Gaussian elimination with partial pivoting on the tridiagonal system
      std::vector<double> M(m * m, 0.0);
      for (int i = 0; i < m; ++i) {
        M[i * m + i] = diag[i] - shift;
        if (i + 1 < m) M[i * m + i + 1] = M[(i + 1) * m + i] = off[i];
      }
      for (int i = 0; i < m; ++i) y[i] = rhs[i];
      for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < std::min(m, c + 2); ++r)
          if (std::fabs(M[r * m + c]) > std::fabs(M[piv * m + c])) piv = r;
        if (piv != c) {
          for (int j = 0; j < m; ++j) std::swap(M[c * m + j], M[piv * m + j]);
          std::swap(y[c], y[piv]);
        }
        double pv = M[c * m + c];
        if (pv == 0.0) pv = M[c * m + c] = 1e-300;
        for (int r = c + 1; r < std::min(m, c + 2); ++r) {
          double f = M[r * m + c] / pv;
          for (int j = c; j < m; ++j) M[r * m + j] -= f * M[c * m + j];
          y[r] -= f * y[c];
        }
      }
      for (int c = m - 1; c >= 0; --c) {
        double s = y[c];
        for (int j = c + 1; j < m; ++j) s -= M[c * m + j] * y[j];
        y[c] = s / M[c * m + c];
      }
      double nrm = 0.0;
      for (int i = 0; i < m; ++i) nrm += y[i] * y[i];
      nrm = std::sqrt(nrm);
      for (int i = 0; i < m; ++i) rhs[i] = y[i] / nrm;
    }
    // orthogonalise against previous vectors (eigenvalues are distinct; this
    // only removes rounding)
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += Y[i * m + j] * rhs[i];
      for (int i = 0; i < m; ++i) rhs[i] -= s * Y[i * m + j];
    }
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += rhs[i] * rhs[i];
    nrm = std::sqrt(nrm);
    for (int i = 0; i < m; ++i) Y[i * m + k] = rhs[i] / nrm;
  }
  for (int i = 0; i < m; ++i)  // a = Q Y
    for (int k = 0; k < m; ++k) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += Q[i * m + j] * Y[j * m + k];
      a[i * m + k] = s;
    }
}

// In-place lower Cholesky of an m x m row-major SPD matrix.
void chol_lower(int m, std::vector<double> &a) {
  for (int j = 0; j < m; ++j) {
    for (int k = 0; k < j; ++k)
      for (int i = j; i < m; ++i) a[i * m + j] -= a[i * m + k] * a[j * m + k];
    if (!(a[j * m + j] > 0.0)) fail(FDM_ENOTSPD, "basis: interior mass matrix not SPD");
    double s = std::sqrt(a[j * m + j]);
    for (int i = j; i < m; ++i) a[i * m + j] /= s;
    for (int i = 0; i < j; ++i) a[i * m + j] = 0.0;
  }
}

}  // namespace

// The generalised eigenpairs of the whole-element pencil (A, B): A s = lam B s,
// S^T B S = I (Section 2.3's fast diagonalisation on all n nodes), as the rows
// of V = S^T B (so that A = V^T diag(lam) V and B = V^T V).  A and B are
// symmetric about the element centre, so every mode is even or odd there; the
// modes are ordered even first (ascending lam within each group), and each row
// of V is made exactly even or odd (averaged with its mirror image), since the
// kernels read only its first ceil(n/2) entries.
void cell_modes(Basis1D &b) {
  const int n = b.n;
  std::vector<double> L = b.B, C(n * n, 0.0), W(n * n, 0.0);
  chol_lower(n, L);
  for (int c = 0; c < n; ++c)  // W = L^{-1} A
    for (int i = 0; i < n; ++i) {
      double s = b.A[i * n + c];
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * W[k * n + c];
      W[i * n + c] = s / L[i * n + i];
    }
  for (int c = 0; c < n; ++c)  // C = L^{-1} W^T = L^{-1} A L^{-T}
    for (int i = 0; i < n; ++i) {
      double s = W[c * n + i];
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * C[k * n + c];
      C[i * n + c] = s / L[i * n + i];
    }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < i; ++j) C[i * n + j] = C[j * n + i] = 0.5 * (C[i * n + j] + C[j * n + i]);
  std::vector<double> ev;
  sym_eig(n, C, ev);  // eigenvectors q in the columns of C
  std::vector<double> S(n * n);
  for (int j = 0; j < n; ++j)  // s = L^{-T} q
    for (int i = n - 1; i >= 0; --i) {
      double v = C[i * n + j];
      for (int k = i + 1; k < n; ++k) v -= L[k * n + i] * S[k * n + j];
      S[i * n + j] = v / L[i * n + i];
    }
  std::vector<int> even, odd;
  for (int j = 0; j < n; ++j) {
    double sym = 0.0, nrm = 0.0;
    for (int i = 0; i < n; ++i) {
      sym += S[i * n + j] * S[(n - 1 - i) * n + j];
      nrm += S[i * n + j] * S[i * n + j];
    }
    if (std::fabs(std::fabs(sym) - nrm) > 1e-8 * nrm) fail(FDM_EINVAL, "basis: an element mode is neither even nor odd");
    (sym > 0 ? even : odd).push_back(j);
  }
  auto by_lam = [&](int a, int c) { return ev[a] < ev[c]; };
  std::sort(even.begin(), even.end(), by_lam);
  std::sort(odd.begin(), odd.end(), by_lam);
  if ((int)even.size() != (n + 1) / 2) fail(FDM_EINVAL, "basis: unexpected number of even element modes");
  std::vector<int> ord = even;
  ord.insert(ord.end(), odd.begin(), odd.end());
  b.Ve.assign(n * n, 0.0);
  b.lame.assign(n, 0.0);
  for (int k = 0; k < n; ++k) {
    const int j = ord[k];
    const double par = k < (n + 1) / 2 ? 1.0 : -1.0;
    b.lame[k] = ev[j];
    std::vector<double> v(n, 0.0);
    for (int c = 0; c < n; ++c)
      for (int i = 0; i < n; ++i) v[c] += S[i * n + j] * b.B[i * n + c];
    for (int c = 0; c < n; ++c) {
      const int cm = n - 1 - c;
      b.Ve[k * n + c] = c == cm ? (par > 0 ? v[c] : 0.0) : 0.5 * (v[c] + par * v[cm]);
    }
  }
}

Basis1D make_basis(int p) {
  if (p < 1 || p > PMAX) fail(FDM_EINVAL, "degree p must be in [1, 31]");
  Basis1D b;
  b.p = p;
  b.n = p + 1;
  const int n = b.n, m = p - 1;
  gll_rule(p, b.xi, b.wgll);
  gauss_rule(n, b.xq, b.wq);
  lagrange_eval(b.xi, b.xq, b.Vq, b.Dq);
  b.A.assign(n * n, 0.0);
  b.B.assign(n * n, 0.0);
  for (int t = 0; t < n; ++t)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        b.A[i * n + j] += b.wq[t] * b.Dq[t * n + i] * b.Dq[t * n + j];
        b.B[i * n + j] += b.wq[t] * b.Vq[t * n + i] * b.Vq[t * n + j];
      }
  b.T.assign(n * n, 0.0);
  b.T[0] = 1.0;
  b.T[p * n + p] = 1.0;
  if (m > 0) {
    std::vector<double> L(m * m), C(m * m, 0.0), W(m * m, 0.0);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) L[i * m + j] = b.B[(i + 1) * n + j + 1];
    chol_lower(m, L);
    // C = L^{-1} A_II L^{-T}: W = L^{-1} A_II, C = (L^{-1} W^T)
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < m; ++i) {
        double s = b.A[(i + 1) * n + c + 1];
        for (int k = 0; k < i; ++k) s -= L[i * m + k] * W[k * m + c];
        W[i * m + c] = s / L[i * m + i];
      }
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < m; ++i) {
        double s = W[c * m + i];
        for (int k = 0; k < i; ++k) s -= L[i * m + k] * C[k * m + c];
        C[i * m + c] = s / L[i * m + i];
      }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < i; ++j) C[i * m + j] = C[j * m + i] = 0.5 * (C[i * m + j] + C[j * m + i]);
    std::vector<double> ev;
    sym_eig(m, C, ev);  // C now holds eigenvectors Q in columns
    std::vector<int> ord(m);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int c) { return ev[a] < ev[c]; });
    b.S.assign(m * m, 0.0);
    b.lam.assign(m, 0.0);
    for (int jj = 0; jj < m; ++jj) {
      int j = ord[jj];
      b.lam[jj] = ev[j];
      // s = L^{-T} q
      std::vector<double> s(m);
      for (int i = m - 1; i >= 0; --i) {
        double v = C[i * m + j];
        for (int k = i + 1; k < m; ++k) v -= L[k * m + i] * s[k];
        s[i] = v / L[i * m + i];
      }
      double sg = s[0] < 0 ? -1.0 : 1.0;
      for (int i = 0; i < m; ++i) b.S[i * m + jj] = sg * s[i];
    }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) b.T[(i + 1) * n + j + 1] = b.S[i * m + j];
    // interface functions: T[I,e] = -B_II^{-1} B_{I,e}
    for (int e = 0; e <= p; e += p) {
      std::vector<double> y(m);
      for (int i = 0; i < m; ++i) {
        double v = -b.B[(i + 1) * n + e];
        for (int k = 0; k < i; ++k) v -= L[i * m + k] * y[k];
        y[i] = v / L[i * m + i];
      }
      for (int i = m - 1; i >= 0; --i) {
        double v = y[i];
        for (int k = i + 1; k < m; ++k) v -= L[k * m + i] * y[k];
        y[i] = v / L[i * m + i];
      }
      for (int i = 0; i < m; ++i) b.T[(i + 1) * n + e] = y[i];
    }
  }
  // FDM-basis matrices
  std::vector<double> AT(n * n, 0.0), BT(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        AT[i * n + j] += b.A[i * n + k] * b.T[k * n + j];
        BT[i * n + j] += b.B[i * n + k] * b.T[k * n + j];
      }
  b.Af.assign(n * n, 0.0);
  b.Bf.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int k = 0; k < n; ++k) {
        b.Af[i * n + j] += b.T[k * n + i] * AT[k * n + j];
        b.Bf[i * n + j] += b.T[k * n + i] * BT[k * n + j];
      }
  double amax = 0.0, bmax = 0.0;
  for (int i = 0; i < n * n; ++i) {
    amax = std::max(amax, std::fabs(b.Af[i]));
    bmax = std::max(bmax, std::fabs(b.Bf[i]));
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      bool ii = i > 0 && i < p, jj = j > 0 && j < p;
      if (ii && jj && i != j) {
        if (std::fabs(b.Af[i * n + j]) > 1e-12 * amax || std::fabs(b.Bf[i * n + j]) > 1e-12 * bmax)
          fail(FDM_EINVAL, "basis: FDM interior block is not diagonal");
        b.Af[i * n + j] = b.Bf[i * n + j] = 0.0;
      }
      if (ii != jj) {
        if (std::fabs(b.Bf[i * n + j]) > 1e-12 * bmax) fail(FDM_EINVAL, "basis: FDM mass coupling");
        b.Bf[i * n + j] = 0.0;
      }
    }
  cell_modes(b);
  return b;
}

}  // namespace fdm
