// Host set-up of the SIPG star solves (Section 5): the 1D two-cell pencils of
// a Cartesian vertex star and their generalized eigendecompositions.
//
// Along one axis a star holds cells c0 = k - 1 and c1 = k of the vertex k.
// In the GLL basis of each cell (reference interval [-1, 1], half-widths h)
// the pencil's stiffness is blockdiag(A_hat / h0, A_hat / h1) plus the 1D
// normal parts of the facet terms of the weak form: the facet between the two
// cells in full, and at each outer end the star cell's own block only (the
// principal submatrix: the cell beyond contributes no values).  Per facet,
// with J the jump of the traces along the facet normal and G the normal
// derivative, averaged on an interior facet, the 1D term is
// sigma J J^T - J G^T - G J^T, sigma = eta h_e^{-1}: eta (1/h^- + 1/h^+) / 4
// on an interior facet, eta / (2 h) on a boundary one.  The mass is
// blockdiag(h0 B_hat, h1 B_hat).
#include <cmath>
#include <string>
#include <vector>

#include "internal.h"

namespace fdm {

void sipg_end_derivatives(const std::vector<double> &xi, std::vector<double> &dm, std::vector<double> &dp) {
  // derivatives of the Lagrange polynomials at the first and last node from
  // the barycentric form: l_j'(x_i) = (w_j / w_i) / (x_i - x_j), i != j,
  // l_i'(x_i) = -sum_{j != i} l_j'(x_i)
  const int n = (int)xi.size();
  std::vector<double> w(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) w[j] /= xi[j] - xi[k];
  dm.assign(n, 0.0);
  dp.assign(n, 0.0);
  for (int e = 0; e < 2; ++e) {
    const int i = e ? n - 1 : 0;
    std::vector<double> &d = e ? dp : dm;
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      d[j] = (w[j] / w[i]) / (xi[i] - xi[j]);
      diag -= d[j];
    }
    d[i] = diag;
  }
}

void sipg_star_pencil(int n, const double *A1, const double *B1, const double *dm, const double *dp, double eta,
                      double h0, double h1, double hl, double hr, double *A, double *M) {
  const int m = 2 * n;
  for (int t = 0; t < m * m; ++t) A[t] = M[t] = 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      A[i * m + j] = A1[i * n + j] / h0;
      A[(n + i) * m + n + j] = A1[i * n + j] / h1;
      M[i * m + j] = B1[i * n + j] * h0;
      M[(n + i) * m + n + j] = B1[i * n + j] * h1;
    }
  std::vector<double> J(m), G(m);
  auto add = [&](double sigma) {
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) A[i * m + j] += sigma * J[i] * J[j] - J[i] * G[j] - G[i] * J[j];
  };
  // the facet between the star's cells: J = [e_end; -e_0], G = ([l'(1)/h0; l'(-1)/h1]) / 2
  std::fill(J.begin(), J.end(), 0.0);
  std::fill(G.begin(), G.end(), 0.0);
  J[n - 1] = 1.0;
  J[n] = -1.0;
  for (int i = 0; i < n; ++i) {
    G[i] = 0.5 * dp[i] / h0;
    G[n + i] = 0.5 * dm[i] / h1;
  }
  add(eta * 0.25 * (1.0 / h0 + 1.0 / h1));
  // the low end of c0: a boundary facet (hl <= 0) or an interior one with the cell beyond
  std::fill(J.begin(), J.end(), 0.0);
  std::fill(G.begin(), G.end(), 0.0);
  J[0] = -1.0;
  for (int i = 0; i < n; ++i) G[i] = (hl > 0.0 ? 0.5 : 1.0) * dm[i] / h0;
  add(hl > 0.0 ? eta * 0.25 * (1.0 / hl + 1.0 / h0) : eta / (2.0 * h0));
  // the high end of c1
  std::fill(J.begin(), J.end(), 0.0);
  std::fill(G.begin(), G.end(), 0.0);
  J[m - 1] = 1.0;
  for (int i = 0; i < n; ++i) G[n + i] = (hr > 0.0 ? 0.5 : 1.0) * dp[i] / h1;
  add(hr > 0.0 ? eta * 0.25 * (1.0 / h1 + 1.0 / hr) : eta / (2.0 * h1));
}

void sym_gen_eig(int m, const double *A, const double *M, double *S, double *lam) {
  // M = L L^T (Cholesky), C = L^{-1} A L^{-T}, C = Q diag(lam) Q^T by cyclic
  // Jacobi rotations, S = L^{-T} Q: S^T A S = diag(lam), S^T M S = I
  std::vector<double> L(M, M + (size_t)m * m);
  for (int j = 0; j < m; ++j) {
    double d = L[j * m + j];
    for (int k = 0; k < j; ++k) d -= L[j * m + k] * L[j * m + k];
    if (!(d > 0.0)) fail(FDM_ENOTSPD, "SIPG star pencil: mass matrix is not positive definite");
    d = std::sqrt(d);
    L[j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double s = L[i * m + j];
      for (int k = 0; k < j; ++k) s -= L[i * m + k] * L[j * m + k];
      L[i * m + j] = s / d;
    }
    for (int i = 0; i < j; ++i) L[i * m + j] = 0.0;
  }
  // C = L^{-1} A L^{-T}: forward substitution on the columns, then on the rows
  std::vector<double> W(A, A + (size_t)m * m), C((size_t)m * m);
  for (int c = 0; c < m; ++c)
    for (int i = 0; i < m; ++i) {
      double s = W[i * m + c];
      for (int k = 0; k < i; ++k) s -= L[i * m + k] * W[k * m + c];
      W[i * m + c] = s / L[i * m + i];
    }
  for (int r = 0; r < m; ++r)
    for (int j = 0; j < m; ++j) {
      double s = W[r * m + j];
      for (int k = 0; k < j; ++k) s -= L[j * m + k] * C[r * m + k];
      C[r * m + j] = s / L[j * m + j];
    }
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < i; ++j) C[i * m + j] = C[j * m + i] = 0.5 * (C[i * m + j] + C[j * m + i]);
  std::vector<double> Q((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[i * m + i] = 1.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < m; ++i) {
      diag += C[i * m + i] * C[i * m + i];
      for (int j = i + 1; j < m; ++j) off += C[i * m + j] * C[i * m + j];
    }
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = C[p * m + q];
        if (apq == 0.0) continue;
        const double theta = (C[q * m + q] - C[p * m + p]) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < m; ++r) {
          if (r == p || r == q) continue;
          const double crp = C[r * m + p], crq = C[r * m + q];
          C[r * m + p] = C[p * m + r] = c * crp - s * crq;
          C[r * m + q] = C[q * m + r] = s * crp + c * crq;
        }
        C[p * m + p] -= t * apq;
        C[q * m + q] += t * apq;
        C[p * m + q] = C[q * m + p] = 0.0;
        for (int r = 0; r < m; ++r) {
          const double qrp = Q[r * m + p], qrq = Q[r * m + q];
          Q[r * m + p] = c * qrp - s * qrq;
          Q[r * m + q] = s * qrp + c * qrq;
        }
      }
  }
  for (int i = 0; i < m; ++i) {
    lam[i] = C[i * m + i];
    if (!(lam[i] > 0.0)) fail(FDM_ENOTSPD, "SIPG star pencil: stiffness is not positive definite");
  }
  // S = L^{-T} Q: back substitution with L^T per column
  for (int c = 0; c < m; ++c)
    for (int i = m - 1; i >= 0; --i) {
      double s = Q[i * m + c];
      for (int k = i + 1; k < m; ++k) s -= L[k * m + i] * S[k * m + c];
      S[i * m + c] = s / L[i * m + i];
    }
}

}  // namespace fdm
