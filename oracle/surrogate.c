/*
 * surrogate.c -- FP64 CPU reference of the learned separable surrogate
 * (TEST INFRASTRUCTURE ONLY; see oracle.h).
 *
 * The paper (Section 2.7) replaces the stiffness of a curved cell by a
 * separable surrogate with one scaling mu_j per reference direction, and
 * Theorem 1 bounds the spectrum of the true cell stiffness against the
 * surrogate by the extreme eigenvalues, over the cell's quadrature points,
 * of D^{-1/2} (kappa Ghat) D^{-1/2}, D = diag(mu).  The paper takes mu_j as
 * the cell average of kappa Ghat_jj.  Here a small network predicts a
 * per-direction correction c, mu = mu_avg exp(c), from 27 samples of kappa
 * and the Jacobian per cell; its training label is the mu that minimises
 * the Theorem 1 bound ratio of the cell.  Every function below is the plain
 * definition, written out.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

/* kappa |det J| J^{-1} J^{-T} at one point (Section 2.7), 6 entries
 * (00, 11, 22, 01, 02, 12).  Returns -1 for a singular J. */
static int ghat(const double *J, double kap, double *G) {
  double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
               J[2] * (J[3] * J[7] - J[4] * J[6]);
  if (!(det != 0.0)) return -1;
  double Ji[9];
  Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
  Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
  Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
  double M[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double s = 0.0;
      for (int r = 0; r < 3; ++r) s += Ji[a * 3 + r] * Ji[b * 3 + r];
      M[a][b] = kap * fabs(det) * s;
    }
  G[0] = M[0][0]; G[1] = M[1][1]; G[2] = M[2][2];
  G[3] = M[0][1]; G[4] = M[0][2]; G[5] = M[1][2];
  return 0;
}

/* eigenpairs of a symmetric 3x3 matrix by cyclic Jacobi rotations (until the
 * off-diagonal part is negligible); lam[i] with unit eigenvector V[.][i] */
static void eig3(double a[3][3], double lam[3], double V[3][3]) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-34 * dia) break;
    for (int p = 0; p < 2; ++p)
      for (int q = p + 1; q < 3; ++q) {
        if (a[p][q] == 0.0) continue;
        double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < 3; ++k) { /* A <- A R, V <- V R */
          double x = a[k][p], y = a[k][q];
          a[k][p] = cs * x - sn * y;
          a[k][q] = sn * x + cs * y;
          x = V[k][p]; y = V[k][q];
          V[k][p] = cs * x - sn * y;
          V[k][q] = sn * x + cs * y;
        }
        for (int k = 0; k < 3; ++k) { /* A <- R^T A */
          double x = a[p][k], y = a[q][k];
          a[p][k] = cs * x - sn * y;
          a[q][k] = sn * x + cs * y;
        }
      }
  }
  lam[0] = a[0][0]; lam[1] = a[1][1]; lam[2] = a[2][2];
}

/* the bound over the points, with unit eigenvectors of the extreme pairs
 * (first point attaining the extreme, in point order) */
static double bound_vec(int nq, const double *G, const double *mu, double *lo_o, double *hi_o,
                        double vlo[3], double vhi[3]) {
  double lo = INFINITY, hi = -INFINITY;
  double s[3] = {1.0 / sqrt(mu[0]), 1.0 / sqrt(mu[1]), 1.0 / sqrt(mu[2])};
  for (int q = 0; q < nq; ++q) {
    const double *g = G + 6 * (size_t)q;
    double a[3][3] = {{g[0] * s[0] * s[0], g[3] * s[0] * s[1], g[4] * s[0] * s[2]},
                      {g[3] * s[0] * s[1], g[1] * s[1] * s[1], g[5] * s[1] * s[2]},
                      {g[4] * s[0] * s[2], g[5] * s[1] * s[2], g[2] * s[2] * s[2]}};
    double lam[3], V[3][3];
    eig3(a, lam, V);
    for (int i = 0; i < 3; ++i) {
      if (lam[i] < lo) {
        lo = lam[i];
        if (vlo) for (int k = 0; k < 3; ++k) vlo[k] = V[k][i];
      }
      if (lam[i] > hi) {
        hi = lam[i];
        if (vhi) for (int k = 0; k < 3; ++k) vhi[k] = V[k][i];
      }
    }
  }
  if (lo_o) *lo_o = lo;
  if (hi_o) *hi_o = hi;
  return log(hi / lo);
}

double or_surr_bound(int nq, const double *G, const double *mu, double *lo_o, double *hi_o) {
  return bound_vec(nq, G, mu, lo_o, hi_o, NULL, NULL);
}

/* Theorem 1 optimum.  With mu = mubar exp(u) the ratio F(u) = log(hi/lo) is
 * convex in u (log hi is a maximum of log-sum-exp functions of -u, -log lo
 * one of u) and invariant to u -> u + t (1,1,1), so u = (0, x1, x2) and F is
 * minimised over x by the central-cut ellipsoid method: a subgradient of
 * log lambda in u_a is -v_a^2 for the unit eigenvector v of the scaled
 * matrix, so g_a = v_lo,a^2 - v_hi,a^2.  Start: x = 0 in the disc of radius
 * OR_SURR_RADIUS; stop when sqrt(g^T P g), a bound on F(x) - min F inside
 * the ellipsoid, falls below OR_SURR_TOL or after OR_SURR_MAXIT steps.  The
 * best point seen (strict improvement) is returned. */
static double label_one(int nq, const double *G, const double *mubar, double *u) {
  /* the ellipsoid {x + B z : |z| <= 1} is kept through its factor B (P = B B^T),
   * updated as B <- (2/sqrt(3)) B (I + (1/sqrt(3) - 1) e e^T), e = B^T g / |B^T g|,
   * the n = 2 central cut, which keeps P positive semi-definite in rounding */
  double x[2] = {0.0, 0.0};
  double B[2][2] = {{OR_SURR_RADIUS, 0.0}, {0.0, OR_SURR_RADIUS}};
  double best = INFINITY, bx[2] = {0.0, 0.0};
  const double a = 2.0 / sqrt(3.0), b = 1.0 / sqrt(3.0) - 1.0;
  for (int it = 0; it < OR_SURR_MAXIT; ++it) {
    double mu[3] = {mubar[0], mubar[1] * exp(x[0]), mubar[2] * exp(x[1])};
    double vlo[3], vhi[3];
    double F = bound_vec(nq, G, mu, NULL, NULL, vlo, vhi);
    if (F < best) { best = F; bx[0] = x[0]; bx[1] = x[1]; }
    double g[2] = {vlo[1] * vlo[1] - vhi[1] * vhi[1], vlo[2] * vlo[2] - vhi[2] * vhi[2]};
    double Bg[2] = {B[0][0] * g[0] + B[1][0] * g[1], B[0][1] * g[0] + B[1][1] * g[1]}; /* B^T g */
    double r = sqrt(Bg[0] * Bg[0] + Bg[1] * Bg[1]);
    if (!(r > OR_SURR_TOL)) break;
    double e[2] = {Bg[0] / r, Bg[1] / r};
    double Be[2] = {B[0][0] * e[0] + B[0][1] * e[1], B[1][0] * e[0] + B[1][1] * e[1]};
    x[0] -= Be[0] / 3.0;
    x[1] -= Be[1] / 3.0;
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) B[i][j] = a * (B[i][j] + b * Be[i] * e[j]);
  }
  u[0] = 0.0; u[1] = bx[0]; u[2] = bx[1];
  return best;
}

int or_surr_cell_ghat(int p, int ncell, const double *jac, const double *kappa, double *G,
                      double *mubar) {
  int n = p + 1, nq = n * n * n;
  double xg[OR_PMAX + 1], wg[OR_PMAX + 1];
  if (p < 1 || p > OR_PMAX) return -1;
  or_gauss(n, xg, wg);
  for (int e = 0; e < ncell; ++e) {
    double avg[3] = {0, 0, 0};
    for (int k = 0; k < n; ++k)
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          int q = i + n * (j + n * k);
          double *g = G + ((size_t)e * nq + q) * 6;
          if (ghat(jac + ((size_t)e * nq + q) * 9, kappa ? kappa[(size_t)e * nq + q] : 1.0, g)) return -1;
          double w = wg[i] * wg[j] * wg[k];
          for (int a = 0; a < 3; ++a) avg[a] += w * g[a];
        }
    for (int a = 0; a < 3; ++a) mubar[3 * e + a] = avg[a] / 8.0; /* |K_hat| = 8 */
  }
  return 0;
}

int or_surr_label(int p, int ncell, const double *jac, const double *kappa, double *mubar,
                  double *cstar, double *F0, double *F1) {
  int n = p + 1, nq = n * n * n;
  double *G = (double *)malloc(sizeof(double) * 6 * (size_t)nq * ncell);
  if (!G) return -1;
  if (or_surr_cell_ghat(p, ncell, jac, kappa, G, mubar)) { free(G); return -1; }
#pragma omp parallel for schedule(dynamic)
  for (int e = 0; e < ncell; ++e) {
    const double *Ge = G + (size_t)e * nq * 6;
    double u[3], lo, hi, mu[3];
    F0[e] = or_surr_bound(nq, Ge, mubar + 3 * e, NULL, NULL);
    F1[e] = label_one(nq, Ge, mubar + 3 * e, u);
    for (int a = 0; a < 3; ++a) mu[a] = mubar[3 * e + a] * exp(u[a]);
    or_surr_bound(nq, Ge, mu, &lo, &hi);
    /* scale so that the bound's spectrum is centred (lo * hi = 1) */
    for (int a = 0; a < 3; ++a) cstar[3 * e + a] = u[a] + 0.5 * log(lo * hi);
  }
  free(G);
  return 0;
}

int or_surr_features(int ncell, const double *s27, double *feat) {
  double xg[3], wg[3];
  or_gauss(3, xg, wg);
  for (int e = 0; e < ncell; ++e) {
    double G[27][6], lk[27], nu[3] = {0, 0, 0}, lbar = 0.0;
    for (int q = 0; q < 27; ++q) {
      const double *s = s27 + ((size_t)e * 27 + q) * 10;
      if (!(s[0] > 0.0)) return -1;
      if (ghat(s + 1, s[0], G[q])) return -1;
      lk[q] = log(s[0]);
      double w = wg[q % 3] * wg[(q / 3) % 3] * wg[q / 9];
      for (int a = 0; a < 3; ++a) nu[a] += w * G[q][a] / 8.0;
      lbar += w * lk[q] / 8.0;
    }
    double *f = feat + (size_t)e * OR_MLP_NIN;
    for (int q = 0; q < 27; ++q) {
      f[7 * q + 0] = lk[q] - lbar;
      for (int a = 0; a < 3; ++a) f[7 * q + 1 + a] = log(G[q][a] / nu[a]);
      f[7 * q + 4] = G[q][3] / sqrt(G[q][0] * G[q][1]);
      f[7 * q + 5] = G[q][4] / sqrt(G[q][0] * G[q][2]);
      f[7 * q + 6] = G[q][5] / sqrt(G[q][1] * G[q][2]);
    }
  }
  return 0;
}

/* parameter blocks, in storage order */
#define W1 0
#define B1 (W1 + OR_MLP_NH * OR_MLP_NIN)
#define W2 (B1 + OR_MLP_NH)
#define B2 (W2 + OR_MLP_NH * OR_MLP_NH)
#define W3 (B2 + OR_MLP_NH)
#define B3 (W3 + OR_MLP_NOUT * OR_MLP_NH)

/* one cell: hidden activations and outputs */
static void forward_one(const double *P, const double *f, double *h1, double *h2, double *c) {
  for (int j = 0; j < OR_MLP_NH; ++j) {
    double s = P[B1 + j];
    for (int k = 0; k < OR_MLP_NIN; ++k) s += P[W1 + j * OR_MLP_NIN + k] * f[k];
    h1[j] = tanh(s);
  }
  for (int j = 0; j < OR_MLP_NH; ++j) {
    double s = P[B2 + j];
    for (int k = 0; k < OR_MLP_NH; ++k) s += P[W2 + j * OR_MLP_NH + k] * h1[k];
    h2[j] = tanh(s);
  }
  for (int o = 0; o < OR_MLP_NOUT; ++o) {
    double s = P[B3 + o];
    for (int k = 0; k < OR_MLP_NH; ++k) s += P[W3 + o * OR_MLP_NH + k] * h2[k];
    c[o] = s;
  }
}

void or_mlp_forward(int ncell, const double *P, const double *feat, double *c) {
  double h1[OR_MLP_NH], h2[OR_MLP_NH];
  for (int e = 0; e < ncell; ++e)
    forward_one(P, feat + (size_t)e * OR_MLP_NIN, h1, h2, c + 3 * (size_t)e);
}

/* loss = (1 / (2 ncell)) sum_e sum_o (c_eo - label_eo)^2 and its gradient,
 * by the chain rule through the three layers (d tanh(s)/ds = 1 - tanh^2) */
double or_mlp_loss_grad(int ncell, const double *P, const double *feat, const double *label,
                        double *grad) {
  double h1[OR_MLP_NH], h2[OR_MLP_NH], c[OR_MLP_NOUT], d1[OR_MLP_NH], d2[OR_MLP_NH], d3[OR_MLP_NOUT];
  double loss = 0.0;
  if (grad) memset(grad, 0, sizeof(double) * OR_MLP_NPARAM);
  for (int e = 0; e < ncell; ++e) {
    const double *f = feat + (size_t)e * OR_MLP_NIN;
    forward_one(P, f, h1, h2, c);
    for (int o = 0; o < OR_MLP_NOUT; ++o) {
      double r = c[o] - label[3 * (size_t)e + o];
      loss += 0.5 * r * r / ncell;
      d3[o] = r / ncell;
    }
    if (!grad) continue;
    for (int k = 0; k < OR_MLP_NH; ++k) {
      double s = 0.0;
      for (int o = 0; o < OR_MLP_NOUT; ++o) s += P[W3 + o * OR_MLP_NH + k] * d3[o];
      d2[k] = s * (1.0 - h2[k] * h2[k]);
    }
    for (int k = 0; k < OR_MLP_NH; ++k) {
      double s = 0.0;
      for (int j = 0; j < OR_MLP_NH; ++j) s += P[W2 + j * OR_MLP_NH + k] * d2[j];
      d1[k] = s * (1.0 - h1[k] * h1[k]);
    }
    for (int o = 0; o < OR_MLP_NOUT; ++o) {
      grad[B3 + o] += d3[o];
      for (int k = 0; k < OR_MLP_NH; ++k) grad[W3 + o * OR_MLP_NH + k] += d3[o] * h2[k];
    }
    for (int j = 0; j < OR_MLP_NH; ++j) {
      grad[B2 + j] += d2[j];
      for (int k = 0; k < OR_MLP_NH; ++k) grad[W2 + j * OR_MLP_NH + k] += d2[j] * h1[k];
    }
    for (int j = 0; j < OR_MLP_NH; ++j) {
      grad[B1 + j] += d1[j];
      for (int k = 0; k < OR_MLP_NIN; ++k) grad[W1 + j * OR_MLP_NIN + k] += d1[j] * f[k];
    }
  }
  return loss;
}

/* Adam (Kingma & Ba, 2015), step t >= 1, with bias-corrected moments */
void or_mlp_adam(int nparam, double *P, const double *g, double *m, double *v, int t, double lr) {
  const double b1 = OR_ADAM_BETA1, b2 = OR_ADAM_BETA2, eps = OR_ADAM_EPS;
  double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int i = 0; i < nparam; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    P[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

int or_surr_apply(int ncell, const double *mubar, const double *c, double *mu) {
  int nfall = 0;
  for (int e = 0; e < ncell; ++e) {
    int ok = 1;
    for (int a = 0; a < 3; ++a)
      if (!isfinite(c[3 * e + a]) || fabs(c[3 * e + a]) > OR_SURR_CMAX) ok = 0;
    for (int a = 0; a < 3; ++a) mu[3 * e + a] = ok ? mubar[3 * e + a] * exp(c[3 * e + a]) : mubar[3 * e + a];
    nfall += !ok;
  }
  return nfall;
}
