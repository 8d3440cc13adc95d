/*
 * oracle.c -- plain FP64 CPU reference of the vertex-star FDM/sparse
 * relaxation (arXiv 2107.14758).  TEST INFRASTRUCTURE ONLY: see oracle.h.
 *
 * Every routine follows the paper's definitions directly, in its order and
 * notation, with no blocking or fusion beyond applying a Kronecker product
 * one axis at a time (the meaning of the Kronecker symbol in eq. (kron)).
 */
#include "oracle.h"

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static char g_err[512];
static void set_err(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
const char *or_last_error(void) { return g_err; }

/* ======================================================================
 * 1D: Legendre polynomials, Gauss and Gauss-Lobatto rules (Section 2.1)
 * ====================================================================== */

/* P_k(x) and P_k'(x) by the three-term recurrence; the derivative from
 * (1-x^2) P_k' = k (P_{k-1} - x P_k), with the closed form at x = +-1. */
static void legendre(int k, double x, double *P, double *dP) {
  if (k == 0) { *P = 1.0; *dP = 0.0; return; }
  double pm1 = 1.0, pk = x;
  for (int j = 1; j < k; ++j) {
    double pn = ((2.0 * j + 1.0) * x * pk - j * pm1) / (j + 1.0);
    pm1 = pk;
    pk = pn;
  }
  *P = pk;
  double omx2 = 1.0 - x * x;
  if (fabs(omx2) < 1e-14) {
    double s = (x > 0 || (k - 1) % 2 == 0) ? 1.0 : -1.0;
    *dP = s * 0.5 * k * (k + 1.0);
  } else {
    *dP = k * (pm1 - x * pk) / omx2;
  }
}

int or_gauss(int q, double *x, double *w) {
  if (q < 1 || q > 64) { set_err("gauss: bad q=%d", q); return -1; }
  for (int i = 0; i < q; ++i) {
    /* root i (descending) of P_q: Newton from a Chebyshev-type guess */
    double t = cos(M_PI * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    double P, dP;
    legendre(q, t, &P, &dP);
    x[q - 1 - i] = t;
    w[q - 1 - i] = 2.0 / ((1.0 - t * t) * dP * dP);
  }
  return 0;
}

int or_gll(int p, double *xi, double *w) {
  if (p < 1 || p > OR_PMAX) { set_err("gll: bad p=%d", p); return -1; }
  xi[0] = -1.0;
  xi[p] = 1.0;
  for (int i = 1; i < p; ++i) {
    /* interior roots of P_p': Newton with P_p'' = (2x P_p' - p(p+1) P_p)/(1-x^2) */
    double t = -cos(M_PI * i / p);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(p, t, &P, &dP);
      double d2P = (2.0 * t * dP - p * (p + 1.0) * P) / (1.0 - t * t);
      double dt = dP / d2P;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    xi[i] = t;
  }
  for (int i = 0; i <= p; ++i) {
    double P, dP;
    legendre(p, xi[i], &P, &dP);
    w[i] = 2.0 / (p * (p + 1.0) * P * P);
  }
  return 0;
}

void or_lagrange(int p, const double *xi, int m, const double *x, double *V, double *D) {
  int n = p + 1;
  for (int t = 0; t < m; ++t) {
    for (int j = 0; j < n; ++j) {
      double v = 1.0;
      for (int k = 0; k < n; ++k)
        if (k != j) v *= (x[t] - xi[k]) / (xi[j] - xi[k]);
      double d = 0.0;
      for (int mm = 0; mm < n; ++mm) {
        if (mm == j) continue;
        double term = 1.0 / (xi[j] - xi[mm]);
        for (int k = 0; k < n; ++k)
          if (k != j && k != mm) term *= (x[t] - xi[k]) / (xi[j] - xi[k]);
        d += term;
      }
      if (V) V[t * n + j] = v;
      if (D) D[t * n + j] = d;
    }
  }
}

/* ======================================================================
 * small dense linear algebra (row-major)
 * ====================================================================== */

int or_cholesky(int m, double *S) {
  for (int j = 0; j < m; ++j) {
    double d = S[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= S[(size_t)j * m + k] * S[(size_t)j * m + k];
    if (!(d > 0.0)) { set_err("cholesky: pivot %d = %g <= 0", j, d); return -1; }
    double ljj = sqrt(d);
    S[(size_t)j * m + j] = ljj;
    for (int i = j + 1; i < m; ++i) {
      double s = S[(size_t)i * m + j];
      const double *Li = S + (size_t)i * m, *Lj = S + (size_t)j * m;
      for (int k = 0; k < j; ++k) s -= Li[k] * Lj[k];
      S[(size_t)i * m + j] = s / ljj;
    }
  }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) S[(size_t)i * m + j] = 0.0;
  return 0;
}

/* solve L y = b then L^T x = y in place (L lower, row-major m x m) */
static void chol_solve(int m, const double *L, double *b) {
  for (int i = 0; i < m; ++i) {
    double s = b[i];
    for (int k = 0; k < i; ++k) s -= L[(size_t)i * m + k] * b[k];
    b[i] = s / L[(size_t)i * m + i];
  }
  for (int i = m - 1; i >= 0; --i) {
    double s = b[i];
    for (int k = i + 1; k < m; ++k) s -= L[(size_t)k * m + i] * b[k];
    b[i] = s / L[(size_t)i * m + i];
  }
}

/* cyclic Jacobi eigenvalue algorithm for a symmetric m x m matrix C;
 * on return C is (numerically) diagonal and Q holds the eigenvectors
 * in its columns: C_in = Q diag Q^T. */
static void jacobi_eig(int m, double *C, double *Q) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Q[i * m + j] = (i == j) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        tot += C[i * m + j] * C[i * m + j];
        if (i != j) off += C[i * m + j] * C[i * m + j];
      }
    if (off <= 1e-32 * tot) break;
    for (int a = 0; a < m; ++a)
      for (int b = a + 1; b < m; ++b) {
        double apq = C[a * m + b];
        if (apq == 0.0) continue;
        double theta = (C[b * m + b] - C[a * m + a]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < m; ++k) { /* columns a, b */
          double ca = C[k * m + a], cb = C[k * m + b];
          C[k * m + a] = cs * ca - sn * cb;
          C[k * m + b] = sn * ca + cs * cb;
        }
        for (int k = 0; k < m; ++k) { /* rows a, b */
          double ra = C[a * m + k], rb = C[b * m + k];
          C[a * m + k] = cs * ra - sn * rb;
          C[b * m + k] = sn * ra + cs * rb;
        }
        for (int k = 0; k < m; ++k) {
          double qa = Q[k * m + a], qb = Q[k * m + b];
          Q[k * m + a] = cs * qa - sn * qb;
          Q[k * m + b] = sn * qa + cs * qb;
        }
      }
  }
}

/* ======================================================================
 * 1D basis, interior eigenproblem and FDM basis (Sections 2.1, 2.3, 2.4)
 * ====================================================================== */

int or_basis1d(int p, double *xi_o, double *A_o, double *B_o, double *S_o, double *lam_o,
               double *T_o, double *Af_o, double *Bf_o) {
  if (p < 1 || p > OR_PMAX) { set_err("basis1d: bad p=%d", p); return -1; }
  const int n = p + 1, m = p - 1;
  double xi[OR_PMAX + 1], wl[OR_PMAX + 1], xq[OR_PMAX + 1], wq[OR_PMAX + 1];
  double V[(OR_PMAX + 1) * (OR_PMAX + 1)], D[(OR_PMAX + 1) * (OR_PMAX + 1)];
  double A[(OR_PMAX + 1) * (OR_PMAX + 1)], B[(OR_PMAX + 1) * (OR_PMAX + 1)];
  if (or_gll(p, xi, wl) || or_gauss(n, xq, wq)) return -1;
  or_lagrange(p, xi, n, xq, V, D);
  /* A_ij = int l_i' l_j', B_ij = int l_i l_j: Gauss with n points is exact
   * for the degree-2p integrands */
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = 0.0, b = 0.0;
      for (int t = 0; t < n; ++t) {
        a += wq[t] * D[t * n + i] * D[t * n + j];
        b += wq[t] * V[t * n + i] * V[t * n + j];
      }
      A[i * n + j] = a;
      B[i * n + j] = b;
    }
  double S[OR_PMAX * OR_PMAX], lam[OR_PMAX], T[(OR_PMAX + 1) * (OR_PMAX + 1)];
  memset(T, 0, sizeof T);
  T[0] = 1.0;
  T[p * n + p] = 1.0;
  if (m >= 1) {
    /* eq:eig: A_II S = B_II S Lambda with S^T B_II S = I.  Reduce with the
     * Cholesky factor of B_II: C = L^{-1} A_II L^{-T} = Q Lambda Q^T and
     * S = L^{-T} Q. */
    double Lb[OR_PMAX * OR_PMAX], C[OR_PMAX * OR_PMAX], X[OR_PMAX * OR_PMAX], Q[OR_PMAX * OR_PMAX];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) Lb[i * m + j] = B[(i + 1) * n + (j + 1)];
    if (or_cholesky(m, Lb)) return -1;
    /* X = L^{-1} A_II (column by column) */
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) {
        double s = A[(i + 1) * n + (j + 1)];
        for (int k = 0; k < i; ++k) s -= Lb[i * m + k] * X[k * m + j];
        X[i * m + j] = s / Lb[i * m + i];
      }
    /* C = L^{-1} X^T */
    for (int j = 0; j < m; ++j)
      for (int i = 0; i < m; ++i) {
        double s = X[j * m + i];
        for (int k = 0; k < i; ++k) s -= Lb[i * m + k] * C[k * m + j];
        C[i * m + j] = s / Lb[i * m + i];
      }
    for (int i = 0; i < m; ++i) /* symmetrise rounding */
      for (int j = i + 1; j < m; ++j) {
        double s = 0.5 * (C[i * m + j] + C[j * m + i]);
        C[i * m + j] = C[j * m + i] = s;
      }
    jacobi_eig(m, C, Q);
    /* S = L^{-T} Q */
    double Sraw[OR_PMAX * OR_PMAX], lraw[OR_PMAX];
    for (int j = 0; j < m; ++j) {
      lraw[j] = C[j * m + j];
      for (int i = m - 1; i >= 0; --i) {
        double s = Q[i * m + j];
        for (int k = i + 1; k < m; ++k) s -= Lb[k * m + i] * Sraw[k * m + j];
        Sraw[i * m + j] = s / Lb[i * m + i];
      }
    }
    /* order eigenpairs by ascending lambda; sign: first interior node > 0 */
    int ord[OR_PMAX];
    for (int j = 0; j < m; ++j) ord[j] = j;
    for (int a = 0; a < m; ++a)
      for (int b = a + 1; b < m; ++b)
        if (lraw[ord[b]] < lraw[ord[a]]) { int t = ord[a]; ord[a] = ord[b]; ord[b] = t; }
    for (int j = 0; j < m; ++j) {
      int o = ord[j];
      double sg = Sraw[0 * m + o] < 0 ? -1.0 : 1.0;
      lam[j] = lraw[o];
      for (int i = 0; i < m; ++i) S[i * m + j] = sg * Sraw[i * m + o];
    }
    /* interior FDM shape functions: nodal values S on the interior nodes */
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) T[(i + 1) * n + (j + 1)] = S[i * m + j];
    /* interface shape functions: value 1 at their vertex, 0 at the other,
     * and zero moments against every s_j, i.e. B-orthogonal to the interior:
     * T[I, e] = -B_II^{-1} B_{I,e} for e in {0, p}. */
    for (int e = 0; e <= p; e += p) {
      double rhs[OR_PMAX];
      for (int i = 0; i < m; ++i) rhs[i] = -B[(i + 1) * n + e];
      chol_solve(m, Lb, rhs);
      for (int i = 0; i < m; ++i) T[(i + 1) * n + e] = rhs[i];
    }
  }
  /* Af = T^T A T, Bf = T^T B T */
  double Af[(OR_PMAX + 1) * (OR_PMAX + 1)], Bf[(OR_PMAX + 1) * (OR_PMAX + 1)];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double a = 0.0, b = 0.0;
      for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
          a += T[k * n + i] * A[k * n + l] * T[l * n + j];
          b += T[k * n + i] * B[k * n + l] * T[l * n + j];
        }
      Af[i * n + j] = a;
      Bf[i * n + j] = b;
    }
  /* Section 2.4: A_II and B_II diagonal, B_{I,Gamma} = 0 in the FDM basis.
   * Check the rounding residue, then make those zeros exact. */
  double sa = 0.0, sb = 0.0;
  for (int i = 0; i < n * n; ++i) {
    if (fabs(Af[i]) > sa) sa = fabs(Af[i]);
    if (fabs(Bf[i]) > sb) sb = fabs(Bf[i]);
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      int ii = (i > 0 && i < p), jj = (j > 0 && j < p);
      if (ii && jj && i != j) {
        if (fabs(Af[i * n + j]) > 1e-12 * sa || fabs(Bf[i * n + j]) > 1e-12 * sb) {
          set_err("basis1d: interior block not diagonal (%g, %g)", Af[i * n + j], Bf[i * n + j]);
          return -2;
        }
        Af[i * n + j] = 0.0;
        Bf[i * n + j] = 0.0;
      }
      if (ii != jj) {
        if (fabs(Bf[i * n + j]) > 1e-12 * sb) {
          set_err("basis1d: B interior/interface coupling %g", Bf[i * n + j]);
          return -2;
        }
        Bf[i * n + j] = 0.0;
      }
    }
  if (xi_o) memcpy(xi_o, xi, sizeof(double) * n);
  if (A_o) memcpy(A_o, A, sizeof(double) * n * n);
  if (B_o) memcpy(B_o, B, sizeof(double) * n * n);
  if (S_o && m > 0) memcpy(S_o, S, sizeof(double) * m * m);
  if (lam_o && m > 0) memcpy(lam_o, lam, sizeof(double) * m);
  if (T_o) memcpy(T_o, T, sizeof(double) * n * n);
  if (Af_o) memcpy(Af_o, Af, sizeof(double) * n * n);
  if (Bf_o) memcpy(Bf_o, Bf, sizeof(double) * n * n);
  return 0;
}

/* ======================================================================
 * problem context
 * ====================================================================== */

typedef struct {
  int built;
  int vx, vy, vz;
  int lo[3], hi[3], dim[3]; /* star box in grid indices (inclusive) */
  int nd, nI, nG;
  long *gidx;   /* [nd] */
  int *kind;    /* [nd]: position in I list (>=0) or -(1+position in G list) */
  int *listI, *listG;
  double *D;    /* [nI] diagonal of A_II */
  int *gi_ptr, *gi_col; /* CSR of A_{Gamma I}: rows = Gamma, cols = I */
  double *gi_val;
  double *L;    /* [nG*nG] Cholesky factor of the Schur complement */
} or_patch;

struct or_ctx {
  int p, n, nx, ny, nz, N[3];
  long ndof;
  int ncell;
  double *xv, *yv, *zv;
  /* 1D data */
  double xi[OR_PMAX + 1], A[(OR_PMAX + 1) * (OR_PMAX + 1)], B[(OR_PMAX + 1) * (OR_PMAX + 1)];
  double T[(OR_PMAX + 1) * (OR_PMAX + 1)], Af[(OR_PMAX + 1) * (OR_PMAX + 1)], Bf[(OR_PMAX + 1) * (OR_PMAX + 1)];
  double xq[OR_PMAX + 1], wq[OR_PMAX + 1];
  double Vq[(OR_PMAX + 1) * (OR_PMAX + 1)], Dq[(OR_PMAX + 1) * (OR_PMAX + 1)];
  /* geometry */
  int general;
  double *Gw;     /* general: [cell][q^3][6] w_q kappa |det J| J^{-1} J^{-T}  (xx,yy,zz,xy,xz,yz) */
  double *detw;   /* general: [cell][q^3] w_q |det J| (mass) */
  double *mu_box; /* box: [cell][3] exact Kronecker coefficients */
  double *mu;     /* [cell][3] coefficients of the separable surrogate used by the relaxation */
  double omega;
  int npatch;
  or_patch *patches;
  /* coarse */
  int nc;          /* number of free coarse dofs */
  int *cfree;      /* vertex -> free index or -1 */
  double *Lc;      /* dense Cholesky of A_c */
  double *Ac;      /* A_c itself (before factorisation) */
  /* geometric multigrid on the Q1 problem (0 levels: exact solve with Lc) */
  int gmg_levels, gmg_nu;
  double gmg_omega;
  struct or_level *lev; /* gmg_levels + 1 levels, level 0 = the Q1 problem on the mesh */
};

/* one level of the Q1 hierarchy: vertex grid nv[3] (free = interior vertices),
 * dense operator A (nf x nf), prolongation P from the next coarser level
 * (nf x nf_coarse, dense), Cholesky factor on the coarsest level */
struct or_level {
  int n[3];        /* cells per axis */
  double *x[3];    /* vertex coordinates per axis */
  int nf;          /* free vertices */
  double *A, *P, *L;
};

static void set_mu_box(or_ctx *c);

long or_ndof(const or_ctx *c) { return c->ndof; }
int or_npatch(const or_ctx *c) { return c->npatch; }

or_ctx *or_create(int p, int nx, int ny, int nz, const double *xv, const double *yv,
                  const double *zv, const double *jac, const double *kappa) {
  if (p < 1 || p > OR_PMAX || nx < 1 || ny < 1 || nz < 1) { set_err("create: bad sizes"); return NULL; }
  or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
  c->p = p;
  c->n = p + 1;
  c->nx = nx; c->ny = ny; c->nz = nz;
  c->N[0] = nx * p + 1; c->N[1] = ny * p + 1; c->N[2] = nz * p + 1;
  c->ndof = (long)c->N[0] * c->N[1] * c->N[2];
  c->ncell = nx * ny * nz;
  c->xv = (double *)malloc(sizeof(double) * (nx + 1));
  c->yv = (double *)malloc(sizeof(double) * (ny + 1));
  c->zv = (double *)malloc(sizeof(double) * (nz + 1));
  memcpy(c->xv, xv, sizeof(double) * (nx + 1));
  memcpy(c->yv, yv, sizeof(double) * (ny + 1));
  memcpy(c->zv, zv, sizeof(double) * (nz + 1));
  if (or_basis1d(p, c->xi, c->A, c->B, NULL, NULL, c->T, c->Af, c->Bf)) { or_free(c); return NULL; }
  int n = c->n;
  or_gauss(n, c->xq, c->wq);
  or_lagrange(p, c->xi, n, c->xq, c->Vq, c->Dq);
  c->mu_box = (double *)calloc((size_t)3 * c->ncell, sizeof(double));
  c->mu = (double *)calloc((size_t)3 * c->ncell, sizeof(double));
  c->omega = 1.0;
  set_mu_box(c);
  if (jac) {
    /* Section 2.7: Ghat = |det J| J^{-1} J^{-T} (times kappa), and the
     * surrogate's mu_j = cell average of Ghat_jj. */
    c->general = 1;
    int nq = n * n * n;
    c->Gw = (double *)malloc(sizeof(double) * 6 * nq * c->ncell);
    c->detw = (double *)malloc(sizeof(double) * nq * c->ncell);
    for (int e = 0; e < c->ncell; ++e) {
      double avg[3] = {0, 0, 0};
      for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
          for (int i = 0; i < n; ++i) {
            int qp = i + n * (j + n * k);
            const double *J = jac + ((size_t)e * nq + qp) * 9;
            double det = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
                         J[2] * (J[3] * J[7] - J[4] * J[6]);
            if (!(det != 0.0)) { set_err("create: singular Jacobian in cell %d", e); or_free(c); return NULL; }
            double Ji[9]; /* inverse by cofactors */
            Ji[0] = (J[4] * J[8] - J[5] * J[7]) / det;
            Ji[1] = (J[2] * J[7] - J[1] * J[8]) / det;
            Ji[2] = (J[1] * J[5] - J[2] * J[4]) / det;
            Ji[3] = (J[5] * J[6] - J[3] * J[8]) / det;
            Ji[4] = (J[0] * J[8] - J[2] * J[6]) / det;
            Ji[5] = (J[2] * J[3] - J[0] * J[5]) / det;
            Ji[6] = (J[3] * J[7] - J[4] * J[6]) / det;
            Ji[7] = (J[1] * J[6] - J[0] * J[7]) / det;
            Ji[8] = (J[0] * J[4] - J[1] * J[3]) / det;
            double kap = kappa ? kappa[(size_t)e * nq + qp] : 1.0;
            double w = c->wq[i] * c->wq[j] * c->wq[k];
            double G[3][3];
            for (int a = 0; a < 3; ++a)
              for (int b = 0; b < 3; ++b) {
                double s = 0.0;
                for (int r = 0; r < 3; ++r) s += Ji[a * 3 + r] * Ji[b * 3 + r];
                G[a][b] = kap * fabs(det) * s;
              }
            double *g = c->Gw + ((size_t)e * nq + qp) * 6;
            g[0] = w * G[0][0]; g[1] = w * G[1][1]; g[2] = w * G[2][2];
            g[3] = w * G[0][1]; g[4] = w * G[0][2]; g[5] = w * G[1][2];
            c->detw[(size_t)e * nq + qp] = w * fabs(det);
            for (int a = 0; a < 3; ++a) avg[a] += w * G[a][a];
          }
      for (int a = 0; a < 3; ++a) c->mu[3 * e + a] = avg[a] / 8.0;
    }
  } else {
    memcpy(c->mu, c->mu_box, sizeof(double) * 3 * c->ncell);
  }
  c->npatch = (nx + 1) * (ny + 1) * (nz + 1);
  c->patches = (or_patch *)calloc(c->npatch, sizeof(or_patch));
  return c;
}

static void free_patch(or_patch *P) {
  free(P->gidx); free(P->kind); free(P->listI); free(P->listG); free(P->D);
  free(P->gi_ptr); free(P->gi_col); free(P->gi_val); free(P->L);
  memset(P, 0, sizeof *P);
}

void or_free(or_ctx *c) {
  if (!c) return;
  if (c->patches)
    for (int i = 0; i < c->npatch; ++i) free_patch(&c->patches[i]);
  free(c->patches);
  free(c->xv); free(c->yv); free(c->zv);
  free(c->Gw); free(c->detw); free(c->mu_box); free(c->mu);
  free(c->cfree); free(c->Lc); free(c->Ac);
  if (c->lev) {
    for (int l = 0; l <= c->gmg_levels; ++l) {
      for (int a = 0; a < 3; ++a) free(c->lev[l].x[a]);
      free(c->lev[l].A); free(c->lev[l].P); free(c->lev[l].L);
    }
    free(c->lev);
  }
  free(c);
}

/* Section 2.2: mu_j = L_j^{-2} prod_i L_i with L = edge length / 2 */
static void set_mu_box(or_ctx *c) {
  for (int cz = 0; cz < c->nz; ++cz)
    for (int cy = 0; cy < c->ny; ++cy)
      for (int cx = 0; cx < c->nx; ++cx) {
        int e = cx + c->nx * (cy + c->ny * cz);
        double L[3] = {0.5 * (c->xv[cx + 1] - c->xv[cx]), 0.5 * (c->yv[cy + 1] - c->yv[cy]),
                       0.5 * (c->zv[cz + 1] - c->zv[cz])};
        double vol = L[0] * L[1] * L[2];
        for (int a = 0; a < 3; ++a) c->mu_box[3 * e + a] = vol / (L[a] * L[a]);
      }
}

void or_get_mu(const or_ctx *c, double *mu) { memcpy(mu, c->mu, sizeof(double) * 3 * c->ncell); }
void or_set_mu(or_ctx *c, const double *mu) { memcpy(c->mu, mu, sizeof(double) * 3 * c->ncell); }
void or_set_omega(or_ctx *c, double omega) { c->omega = omega; }
double or_get_omega(const or_ctx *c) { return c->omega; }

/* ---- grid helpers ---- */
static inline long gid(const or_ctx *c, int gx, int gy, int gz) {
  return gx + (long)c->N[0] * (gy + (long)c->N[1] * gz);
}
static inline int is_dirichlet(const or_ctx *c, int gx, int gy, int gz) {
  return gx == 0 || gy == 0 || gz == 0 || gx == c->N[0] - 1 || gy == c->N[1] - 1 || gz == c->N[2] - 1;
}

/* out = (M3 kron M2 kron M1) in, with in of dims (n1,n2,n3) (first fastest)
 * and M_a of size m_a x n_a row-major; out of dims (m1,m2,m3). */
static void kron3(const double *M3, const double *M2, const double *M1, int n1, int n2, int n3,
                  int m1, int m2, int m3, const double *in, double *out) {
  double *t1 = (double *)malloc(sizeof(double) * m1 * n2 * n3);
  double *t2 = (double *)malloc(sizeof(double) * m1 * m2 * n3);
  for (int k = 0; k < n3; ++k)
    for (int j = 0; j < n2; ++j)
      for (int a = 0; a < m1; ++a) {
        double s = 0.0;
        for (int b = 0; b < n1; ++b) s += M1[a * n1 + b] * in[b + n1 * (j + n2 * k)];
        t1[a + m1 * (j + n2 * k)] = s;
      }
  for (int k = 0; k < n3; ++k)
    for (int a2 = 0; a2 < m2; ++a2)
      for (int i = 0; i < m1; ++i) {
        double s = 0.0;
        for (int b = 0; b < n2; ++b) s += M2[a2 * n2 + b] * t1[i + m1 * (b + n2 * k)];
        t2[i + m1 * (a2 + m2 * k)] = s;
      }
  for (int a3 = 0; a3 < m3; ++a3)
    for (int j = 0; j < m2; ++j)
      for (int i = 0; i < m1; ++i) {
        double s = 0.0;
        for (int b = 0; b < n3; ++b) s += M3[a3 * n3 + b] * t2[i + m1 * (j + m2 * b)];
        out[i + m1 * (j + m2 * a3)] = s;
      }
  free(t1);
  free(t2);
}

static void transpose(int m, int n, const double *M, double *Mt) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) Mt[j * m + i] = M[i * n + j];
}

/* y_K = A^K u_K for one cell (true operator: eq. (kron) on box cells,
 * Gauss quadrature with Ghat on curved cells, Section 2.7). */
static void cell_stiffness(const or_ctx *c, int e, const double *u, double *y) {
  int n = c->n, n3 = n * n * n;
  double *t = (double *)malloc(sizeof(double) * n3);
  if (!c->general) {
    const double *mu = c->mu_box + 3 * e;
    kron3(c->B, c->B, c->A, n, n, n, n, n, n, u, y);
    for (int i = 0; i < n3; ++i) y[i] *= mu[0];
    kron3(c->B, c->A, c->B, n, n, n, n, n, n, u, t);
    for (int i = 0; i < n3; ++i) y[i] += mu[1] * t[i];
    kron3(c->A, c->B, c->B, n, n, n, n, n, n, u, t);
    for (int i = 0; i < n3; ++i) y[i] += mu[2] * t[i];
  } else {
    double *gx = (double *)malloc(sizeof(double) * n3), *gy = (double *)malloc(sizeof(double) * n3),
           *gz = (double *)malloc(sizeof(double) * n3);
    double Vt[(OR_PMAX + 1) * (OR_PMAX + 1)], Dt[(OR_PMAX + 1) * (OR_PMAX + 1)];
    transpose(n, n, c->Vq, Vt);
    transpose(n, n, c->Dq, Dt);
    /* reference gradient at the Gauss points */
    kron3(c->Vq, c->Vq, c->Dq, n, n, n, n, n, n, u, gx);
    kron3(c->Vq, c->Dq, c->Vq, n, n, n, n, n, n, u, gy);
    kron3(c->Dq, c->Vq, c->Vq, n, n, n, n, n, n, u, gz);
    const double *G = c->Gw + (size_t)e * n3 * 6;
    for (int q = 0; q < n3; ++q) {
      const double *g = G + 6 * q;
      double a = gx[q], b = gy[q], d = gz[q];
      gx[q] = g[0] * a + g[3] * b + g[4] * d;
      gy[q] = g[3] * a + g[1] * b + g[5] * d;
      gz[q] = g[4] * a + g[5] * b + g[2] * d;
    }
    kron3(Vt, Vt, Dt, n, n, n, n, n, n, gx, y);
    kron3(Vt, Dt, Vt, n, n, n, n, n, n, gy, t);
    for (int i = 0; i < n3; ++i) y[i] += t[i];
    kron3(Dt, Vt, Vt, n, n, n, n, n, n, gz, t);
    for (int i = 0; i < n3; ++i) y[i] += t[i];
    free(gx); free(gy); free(gz);
  }
  free(t);
}

static void cell_mass(const or_ctx *c, int e, const double *u, double *y) {
  int n = c->n, n3 = n * n * n;
  if (!c->general) {
    const double *mu = c->mu_box + 3 * e;
    /* mu1 mu2 mu3 = (L1 L2 L3)^3 / (L1 L2 L3)^2 = L1 L2 L3 */
    double vol = mu[0] * mu[1] * mu[2];
    kron3(c->B, c->B, c->B, n, n, n, n, n, n, u, y);
    for (int i = 0; i < n3; ++i) y[i] *= vol;
  } else {
    double *g = (double *)malloc(sizeof(double) * n3);
    double Vt[(OR_PMAX + 1) * (OR_PMAX + 1)];
    transpose(n, n, c->Vq, Vt);
    kron3(c->Vq, c->Vq, c->Vq, n, n, n, n, n, n, u, g);
    for (int q = 0; q < n3; ++q) g[q] *= c->detw[(size_t)e * n3 + q];
    kron3(Vt, Vt, Vt, n, n, n, n, n, n, g, y);
    free(g);
  }
}

typedef void (*cell_op)(const or_ctx *, int, const double *, double *);

/* A = sum_K R_K^T A^K R_K (direct stiffness summation), Dirichlet removed */
static void assemble_apply(const or_ctx *c, cell_op op, const double *u, double *y) {
  int n = c->n, p = c->p, n3 = n * n * n;
  double *uk = (double *)malloc(sizeof(double) * n3), *yk = (double *)malloc(sizeof(double) * n3);
  memset(y, 0, sizeof(double) * c->ndof);
  for (int cz = 0; cz < c->nz; ++cz)
    for (int cy = 0; cy < c->ny; ++cy)
      for (int cx = 0; cx < c->nx; ++cx) {
        int e = cx + c->nx * (cy + c->ny * cz);
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              int gx = cx * p + i, gy = cy * p + j, gz = cz * p + k;
              uk[i + n * (j + n * k)] = is_dirichlet(c, gx, gy, gz) ? 0.0 : u[gid(c, gx, gy, gz)];
            }
        op(c, e, uk, yk);
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
              y[gid(c, cx * p + i, cy * p + j, cz * p + k)] += yk[i + n * (j + n * k)];
      }
  for (int gz = 0; gz < c->N[2]; ++gz)
    for (int gy = 0; gy < c->N[1]; ++gy)
      for (int gx = 0; gx < c->N[0]; ++gx)
        if (is_dirichlet(c, gx, gy, gz)) y[gid(c, gx, gy, gz)] = 0.0;
  free(uk);
  free(yk);
}

void or_stiffness_apply(const or_ctx *c, const double *u, double *y) { assemble_apply(c, cell_stiffness, u, y); }
void or_mass_apply(const or_ctx *c, const double *f, double *b) { assemble_apply(c, cell_mass, f, b); }

/* ======================================================================
 * global basis change (Section 2.4: interpolation and restriction)
 * ====================================================================== */

/* number of cells sharing grid index g along an axis with N nodes */
static inline int mult1(int g, int p, int N) { return (g % p == 0 && g > 0 && g < N - 1) ? 2 : 1; }

void or_restrict_fdm(const or_ctx *c, const double *r, double *r_fdm) {
  /* T_g = sum_K R_K^T W_K T_K R_K with W_K = 1/multiplicity, hence
   * T_g^T r = sum_K R_K^T T_K^T (W_K r_K) */
  int n = c->n, p = c->p, n3 = n * n * n;
  double Tt[(OR_PMAX + 1) * (OR_PMAX + 1)];
  transpose(n, n, c->T, Tt);
  double *w = (double *)malloc(sizeof(double) * n3), *t = (double *)malloc(sizeof(double) * n3);
  memset(r_fdm, 0, sizeof(double) * c->ndof);
  for (int cz = 0; cz < c->nz; ++cz)
    for (int cy = 0; cy < c->ny; ++cy)
      for (int cx = 0; cx < c->nx; ++cx) {
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              int gx = cx * p + i, gy = cy * p + j, gz = cz * p + k;
              double m = mult1(gx, p, c->N[0]) * mult1(gy, p, c->N[1]) * mult1(gz, p, c->N[2]);
              w[i + n * (j + n * k)] = is_dirichlet(c, gx, gy, gz) ? 0.0 : r[gid(c, gx, gy, gz)] / m;
            }
        kron3(Tt, Tt, Tt, n, n, n, n, n, n, w, t);
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
              r_fdm[gid(c, cx * p + i, cy * p + j, cz * p + k)] += t[i + n * (j + n * k)];
      }
  free(w);
  free(t);
}

void or_interp_fdm(const or_ctx *c, const double *u_fdm, double *u) {
  int n = c->n, p = c->p, n3 = n * n * n;
  double *w = (double *)malloc(sizeof(double) * n3), *t = (double *)malloc(sizeof(double) * n3);
  unsigned char *done = (unsigned char *)calloc(c->ndof, 1);
  for (int cz = 0; cz < c->nz; ++cz)
    for (int cy = 0; cy < c->ny; ++cy)
      for (int cx = 0; cx < c->nx; ++cx) {
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
              w[i + n * (j + n * k)] = u_fdm[gid(c, cx * p + i, cy * p + j, cz * p + k)];
        kron3(c->T, c->T, c->T, n, n, n, n, n, n, w, t);
        for (int k = 0; k < n; ++k)
          for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
              long g = gid(c, cx * p + i, cy * p + j, cz * p + k);
              if (!done[g]) { u[g] = t[i + n * (j + n * k)]; done[g] = 1; }
            }
      }
  for (int gz = 0; gz < c->N[2]; ++gz)
    for (int gy = 0; gy < c->N[1]; ++gy)
      for (int gx = 0; gx < c->N[0]; ++gx)
        if (is_dirichlet(c, gx, gy, gz)) u[gid(c, gx, gy, gz)] = 0.0;
  free(done);
  free(w);
  free(t);
}

/* ======================================================================
 * vertex-star patches (Sections 2.5, 2.6)
 * ====================================================================== */

/* Star of vertex v: all dofs on entities whose closure contains v, i.e. the
 * grid box [p v - (p-1), p v + (p-1)] per axis, minus Dirichlet nodes. */
static void star_box(const or_ctx *c, int v, int *vv, int *lo, int *hi) {
  vv[0] = v % (c->nx + 1);
  vv[1] = (v / (c->nx + 1)) % (c->ny + 1);
  vv[2] = v / ((c->nx + 1) * (c->ny + 1));
  for (int a = 0; a < 3; ++a) {
    int cen = c->p * vv[a];
    lo[a] = cen - (c->p - 1);
    hi[a] = cen + (c->p - 1);
    if (lo[a] < 1) lo[a] = 1;
    if (hi[a] > c->N[a] - 2) hi[a] = c->N[a] - 2;
  }
}

static int patch_dofs(const or_ctx *c, int v, or_patch *P) {
  int vv[3];
  star_box(c, v, vv, P->lo, P->hi);
  P->vx = vv[0]; P->vy = vv[1]; P->vz = vv[2];
  P->nd = 1;
  for (int a = 0; a < 3; ++a) {
    P->dim[a] = P->hi[a] - P->lo[a] + 1;
    if (P->dim[a] < 0) P->dim[a] = 0;
    P->nd *= P->dim[a];
  }
  P->gidx = (long *)malloc(sizeof(long) * (P->nd > 0 ? P->nd : 1));
  P->kind = (int *)malloc(sizeof(int) * (P->nd > 0 ? P->nd : 1));
  P->nI = P->nG = 0;
  int s = 0;
  for (int gz = P->lo[2]; gz <= P->hi[2]; ++gz)
    for (int gy = P->lo[1]; gy <= P->hi[1]; ++gy)
      for (int gx = P->lo[0]; gx <= P->hi[0]; ++gx, ++s) {
        P->gidx[s] = gid(c, gx, gy, gz);
        /* cell-interior dof: on no vertex plane in any direction */
        int interior = (gx % c->p) && (gy % c->p) && (gz % c->p);
        P->kind[s] = interior ? P->nI++ : -(1 + P->nG++);
      }
  P->listI = (int *)malloc(sizeof(int) * (P->nI > 0 ? P->nI : 1));
  P->listG = (int *)malloc(sizeof(int) * (P->nG > 0 ? P->nG : 1));
  for (s = 0; s < P->nd; ++s) {
    if (P->kind[s] >= 0) P->listI[P->kind[s]] = s;
    else P->listG[-P->kind[s] - 1] = s;
  }
  return 0;
}

/* row a (star index) of A_j = R_j A R_j^T in the FDM basis:
 * sum over the star's cells K containing dof a of the entries of the
 * separable cell matrix mu1 Bf(x)Bf(x)Af + mu2 Bf(x)Af(x)Bf + mu3 Af(x)Bf(x)Bf. */
static void patch_row(const or_ctx *c, const or_patch *P, int a, double *row) {
  int p = c->p, n = c->n;
  memset(row, 0, sizeof(double) * P->nd);
  int ax = P->lo[0] + a % P->dim[0];
  int ay = P->lo[1] + (a / P->dim[0]) % P->dim[1];
  int az = P->lo[2] + a / (P->dim[0] * P->dim[1]);
  for (int cz = P->vz - 1; cz <= P->vz; ++cz)
    for (int cy = P->vy - 1; cy <= P->vy; ++cy)
      for (int cx = P->vx - 1; cx <= P->vx; ++cx) {
        if (cx < 0 || cy < 0 || cz < 0 || cx >= c->nx || cy >= c->ny || cz >= c->nz) continue;
        int ia = ax - cx * p, ja = ay - cy * p, ka = az - cz * p;
        if (ia < 0 || ia > p || ja < 0 || ja > p || ka < 0 || ka > p) continue;
        const double *mu = c->mu + 3 * (cx + c->nx * (cy + c->ny * cz));
        for (int gz = cz * p; gz <= cz * p + p; ++gz) {
          if (gz < P->lo[2] || gz > P->hi[2]) continue;
          for (int gy = cy * p; gy <= cy * p + p; ++gy) {
            if (gy < P->lo[1] || gy > P->hi[1]) continue;
            for (int gx = cx * p; gx <= cx * p + p; ++gx) {
              if (gx < P->lo[0] || gx > P->hi[0]) continue;
              int ib = gx - cx * p, jb = gy - cy * p, kb = gz - cz * p;
              double v = mu[0] * c->Bf[ka * n + kb] * c->Bf[ja * n + jb] * c->Af[ia * n + ib] +
                         mu[1] * c->Bf[ka * n + kb] * c->Af[ja * n + jb] * c->Bf[ia * n + ib] +
                         mu[2] * c->Af[ka * n + kb] * c->Bf[ja * n + jb] * c->Bf[ia * n + ib];
              int b = (gx - P->lo[0]) + P->dim[0] * ((gy - P->lo[1]) + P->dim[1] * (gz - P->lo[2]));
              row[b] += v;
            }
          }
        }
      }
}

int or_patch_matrix(const or_ctx *c, int v, double *Aj) {
  if (v < 0 || v >= c->npatch) { set_err("patch id"); return -1; }
  or_patch P;
  memset(&P, 0, sizeof P);
  patch_dofs(c, v, &P);
  for (int a = 0; a < P.nd; ++a) patch_row(c, &P, a, Aj + (size_t)a * P.nd);
  free_patch(&P);
  return 0;
}

int or_patch_dofs(const or_ctx *c, int v, int *nd, int *nI, long *gidx) {
  if (v < 0 || v >= c->npatch) { set_err("patch id"); return -1; }
  or_patch P;
  memset(&P, 0, sizeof P);
  patch_dofs(c, v, &P);
  if (nd) *nd = P.nd;
  if (nI) *nI = P.nI;
  if (gidx) memcpy(gidx, P.gidx, sizeof(long) * P.nd);
  free_patch(&P);
  return 0;
}

/* Section 2.6: A_II diagonal; S_G = A_GG - A_GI A_II^{-1} A_IG.
 * Builds D, the CSR of A_GI and (if S != NULL) the dense S_G. */
static int patch_schur(const or_ctx *c, or_patch *P, double *S) {
  int nd = P->nd, nI = P->nI, nG = P->nG;
  double *row = (double *)malloc(sizeof(double) * (nd > 0 ? nd : 1));
  P->D = (double *)malloc(sizeof(double) * (nI > 0 ? nI : 1));
  for (int m = 0; m < nI; ++m) {
    int a = P->listI[m];
    patch_row(c, P, a, row);
    for (int b = 0; b < nd; ++b)
      if (P->kind[b] >= 0 && b != a && row[b] != 0.0) {
        set_err("patch %d: A_II not diagonal", (int)(P - c->patches));
        free(row);
        return -2;
      }
    P->D[m] = row[a];
    if (!(P->D[m] > 0.0)) { set_err("patch: nonpositive interior diagonal"); free(row); return -3; }
  }
  /* Gamma rows: A_GG part into S, A_GI part into CSR */
  int cap = 64 > nG ? 64 : nG, nnz = 0;
  P->gi_ptr = (int *)malloc(sizeof(int) * (nG + 1));
  P->gi_col = (int *)malloc(sizeof(int) * cap);
  P->gi_val = (double *)malloc(sizeof(double) * cap);
  if (S) memset(S, 0, sizeof(double) * (size_t)nG * nG);
  for (int g = 0; g < nG; ++g) {
    P->gi_ptr[g] = nnz;
    patch_row(c, P, P->listG[g], row);
    for (int b = 0; b < nd; ++b) {
      if (row[b] == 0.0) continue;
      if (P->kind[b] >= 0) {
        if (nnz == cap) {
          cap *= 2;
          P->gi_col = (int *)realloc(P->gi_col, sizeof(int) * cap);
          P->gi_val = (double *)realloc(P->gi_val, sizeof(double) * cap);
        }
        P->gi_col[nnz] = P->kind[b];
        P->gi_val[nnz++] = row[b];
      } else if (S) {
        S[(size_t)g * nG + (-P->kind[b] - 1)] = row[b];
      }
    }
  }
  P->gi_ptr[nG] = nnz;
  free(row);
  if (S) {
    /* S -= sum_m A_{G m} A_{m G} / D_m, interior dof by interior dof */
    int *cnt = (int *)calloc(nI + 1, sizeof(int));
    for (int k = 0; k < nnz; ++k) cnt[P->gi_col[k] + 1]++;
    for (int m = 0; m < nI; ++m) cnt[m + 1] += cnt[m];
    int *fill = (int *)malloc(sizeof(int) * (nI + 1));
    memcpy(fill, cnt, sizeof(int) * (nI + 1));
    int *rg = (int *)malloc(sizeof(int) * (nnz > 0 ? nnz : 1));
    double *rv = (double *)malloc(sizeof(double) * (nnz > 0 ? nnz : 1));
    for (int g = 0; g < nG; ++g)
      for (int k = P->gi_ptr[g]; k < P->gi_ptr[g + 1]; ++k) {
        int m = P->gi_col[k];
        rg[fill[m]] = g;
        rv[fill[m]++] = P->gi_val[k];
      }
    for (int m = 0; m < nI; ++m)
      for (int s = cnt[m]; s < cnt[m + 1]; ++s)
        for (int t = cnt[m]; t < cnt[m + 1]; ++t)
          S[(size_t)rg[s] * nG + rg[t]] -= rv[s] * rv[t] / P->D[m];
    free(cnt); free(fill); free(rg); free(rv);
  }
  return 0;
}

static int setup_one(const or_ctx *c, int v, or_patch *P) {
  free_patch(P);
  patch_dofs(c, v, P);
  double *S = (double *)malloc(sizeof(double) * ((size_t)P->nG * P->nG > 0 ? (size_t)P->nG * P->nG : 1));
  int rc = patch_schur(c, P, S);
  if (!rc && P->nG > 0) rc = or_cholesky(P->nG, S);
  if (rc) { free(S); return rc; }
  P->L = S;
  P->built = 1;
  return 0;
}

int or_setup_patches(or_ctx *c, const int *vertices, int nvert, int nthreads) {
  int cnt = vertices ? nvert : c->npatch;
  int err = 0;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int i = 0; i < cnt; ++i) {
    int v = vertices ? vertices[i] : i;
    if (v < 0 || v >= c->npatch) { err = -1; continue; }
    int rc = setup_one(c, v, &c->patches[v]);
    if (rc) err = rc;
  }
  (void)nthreads;
  return err;
}

int or_patch_schur(const or_ctx *c, int v, double *S) {
  if (v < 0 || v >= c->npatch) { set_err("patch id"); return -1; }
  or_patch P;
  memset(&P, 0, sizeof P);
  patch_dofs(c, v, &P);
  int rc = patch_schur(c, &P, S);
  free_patch(&P);
  return rc;
}

/* eq:LDLT: g_G = r_G - A_GI A_II^{-1} r_I; x_G = S_G^{-1} g_G;
 * x_I = A_II^{-1} (r_I - A_IG x_G) */
static void patch_solve(const or_patch *P, const double *r, double *x) {
  int nI = P->nI, nG = P->nG;
  double *g = (double *)malloc(sizeof(double) * (nG > 0 ? nG : 1));
  double *t = (double *)calloc(nI > 0 ? nI : 1, sizeof(double));
  for (int a = 0; a < nG; ++a) {
    double s = r[P->listG[a]];
    for (int k = P->gi_ptr[a]; k < P->gi_ptr[a + 1]; ++k)
      s -= P->gi_val[k] * r[P->listI[P->gi_col[k]]] / P->D[P->gi_col[k]];
    g[a] = s;
  }
  if (nG > 0) chol_solve(nG, P->L, g);
  for (int a = 0; a < nG; ++a)
    for (int k = P->gi_ptr[a]; k < P->gi_ptr[a + 1]; ++k) t[P->gi_col[k]] += P->gi_val[k] * g[a];
  for (int m = 0; m < nI; ++m) x[P->listI[m]] = (r[P->listI[m]] - t[m]) / P->D[m];
  for (int a = 0; a < nG; ++a) x[P->listG[a]] = g[a];
  free(g);
  free(t);
}

int or_patch_solve(const or_ctx *c, int v, const double *r, double *x) {
  if (v < 0 || v >= c->npatch || !c->patches[v].built) { set_err("patch %d not set up", v); return -1; }
  patch_solve(&c->patches[v], r, x);
  return 0;
}

void or_symbolic_fill(int m, unsigned char *pat) {
  /* eliminating column k connects every pair of its later neighbours */
  for (int k = 0; k < m; ++k)
    for (int i = k + 1; i < m; ++i) {
      if (!pat[(size_t)i * m + k]) continue;
      for (int j = k + 1; j <= i; ++j)
        if (pat[(size_t)j * m + k]) pat[(size_t)i * m + j] = pat[(size_t)j * m + i] = 1;
    }
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j) pat[(size_t)i * m + j] = 0;
}

/* z = omega sum_j R_j^T A_j^{-1} R_j r, with R_j acting on FDM coefficients */
int or_asm_apply(const or_ctx *c, const double *r, double *z) {
  double *rf = (double *)malloc(sizeof(double) * c->ndof);
  double *zf = (double *)calloc(c->ndof, sizeof(double));
  or_restrict_fdm(c, r, rf);
  double **xs = (double **)calloc(c->npatch, sizeof(double *));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int v = 0; v < c->npatch; ++v) {
    const or_patch *P = &c->patches[v];
    if (!P->built || P->nd == 0) continue;
    double *rs = (double *)malloc(sizeof(double) * P->nd);
    xs[v] = (double *)malloc(sizeof(double) * P->nd);
    for (int s = 0; s < P->nd; ++s) rs[s] = rf[P->gidx[s]];
    patch_solve(P, rs, xs[v]);
    free(rs);
  }
  for (int v = 0; v < c->npatch; ++v) { /* additive, in patch order */
    if (!xs[v]) continue;
    const or_patch *P = &c->patches[v];
    for (int s = 0; s < P->nd; ++s) zf[P->gidx[s]] += xs[v][s];
    free(xs[v]);
  }
  free(xs);
  or_interp_fdm(c, zf, z);
  for (long i = 0; i < c->ndof; ++i) z[i] *= c->omega;
  free(rf);
  free(zf);
  return 0;
}

/* ======================================================================
 * Q1 coarse space on the same mesh (Section 2.5)
 * ====================================================================== */

/* 1D hat function of coarse vertex v at fine grid index g */
static double hat1(const or_ctx *c, int g, int v) {
  int p = c->p;
  if (g % p == 0) return (g / p == v) ? 1.0 : 0.0;
  int cell = g / p, i = g % p;
  if (v == cell) return 0.5 * (1.0 - c->xi[i]);
  if (v == cell + 1) return 0.5 * (1.0 + c->xi[i]);
  return 0.0;
}

int or_setup_coarse(or_ctx *c) {
  int nvx = c->nx + 1, nvy = c->ny + 1, nvz = c->nz + 1, nv = nvx * nvy * nvz;
  free(c->cfree);
  free(c->Lc);
  c->cfree = (int *)malloc(sizeof(int) * nv);
  c->nc = 0;
  for (int vz = 0; vz < nvz; ++vz)
    for (int vy = 0; vy < nvy; ++vy)
      for (int vx = 0; vx < nvx; ++vx) {
        int v = vx + nvx * (vy + nvy * vz);
        int fr = vx > 0 && vy > 0 && vz > 0 && vx < c->nx && vy < c->ny && vz < c->nz;
        c->cfree[v] = fr ? c->nc++ : -1;
      }
  int nc = c->nc, n = c->n, n3 = n * n * n;
  c->Lc = (double *)calloc((size_t)(nc > 0 ? nc : 1) * (nc > 0 ? nc : 1), sizeof(double));
  if (nc == 0) return 0;
  /* A_c = P^T A P assembled cell by cell: A_c^K = P_K^T A^K P_K */
  double *u = (double *)malloc(sizeof(double) * 8 * n3), *y = (double *)malloc(sizeof(double) * 8 * n3);
  for (int cz = 0; cz < c->nz; ++cz)
    for (int cy = 0; cy < c->ny; ++cy)
      for (int cx = 0; cx < c->nx; ++cx) {
        int e = cx + c->nx * (cy + c->ny * cz);
        int vid[8];
        for (int s = 0; s < 8; ++s) {
          int ox = s & 1, oy = (s >> 1) & 1, oz = (s >> 2) & 1;
          vid[s] = c->cfree[(cx + ox) + nvx * ((cy + oy) + nvy * (cz + oz))];
          for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
              for (int i = 0; i < n; ++i) {
                double hx = ox ? 0.5 * (1 + c->xi[i]) : 0.5 * (1 - c->xi[i]);
                double hy = oy ? 0.5 * (1 + c->xi[j]) : 0.5 * (1 - c->xi[j]);
                double hz = oz ? 0.5 * (1 + c->xi[k]) : 0.5 * (1 - c->xi[k]);
                u[s * n3 + i + n * (j + n * k)] = hx * hy * hz;
              }
          cell_stiffness(c, e, u + s * n3, y + s * n3);
        }
        for (int s = 0; s < 8; ++s) {
          if (vid[s] < 0) continue;
          for (int t = 0; t < 8; ++t) {
            if (vid[t] < 0) continue;
            double d = 0.0;
            for (int l = 0; l < n3; ++l) d += u[s * n3 + l] * y[t * n3 + l];
            c->Lc[(size_t)vid[s] * nc + vid[t]] += d;
          }
        }
      }
  free(u);
  free(y);
  free(c->Ac);
  c->Ac = (double *)malloc(sizeof(double) * (size_t)nc * nc);
  memcpy(c->Ac, c->Lc, sizeof(double) * (size_t)nc * nc);
  return or_cholesky(nc, c->Lc);
}

/* ---- geometric multigrid on the Q1 problem (the paper's solver for the
 * p-coarse problem: damped point-Jacobi on every level, Cholesky on the
 * coarsest).  Levels are nested: level l+1 keeps every other vertex of level l
 * along each axis; P interpolates linearly along each axis in the level's own
 * vertex coordinates (exact for Q1 on nested meshes), and A_{l+1} = P^T A_l P. */
static int lev_index(const struct or_level *L, int vx, int vy, int vz) {
  if (vx <= 0 || vy <= 0 || vz <= 0 || vx >= L->n[0] || vy >= L->n[1] || vz >= L->n[2]) return -1;
  return (vx - 1) + (L->n[0] - 1) * ((vy - 1) + (L->n[1] - 1) * (vz - 1));
}

/* weight of coarse vertex I (coordinates xc) at fine vertex i (coordinates xf), one axis */
static double interp1(const double *xf, int i, int I) {
  if (i % 2 == 0) return i / 2 == I ? 1.0 : 0.0;
  const int l = (i - 1) / 2, r = (i + 1) / 2;
  const double t = (xf[i] - xf[i - 1]) / (xf[i + 1] - xf[i - 1]);
  if (I == l) return 1.0 - t;
  if (I == r) return t;
  return 0.0;
}

int or_setup_coarse_gmg(or_ctx *c, int levels, int nu, double omega) {
  if (!c->Ac) { set_err("gmg: set up the coarse space first"); return -1; }
  if (c->lev) {
    for (int l = 0; l <= c->gmg_levels; ++l) {
      for (int a = 0; a < 3; ++a) free(c->lev[l].x[a]);
      free(c->lev[l].A); free(c->lev[l].P); free(c->lev[l].L);
    }
    free(c->lev);
    c->lev = NULL;
  }
  c->gmg_levels = 0;
  if (levels <= 0) return 0;
  c->lev = (struct or_level *)calloc(levels + 1, sizeof(struct or_level));
  struct or_level *L0 = &c->lev[0];
  L0->n[0] = c->nx; L0->n[1] = c->ny; L0->n[2] = c->nz;
  const double *v0[3] = {c->xv, c->yv, c->zv};
  for (int a = 0; a < 3; ++a) {
    L0->x[a] = (double *)malloc(sizeof(double) * (L0->n[a] + 1));
    memcpy(L0->x[a], v0[a], sizeof(double) * (L0->n[a] + 1));
  }
  L0->nf = c->nc;
  L0->A = (double *)malloc(sizeof(double) * (size_t)c->nc * c->nc);
  memcpy(L0->A, c->Ac, sizeof(double) * (size_t)c->nc * c->nc);
  int l = 0;
  for (; l < levels; ++l) {
    struct or_level *F = &c->lev[l], *C = &c->lev[l + 1];
    if (F->n[0] % 2 || F->n[1] % 2 || F->n[2] % 2 || F->n[0] < 4 || F->n[1] < 4 || F->n[2] < 4) break;
    for (int a = 0; a < 3; ++a) {
      C->n[a] = F->n[a] / 2;
      C->x[a] = (double *)malloc(sizeof(double) * (C->n[a] + 1));
      for (int i = 0; i <= C->n[a]; ++i) C->x[a][i] = F->x[a][2 * i];
    }
    C->nf = (C->n[0] - 1) * (C->n[1] - 1) * (C->n[2] - 1);
    /* P (F->nf x C->nf): tensor product of the 1D linear interpolation weights */
    F->P = (double *)calloc((size_t)F->nf * C->nf, sizeof(double));
    for (int vz = 1; vz < F->n[2]; ++vz)
      for (int vy = 1; vy < F->n[1]; ++vy)
        for (int vx = 1; vx < F->n[0]; ++vx) {
          const int i = lev_index(F, vx, vy, vz);
          for (int Vz = 1; Vz < C->n[2]; ++Vz)
            for (int Vy = 1; Vy < C->n[1]; ++Vy)
              for (int Vx = 1; Vx < C->n[0]; ++Vx) {
                const double w = interp1(F->x[0], vx, Vx) * interp1(F->x[1], vy, Vy) * interp1(F->x[2], vz, Vz);
                if (w != 0.0) F->P[(size_t)i * C->nf + lev_index(C, Vx, Vy, Vz)] = w;
              }
        }
    /* A_c = P^T A P */
    double *AP = (double *)calloc((size_t)F->nf * C->nf, sizeof(double));
    for (int i = 0; i < F->nf; ++i)
      for (int k = 0; k < F->nf; ++k) {
        const double a = F->A[(size_t)i * F->nf + k];
        if (a == 0.0) continue;
        for (int J = 0; J < C->nf; ++J) AP[(size_t)i * C->nf + J] += a * F->P[(size_t)k * C->nf + J];
      }
    C->A = (double *)calloc((size_t)C->nf * C->nf, sizeof(double));
    for (int i = 0; i < F->nf; ++i)
      for (int I = 0; I < C->nf; ++I) {
        const double pi = F->P[(size_t)i * C->nf + I];
        if (pi == 0.0) continue;
        for (int J = 0; J < C->nf; ++J) C->A[(size_t)I * C->nf + J] += pi * AP[(size_t)i * C->nf + J];
      }
    free(AP);
  }
  c->gmg_levels = l;
  c->gmg_nu = nu;
  c->gmg_omega = omega;
  struct or_level *B = &c->lev[l];
  B->L = (double *)malloc(sizeof(double) * (size_t)B->nf * B->nf);
  memcpy(B->L, B->A, sizeof(double) * (size_t)B->nf * B->nf);
  return or_cholesky(B->nf, B->L) ? -1 : l;
}

/* x = V-cycle on level l applied to b (x starts at zero) */
static void gmg_vcycle(const or_ctx *c, int l, const double *b, double *x) {
  const struct or_level *F = &c->lev[l];
  const int n = F->nf;
  if (l == c->gmg_levels) {
    memcpy(x, b, sizeof(double) * n);
    chol_solve(n, F->L, x);
    return;
  }
  const struct or_level *C = &c->lev[l + 1];
  double *r = (double *)malloc(sizeof(double) * n), *bc = (double *)calloc(C->nf, sizeof(double));
  double *xc = (double *)calloc(C->nf, sizeof(double));
  memset(x, 0, sizeof(double) * n);
  for (int sweep = 0; sweep < 2 * c->gmg_nu + 1; ++sweep) {
    if (sweep == c->gmg_nu) { /* coarse-grid correction between the pre- and post-sweeps */
      for (int i = 0; i < n; ++i) {
        double s = b[i];
        for (int k = 0; k < n; ++k) s -= F->A[(size_t)i * n + k] * x[k];
        r[i] = s;
      }
      for (int I = 0; I < C->nf; ++I) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += F->P[(size_t)i * C->nf + I] * r[i];
        bc[I] = s;
      }
      gmg_vcycle(c, l + 1, bc, xc);
      for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int I = 0; I < C->nf; ++I) s += F->P[(size_t)i * C->nf + I] * xc[I];
        x[i] += s;
      }
      continue;
    }
    /* damped point-Jacobi: x += omega D^{-1} (b - A x) */
    for (int i = 0; i < n; ++i) {
      double s = b[i];
      for (int k = 0; k < n; ++k) s -= F->A[(size_t)i * n + k] * x[k];
      r[i] = s;
    }
    for (int i = 0; i < n; ++i) x[i] += c->gmg_omega * r[i] / F->A[(size_t)i * n + i];
  }
  free(r); free(bc); free(xc);
}

int or_gmg_level(const or_ctx *c, int l, int *nf, double *A) {
  if (!c->lev || l < 0 || l > c->gmg_levels) { set_err("gmg: no such level"); return -1; }
  *nf = c->lev[l].nf;
  if (A) memcpy(A, c->lev[l].A, sizeof(double) * (size_t)c->lev[l].nf * c->lev[l].nf);
  return 0;
}

int or_gmg_vcycle(const or_ctx *c, const double *b, double *x) {
  if (!c->lev) { set_err("gmg not set up"); return -1; }
  gmg_vcycle(c, 0, b, x);
  return 0;
}

int or_coarse_matrix(const or_ctx *c, int *nc, double *Ac) {
  /* re-multiplies L L^T (for tests) */
  *nc = c->nc;
  if (!Ac) return 0;
  int m = c->nc;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      double s = 0.0;
      for (int k = 0; k < m; ++k) s += c->Lc[(size_t)i * m + k] * c->Lc[(size_t)j * m + k];
      Ac[(size_t)i * m + j] = s;
    }
  return 0;
}

int or_coarse_apply(const or_ctx *c, const double *r, double *z) {
  if (!c->cfree) { set_err("coarse not set up"); return -1; }
  int nvx = c->nx + 1, nvy = c->ny + 1, nvz = c->nz + 1, p = c->p;
  double *rc = (double *)calloc(c->nc > 0 ? c->nc : 1, sizeof(double));
  /* r_c = P^T r over the support box of each coarse hat function */
  for (int vz = 0; vz < nvz; ++vz)
    for (int vy = 0; vy < nvy; ++vy)
      for (int vx = 0; vx < nvx; ++vx) {
        int f = c->cfree[vx + nvx * (vy + nvy * vz)];
        if (f < 0) continue;
        double s = 0.0;
        for (int gz = p * (vz - 1); gz <= p * (vz + 1); ++gz)
          for (int gy = p * (vy - 1); gy <= p * (vy + 1); ++gy)
            for (int gx = p * (vx - 1); gx <= p * (vx + 1); ++gx) {
              if (gx < 0 || gy < 0 || gz < 0 || gx >= c->N[0] || gy >= c->N[1] || gz >= c->N[2]) continue;
              if (is_dirichlet(c, gx, gy, gz)) continue;
              s += hat1(c, gx, vx) * hat1(c, gy, vy) * hat1(c, gz, vz) * r[gid(c, gx, gy, gz)];
            }
        rc[f] = s;
      }
  if (c->nc > 0) {
    if (c->gmg_levels > 0) { /* one geometric multigrid V-cycle on the Q1 problem */
      double *xc = (double *)calloc(c->nc, sizeof(double));
      gmg_vcycle(c, 0, rc, xc);
      memcpy(rc, xc, sizeof(double) * c->nc);
      free(xc);
    } else {
      chol_solve(c->nc, c->Lc, rc);
    }
  }
  /* z = P x_c */
  for (int gz = 0; gz < c->N[2]; ++gz)
    for (int gy = 0; gy < c->N[1]; ++gy)
      for (int gx = 0; gx < c->N[0]; ++gx) {
        double s = 0.0;
        if (!is_dirichlet(c, gx, gy, gz)) {
          int v0x = gx / p, v0y = gy / p, v0z = gz / p;
          for (int vz = v0z - 1; vz <= v0z + 1; ++vz)
            for (int vy = v0y - 1; vy <= v0y + 1; ++vy)
              for (int vx = v0x - 1; vx <= v0x + 1; ++vx) {
                if (vx < 0 || vy < 0 || vz < 0 || vx >= nvx || vy >= nvy || vz >= nvz) continue;
                int f = c->cfree[vx + nvx * (vy + nvy * vz)];
                if (f < 0) continue;
                s += hat1(c, gx, vx) * hat1(c, gy, vy) * hat1(c, gz, vz) * rc[f];
              }
        }
        z[gid(c, gx, gy, gz)] = s;
      }
  free(rc);
  return 0;
}

/* ======================================================================
 * hybrid V(1,1), Lanczos damping, PCG (Sections 2.5, 2.8)
 * ====================================================================== */

static double dot(long n, const double *a, const double *b) {
  double s = 0.0;
  for (long i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

int or_pc_apply(const or_ctx *c, const double *r, double *z) {
  long N = c->ndof;
  double *x1 = (double *)malloc(sizeof(double) * N), *t = (double *)malloc(sizeof(double) * N);
  double *r1 = (double *)malloc(sizeof(double) * N);
  int rc = or_asm_apply(c, r, x1); /* pre-relaxation */
  if (rc) goto out;
  or_stiffness_apply(c, x1, t);
  for (long i = 0; i < N; ++i) r1[i] = r[i] - t[i];
  rc = or_coarse_apply(c, r1, t); /* coarse correction */
  if (rc) goto out;
  for (long i = 0; i < N; ++i) x1[i] += t[i];
  or_stiffness_apply(c, x1, t);
  for (long i = 0; i < N; ++i) r1[i] = r[i] - t[i];
  rc = or_asm_apply(c, r1, t); /* post-relaxation */
  if (rc) goto out;
  for (long i = 0; i < N; ++i) z[i] = x1[i] + t[i];
out:
  free(x1); free(t); free(r1);
  return rc;
}

static void zero_dirichlet(const or_ctx *c, double *v) {
  for (int gz = 0; gz < c->N[2]; ++gz)
    for (int gy = 0; gy < c->N[1]; ++gy)
      for (int gx = 0; gx < c->N[0]; ++gx)
        if (is_dirichlet(c, gx, gy, gz)) v[gid(c, gx, gy, gz)] = 0.0;
}

static int apply_pc(const or_ctx *c, int pc, const double *r, double *z) {
  if (pc == 0) { memcpy(z, r, sizeof(double) * c->ndof); zero_dirichlet(c, z); return 0; }
  if (pc == 1) return or_asm_apply(c, r, z);
  return or_pc_apply(c, r, z);
}

int or_pcg(const or_ctx *c, const double *b, double *x, double rtol, int maxit, int pc, int *iters,
           double *hist) {
  long N = c->ndof;
  double *r = (double *)malloc(sizeof(double) * N), *z = (double *)malloc(sizeof(double) * N);
  double *d = (double *)malloc(sizeof(double) * N), *q = (double *)malloc(sizeof(double) * N);
  memset(x, 0, sizeof(double) * N);
  memcpy(r, b, sizeof(double) * N);
  zero_dirichlet(c, r);
  double nb = sqrt(dot(N, r, r)), nr = nb;
  int k = 0, rc = 0, conv = 0;
  if (hist) hist[0] = nr;
  if (nb == 0.0) { conv = 1; goto done; }
  rc = apply_pc(c, pc, r, z);
  if (rc) goto done;
  memcpy(d, z, sizeof(double) * N);
  double rz = dot(N, r, z);
  for (k = 0; k < maxit;) {
    or_stiffness_apply(c, d, q);
    double alpha = rz / dot(N, d, q);
    for (long i = 0; i < N; ++i) { x[i] += alpha * d[i]; r[i] -= alpha * q[i]; }
    ++k;
    nr = sqrt(dot(N, r, r));
    if (hist) hist[k] = nr;
    if (nr <= rtol * nb) { conv = 1; break; }
    rc = apply_pc(c, pc, r, z);
    if (rc) goto done;
    double rz1 = dot(N, r, z), beta = rz1 / rz;
    rz = rz1;
    for (long i = 0; i < N; ++i) d[i] = z[i] + beta * d[i];
  }
done:
  if (iters) *iters = k;
  free(r); free(z); free(d); free(q);
  if (rc) return rc;
  return conv ? 0 : 1;
}

int or_lanczos_omega(or_ctx *c, const double *b0, int kmax, double *lmin, double *lmax, double *omega) {
  /* CG on A x = b0 preconditioned by P_ASM^{-1} (undamped); the CG
   * coefficients give the Lanczos tridiagonal matrix of P_ASM^{-1} A. */
  long N = c->ndof;
  double om = c->omega;
  c->omega = 1.0;
  double *r = (double *)malloc(sizeof(double) * N), *z = (double *)malloc(sizeof(double) * N);
  double *d = (double *)malloc(sizeof(double) * N), *q = (double *)malloc(sizeof(double) * N);
  double *al = (double *)calloc(kmax + 1, sizeof(double)), *be = (double *)calloc(kmax + 1, sizeof(double));
  memcpy(r, b0, sizeof(double) * N);
  zero_dirichlet(c, r);
  int rc = or_asm_apply(c, r, z), k = 0;
  if (rc) goto out;
  memcpy(d, z, sizeof(double) * N);
  double rz = dot(N, r, z);
  for (k = 0; k < kmax; ++k) {
    if (!(rz > 0.0)) break;
    or_stiffness_apply(c, d, q);
    double dq = dot(N, d, q);
    if (!(dq > 0.0)) break;
    al[k] = rz / dq;
    for (long i = 0; i < N; ++i) r[i] -= al[k] * q[i];
    rc = or_asm_apply(c, r, z);
    if (rc) goto out;
    double rz1 = dot(N, r, z);
    be[k] = rz1 / rz;
    rz = rz1;
    for (long i = 0; i < N; ++i) d[i] = z[i] + be[k] * d[i];
  }
  {
    int m = k;
    if (m < 1) { set_err("lanczos: no steps"); rc = -1; goto out; }
    double *Tm = (double *)calloc((size_t)m * m, sizeof(double)), *Q = (double *)malloc(sizeof(double) * m * m);
    for (int j = 0; j < m; ++j) {
      Tm[j * m + j] = 1.0 / al[j] + (j > 0 ? be[j - 1] / al[j - 1] : 0.0);
      if (j + 1 < m) Tm[j * m + j + 1] = Tm[(j + 1) * m + j] = sqrt(be[j]) / al[j];
    }
    jacobi_eig(m, Tm, Q);
    double lo = Tm[0], hi = Tm[0];
    for (int j = 1; j < m; ++j) {
      if (Tm[j * m + j] < lo) lo = Tm[j * m + j];
      if (Tm[j * m + j] > hi) hi = Tm[j * m + j];
    }
    free(Tm);
    free(Q);
    const double a = 0.25;
    om = 2.0 / ((1.0 + a) * hi + (1.0 - a) * lo);
    if (lmin) *lmin = lo;
    if (lmax) *lmax = hi;
    if (omega) *omega = om;
  }
out:
  c->omega = om;
  free(r); free(z); free(d); free(q); free(al); free(be);
  return rc;
}
