// Levels of the geometric multigrid for the Q1 problem (Section 3: the
// p-coarse problem is solved by multigrid).  Level l+1 keeps every other
// vertex of level l along each axis.  The prolongation P interpolates linearly
// along each axis in the vertex coordinates of level l, which is exact on
// nested Q1 spaces, so the Galerkin operator P^T A_l P is the Q1 operator of
// the coarser mesh whenever A_l is a Q1 operator.  Both operators are 27-point
// stencils: a coarse vertex's basis function reaches one fine vertex beyond
// each of its fine children, so two coarse vertices interact only when they
// are stencil neighbours themselves.
#include <cmath>

#include "internal.h"

namespace fdm {

namespace {

// parents of fine vertex v along one axis of a transfer to nc coarse cells:
// (coarse vertex, weight) pairs, Dirichlet vertices (0, nc) dropped
int axis_parents(const std::vector<double> &t, int v, int nc, int V[2], double w[2]) {
  if (v % 2 == 0) {
    V[0] = v / 2;
    w[0] = 1.0;
    return (V[0] >= 1 && V[0] <= nc - 1) ? 1 : 0;
  }
  int k = 0;
  if ((v - 1) / 2 >= 1) { V[k] = (v - 1) / 2; w[k] = 1.0 - t[v]; ++k; }
  if ((v + 1) / 2 <= nc - 1) { V[k] = (v + 1) / 2; w[k] = t[v]; ++k; }
  return k;
}

}  // namespace

void gmg_coarsen(std::vector<GmgHostLevel> &lev, int max_levels) {
  while ((int)lev.size() - 1 < max_levels) {
    GmgHostLevel &F = lev.back();
    bool ok = true;
    for (int a = 0; a < 3; ++a) ok = ok && F.n[a] % 2 == 0 && F.n[a] >= 4;
    if (!ok) break;
    GmgHostLevel C;
    for (int a = 0; a < 3; ++a) {
      C.n[a] = F.n[a] / 2;
      C.m[a] = C.n[a] - 1;
      C.x[a].resize(C.n[a] + 1);
      for (int i = 0; i <= C.n[a]; ++i) C.x[a][i] = F.x[a][2 * i];
      F.t[a].assign(F.n[a] + 1, 0.0);
      for (int v = 1; v < F.n[a]; v += 2)
        F.t[a][v] = (F.x[a][v] - F.x[a][v - 1]) / (F.x[a][v + 1] - F.x[a][v - 1]);
    }
    C.nf = C.m[0] * C.m[1] * C.m[2];
    C.A.assign((size_t)27 * C.nf, 0.0);
    // A_c[I][J] = sum over children i of I, stencil neighbours k of i and
    // parents J of k of P[i][I] A[i][k] P[k][J]
    for (int IZ = 0; IZ < C.m[2]; ++IZ)
      for (int IY = 0; IY < C.m[1]; ++IY)
        for (int IX = 0; IX < C.m[0]; ++IX) {
          const int I = IX + C.m[0] * (IY + C.m[1] * IZ);
          const int Vc[3] = {IX + 1, IY + 1, IZ + 1};
          for (int cz = -1; cz <= 1; ++cz)
            for (int cy = -1; cy <= 1; ++cy)
              for (int cx = -1; cx <= 1; ++cx) {
                const int v[3] = {2 * Vc[0] + cx, 2 * Vc[1] + cy, 2 * Vc[2] + cz};
                const int cc[3] = {cx, cy, cz};
                double wI = 1.0;
                for (int a = 0; a < 3; ++a)
                  wI *= cc[a] == 0 ? 1.0 : (cc[a] < 0 ? F.t[a][v[a]] : 1.0 - F.t[a][v[a]]);
                if (wI == 0.0) continue;
                const int i = (v[0] - 1) + F.m[0] * ((v[1] - 1) + F.m[1] * (v[2] - 1));
                for (int k = 0; k < 27; ++k) {
                  const double aik = F.A[(size_t)k * F.nf + i];
                  if (aik == 0.0) continue;
                  const int u[3] = {v[0] + k % 3 - 1, v[1] + (k / 3) % 3 - 1, v[2] + k / 9 - 1};
                  int Vp[3][2];
                  double wp[3][2];
                  int np[3];
                  for (int a = 0; a < 3; ++a) np[a] = axis_parents(F.t[a], u[a], C.n[a], Vp[a], wp[a]);
                  for (int pz = 0; pz < np[2]; ++pz)
                    for (int py = 0; py < np[1]; ++py)
                      for (int px = 0; px < np[0]; ++px) {
                        const int kc = (Vp[0][px] - Vc[0] + 1) + 3 * (Vp[1][py] - Vc[1] + 1) + 9 * (Vp[2][pz] - Vc[2] + 1);
                        C.A[(size_t)kc * C.nf + I] += wI * aik * (wp[0][px] * wp[1][py] * wp[2][pz]);
                      }
                }
              }
        }
    lev.push_back(std::move(C));
  }
}

}  // namespace fdm
