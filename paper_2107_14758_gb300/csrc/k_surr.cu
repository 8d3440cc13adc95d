// Learned separable surrogate (Section 2.7, Theorem 1): network inputs from
// 27 samples per cell, the per-cell Theorem 1 optimum used as training label,
// and the training / inference kernels of a 189-64-64-3 tanh network.
//
// The bound: for the true cell stiffness with coefficient M_q = kappa Ghat_q at
// the quadrature points q and the separable surrogate with scalings
// D = diag(mu), lo a~(v,v) <= a(v,v) <= hi a~(v,v) where lo (hi) is the smallest
// (largest) eigenvalue of D^{-1/2} M_q D^{-1/2} over q.  The label is the mu
// minimising hi/lo, scaled so that lo * hi = 1, written as c = log(mu/mu_avg).
// The ratio is convex in log mu: log hi is a maximum over unit vectors of
// log-sum-exp functions of -log mu, and -log lo one of log mu.
#include <cmath>

#include "kernels.h"

namespace fdm {
namespace {

// eigenpairs of a symmetric 3x3 matrix by cyclic Jacobi rotations until the
// off-diagonal mass is negligible (at most 12 sweeps): lam[i], column V[.][i]
__device__ void sym3_eig(double a[3][3], double lam[3], double V[3][3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) V[i][j] = i == j ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 12; ++sweep) {
    const double off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const double dia = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2];
    if (off <= 1e-34 * dia) break;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;  // (0,1), (0,2), (1,2)
      const double apq = a[p][q];
      if (apq == 0.0) continue;
      const double th = (a[q][q] - a[p][p]) / (2.0 * apq);
      const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
      const double cs = 1.0 / sqrt(t * t + 1.0), sn = t * cs;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double x = a[k][p], y = a[k][q];
        a[k][p] = cs * x - sn * y;
        a[k][q] = sn * x + cs * y;
        x = V[k][p];
        y = V[k][q];
        V[k][p] = cs * x - sn * y;
        V[k][q] = sn * x + cs * y;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double x = a[p][k], y = a[q][k];
        a[p][k] = cs * x - sn * y;
        a[q][k] = sn * x + cs * y;
      }
    }
  }
  lam[0] = a[0][0];
  lam[1] = a[1][1];
  lam[2] = a[2][2];
}

// extreme eigenpair over the warp: the smallest (largest) value, ties to the
// lower point index; the eigenvector travels with it
struct Extreme {
  double val;
  int q;
  double v[3];
};
template <bool MIN>
__device__ void warp_extreme(Extreme &e) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, e.val, o);
    const int oq = __shfl_xor_sync(0xffffffffu, e.q, o);
    const double o0 = __shfl_xor_sync(0xffffffffu, e.v[0], o), o1 = __shfl_xor_sync(0xffffffffu, e.v[1], o),
                 o2 = __shfl_xor_sync(0xffffffffu, e.v[2], o);
    const bool take = (MIN ? ov < e.val : ov > e.val) || (ov == e.val && oq < e.q);
    if (take) {
      e.val = ov;
      e.q = oq;
      e.v[0] = o0;
      e.v[1] = o1;
      e.v[2] = o2;
    }
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Theorem 1 bound of a cell for the scalings mu, over its nq points (whole
// warp; every lane gets the same result): lo/hi with unit eigenvectors.  Gw
// holds w_q * kappa Ghat_q, divided back by the Gauss weight w_q.
__device__ void cell_bound(const double *Gw, const double *wq, int n, int nq, const double mu[3], Extreme &lo,
                           Extreme &hi) {
  const int lane = threadIdx.x & 31;
  const double s0 = 1.0 / sqrt(mu[0]), s1 = 1.0 / sqrt(mu[1]), s2 = 1.0 / sqrt(mu[2]);
  lo.val = INFINITY;
  hi.val = -INFINITY;
  lo.q = hi.q = 0x7fffffff;
  lo.v[0] = lo.v[1] = lo.v[2] = hi.v[0] = hi.v[1] = hi.v[2] = 0.0;
  for (int q = lane; q < nq; q += 32) {
    const int i = q % n, j = (q / n) % n, k = q / (n * n);
    const double iw = 1.0 / (wq[i] * wq[j] * wq[k]);
    const double *g = Gw + 6 * (size_t)q;
    double a[3][3] = {{g[0] * iw * s0 * s0, g[3] * iw * s0 * s1, g[4] * iw * s0 * s2},
                      {g[3] * iw * s0 * s1, g[1] * iw * s1 * s1, g[5] * iw * s1 * s2},
                      {g[4] * iw * s0 * s2, g[5] * iw * s1 * s2, g[2] * iw * s2 * s2}};
    double lam[3], V[3][3];
    sym3_eig(a, lam, V);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      if (lam[t] < lo.val) {
        lo.val = lam[t];
        lo.q = q;
        lo.v[0] = V[0][t]; lo.v[1] = V[1][t]; lo.v[2] = V[2][t];
      }
      if (lam[t] > hi.val) {
        hi.val = lam[t];
        hi.q = q;
        hi.v[0] = V[0][t]; hi.v[1] = V[1][t]; hi.v[2] = V[2][t];
      }
    }
  }
  warp_extreme<true>(lo);
  warp_extreme<false>(hi);
}

struct SurrArgs {
  int ncell, n, nq;
  const double *Gw;    // [cell][nq][6] weighted kappa Ghat (FP64)
  const double *wq;    // n Gauss weights
  const double *mubar; // [cell][3] averaged surrogate
};

// One warp per cell.  With mu = mubar exp(u), u = (0, x1, x2) (the ratio is
// invariant to a common scaling), F(x) = log(hi/lo) is convex in x and is
// minimised by the central-cut ellipsoid method: subgradient
// g_a = v_lo,a^2 - v_hi,a^2 (d log lambda / d u_a = -v_a^2 for the unit
// eigenvector v of the scaled matrix), ellipsoid {x + B z : |z| <= 1} from the
// disc of radius SURR_RADIUS, factor update B <- (2/sqrt 3) B (I + (1/sqrt 3 - 1)
// e e^T) with e = B^T g / |B^T g|, stop when |B^T g| <= SURR_TOL (a bound on the
// gap to the minimum) or after SURR_MAXIT steps; the best point seen is kept.
__global__ void __launch_bounds__(128) k_surr_label(SurrArgs a, double *cstar, double *F0, double *F1) {
  const int e = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (e >= a.ncell) return;  // warp-uniform
  const double *Gw = a.Gw + (size_t)e * a.nq * 6;
  const double mb[3] = {a.mubar[3 * e], a.mubar[3 * e + 1], a.mubar[3 * e + 2]};
  const double ca = 2.0 / sqrt(3.0), cb = 1.0 / sqrt(3.0) - 1.0;
  double x0 = 0.0, x1 = 0.0;
  double B00 = SURR_RADIUS, B01 = 0.0, B10 = 0.0, B11 = SURR_RADIUS;
  double best = INFINITY, bx0 = 0.0, bx1 = 0.0, f0 = 0.0;
  Extreme lo, hi;
  for (int it = 0; it < SURR_MAXIT; ++it) {
    const double mu[3] = {mb[0], mb[1] * exp(x0), mb[2] * exp(x1)};
    cell_bound(Gw, a.wq, a.n, a.nq, mu, lo, hi);
    const double F = log(hi.val / lo.val);
    if (it == 0) f0 = F;
    if (F < best) {
      best = F;
      bx0 = x0;
      bx1 = x1;
    }
    const double g0 = lo.v[1] * lo.v[1] - hi.v[1] * hi.v[1], g1 = lo.v[2] * lo.v[2] - hi.v[2] * hi.v[2];
    const double bg0 = B00 * g0 + B10 * g1, bg1 = B01 * g0 + B11 * g1;  // B^T g
    const double r = sqrt(bg0 * bg0 + bg1 * bg1);
    if (!(r > SURR_TOL)) break;
    const double e0 = bg0 / r, e1 = bg1 / r;
    const double be0 = B00 * e0 + B01 * e1, be1 = B10 * e0 + B11 * e1;  // B e
    x0 -= be0 / 3.0;
    x1 -= be1 / 3.0;
    B00 = ca * (B00 + cb * be0 * e0);
    B01 = ca * (B01 + cb * be0 * e1);
    B10 = ca * (B10 + cb * be1 * e0);
    B11 = ca * (B11 + cb * be1 * e1);
  }
  const double mu[3] = {mb[0], mb[1] * exp(bx0), mb[2] * exp(bx1)};
  cell_bound(Gw, a.wq, a.n, a.nq, mu, lo, hi);
  if ((threadIdx.x & 31) == 0) {
    const double sh = 0.5 * log(lo.val * hi.val);  // centre the bound's spectrum: lo * hi = 1
    cstar[3 * e] = sh;
    cstar[3 * e + 1] = bx0 + sh;
    cstar[3 * e + 2] = bx1 + sh;
    F0[e] = f0;
    F1[e] = best;
  }
}

__global__ void __launch_bounds__(128) k_surr_bound(SurrArgs a, const double *mu, double *F) {
  const int e = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (e >= a.ncell) return;
  const double m[3] = {mu[3 * e], mu[3 * e + 1], mu[3 * e + 2]};
  Extreme lo, hi;
  cell_bound(a.Gw + (size_t)e * a.nq * 6, a.wq, a.n, a.nq, m, lo, hi);
  if ((threadIdx.x & 31) == 0) F[e] = log(hi.val / lo.val);
}

// one warp per cell, lane q < 27 handles sample q of the 3x3x3 Gauss rule
__global__ void __launch_bounds__(128) k_surr_features(int ncell, const double *s27, double w0, double w1,
                                                       float *feat) {
  const int e = blockIdx.x * 4 + (threadIdx.x >> 5);
  const int q = threadIdx.x & 31;
  if (e >= ncell) return;
  const bool on = q < 27;
  double G[6] = {1, 1, 1, 0, 0, 0}, lk = 0.0, w = 0.0;
  if (on) {
    const double *s = s27 + ((size_t)e * 27 + q) * 10;
    const double *J = s + 1;
    const double a00 = J[4] * J[8] - J[5] * J[7], a01 = J[2] * J[7] - J[1] * J[8], a02 = J[1] * J[5] - J[2] * J[4];
    const double a10 = J[5] * J[6] - J[3] * J[8], a11 = J[0] * J[8] - J[2] * J[6], a12 = J[2] * J[3] - J[0] * J[5];
    const double a20 = J[3] * J[7] - J[4] * J[6], a21 = J[1] * J[6] - J[0] * J[7], a22 = J[0] * J[4] - J[1] * J[3];
    const double det = J[0] * a00 + J[1] * a10 + J[2] * a20;
    const double Ji[9] = {a00 / det, a01 / det, a02 / det, a10 / det, a11 / det,
                          a12 / det, a20 / det, a21 / det, a22 / det};
    const double sc = s[0] * fabs(det);
    auto gg = [&](int r, int t) {
      return sc * (Ji[3 * r] * Ji[3 * t] + Ji[3 * r + 1] * Ji[3 * t + 1] + Ji[3 * r + 2] * Ji[3 * t + 2]);
    };
    G[0] = gg(0, 0); G[1] = gg(1, 1); G[2] = gg(2, 2);
    G[3] = gg(0, 1); G[4] = gg(0, 2); G[5] = gg(1, 2);
    lk = log(s[0]);
    auto wt = [&](int i) { return i == 1 ? w1 : w0; };
    w = wt(q % 3) * wt((q / 3) % 3) * wt(q / 9);
  }
  const double nu0 = warp_sum_d(w * G[0]) / 8.0, nu1 = warp_sum_d(w * G[1]) / 8.0, nu2 = warp_sum_d(w * G[2]) / 8.0;
  const double lbar = warp_sum_d(w * lk) / 8.0;
  if (on) {
    float *f = feat + (size_t)e * MLP_NIN + 7 * q;
    f[0] = (float)(lk - lbar);
    f[1] = (float)log(G[0] / nu0);
    f[2] = (float)log(G[1] / nu1);
    f[3] = (float)log(G[2] / nu2);
    f[4] = (float)(G[3] / sqrt(G[0] * G[1]));
    f[5] = (float)(G[4] / sqrt(G[0] * G[2]));
    f[6] = (float)(G[5] / sqrt(G[1] * G[2]));
  }
}

// ---- network: 189 -> 64 tanh -> 64 tanh -> 3, FP32 ------------------------
constexpr int NIN = MLP_NIN, NH = MLP_NH, NOUT = MLP_NOUT;
constexpr int OFF_B1 = NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH, OFF_W3 = OFF_B2 + NH,
              OFF_B3 = OFF_W3 + NOUT * NH;
static_assert(OFF_B3 + NOUT == MLP_NPARAM, "parameter layout");
constexpr int CB = 32;   // cells per CTA
constexpr int MT = 128;  // threads per CTA: 64 units x 2 halves of the cells
constexpr int LD = NH + 1;  // padded rows of the transposed weights (conflict-free both ways)
constexpr int SM_W1T = 0, SM_W2T = SM_W1T + NIN * LD, SM_W3 = SM_W2T + NH * LD, SM_B1 = SM_W3 + NOUT * NH,
              SM_B2 = SM_B1 + NH, SM_B3 = SM_B2 + NH, SM_X = SM_B3 + 4, SM_H1 = SM_X + CB * NIN,
              SM_H2 = SM_H1 + CB * NH, SM_D1 = SM_H2 + CB * NH, SM_D2 = SM_D1 + CB * NH, SM_O = SM_D2 + CB * NH,
              SM_D3 = SM_O + CB * 4, SM_RED = SM_D3 + CB * 4, SM_TOTAL = SM_RED + MT;
constexpr size_t MLP_SMEM = sizeof(float) * SM_TOTAL;

// Forward pass of CB cells; with labels also the loss share and this CTA's
// partial gradient (backpropagation through the three layers, tanh' = 1 - tanh^2).
__global__ void __launch_bounds__(MT) k_mlp(int ncell, const float *__restrict__ P, const float *__restrict__ feat,
                                            const float *__restrict__ label, float inv_n, float *__restrict__ out,
                                            float *__restrict__ partial, float *__restrict__ lossp) {
  extern __shared__ float sm[];
  float *w1t = sm + SM_W1T, *w2t = sm + SM_W2T, *w3 = sm + SM_W3, *b1 = sm + SM_B1, *b2 = sm + SM_B2,
        *b3 = sm + SM_B3, *x = sm + SM_X, *h1 = sm + SM_H1, *h2 = sm + SM_H2, *d1 = sm + SM_D1, *d2 = sm + SM_D2,
        *o = sm + SM_O, *d3 = sm + SM_D3, *red = sm + SM_RED;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * CB;
  const int nc = min(CB, ncell - c0);
  for (int i = tid; i < NH * NIN; i += MT) {
    const int j = i / NIN, k = i - j * NIN;
    w1t[k * LD + j] = P[i];
  }
  for (int i = tid; i < NH * NH; i += MT) {
    const int j = i / NH, k = i - j * NH;
    w2t[k * LD + j] = P[OFF_W2 + i];
  }
  for (int i = tid; i < NOUT * NH; i += MT) w3[i] = P[OFF_W3 + i];
  if (tid < NH) {
    b1[tid] = P[OFF_B1 + tid];
    b2[tid] = P[OFF_B2 + tid];
  }
  if (tid < NOUT) b3[tid] = P[OFF_B3 + tid];
  for (int i = tid; i < CB * NIN; i += MT) x[i] = i < nc * NIN ? feat[(size_t)c0 * NIN + i] : 0.f;
  __syncthreads();

  const int j = tid & (NH - 1), cb = (tid >> 6) * (CB / 2);
  float acc[CB / 2];
#pragma unroll
  for (int t = 0; t < CB / 2; ++t) acc[t] = b1[j];
  for (int k = 0; k < NIN; ++k) {
    const float w = w1t[k * LD + j];
#pragma unroll
    for (int t = 0; t < CB / 2; ++t) acc[t] = fmaf(w, x[(cb + t) * NIN + k], acc[t]);
  }
#pragma unroll
  for (int t = 0; t < CB / 2; ++t) h1[(cb + t) * NH + j] = tanhf(acc[t]);
  __syncthreads();
#pragma unroll
  for (int t = 0; t < CB / 2; ++t) acc[t] = b2[j];
  for (int k = 0; k < NH; ++k) {
    const float w = w2t[k * LD + j];
#pragma unroll
    for (int t = 0; t < CB / 2; ++t) acc[t] = fmaf(w, h1[(cb + t) * NH + k], acc[t]);
  }
#pragma unroll
  for (int t = 0; t < CB / 2; ++t) h2[(cb + t) * NH + j] = tanhf(acc[t]);
  __syncthreads();
  if (tid < CB * NOUT) {
    const int c = tid / NOUT, oo = tid - c * NOUT;
    float s = b3[oo];
    for (int k = 0; k < NH; ++k) s = fmaf(w3[oo * NH + k], h2[c * NH + k], s);
    o[c * 4 + oo] = s;
    if (c < nc) out[(size_t)(c0 + c) * NOUT + oo] = s;
  }
  if (!label) return;  // inference only (uniform over the CTA)
  __syncthreads();
  float ls = 0.f;
  if (tid < CB * NOUT) {
    const int c = tid / NOUT, oo = tid - c * NOUT;
    const float r = c < nc ? o[c * 4 + oo] - label[(size_t)(c0 + c) * NOUT + oo] : 0.f;
    d3[c * 4 + oo] = r * inv_n;
    ls = 0.5f * r * r * inv_n;
  }
  red[tid] = ls;
  __syncthreads();
#pragma unroll
  for (int t = 0; t < CB / 2; ++t) {
    const int c = cb + t;
    float s = 0.f;
#pragma unroll
    for (int oo = 0; oo < NOUT; ++oo) s = fmaf(w3[oo * NH + j], d3[c * 4 + oo], s);
    const float hv = h2[c * NH + j];
    d2[c * NH + j] = s * (1.f - hv * hv);
  }
  if (tid == 0) {
    float s = 0.f;
    for (int i = 0; i < MT; ++i) s += red[i];
    lossp[blockIdx.x] = s;
  }
  __syncthreads();
#pragma unroll 4
  for (int t = 0; t < CB / 2; ++t) {
    const int c = cb + t;
    float s = 0.f;
    for (int i = 0; i < NH; ++i) s = fmaf(w2t[j * LD + i], d2[c * NH + i], s);  // sum_i W2[i][j] d2[c][i]
    const float hv = h1[c * NH + j];
    d1[c * NH + j] = s * (1.f - hv * hv);
  }
  __syncthreads();
  float *pp = partial + (size_t)blockIdx.x * MLP_NPARAM;
  for (int i = tid; i < MLP_NPARAM; i += MT) {
    float s = 0.f;
    if (i < OFF_B1) {
      const int u = i / NIN, k = i - u * NIN;
      for (int c = 0; c < CB; ++c) s = fmaf(d1[c * NH + u], x[c * NIN + k], s);
    } else if (i < OFF_W2) {
      for (int c = 0; c < CB; ++c) s += d1[c * NH + (i - OFF_B1)];
    } else if (i < OFF_B2) {
      const int r = i - OFF_W2, u = r / NH, k = r - u * NH;
      for (int c = 0; c < CB; ++c) s = fmaf(d2[c * NH + u], h1[c * NH + k], s);
    } else if (i < OFF_W3) {
      for (int c = 0; c < CB; ++c) s += d2[c * NH + (i - OFF_B2)];
    } else if (i < OFF_B3) {
      const int r = i - OFF_W3, u = r / NH, k = r - u * NH;
      for (int c = 0; c < CB; ++c) s = fmaf(d3[c * 4 + u], h2[c * NH + k], s);
    } else {
      for (int c = 0; c < CB; ++c) s += d3[c * 4 + (i - OFF_B3)];
    }
    pp[i] = s;
  }
}

// grad[i] = sum over CTAs of the partial gradients, in CTA order (FP64 sum)
__global__ void k_mlp_reduce(int nblk, const float *__restrict__ partial, const float *__restrict__ lossp,
                             float *__restrict__ grad, double *__restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < MLP_NPARAM) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * MLP_NPARAM + i];
    grad[i] = (float)s;
  }
  if (i == 0 && loss) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += lossp[b];
    *loss = s;
  }
}

// Adam with bias-corrected moments (Kingma & Ba, 2015) and decoupled weight decay
__global__ void k_adam(int n, float *__restrict__ P, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float c1, float c2, float wd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = ADAM_BETA1 * m[i] + (1.f - ADAM_BETA1) * gi;
  const float vi = ADAM_BETA2 * v[i] + (1.f - ADAM_BETA2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * ((mi / c1) / (sqrtf(vi / c2) + ADAM_EPS) + wd * P[i]);
}

// mu = mubar exp(c), or mubar for the whole cell where c is not finite or |c| > SURR_CMAX
__global__ void k_surr_apply(int ncell, const float *__restrict__ c, const double *__restrict__ mubar,
                             double *__restrict__ mu, int *__restrict__ nfall) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ncell) return;
  bool ok = true;
  for (int a = 0; a < 3; ++a) {
    const float v = c[3 * e + a];
    ok = ok && isfinite(v) && fabsf(v) <= SURR_CMAX;
  }
  for (int a = 0; a < 3; ++a) mu[3 * e + a] = ok ? mubar[3 * e + a] * exp((double)c[3 * e + a]) : mubar[3 * e + a];
  if (!ok) atomicAdd(nfall, 1);
}

}  // namespace

size_t mlp_smem_bytes() { return MLP_SMEM; }

void launch_surr_features(int ncell, const double *s27, const double w3[3], float *feat, cudaStream_t st) {
  k_surr_features<<<(ncell + 3) / 4, 128, 0, st>>>(ncell, s27, w3[0], w3[1], feat);
  FDM_CUDA(cudaGetLastError());
}

void launch_surr_label(int ncell, int n, const double *Gw, const double *wq, const double *mubar, double *cstar,
                       double *F0, double *F1, cudaStream_t st) {
  SurrArgs a{ncell, n, n * n * n, Gw, wq, mubar};
  k_surr_label<<<(ncell + 3) / 4, 128, 0, st>>>(a, cstar, F0, F1);
  FDM_CUDA(cudaGetLastError());
}

void launch_surr_bound(int ncell, int n, const double *Gw, const double *wq, const double *mu, double *F,
                       cudaStream_t st) {
  SurrArgs a{ncell, n, n * n * n, Gw, wq, nullptr};
  k_surr_bound<<<(ncell + 3) / 4, 128, 0, st>>>(a, mu, F);
  FDM_CUDA(cudaGetLastError());
}

int mlp_blocks(int ncell) { return (ncell + CB - 1) / CB; }

void launch_mlp(int ncell, const float *P, const float *feat, const float *label, float *out, float *partial,
                float *lossp, cudaStream_t st) {
  if (ncell <= 0) return;
  FDM_CUDA(cudaFuncSetAttribute(k_mlp, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MLP_SMEM));
  k_mlp<<<mlp_blocks(ncell), MT, MLP_SMEM, st>>>(ncell, P, feat, label, 1.f / (float)ncell, out, partial, lossp);
  FDM_CUDA(cudaGetLastError());
}

void launch_mlp_reduce(int nblk, const float *partial, const float *lossp, float *grad, double *loss,
                       cudaStream_t st) {
  k_mlp_reduce<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(nblk, partial, lossp, grad, loss);
  FDM_CUDA(cudaGetLastError());
}

void launch_adam(float *P, const float *g, float *m, float *v, int t, double lr, double wd, cudaStream_t st) {
  const double c1 = 1.0 - std::pow((double)ADAM_BETA1, t), c2 = 1.0 - std::pow((double)ADAM_BETA2, t);
  k_adam<<<(MLP_NPARAM + 255) / 256, 256, 0, st>>>(MLP_NPARAM, P, g, m, v, (float)lr, (float)c1, (float)c2,
                                                   (float)wd);
  FDM_CUDA(cudaGetLastError());
}

void launch_surr_apply(int ncell, const float *c, const double *mubar, double *mu, int *nfall, cudaStream_t st) {
  k_surr_apply<<<(ncell + 127) / 128, 128, 0, st>>>(ncell, c, mubar, mu, nfall);
  FDM_CUDA(cudaGetLastError());
}

}  // namespace fdm
