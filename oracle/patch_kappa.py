"""Surrogate labels scored by the condition number of a patch (FP64 CPU
reference; TEST INFRASTRUCTURE ONLY: the product path never imports it).

Section 2.7 replaces the stiffness of a curved cell by a separable surrogate
with one scaling mu_a per reference direction, and Theorem 1 bounds the
spectrum of the true stiffness against it.  Here each candidate mu is scored by
the quantity the relaxation feels: the condition number of the surrogate-
preconditioned patch matrix, kappa(A~_P(mu)^{-1} A_P), estimated by Lanczos,
with P the patch of the cell's interior functions (homogeneous Dirichlet on
the cell boundary).  Plain definitions throughout:

* A_P: the true cell stiffness sum_q w_q grad phi_i . (kappa Ghat_q) grad phi_j
  on the interior GLL functions, assembled densely from the Gauss points;
* A~_P(mu) = mu_x B (x) B (x) A + mu_y B (x) A (x) B + mu_z A (x) B (x) B on the
  interior block of the reference 1D stiffness A and mass B;
* the estimate: Lanczos with full reorthogonalisation (two classical
  Gram-Schmidt passes per step), K = min(48, m) steps from the fixed start
  vector r0 below, on the symmetric form C = D^{-1/2} S^T A_P S D^{-1/2} of
  A~_P^{-1} A_P, where S = S_1 (x) S_1 (x) S_1 is the interior FDM basis
  (A_II S_1 = B_II S_1 Lam, S_1^T B_II S_1 = I, Section 2.3) and
  D = mu_x lam_i + mu_y lam_j + mu_z lam_k, so that A~_P = S^{-T} D S^{-1};
  the run stops early once the next Lanczos vector's norm falls below 1e-10
  times the largest diagonal entry; the extreme eigenvalues of the Lanczos
  tridiagonal matrix (numpy's symmetric routine) estimate lambda_min and
  lambda_max;
* the label: mu = mubar exp(c), c = (0, t1, t2) + gamma (1, 1, 1); (t1, t2)
  minimises log(lambda_max / lambda_min) by compass search from 0 (the four
  moves +-s along t1 then t2 are scored, the best one that lowers it by more
  than 1e-9 is taken, else s is halved; s from 1/2 down to below 1/256, at
  most 48 rounds),
  and gamma = log(lambda_min lambda_max) / 2 centres the spectrum of the
  labelled patch (lambda_min lambda_max = 1), as the Theorem 1 labels centre
  their bound.
"""
import numpy as np

from . import basis1d, gauss, lagrange

LANCZOS_STEPS = 48
SEARCH_S0 = 0.5
SEARCH_SMIN = 1.0 / 256.0
SEARCH_ROUNDS = 48
IMPROVE = 1e-9  # a move must lower log kappa by more than this
BREAKDOWN = 1e-10  # relative norm of the next Lanczos vector that ends the run


def start_vector(m):
    """r0[i] = frac(i * 0.6180339887...) - 1/2, the fractional part of i times the
    golden ratio conjugate taken in exact integer arithmetic: (i * 2654435769
    mod 2^32) / 2^32 - 1/2."""
    i = np.arange(m, dtype=np.uint64)
    return ((i * np.uint64(2654435769)) % np.uint64(1 << 32)).astype(np.float64) / float(1 << 32) - 0.5


class CellPatches:
    """The interior patches of the cells: G[cell][q][6] the unweighted kappa
    Ghat at the (p+1)^3 Gauss points (00, 11, 22, 01, 02, 12; q = i + n (j + n k)),
    mubar[cell][3] the averaged surrogate."""

    def __init__(self, p, G, mubar):
        if p < 2:
            raise ValueError("interior patches need p >= 2")
        self.p, n = p, p + 1
        self.G = np.asarray(G, dtype=np.float64).reshape(-1, n ** 3, 6)
        self.mubar = np.asarray(mubar, dtype=np.float64).reshape(-1, 3)
        b = basis1d(p)
        xg, wg = gauss(n)
        V, D = lagrange(p, b["xi"], xg)
        Vi, Di = V[:, 1:p], D[:, 1:p]  # interior functions at the Gauss points
        # reference gradients of the interior functions at the Gauss points, [3][q][m]
        self.grad = np.stack([np.kron(Vi, np.kron(Vi, Di)), np.kron(Vi, np.kron(Di, Vi)),
                              np.kron(Di, np.kron(Vi, Vi))])
        self.w = np.kron(wg, np.kron(wg, wg))
        Ai, Bi = b["A"][1:p, 1:p], b["B"][1:p, 1:p]
        self.K = [np.kron(Bi, np.kron(Bi, Ai)), np.kron(Bi, np.kron(Ai, Bi)), np.kron(Ai, np.kron(Bi, Bi))]
        self.S3 = np.kron(b["S"], np.kron(b["S"], b["S"]))
        lam = b["lam"]
        self.lam3 = [np.kron(np.ones(p - 1), np.kron(np.ones(p - 1), lam)),
                     np.kron(np.ones(p - 1), np.kron(lam, np.ones(p - 1))),
                     np.kron(lam, np.kron(np.ones(p - 1), np.ones(p - 1)))]
        self.m = (p - 1) ** 3
        self.r0 = start_vector(self.m)

    def true_matrix(self, e):
        G = self.G[e]
        idx = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
        A = np.zeros((self.m, self.m))
        for a in range(3):
            for c in range(3):
                A += self.grad[a].T @ ((self.w * G[:, idx[(a, c)]])[:, None] * self.grad[c])
        return A

    def surrogate_matrix(self, mu):
        return mu[0] * self.K[0] + mu[1] * self.K[1] + mu[2] * self.K[2]

    def symmetric_form(self, A, mu):
        """C = D^{-1/2} S^T A S D^{-1/2}, similar to A~(mu)^{-1} A."""
        D = mu[0] * self.lam3[0] + mu[1] * self.lam3[1] + mu[2] * self.lam3[2]
        R = self.S3 / np.sqrt(D)[None, :]
        return R.T @ A @ R

    def lanczos(self, A, mu, steps=LANCZOS_STEPS):
        """(lambda_min, lambda_max) estimates of A~(mu)^{-1} A."""
        C = self.symmetric_form(A, mu)
        K = min(steps, self.m)
        V = [self.r0 / np.linalg.norm(self.r0)]
        al, be = [], []
        for k in range(K):
            w = C @ V[k]
            al.append(w @ V[k])
            w = w - al[k] * V[k] - (be[k - 1] * V[k - 1] if k > 0 else 0.0)
            for _ in range(2):
                Vm = np.array(V)
                w = w - Vm.T @ (Vm @ w)
            b = np.linalg.norm(w)
            if k == K - 1 or not b > BREAKDOWN * max(abs(x) for x in al):
                break
            be.append(b)
            V.append(w / b)
        k = len(al)
        T = np.diag(al) + np.diag(be[:k - 1], 1) + np.diag(be[:k - 1], -1)
        ev = np.linalg.eigvalsh(T)
        return ev[0], ev[-1]

    def log_kappa(self, e, c, A=None):
        A = self.true_matrix(e) if A is None else A
        lo, hi = self.lanczos(A, self.mubar[e] * np.exp(c))
        return np.log(hi / lo), lo, hi

    def label(self, e):
        """(c[3], log kappa at mubar, log kappa at the label, evaluations)."""
        A = self.true_matrix(e)
        t = np.zeros(2)
        f, _, _ = self.log_kappa(e, np.array([0.0, 0.0, 0.0]), A)
        f0, s, evals = f, SEARCH_S0, 1
        for _ in range(SEARCH_ROUNDS):
            if s < SEARCH_SMIN:
                break
            best, bt = f, None
            for dt in ((s, 0.0), (-s, 0.0), (0.0, s), (0.0, -s)):
                tt = t + np.array(dt)
                ft, _, _ = self.log_kappa(e, np.array([0.0, tt[0], tt[1]]), A)
                evals += 1
                if ft < best - IMPROVE:
                    best, bt = ft, tt
            if bt is None:
                s *= 0.5
            else:
                t, f = bt, best
        c = np.array([0.0, t[0], t[1]])
        f1, lo, hi = self.log_kappa(e, c, A)
        gamma = 0.5 * np.log(lo * hi)
        return c + gamma, f0, f1, evals

    def labels(self):
        out = [self.label(e) for e in range(self.G.shape[0])]
        return (np.array([o[0] for o in out]), np.array([o[1] for o in out]), np.array([o[2] for o in out]))
