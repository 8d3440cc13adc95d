"""Primal linear elasticity with the SDC/FDM/sparse relaxation (Section 4.1):
the FP64 CPU oracle, in numpy on top of the scalar oracle.  Test
infrastructure only: only the test suite, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may use it.

Discretisation.  Each displacement component is a Q_p function on the
tensor GLL grid of the scalar problem; vectors are component-major [3, N]
(N grid nodes, x fastest).  Box cells, homogeneous isotropic material with
Lame parameters mu, lam:

    a(v, u) = int 2 mu eps(v):eps(u) + lam div v div u.

Block (i, i) of the stiffness is mu grad v_i . grad u_i + (mu + lam) d_i v_i
d_i u_i; block (i, j), i != j, is mu d_j v_i d_i u_j + lam d_i v_i d_j u_j.
On a box cell with half-widths L and volume factor vol = L_x L_y L_z every
term is a Kronecker product of 1D matrices: A_hat (int l' l'), B_hat
(int l l) and C_hat (int l_k' l_l: test derivative, trial value), scaled by
vol / (L_a L_b).  The Dirichlet boundary is the whole of the boundary (all
three components), as for the scalar problem.

SDC relaxation: the block-diagonal A_SDC = diag(A_11, A_22, A_33) (Section
4.1).  Block A_jj is the scalar operator with per-axis coefficients
mu + (mu + lam) delta_aj, which is separable on box cells, so it takes the
scalar vertex-star FDM/sparse relaxation with the per-cell surrogate
mu_a^(j) = (mu + (mu + lam) delta_aj) vol / L_a^2, exactly.

Preconditioner: the hybrid V(1,1) of the scalar problem (Section 2.5) with
the SDC relaxation, the elasticity residual, and the vector Q1 Galerkin
coarse problem P^T A P (P the trilinear interpolation of each component)
solved exactly.  Damping omega from 20 CG-Lanczos steps on A_SDC^{-1} A.
"""
import numpy as np

from . import Problem, basis1d, gauss, lagrange


def c_hat(p):
    """C_hat[k, l] = int_{-1}^{1} l_k'(s) l_l(s) ds (Gauss, q = p + 1: exact)."""
    xi = basis1d(p)["xi"]
    xq, wq = gauss(p + 1)
    V, D = lagrange(p, xi, xq)
    return D.T @ (wq[:, None] * V)


def _kron_cells(M, U):
    """Applies Mz (x) My (x) Mx to cell arrays U[c, z, y, x]."""
    Mx, My, Mz = M
    U = np.einsum("ij,czyj->czyi", Mx, U)
    U = np.einsum("ij,czjx->czix", My, U)
    return np.einsum("ij,cjyx->ciyx", Mz, U)


class Elasticity:
    """Q_p elasticity on a tensor mesh of box cells, clamped on the boundary."""

    def __init__(self, p, xv, yv, zv, mu, lam):
        self.p, self.mu, self.lam = p, float(mu), float(lam)
        self.v = [np.asarray(a, dtype=np.float64) for a in (xv, yv, zv)]
        self.nc = [len(a) - 1 for a in self.v]
        self.Nn = [c * p + 1 for c in self.nc]
        self.N = self.Nn[0] * self.Nn[1] * self.Nn[2]
        b = basis1d(p)
        self.A1, self.B1, self.C1 = b["A"], b["B"], c_hat(p)
        self.xi = b["xi"]
        # half-widths per cell and axis, cells x fastest
        h = [0.5 * np.diff(a) for a in self.v]
        L = np.stack(np.meshgrid(h[0], h[1], h[2], indexing="ij"), axis=-1)   # [cx, cy, cz, 3]
        self.L = np.transpose(L, (2, 1, 0, 3)).reshape(-1, 3)                # [cell, 3]
        self.vol = self.L.prod(axis=1)
        m = np.ones(self.Nn[::-1], dtype=bool)
        m[0], m[-1], m[:, 0], m[:, -1], m[:, :, 0], m[:, :, -1] = (False,) * 6
        self.free = m.ravel()
        # cell -> grid node index table [cell, z, y, x]
        n = p + 1
        idx = []
        for cz in range(self.nc[2]):
            for cy in range(self.nc[1]):
                for cx in range(self.nc[0]):
                    g = (np.arange(n)[None, None, :] + cx * p) + self.Nn[0] * (
                        (np.arange(n)[None, :, None] + cy * p) + self.Nn[1] * (np.arange(n)[:, None, None] + cz * p))
                    idx.append(g)
        self.cidx = np.array(idx)
        self.comps = None
        self.Ac = None
        self.omega = 1.0

    # ------------------------------------------------------------ operator
    def sdc_mu(self, j):
        """Per-cell surrogate [cell, 3] of the diagonal block A_jj (exact on box cells)."""
        c = np.full(3, self.mu)
        c[j] += self.mu + self.lam
        return c[None, :] * self.vol[:, None] / self.L ** 2

    def apply(self, u):
        """y = A u, u and y [3, N]; Dirichlet entries of u ignored, of y zero."""
        u = np.where(self.free, np.asarray(u, dtype=np.float64).reshape(3, self.N), 0.0)
        Uc = [u[a][self.cidx] for a in range(3)]
        A, B, C = self.A1, self.B1, self.C1
        y = np.zeros((3, self.N))
        for a in range(3):
            Ya = np.zeros_like(Uc[0])
            for b in range(3):
                if a == b:
                    for d in range(3):
                        coef = (self.mu + (self.mu + self.lam) * (d == a)) * self.vol / self.L[:, d] ** 2
                        M = [B, B, B]
                        M[d] = A
                        Ya += coef[:, None, None, None] * _kron_cells(M, Uc[b])
                else:
                    s = self.vol / (self.L[:, a] * self.L[:, b])
                    t = 3 - a - b
                    Mmu = [None] * 3
                    Mmu[b], Mmu[a], Mmu[t] = C, C.T, B          # mu d_b v_a d_a u_b
                    Mla = [None] * 3
                    Mla[a], Mla[b], Mla[t] = C, C.T, B          # lam d_a v_a d_b u_b
                    Ya += s[:, None, None, None] * (self.mu * _kron_cells(Mmu, Uc[b]) +
                                                    self.lam * _kron_cells(Mla, Uc[b]))
            np.add.at(y[a], self.cidx.ravel(), Ya.ravel())
        return np.where(self.free, y, 0.0)

    def body_force(self, f):
        """Load vector of a constant body force f (3 components): b_a = f_a int phi."""
        b1 = self.B1.sum(axis=1)
        w = np.einsum("k,j,i->kji", b1, b1, b1)[None] * self.vol[:, None, None, None]
        m = np.zeros(self.N)
        np.add.at(m, self.cidx.ravel(), np.broadcast_to(w, self.cidx.shape).ravel())
        return np.where(self.free, np.outer(np.asarray(f, dtype=np.float64), m), 0.0)

    # ------------------------------------------------------------ SDC relaxation
    def setup_sdc(self):
        self.comps = []
        for j in range(3):
            P = Problem(self.p, *self.v)
            P.set_mu(self.sdc_mu(j))
            P.setup_patches()
            P.set_omega(1.0)
            self.comps.append(P)

    def sdc(self, r):
        """Undamped additive Schwarz with the SDC blocks: [ASM_j(r_j)]."""
        r = np.asarray(r, dtype=np.float64).reshape(3, self.N)
        return np.stack([self.comps[j].asm_apply(r[j]) for j in range(3)])

    # ------------------------------------------------------------ coarse space
    def _hat(self, a):
        """W[g, v]: Q1 hat of vertex v at grid node g along axis a (GLL nodes)."""
        p, nc = self.p, self.nc[a]
        W = np.zeros((self.Nn[a], nc + 1))
        for g in range(self.Nn[a]):
            if g % p == 0:
                W[g, g // p] = 1.0
            else:
                c, i = divmod(g, p)
                W[g, c] = 0.5 * (1.0 - self.xi[i])
                W[g, c + 1] = 0.5 * (1.0 + self.xi[i])
        return W

    def prolong(self, xc):
        """Fine [3, N] from coarse [3, nq] (free Q1 vertices, x fastest)."""
        W = [self._hat(a) for a in range(3)]
        nv = [c + 1 for c in self.nc]
        out = np.zeros((3, self.N))
        for a in range(3):
            X = np.zeros(nv[::-1])
            X[1:-1, 1:-1, 1:-1] = xc[a].reshape(nv[2] - 2, nv[1] - 2, nv[0] - 2)
            out[a] = np.einsum("zc,yb,xa,cba->zyx", W[2], W[1], W[0], X).ravel()
        return np.where(self.free, out, 0.0)

    def restrict(self, r):
        W = [self._hat(a) for a in range(3)]
        r = np.where(self.free, np.asarray(r).reshape(3, self.N), 0.0)
        out = []
        for a in range(3):
            R = r[a].reshape(self.Nn[::-1])
            X = np.einsum("zc,yb,xa,zyx->cba", W[2], W[1], W[0], R)
            out.append(X[1:-1, 1:-1, 1:-1].ravel())
        return np.stack(out)

    def setup_coarse(self):
        """A_c = P^T A P (vector Q1 Galerkin), column by column."""
        nq = (self.nc[0] - 1) * (self.nc[1] - 1) * (self.nc[2] - 1)
        m = 3 * nq
        Ac = np.zeros((m, m))
        for J in range(m):
            e = np.zeros((3, nq))
            e.reshape(-1)[J] = 1.0
            Ac[:, J] = self.restrict(self.apply(self.prolong(e))).ravel()
        self.nq = nq
        self.Ac = Ac
        self.Lc = np.linalg.cholesky(Ac) if m else None

    def coarse_apply(self, r):
        if self.nq == 0:
            return np.zeros((3, self.N))
        import scipy.linalg as sl
        rc = self.restrict(r).ravel()
        xc = sl.cho_solve((self.Lc, True), rc)
        return self.prolong(xc.reshape(3, self.nq))

    # ------------------------------------------------------------ preconditioner and solvers
    def pc_apply(self, r, pc=2):
        """pc 1: omega SDC-ASM; pc 2: hybrid V(1,1) with the vector Q1 coarse solve."""
        r = np.where(self.free, np.asarray(r, dtype=np.float64).reshape(3, self.N), 0.0)
        x1 = self.omega * self.sdc(r)
        if pc == 1:
            return x1
        x1 = x1 + self.coarse_apply(r - self.apply(x1))
        return x1 + self.omega * self.sdc(r - self.apply(x1))

    def lanczos_omega(self, b0, k=20):
        """k CG steps on A x = b0 with the undamped SDC-ASM; the CG coefficients
        give the Lanczos tridiagonal matrix of A_SDC^{-1} A;
        omega = 2 / (1.25 lam_max + 0.75 lam_min) (Section 2.5)."""
        r = np.where(self.free, np.asarray(b0, dtype=np.float64).reshape(3, self.N), 0.0)
        z = self.sdc(r)
        d = z.copy()
        rz = np.vdot(r, z)
        al, be = [], []
        for _ in range(k):
            if not rz > 0:
                break
            q = self.apply(d)
            dq = np.vdot(d, q)
            if not dq > 0:
                break
            a = rz / dq
            r = r - a * q
            z = self.sdc(r)
            rz1 = np.vdot(r, z)
            al.append(a)
            be.append(rz1 / rz)
            rz = rz1
            d = z + be[-1] * d
        m = len(al)
        T = np.zeros((m, m))
        for j in range(m):
            T[j, j] = 1.0 / al[j] + (be[j - 1] / al[j - 1] if j > 0 else 0.0)
            if j + 1 < m:
                T[j, j + 1] = T[j + 1, j] = np.sqrt(be[j]) / al[j]
        ev = np.linalg.eigvalsh(T)
        self.omega = 2.0 / (1.25 * ev[-1] + 0.75 * ev[0])
        return ev[0], ev[-1], self.omega

    def pcg(self, b, rtol=1e-8, maxit=500, pc=2):
        """PCG from x = 0 until ||r||_2 <= rtol ||b||_2.  Returns (x, iterations, converged)."""
        b = np.where(self.free, np.asarray(b, dtype=np.float64).reshape(3, self.N), 0.0)
        x = np.zeros_like(b)
        r = b.copy()
        nb = np.linalg.norm(b)
        if nb == 0.0:
            return x, 0, True
        z = self.pc_apply(r, pc)
        d = z.copy()
        rz = np.vdot(r, z)
        for it in range(1, maxit + 1):
            q = self.apply(d)
            a = rz / np.vdot(d, q)
            x += a * d
            r -= a * q
            if np.linalg.norm(r) <= rtol * nb:
                return x, it, True
            z = self.pc_apply(r, pc)
            rz1 = np.vdot(r, z)
            d = z + (rz1 / rz) * d
            rz = rz1
        return x, maxit, False
