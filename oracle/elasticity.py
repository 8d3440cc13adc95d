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
vol / (L_a L_b).  Dirichlet faces (all three components clamped): the whole
boundary by default, or the faces of the dirichlet_faces mask (bit 2a: the
face at the lower end of axis a, bit 2a + 1: the upper end); the other faces
are traction-free, the natural condition of the weak form (Sec. 4.1 clamps
x_1 = 0 only).

SDC relaxation: the block-diagonal A_SDC = diag(A_11, A_22, A_33) (Section
4.1).  Block A_jj is the scalar operator with per-axis coefficients
mu + (mu + lam) delta_aj, which is separable on box cells, so it takes the
scalar vertex-star FDM/sparse relaxation with the per-cell surrogate
mu_a^(j) = (mu + (mu + lam) delta_aj) vol / L_a^2, exactly.  With traction-free
faces the relaxation is taken as its definition: additive Schwarz over the
vertex stars (the free nodes within p - 1 of the vertex along every axis:
on a traction-free face the star keeps its boundary nodes) with the dense
GLL-basis star matrices of A_jj, which the FDM-basis solve equals on box cells.

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

    def __init__(self, p, xv, yv, zv, mu, lam, dirichlet_faces=63):
        self.p, self.mu, self.lam = p, float(mu), float(lam)
        self.dfaces = int(dirichlet_faces)
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
        m = np.ones(self.Nn[::-1], dtype=bool)   # [z, y, x]
        df = self.dfaces
        if df & 1: m[:, :, 0] = False
        if df & 2: m[:, :, -1] = False
        if df & 4: m[:, 0] = False
        if df & 8: m[:, -1] = False
        if df & 16: m[0] = False
        if df & 32: m[-1] = False
        self.free = m.ravel()
        # free Q1 vertices (not on a Dirichlet face), x fastest
        vm = np.ones([c + 1 for c in self.nc][::-1], dtype=bool)
        if df & 1: vm[:, :, 0] = False
        if df & 2: vm[:, :, -1] = False
        if df & 4: vm[:, 0] = False
        if df & 8: vm[:, -1] = False
        if df & 16: vm[0] = False
        if df & 32: vm[-1] = False
        self.vfree = vm
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
    def block_matrix(self, j):
        """The SDC block A_jj on all grid nodes (sparse CSR, natural boundary)."""
        import scipy.sparse as sp
        n = self.p + 1
        A, B = self.A1, self.B1
        rows, cols, vals = [], [], []
        coef = np.full(3, self.mu)
        coef[j] += self.mu + self.lam
        for e in range(self.cidx.shape[0]):
            K = np.zeros((n ** 3, n ** 3))
            for d in range(3):
                M = [B, B, B]
                M[d] = A
                K += coef[d] * self.vol[e] / self.L[e, d] ** 2 * np.kron(M[2], np.kron(M[1], M[0]))
            g = self.cidx[e].ravel()
            rows.append(np.repeat(g, n ** 3))
            cols.append(np.tile(g, n ** 3))
            vals.append(K.ravel())
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.N, self.N))

    def star_nodes(self, v):
        """Free grid nodes within p - 1 of vertex v = (vx, vy, vz) along every axis."""
        p = self.p
        rng = [np.arange(max(0, p * v[a] - p + 1), min(self.Nn[a] - 1, p * v[a] + p - 1) + 1) for a in range(3)]
        g = (rng[0][None, None, :] + self.Nn[0] * (rng[1][None, :, None] + self.Nn[1] * rng[2][:, None, None])).ravel()
        return g[self.free[g]]

    def setup_sdc(self, definition=False):
        """definition: additive Schwarz with the dense GLL-basis star matrices
        even where the boundary is clamped everywhere (else the scalar FDM
        oracle's star solves, which equal them on box cells)."""
        self.comps = []
        self.stars = None
        if self.dfaces == 63 and not definition:
            for j in range(3):
                P = Problem(self.p, *self.v)
                P.set_mu(self.sdc_mu(j))
                P.setup_patches()
                P.set_omega(1.0)
                self.comps.append(P)
            return
        import scipy.linalg as sl
        self.stars = []
        for j in range(3):
            Aj = self.block_matrix(j)
            facs = []
            for vz in range(self.nc[2] + 1):
                for vy in range(self.nc[1] + 1):
                    for vx in range(self.nc[0] + 1):
                        g = self.star_nodes((vx, vy, vz))
                        if len(g):
                            facs.append((g, sl.cho_factor(Aj[g][:, g].toarray())))
            self.stars.append(facs)

    def sdc(self, r):
        """Undamped additive Schwarz with the SDC blocks: [ASM_j(r_j)]."""
        r = np.asarray(r, dtype=np.float64).reshape(3, self.N)
        if self.stars is None:
            return np.stack([self.comps[j].asm_apply(r[j]) for j in range(3)])
        import scipy.linalg as sl
        z = np.zeros((3, self.N))
        for j in range(3):
            rj = np.where(self.free, r[j], 0.0)
            for g, fac in self.stars[j]:
                z[j, g] += sl.cho_solve(fac, rj[g])
        return z

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
            X[self.vfree] = xc[a]
            out[a] = np.einsum("zc,yb,xa,cba->zyx", W[2], W[1], W[0], X).ravel()
        return np.where(self.free, out, 0.0)

    def restrict(self, r):
        W = [self._hat(a) for a in range(3)]
        r = np.where(self.free, np.asarray(r).reshape(3, self.N), 0.0)
        out = []
        for a in range(3):
            R = r[a].reshape(self.Nn[::-1])
            X = np.einsum("zc,yb,xa,zyx->cba", W[2], W[1], W[0], R)
            out.append(X[self.vfree])
        return np.stack(out)

    def setup_coarse(self):
        """A_c = P^T A P (vector Q1 Galerkin), column by column."""
        nq = int(self.vfree.sum())
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
