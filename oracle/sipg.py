"""Symmetric interior penalty DG (SIPG) for the Poisson equation on DQ_p
(Section 5, Eqs. sipg_lhs, dirichlet_stiffness, interior_stiffness) with
vertex-star Schwarz relaxation: the FP64 CPU oracle, in numpy.  Test
infrastructure only: only the test suite, ``__graft_entry__.smoke()`` and the
CPU legs of ``bench.py`` may use it.

Discretisation.  Each cell carries its own (p+1)^3 GLL Lagrange nodal values;
vectors are cell-major [cell, z, y, x] with cells x fastest.  Box cells of a
tensor mesh with half-widths h (reference interval [-1, 1]), coefficient 1:

    a(v, u) = sum_K int_K grad v . grad u
            + sum_e int_e eta h_e^{-1} [v].[u] - [v].{grad u} - {grad v}.[u],

over the interior facets and the whole boundary (weak homogeneous Dirichlet
condition), with [w] = w^- n^- + w^+ n^+ (w n on the boundary), {w} the mean
of the two traces (the trace on the boundary), and h_e^{-1} = |e| {|K|^{-1}}:
(1/(2h^-) + 1/(2h^+)) / 2 on an interior facet, 1/(2h) on a boundary facet,
h the half-widths normal to e.  eta defaults to p(p+1) (the value the paper
uses for its interior-penalty experiments).

Every cell and facet integral is a Kronecker product of 1D factors: the cell
term sum_d (vol/h_d^2) A_hat (x) B_hat (x) B_hat, the facet term a 2(p+1)
square normal-direction matrix (penalty on the product of the end values,
consistency and adjoint consistency on end value times end derivative) times
the tangential mass h_t1 h_t2 B_hat (x) B_hat.  ``apply`` evaluates them from
the traces; ``matrix`` tabulates ``apply``.

Relaxation: additive Schwarz over the vertex stars of the interior vertices;
a star holds all (2p+2)^3 values of its 8 cells and its matrix is the
principal submatrix of A on them (facets to cells outside the star keep
their own-side block), solved exactly by a dense Cholesky factorisation.

Coarse space: the conforming Q1 functions that vanish on the boundary
(interior vertices), interpolated into each cell's nodes.  Their jumps
vanish on every facet, so the Galerkin operator P^T A P is the Q1 stiffness
matrix.  Preconditioner: the hybrid V(1,1) of the conforming problem
(Section 2.5), damping omega from 20 CG-Lanczos steps on ASM^{-1} A.
"""
import numpy as np

from . import basis1d, gauss, lagrange


def _kron3(U, Mx, My, Mz):
    """Applies Mz (x) My (x) Mx to cell arrays U[..., cz, cy, cx, z, y, x]."""
    U = np.einsum("ij,...j->...i", Mx, U)
    U = np.einsum("ij,...jx->...ix", My, U)
    return np.einsum("ij,...jyx->...iyx", Mz, U)


class Sipg:
    """SIPG Q_p-DG Poisson problem on a tensor mesh of box cells."""

    def __init__(self, p, xv, yv, zv, eta=None):
        self.p, self.n = p, p + 1
        self.eta = float(p * (p + 1)) if eta is None else float(eta)
        self.v = [np.asarray(a, dtype=np.float64) for a in (xv, yv, zv)]
        self.nc = [len(a) - 1 for a in self.v]
        self.ncell = self.nc[0] * self.nc[1] * self.nc[2]
        self.N = self.ncell * self.n ** 3
        b = basis1d(p)
        self.A1, self.B1, self.xi = b["A"], b["B"], b["xi"]
        V, D = lagrange(p, self.xi, np.array([-1.0, 1.0]))
        self.dm, self.dp = D[0].copy(), D[1].copy()   # l_i'(-1), l_i'(+1)
        self.h = [0.5 * np.diff(a) for a in self.v]     # half-widths per axis
        self.shape = (self.nc[2], self.nc[1], self.nc[0], self.n, self.n, self.n)
        self.omega = 1.0
        self.factors = None
        self.Lc = None

    # ------------------------------------------------------------ geometry
    def nodes(self):
        """Physical coordinates [3, N] of every nodal value (x, y, z)."""
        c = [(a[:-1, None] + hh[:, None] * (1.0 + self.xi[None, :])) for a, hh in zip(self.v, self.h)]
        X = np.broadcast_to(c[0][None, None, :, None, None, :], self.shape)
        Y = np.broadcast_to(c[1][None, :, None, None, :, None], self.shape)
        Z = np.broadcast_to(c[2][:, None, None, :, None, None], self.shape)
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()])

    # ------------------------------------------------------------ operator
    def apply(self, u, hcells=None, ghost=None):
        """y = A u.  u is [..., N] for this mesh, or [..., cz, cy, cx, z, y, x]
        for a window of it whose half-widths are hcells (x, y, z lists); ghost
        gives, per axis, the half-widths (left, right) of the cells beyond the
        window (None: the domain boundary).  With a ghost neighbour the facet
        is an interior facet whose other side carries zero values, so the
        result restricted to the window is the principal submatrix of A."""
        h = self.h if hcells is None else [np.asarray(a, dtype=np.float64) for a in hcells]
        ghost = ghost or [(None, None)] * 3
        shape = (len(h[2]), len(h[1]), len(h[0]), self.n, self.n, self.n)
        U = np.asarray(u, dtype=np.float64)
        batch = U.shape[:-1] if U.shape[-6:] != shape else U.shape[:-6]
        U = U.reshape(batch + shape)
        A, B, eta, n = self.A1, self.B1, self.eta, self.n
        hx, hy, hz = h
        # cell terms: (vol / h_d^2) on the d-th factor A_hat
        cx = (hy[None, :, None] * hz[:, None, None]) / hx[None, None, :]
        cy = (hx[None, None, :] * hz[:, None, None]) / hy[None, :, None]
        cz = (hx[None, None, :] * hy[None, :, None]) / hz[:, None, None]
        e = (Ellipsis, slice(None), slice(None), slice(None), None, None, None)
        Y = (cx[e] * _kron3(U, A, B, B) + cy[e] * _kron3(U, B, A, B) + cz[e] * _kron3(U, B, B, A))
        hcell = [hz, hy, hx]                       # in the order of the cell axes of U
        for a in range(3):                         # facets normal to axis a (0 = x)
            ca, na = -6 + (2 - a), -3 + (2 - a)    # its cell and node axes in U
            W = np.moveaxis(U, (ca, na), (-2, -1))  # [..., ct1, ct2, nt1, nt2, c, i]
            YW = np.moveaxis(Y, (ca, na), (-2, -1))
            t = [k for k in range(3) if k != 2 - a]
            s = hcell[t[0]][:, None] * hcell[t[1]][None, :]   # tangential h_t1 h_t2

            def T(X):  # tangential mass on [..., ct1, ct2, nt1, nt2, k]
                X = np.einsum("ab,cd,...ijbdk->...ijack", B, B, X)
                return s[:, :, None, None, None] * X

            ha = h[a]
            val_lo, val_hi = W[..., 0], W[..., n - 1]
            der_lo = np.einsum("...i,i->...", W, self.dm) / ha   # d/dx at the cell's low end
            der_hi = np.einsum("...i,i->...", W, self.dp) / ha
            e0 = np.zeros(n); e0[0] = 1.0
            e1 = np.zeros(n); e1[n - 1] = 1.0
            if len(ha) > 1:                        # interior facets between cells c and c + 1
                sig = eta * 0.25 * (1.0 / ha[:-1] + 1.0 / ha[1:])
                Jt = T(val_hi[..., :-1] - val_lo[..., 1:])
                Gt = T(0.5 * (der_hi[..., :-1] + der_lo[..., 1:]))
                YW[..., :-1, :] += ((sig * Jt - Gt)[..., None] * e1
                                    - 0.5 * Jt[..., None] * (self.dp[None, :] / ha[:-1, None]))
                YW[..., 1:, :] += ((-sig * Jt + Gt)[..., None] * e0
                                   - 0.5 * Jt[..., None] * (self.dm[None, :] / ha[1:, None]))
            # the low face of the first cell and the high face of the last one
            for side in (0, 1):
                c = 0 if side == 0 else len(ha) - 1
                hg = ghost[a][side]
                ub = (val_lo if side == 0 else val_hi)[..., c:c + 1]
                du = (der_lo if side == 0 else der_hi)[..., c:c + 1]
                Ut = T(ub)
                if hg is None:                     # boundary facet: [v] = v n, {grad u} = grad u
                    sig = eta / (2.0 * ha[c])
                    Gt = T(du)
                    sgn = -1.0 if side == 0 else 1.0
                    ev = e0 if side == 0 else e1
                    dv = self.dm if side == 0 else self.dp
                    YW[..., c:c + 1, :] += ((sig * Ut - sgn * Gt)[..., None] * ev
                                            - sgn * Ut[..., None] * (dv / ha[c]))
                else:                              # interior facet, zero values beyond the window
                    sig = eta * 0.25 * (1.0 / ha[c] + 1.0 / hg)
                    Gt = T(0.5 * du)
                    if side == 1:                  # this cell is the facet's minus side
                        YW[..., c:c + 1, :] += ((sig * Ut - Gt)[..., None] * e1
                                                - 0.5 * Ut[..., None] * (self.dp / ha[c]))
                    else:                          # plus side: the jump is -u
                        YW[..., c:c + 1, :] += ((sig * Ut + Gt)[..., None] * e0
                                                + 0.5 * Ut[..., None] * (self.dm / ha[c]))
        return Y.reshape(batch + (-1,))

    def matrix(self):
        """Dense A, column by column from ``apply`` (small meshes)."""
        return self.apply(np.eye(self.N)).T.copy()

    def load(self, f, q=None):
        """b_i = int f phi_i by Gauss quadrature (q points per axis and cell);
        f takes arrays x, y, z."""
        q = q or self.p + 4
        xq, wq = gauss(q)
        V, _ = lagrange(self.p, self.xi, xq)        # [q, n]
        c = [(a[:-1, None] + hh[:, None] * (1.0 + xq[None, :])) for a, hh in zip(self.v, self.h)]
        F = f(c[0][None, None, :, None, None, :], c[1][None, :, None, None, :, None],
              c[2][:, None, None, :, None, None])
        F = np.broadcast_to(F, (self.nc[2], self.nc[1], self.nc[0], q, q, q))
        jac = (self.h[2][:, None, None] * self.h[1][None, :, None] * self.h[0][None, None, :])
        Wq = np.einsum("k,j,i->kji", wq, wq, wq)
        Fw = F * Wq * jac[..., None, None, None]
        return _kron3(Fw, V.T, V.T, V.T).ravel()

    # ------------------------------------------------------------ vertex-star patches
    def vertices(self):
        """Interior vertices (vx, vy, vz), x fastest."""
        return [(vx, vy, vz) for vz in range(1, self.nc[2]) for vy in range(1, self.nc[1])
                for vx in range(1, self.nc[0])]

    def patch_dofs(self, v):
        """Global indices of the star's values in patch tensor order
        [Z][Y][X], X = a (p+1) + i for the cell at x offset a (0 left, 1 right)."""
        n = self.n
        m = 2 * n
        out = np.zeros((m, m, m), dtype=np.int64)
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    cell = (v[0] - 1 + a) + self.nc[0] * ((v[1] - 1 + b) + self.nc[1] * (v[2] - 1 + c))
                    base = cell * n ** 3
                    idx = base + np.arange(n ** 3).reshape(n, n, n)
                    out[c * n:(c + 1) * n, b * n:(b + 1) * n, a * n:(a + 1) * n] = idx
        return out.ravel()

    def patch_matrix(self, v):
        """The star's matrix (principal submatrix of A) in patch tensor order."""
        n, m = self.n, 2 * self.n
        hc, gh = [], []
        for a in range(3):
            k = v[a]
            hc.append(self.h[a][k - 1:k + 1])
            gh.append((self.h[a][k - 2] if k >= 2 else None, self.h[a][k + 1] if k + 1 < self.nc[a] else None))
        M = np.zeros((m ** 3, m ** 3))
        for j0 in range(0, m ** 3, 512):
            j1 = min(m ** 3, j0 + 512)
            E = np.zeros((j1 - j0, m ** 3))
            E[np.arange(j1 - j0), np.arange(j0, j1)] = 1.0
            # patch tensor [Z][Y][X] -> window cells [c][b][a][k][j][i]
            Ew = E.reshape(-1, 2, n, 2, n, 2, n).transpose(0, 1, 3, 5, 2, 4, 6)
            Yw = self.apply(Ew, hcells=hc, ghost=gh).reshape(-1, 2, 2, 2, n, n, n)
            M[:, j0:j1] = Yw.transpose(0, 1, 4, 2, 5, 3, 6).reshape(j1 - j0, m ** 3).T
        return M

    def setup_patches(self, vertices=None):
        import scipy.linalg as sl
        self.factors = {}
        for v in (vertices if vertices is not None else self.vertices()):
            self.factors[v] = sl.cho_factor(self.patch_matrix(v), lower=True)

    def patch_solve(self, v, r):
        """A_v^{-1} R_v r in patch tensor order."""
        import scipy.linalg as sl
        if self.factors is None or v not in self.factors:
            f = sl.cho_factor(self.patch_matrix(v), lower=True)
        else:
            f = self.factors[v]
        return sl.cho_solve(f, np.asarray(r, dtype=np.float64)[self.patch_dofs(v)])

    def asm(self, r):
        """Undamped additive Schwarz: sum_v R_v^T A_v^{-1} R_v r."""
        r = np.asarray(r, dtype=np.float64)
        z = np.zeros(self.N)
        for v in self.vertices():
            z[self.patch_dofs(v)] += self.patch_solve(v, r)
        return z

    # ------------------------------------------------------------ coarse space
    def _hats(self):
        """W[i, s]: 1D Q1 hats of the low (s = 0) and high (s = 1) vertex at the GLL nodes."""
        return np.stack([0.5 * (1.0 - self.xi), 0.5 * (1.0 + self.xi)], axis=1)

    def prolong(self, xc):
        """DG values [N] of the Q1 function with interior vertex values xc (x fastest)."""
        nv = [c + 1 for c in self.nc]
        X = np.zeros(nv[::-1])
        X[1:-1, 1:-1, 1:-1] = np.asarray(xc, dtype=np.float64).reshape(nv[2] - 2, nv[1] - 2, nv[0] - 2)
        W = self._hats()
        U = np.zeros(self.shape)
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    Xc = X[c:c + self.nc[2], b:b + self.nc[1], a:a + self.nc[0]]
                    U += Xc[..., None, None, None] * np.einsum("k,j,i->kji", W[:, c], W[:, b], W[:, a])
        return U.ravel()

    def restrict(self, r):
        """P^T r."""
        nv = [c + 1 for c in self.nc]
        R = np.asarray(r, dtype=np.float64).reshape(self.shape)
        W = self._hats()
        X = np.zeros(nv[::-1])
        for c in range(2):
            for b in range(2):
                for a in range(2):
                    X[c:c + self.nc[2], b:b + self.nc[1], a:a + self.nc[0]] += np.einsum(
                        "zyxkji,k,j,i->zyx", R, W[:, c], W[:, b], W[:, a])
        return X[1:-1, 1:-1, 1:-1].ravel()

    def setup_coarse(self):
        """A_c = P^T A P, column by column, and its Cholesky factor."""
        nq = (self.nc[0] - 1) * (self.nc[1] - 1) * (self.nc[2] - 1)
        self.nq = nq
        Ac = np.zeros((nq, nq))
        for j in range(nq):
            ej = np.zeros(nq)
            ej[j] = 1.0
            Ac[:, j] = self.restrict(self.apply(self.prolong(ej)))
        self.Ac = Ac
        self.Lc = np.linalg.cholesky(Ac) if nq else None

    def coarse_apply(self, r):
        if self.nq == 0:
            return np.zeros(self.N)
        import scipy.linalg as sl
        return self.prolong(sl.cho_solve((self.Lc, True), self.restrict(r)))

    # ------------------------------------------------------------ preconditioner and solvers
    def pc_apply(self, r, pc=2):
        """pc 1: omega ASM; pc 2: hybrid V(1,1) with the Q1 coarse solve."""
        r = np.asarray(r, dtype=np.float64)
        x1 = self.omega * self.asm(r)
        if pc == 1:
            return x1
        x1 = x1 + self.coarse_apply(r - self.apply(x1))
        return x1 + self.omega * self.asm(r - self.apply(x1))

    def lanczos_omega(self, b0, k=20):
        """k CG steps on A x = b0 with the undamped ASM; the CG coefficients give
        the Lanczos tridiagonal matrix of ASM A; omega = 2 / (1.25 lam_max +
        0.75 lam_min) (Section 2.5)."""
        r = np.asarray(b0, dtype=np.float64).copy()
        z = self.asm(r)
        d = z.copy()
        rz = r @ z
        al, be = [], []
        for _ in range(k):
            if not rz > 0:
                break
            q = self.apply(d)
            dq = d @ q
            if not dq > 0:
                break
            a = rz / dq
            r = r - a * q
            z = self.asm(r)
            rz1 = r @ z
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
        b = np.asarray(b, dtype=np.float64)
        x = np.zeros_like(b)
        r = b.copy()
        nb = np.linalg.norm(b)
        if nb == 0.0:
            return x, 0, True
        z = self.pc_apply(r, pc)
        d = z.copy()
        rz = r @ z
        for it in range(1, maxit + 1):
            q = self.apply(d)
            a = rz / (d @ q)
            x += a * d
            r -= a * q
            if np.linalg.norm(r) <= rtol * nb:
                return x, it, True
            z = self.pc_apply(r, pc)
            rz1 = r @ z
            d = z + (rz1 / rz) * d
            rz = rz1
        return x, maxit, False
