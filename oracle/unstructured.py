"""Poisson on a general conforming hexahedral mesh with the vertex-star
FDM/sparse relaxation (Sections 2.1-2.7 on the unstructured meshes of the
paper's Section 3 experiments): the FP64 CPU oracle, in numpy and scipy.
Test infrastructure only: only the test suite, ``__graft_entry__.smoke()``
and the CPU legs of ``bench.py`` may use it.

Mesh.  Vertex coordinates X[nv, 3] and cells[nc, 8]; a cell lists its
vertices at the corners (a, b, c) of the reference cube [-1, 1]^3 (0 for -1,
1 for +1) at index a + 2 b + 4 c, and its geometry is the trilinear map
through them.  Cells may use any orientation of the reference axes.

Space.  Q_p on every cell with the GLL Lagrange basis.  The global nodes are
the cells' GLL nodes merged by physical position: a shared face (edge,
vertex) is the same bilinear patch seen from both cells and the GLL points
are symmetric, so the nodes coincide.  Dirichlet nodes: the nodes on
boundary faces (faces of one cell only), homogeneous.  Vectors hold every
global node; Dirichlet entries are ignored on input and 0 on output.

Operator.  a(v, u) = sum_K int_K kappa grad v . grad u by Gauss quadrature
with q = p + 1 points per axis: per point G = kappa |det J| J^{-1} J^{-T}
in reference coordinates (J = dx/dxi), assembled into a sparse matrix.

Relaxation (Sections 2.6-2.7).  Additive Schwarz over the vertex stars of all
mesh vertices: the star of vertex v holds the free nodes whose cells all
contain v (the interior of the union of v's cells).  The star matrix is the
principal submatrix of the separable surrogate A~ = sum_K R_K^T A~_K R_K,
A~_K = sum_j mu_j^K (A_hat along reference axis j, B_hat along the other
two), mu_j^K = (1/8) sum_q w_q G_jj(q) (the averaged surrogate, exact on box
cells).  Each star is solved exactly (dense Cholesky): z = sum_v R_v^T
A~_v^{-1} R_v r does not depend on the basis the star is solved in.  The FDM
basis of the paper is what makes A~_v sparse; ``star_fdm`` builds it for a
star (the cells' tensor-product FDM functions glued across the shared
entities) so that the sparsity the method relies on can be checked.

Coarse space: the Q1 nodal functions of the interior mesh vertices,
interpolated at each cell's GLL nodes (P); A_c = P^T A P, solved by
Cholesky.  Preconditioner: the hybrid V(1,1) (Section 2.5); omega from 20
CG-Lanczos steps on ASM^{-1} A; PCG from x = 0 to ||r||_2 <= rtol ||b||_2.
"""
import numpy as np
import scipy.linalg as sl
import scipy.sparse as sp
from scipy.spatial import cKDTree

from . import basis1d, gauss, lagrange


def _kron3(Mz, My, Mx):
    """Kronecker product acting on cell arrays indexed i + n (j + n k)."""
    return np.kron(Mz, np.kron(My, Mx))


def _hat(t):
    """The two linear functions of the reference interval at points t."""
    t = np.asarray(t, dtype=np.float64)
    return np.stack([0.5 * (1.0 - t), 0.5 * (1.0 + t)], axis=-1)


def _hat_deriv():
    return np.array([-0.5, 0.5])


class HexProblem:
    """Q_p Poisson problem on a conforming hexahedral mesh (oracle side)."""

    def __init__(self, p, X, cells, kappa=None, tol=1e-10, exact_patches=False):
        """kappa: optional coefficient at the (p+1)^3 Gauss points of every
        cell.  exact_patches: solve the stars with the principal submatrices
        of A itself instead of the separable surrogate (the exact patch
        solves the paper uses on Cartesian meshes)."""
        self.p, self.n = p, p + 1
        self.exact_patches = exact_patches
        self.X = np.asarray(X, dtype=np.float64)
        self.cells = np.asarray(cells, dtype=np.int64)
        self.ncell = self.cells.shape[0]
        n, nc = self.n, self.ncell
        b = basis1d(p)
        self.xi, self.Ah, self.Bh, self.T1 = b["xi"], b["A"], b["B"], b["T"]
        xq, wq = gauss(p + 1)
        self.Vq, self.Dq = lagrange(p, self.xi, xq)   # [q, i]: l_i(x_q), l_i'(x_q)
        self.wq3 = _kron3(wq, wq, wq)                  # weight of point qx + nq (qy + nq qz)

        # ---- geometry at the Gauss points: J[e, q, i, d] = d x_i / d xi_d
        hq, dh = _hat(xq), _hat_deriv()
        corners = self.X[self.cells]                   # [e, 8, 3]
        nq = len(xq)
        J = np.zeros((nc, nq ** 3, 3, 3))
        for c in (0, 1):
            for bb in (0, 1):
                for a in (0, 1):
                    gx = _kron3(hq[:, c], hq[:, bb], np.full(nq, dh[a]))
                    gy = _kron3(hq[:, c], np.full(nq, dh[bb]), hq[:, a])
                    gz = _kron3(np.full(nq, dh[c]), hq[:, bb], hq[:, a])
                    Xv = corners[:, a + 2 * bb + 4 * c, :]  # [e, 3]
                    for d, g in enumerate((gx, gy, gz)):
                        J[:, :, :, d] += Xv[:, None, :] * g[None, :, None]
        det = np.linalg.det(J)
        if np.any(det == 0.0):
            raise ValueError("degenerate cell")
        Jinv = np.linalg.inv(J)
        kap = np.ones((nc, nq ** 3)) if kappa is None else np.asarray(kappa, dtype=np.float64).reshape(nc, nq ** 3)
        self.G = (kap * np.abs(det))[:, :, None, None] * np.einsum("eqdi,eqfi->eqdf", Jinv, Jinv)

        # ---- global nodes: the cells' GLL nodes merged by position
        hn = _hat(self.xi)
        pts = np.zeros((nc, n ** 3, 3))
        for c in (0, 1):
            for bb in (0, 1):
                for a in (0, 1):
                    f = _kron3(hn[:, c], hn[:, bb], hn[:, a])
                    pts += corners[:, a + 2 * bb + 4 * c, None, :] * f[None, :, None]
        flat = pts.reshape(-1, 3)
        scale = max(1.0, np.abs(flat).max())
        pairs = cKDTree(flat).query_pairs(tol * scale, output_type="ndarray")
        parent = np.arange(flat.shape[0])

        def find(i):
            while parent[i] != i:
                parent[i] = parent[parent[i]]
                i = parent[i]
            return i

        for i, j in pairs:
            ri, rj = find(i), find(j)
            if ri != rj:
                parent[max(ri, rj)] = min(ri, rj)
        roots = np.array([find(i) for i in range(flat.shape[0])])
        uniq, first, gid = np.unique(roots, return_index=True, return_inverse=True)
        order = np.argsort(first)                      # number nodes in order of first appearance
        rank = np.empty_like(order)
        rank[order] = np.arange(len(order))
        self.gid = rank[gid].reshape(nc, n ** 3)
        self.ndof = len(uniq)
        self.nodes = np.zeros((self.ndof, 3))
        self.nodes[self.gid.ravel()] = flat

        # ---- Dirichlet nodes: on faces that belong to one cell
        faces = {}
        for e in range(nc):
            for d in range(3):
                for side in (0, 1):
                    key = frozenset(self._face_vertices(e, d, side))
                    faces.setdefault(key, []).append((e, d, side))
        self.dirichlet = np.zeros(self.ndof, dtype=bool)
        idx = np.arange(n)
        I3 = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), axis=-1).reshape(-1, 3)[:, ::-1]  # (i, j, k)
        for lst in faces.values():
            if len(lst) == 1:
                e, d, side = lst[0]
                on = I3[:, d] == (n - 1 if side else 0)
                self.dirichlet[self.gid[e, on]] = True
        self.free = ~self.dirichlet

        # ---- cell matrices and their assembly
        D = [_kron3(self.Vq, self.Vq, self.Dq), _kron3(self.Vq, self.Dq, self.Vq), _kron3(self.Dq, self.Vq, self.Vq)]
        self.Ke = np.zeros((nc, n ** 3, n ** 3))
        for d in range(3):
            for f in range(3):
                W = self.wq3[None, :] * self.G[:, :, d, f]
                self.Ke += np.einsum("qi,eq,qj->eij", D[d], W, D[f])
        self.mu = np.einsum("q,eqdd->ed", self.wq3, self.G) / 8.0
        Kd = [_kron3(self.Bh, self.Bh, self.Ah), _kron3(self.Bh, self.Ah, self.Bh), _kron3(self.Ah, self.Bh, self.Bh)]
        self.Ks = np.einsum("ed,dij->eij", self.mu, np.array(Kd))
        self.A = self._assemble(self.Ke)
        self.As = self._assemble(self.Ks)
        Mq = _kron3(self.Vq, self.Vq, self.Vq)
        self.Me = np.einsum("qi,eq,qj->eij", Mq, self.wq3[None, :] * np.abs(det), Mq)
        self.M = self._assemble(self.Me)

        # ---- cells of every node and of every vertex
        self.node_cells = [[] for _ in range(self.ndof)]
        for e in range(nc):
            for g in set(self.gid[e].tolist()):
                self.node_cells[g].append(e)
        self.vertex_cells = [[] for _ in range(self.X.shape[0])]
        for e in range(nc):
            for v in self.cells[e]:
                self.vertex_cells[v].append(e)
        self.omega = 1.0
        self.stars = None
        self.P = self.Lc = None

    # ------------------------------------------------------------ mesh helpers
    def _face_vertices(self, e, d, side):
        out = []
        for c in (0, 1):
            for b in (0, 1):
                for a in (0, 1):
                    if (a, b, c)[d] == side:
                        out.append(int(self.cells[e, a + 2 * b + 4 * c]))
        return out

    def _assemble(self, Ke):
        n3 = self.n ** 3
        rows = np.repeat(self.gid, n3, axis=1).ravel()
        cols = np.tile(self.gid, (1, n3)).ravel()
        return sp.csr_matrix((Ke.reshape(self.ncell, -1).ravel(), (rows, cols)), shape=(self.ndof, self.ndof))

    def _mask(self, u):
        u = np.asarray(u, dtype=np.float64).copy()
        u[self.dirichlet] = 0.0
        return u

    # ------------------------------------------------------------ operators
    def apply(self, u):
        """y = A u on the free nodes, 0 on the Dirichlet nodes."""
        return self._mask(self.A @ self._mask(u))

    def apply_surrogate(self, u):
        return self._mask(self.As @ self._mask(u))

    def mass_apply(self, f):
        """b = M f on the free nodes (f's Dirichlet entries ignored), 0 on the Dirichlet nodes."""
        return self._mask(self.M @ self._mask(f))

    # ------------------------------------------------------------ vertex stars
    def star_dofs(self, v):
        """Free nodes whose cells all contain vertex v (ascending node order)."""
        cells_v = set(self.vertex_cells[v])
        cand = set()
        for e in cells_v:
            cand.update(self.gid[e].tolist())
        return np.array(sorted(g for g in cand if self.free[g] and set(self.node_cells[g]) <= cells_v),
                        dtype=np.int64)

    def setup_patches(self):
        self.stars = []
        for v in range(self.X.shape[0]):
            dofs = self.star_dofs(v)
            if len(dofs) == 0:
                continue
            Av = self._patch_source()[dofs][:, dofs].toarray()
            self.stars.append((v, dofs, sl.cho_factor(Av, lower=True)))
        return len(self.stars)

    def patch_solve(self, v, r):
        dofs = self.star_dofs(v)
        Av = self._patch_source()[dofs][:, dofs].toarray()
        return dofs, np.linalg.solve(Av, np.asarray(r, dtype=np.float64)[dofs])

    def _patch_source(self):
        return self.A if self.exact_patches else self.As

    def asm(self, r):
        """sum over stars of R_v^T A~_v^{-1} R_v r (undamped)."""
        if self.stars is None:
            self.setup_patches()
        r = np.asarray(r, dtype=np.float64)
        z = np.zeros(self.ndof)
        for _, dofs, fac in self.stars:
            z[dofs] += sl.cho_solve(fac, r[dofs])
        return z

    # ------------------------------------------------------------ FDM basis of a star
    def star_fdm(self, v):
        """The star of vertex v in the FDM basis: returns (dofs, T_v, kind)
        with T_v[len(dofs), len(dofs)] the GLL coefficients (on the star's
        nodes) of the star's FDM functions and kind[k] in {0, 1, 2, 3} the
        number of reference axes along which function k is an interface
        (vertex-end) function of its cells: 0 cell interior, 1 face, 2 edge,
        3 vertex.  Each function is the tensor product of 1D FDM functions
        (columns of T) in every cell that contains its entity; across a
        shared entity the cells' functions are matched by their traces on
        the entity's nodes (a signed permutation: the interior functions s_j
        are even or odd), so the glued function is continuous."""
        dofs = self.star_dofs(v)
        pos = {g: k for k, g in enumerate(dofs)}
        cells_v = self.vertex_cells[v]
        n, p = self.n, self.p
        T3 = _kron3(self.T1, self.T1, self.T1)
        idx = np.arange(n)
        I3 = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), axis=-1).reshape(-1, 3)[:, ::-1]
        end = (I3 == 0) | (I3 == p)
        cols, kind, owner_trace = [], [], {}
        Tv = np.zeros((len(dofs), len(dofs)))
        for e in cells_v:
            for c in range(n ** 3):
                # the entity of local function c: its nodes are the local nodes
                # that agree with c on the end axes and are interior on the others
                on = np.all(np.where(end[c][None, :], I3 == I3[c][None, :], ~end), axis=1)
                ent = self.gid[e, on]
                if not all(g in pos for g in ent):
                    continue  # an entity on the star's boundary
                key = frozenset(ent.tolist())
                vals = T3[on, c]
                order = np.argsort(ent)
                trace = vals[order]
                if key not in owner_trace:
                    owner_trace[key] = []
                matched = None
                for k, tr in owner_trace[key]:
                    if np.allclose(trace, tr, rtol=0, atol=1e-12 * np.abs(tr).max()):
                        matched, sign = k, 1.0
                    elif np.allclose(trace, -tr, rtol=0, atol=1e-12 * np.abs(tr).max()):
                        matched, sign = k, -1.0
                    if matched is not None:
                        break
                if matched is None:
                    matched, sign = len(cols), 1.0
                    owner_trace[key].append((matched, trace))
                    cols.append(key)
                    kind.append(int(end[c].sum()))
                gl = [l for l in range(n ** 3) if self.gid[e, l] in pos]
                rows = [pos[self.gid[e, l]] for l in gl]
                outside = np.setdiff1d(np.arange(n ** 3), gl)
                if np.any(np.abs(T3[outside, c]) > 1e-13):
                    raise RuntimeError("an FDM function of the star reaches a node outside it")
                if matched >= Tv.shape[1]:
                    raise RuntimeError("more FDM functions than star nodes")
                col = sign * T3[gl, c]
                prev = Tv[rows, matched]
                set_before = prev != 0.0
                if np.any(set_before & (np.abs(prev - col) > 1e-12 * max(1.0, np.abs(col).max()))):
                    raise RuntimeError("FDM functions do not agree across a shared entity")
                Tv[rows, matched] = np.where(set_before, prev, col)
        if len(cols) != len(dofs):
            raise RuntimeError("star FDM basis has %d functions for %d nodes" % (len(cols), len(dofs)))
        return dofs, Tv, np.array(kind)

    # ------------------------------------------------------------ coarse space
    def vertex_interpolation(self):
        """P[node, k]: the Q1 function of the k-th interior mesh vertex at
        every node (interior vertex = not on a boundary face)."""
        n = self.n
        hn = _hat(self.xi)
        bnd = np.zeros(self.X.shape[0], dtype=bool)
        vd = {}
        for e in range(self.ncell):
            for d in range(3):
                for side in (0, 1):
                    key = frozenset(self._face_vertices(e, d, side))
                    vd[key] = vd.get(key, 0) + 1
        for key, cnt in vd.items():
            if cnt == 1:
                bnd[list(key)] = True
        interior = np.flatnonzero(~bnd)
        col = -np.ones(self.X.shape[0], dtype=np.int64)
        col[interior] = np.arange(len(interior))
        P = np.zeros((self.ndof, len(interior)))
        for e in range(self.ncell):
            for c in (0, 1):
                for b in (0, 1):
                    for a in (0, 1):
                        k = col[self.cells[e, a + 2 * b + 4 * c]]
                        if k >= 0:
                            P[self.gid[e], k] = _kron3(hn[:, c], hn[:, b], hn[:, a])
        P[self.dirichlet] = 0.0
        return P

    def setup_coarse(self):
        self.P = self.vertex_interpolation()
        if self.P.shape[1] == 0:
            self.Lc = None
            return
        AP = np.column_stack([self.apply(self.P[:, k]) for k in range(self.P.shape[1])])
        self.Ac = self.P.T @ AP
        self.Lc = sl.cho_factor(self.Ac, lower=True)

    def coarse_apply(self, r):
        if self.Lc is None:
            return np.zeros(self.ndof)
        return self.P @ sl.cho_solve(self.Lc, self.P.T @ self._mask(r))

    # ------------------------------------------------------------ preconditioner and solvers
    def pc_apply(self, r, pc=2):
        """pc 1: omega ASM; pc 2: hybrid V(1,1) with the Q1 coarse solve."""
        r = self._mask(r)
        x1 = self.omega * self.asm(r)
        if pc == 1:
            return x1
        if self.P is None:
            self.setup_coarse()
        x1 = x1 + self.coarse_apply(r - self.apply(x1))
        return x1 + self.omega * self.asm(r - self.apply(x1))

    def lanczos_omega(self, b0, k=20):
        """k CG steps on A x = b0 with the undamped ASM; the CG coefficients
        give the Lanczos tridiagonal matrix of ASM^{-1} A; omega = 2 /
        (1.25 lam_max + 0.75 lam_min) (Section 2.5)."""
        r = self._mask(b0)
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
        b = self._mask(b)
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
