"""Independent brute-force references used to pin the oracle.

Everything here is built from numpy polynomials and explicit 3D quadrature
of basis-function gradients on tiny meshes; it shares nothing with
oracle/oracle.c (different node computation, exact polynomial integration for
1D matrices, dense global matrices assembled from 3D gradients).
"""
import numpy as np
from numpy.polynomial import Polynomial as Poly
from numpy.polynomial import legendre as leg


def gll_nodes(p):
    if p == 1:
        return np.array([-1.0, 1.0])
    r = np.sort(leg.Legendre.basis(p).deriv().roots().real)
    return np.concatenate([[-1.0], r, [1.0]])


def lagrange_polys(xi):
    out = []
    for j in range(len(xi)):
        others = np.delete(xi, j)
        pj = Poly.fromroots(others)
        out.append(pj / pj(xi[j]))
    return out


def ref_matrices_exact(p):
    """A_ij = int l_i' l_j', B_ij = int l_i l_j by exact polynomial integration."""
    xi = gll_nodes(p)
    L = lagrange_polys(xi)
    n = p + 1
    A = np.zeros((n, n)); B = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            a = (L[i].deriv() * L[j].deriv()).integ()
            b = (L[i] * L[j]).integ()
            A[i, j] = a(1) - a(-1)
            B[i, j] = b(1) - b(-1)
    return A, B


def _basis_at(p, pts):
    """Lagrange values and derivatives at points that are not GLL nodes:
    product form, derivative as l_j(x) * sum_k 1/(x - xi_k) (log-derivative)."""
    xi = gll_nodes(p)
    pts = np.asarray(pts, dtype=float)
    V = np.zeros((len(pts), p + 1)); D = np.zeros((len(pts), p + 1))
    for a, t in enumerate(pts):
        for j in range(p + 1):
            others = np.delete(xi, j)
            if np.any(np.abs(t - xi) < 1e-13):
                # at a node: fall back to exact polynomials (small p only)
                lj = lagrange_polys(xi)[j]
                V[a, j] = lj(t); D[a, j] = lj.deriv()(t)
                continue
            v = np.prod((t - others) / (xi[j] - others))
            V[a, j] = v
            D[a, j] = v * np.sum(1.0 / (t - others))
    return V, D


def ref_matrices_quad(p):
    """A_hat, B_hat from a Gauss rule with p + 3 points (exact for degree 2p)."""
    x, w = leg.leggauss(p + 3)
    V, D = _basis_at(p, x)
    return D.T @ (w[:, None] * D), V.T @ (w[:, None] * V)


def grid_shape(p, nx, ny, nz):
    return nx * p + 1, ny * p + 1, nz * p + 1


def free_mask(p, nx, ny, nz):
    Nx, Ny, Nz = grid_shape(p, nx, ny, nz)
    m = np.ones((Nz, Ny, Nx), dtype=bool)
    m[0, :, :] = m[-1, :, :] = False
    m[:, 0, :] = m[:, -1, :] = False
    m[:, :, 0] = m[:, :, -1] = False
    return m.ravel()


def dense_matrix(p, xv, yv, zv, jac=None, kappa=None, mass=False, q=None):
    """Dense global matrix on the full grid (Neumann; restrict with free_mask).

    Cell matrices are computed from 3D basis gradients at a tensor Gauss
    rule (q points, default p+1, matching the discretisation's rule), with
    physical gradients J^{-T} grad_hat phi and weight |det J|.
    """
    nx, ny, nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
    n = p + 1
    q = q or n
    xg, wg = leg.leggauss(q)
    V, D = _basis_at(p, xg)
    Nx, Ny, Nz = grid_shape(p, nx, ny, nz)
    M = np.zeros((Nx * Ny * Nz, Nx * Ny * Nz))
    # 3D basis (local index i + n(j + n k)) at points (a + q(b + q c))
    phi = np.einsum("ck,bj,ai->cbakji", V, V, V).reshape(q ** 3, n ** 3)
    gx = np.einsum("ck,bj,ai->cbakji", V, V, D).reshape(q ** 3, n ** 3)
    gy = np.einsum("ck,bj,ai->cbakji", V, D, V).reshape(q ** 3, n ** 3)
    gz = np.einsum("ck,bj,ai->cbakji", D, V, V).reshape(q ** 3, n ** 3)
    w3 = np.einsum("c,b,a->cba", wg, wg, wg).ravel()
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                e = cx + nx * (cy + ny * cz)
                if jac is None:
                    h = np.array([xv[cx + 1] - xv[cx], yv[cy + 1] - yv[cy], zv[cz + 1] - zv[cz]])
                    J = np.tile(np.diag(h / 2), (q ** 3, 1, 1))
                else:
                    J = np.asarray(jac[e]).reshape(q ** 3, 3, 3)
                det = np.abs(np.linalg.det(J))
                kap = np.ones(q ** 3) if kappa is None else np.asarray(kappa[e]).ravel()
                if mass:
                    K = np.einsum("q,qi,qj->ij", w3 * det, phi, phi)
                else:
                    Jinv = np.linalg.inv(J)  # grad = J^{-T} grad_hat
                    G = np.stack([gx, gy, gz], axis=-1)  # q, i, 3
                    Gp = np.einsum("qar,qir->qia", np.transpose(Jinv, (0, 2, 1)), G)
                    K = np.einsum("q,qia,qja->ij", w3 * det * kap, Gp, Gp)
                idx = []
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            idx.append((cx * p + i) + Nx * ((cy * p + j) + Ny * (cz * p + k)))
                idx = np.array(idx)
                M[np.ix_(idx, idx)] += K
    return M


def star_nodes(p, nx, ny, nz, v):
    """Grid nodes (free) within p-1 of vertex v along every axis."""
    Nx, Ny, Nz = grid_shape(p, nx, ny, nz)
    vx = v % (nx + 1); vy = (v // (nx + 1)) % (ny + 1); vz = v // ((nx + 1) * (ny + 1))
    out = []
    for gz in range(max(1, p * vz - p + 1), min(Nz - 2, p * vz + p - 1) + 1):
        for gy in range(max(1, p * vy - p + 1), min(Ny - 2, p * vy + p - 1) + 1):
            for gx in range(max(1, p * vx - p + 1), min(Nx - 2, p * vx + p - 1) + 1):
                out.append(gx + Nx * (gy + Ny * gz))
    return np.array(out, dtype=np.int64)


def asm_gll(p, xv, yv, zv, A_full, r):
    """Additive Schwarz over all vertex stars with dense GLL patch matrices."""
    nx, ny, nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
    z = np.zeros_like(r)
    for v in range((nx + 1) * (ny + 1) * (nz + 1)):
        s = star_nodes(p, nx, ny, nz, v)
        if len(s) == 0:
            continue
        z[s] += np.linalg.solve(A_full[np.ix_(s, s)], r[s])
    return z


def q1_dense(xv, yv, zv):
    """Trilinear (Q1) stiffness on the vertex grid by 2-point Gauss per axis."""
    return dense_matrix(1, xv, yv, zv)


def dense_elasticity(p, xv, yv, zv, mu, lam, q=None):
    """Dense linear-elasticity matrix on the full grid, component-major
    [3 N, 3 N] (Neumann; restrict with free_mask per component).

    Cell matrices from 3D basis gradients at a tensor Gauss rule: for
    v = phi_i e_a, u = phi_j e_b, 2 eps(v):eps(u) = delta_ab grad phi_i . grad
    phi_j + d_b phi_i d_a phi_j and div v div u = d_a phi_i d_b phi_j.
    """
    nx, ny, nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
    n = p + 1
    q = q or n + 1
    xg, wg = leg.leggauss(q)
    V, D = _basis_at(p, xg)
    Nx, Ny, Nz = grid_shape(p, nx, ny, nz)
    N = Nx * Ny * Nz
    M = np.zeros((3 * N, 3 * N))
    gx = np.einsum("ck,bj,ai->cbakji", V, V, D).reshape(q ** 3, n ** 3)
    gy = np.einsum("ck,bj,ai->cbakji", V, D, V).reshape(q ** 3, n ** 3)
    gz = np.einsum("ck,bj,ai->cbakji", D, V, V).reshape(q ** 3, n ** 3)
    w3 = np.einsum("c,b,a->cba", wg, wg, wg).ravel()
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                h = np.array([xv[cx + 1] - xv[cx], yv[cy + 1] - yv[cy], zv[cz + 1] - zv[cz]])
                det = np.prod(h / 2)
                G = np.stack([gx * 2 / h[0], gy * 2 / h[1], gz * 2 / h[2]], axis=-1)   # q, i, 3 (physical)
                w = w3 * det
                lap = np.einsum("q,qia,qja->ij", w, G, G)
                K = np.zeros((3, n ** 3, 3, n ** 3))
                for a in range(3):
                    for b in range(3):
                        blk = mu * np.einsum("q,qi,qj->ij", w, G[:, :, b], G[:, :, a]) + \
                            lam * np.einsum("q,qi,qj->ij", w, G[:, :, a], G[:, :, b])
                        if a == b:
                            blk = blk + mu * lap
                        K[a, :, b, :] = blk
                idx = []
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            idx.append((cx * p + i) + Nx * ((cy * p + j) + Ny * (cz * p + k)))
                idx = np.array(idx)
                full = np.concatenate([idx + a * N for a in range(3)])
                M[np.ix_(full, full)] += K.reshape(3 * n ** 3, 3 * n ** 3)
    return M


def dense_sipg(p, xv, yv, zv, eta, q=None):
    """Dense SIPG matrix of the DQ_p Poisson problem (cell-major values, cells x
    fastest, (z, y, x) inside a cell), weak Dirichlet condition on the whole
    boundary, from explicit quadrature of the weak form in physical
    coordinates: cell integrals of grad v . grad u; on every facet the
    penalty eta |e| mean(1/|K|) [v].[u] and the two consistency terms
    -[v].{grad u} - {grad v}.[u], with [w] = sum over the sides of w n_side
    and {.} the mean of the sides (one side on the boundary)."""
    nc = [len(xv) - 1, len(yv) - 1, len(zv) - 1]
    verts = [np.asarray(a, dtype=float) for a in (xv, yv, zv)]
    n = p + 1
    q = q or n + 1
    xg, wg = leg.leggauss(q)
    polys = lagrange_polys(gll_nodes(p))
    dpolys = [P.deriv() for P in polys]
    ncell = nc[0] * nc[1] * nc[2]
    N = ncell * n ** 3
    M = np.zeros((N, N))

    def cell_id(c):
        return c[0] + nc[0] * (c[1] + nc[1] * c[2])

    def geom(c):
        lo = np.array([verts[a][c[a]] for a in range(3)])
        w = np.array([verts[a][c[a] + 1] - verts[a][c[a]] for a in range(3)])
        return lo, w

    def eval_cell(c, pts):
        """Values [npts, n^3] and physical gradients [npts, n^3, 3] of cell c's basis."""
        lo, w = geom(c)
        ref = 2.0 * (pts - lo) / w - 1.0
        val1 = [np.array([[P(t) for P in polys] for t in ref[:, a]]) for a in range(3)]
        der1 = [np.array([[P(t) for P in dpolys] for t in ref[:, a]]) * (2.0 / w[a]) for a in range(3)]
        phi = np.einsum("qk,qj,qi->qkji", val1[2], val1[1], val1[0]).reshape(len(pts), -1)
        g = np.stack([np.einsum("qk,qj,qi->qkji", val1[2], val1[1], der1[0]).reshape(len(pts), -1),
                      np.einsum("qk,qj,qi->qkji", val1[2], der1[1], val1[0]).reshape(len(pts), -1),
                      np.einsum("qk,qj,qi->qkji", der1[2], val1[1], val1[0]).reshape(len(pts), -1)], axis=-1)
        return phi, g

    cells = [(cx, cy, cz) for cz in range(nc[2]) for cy in range(nc[1]) for cx in range(nc[0])]
    for c in cells:
        lo, w = geom(c)
        g1 = [lo[a] + 0.5 * w[a] * (xg + 1.0) for a in range(3)]
        pts = np.stack(np.meshgrid(g1[0], g1[1], g1[2], indexing="ij"), axis=-1).reshape(-1, 3)
        wt = np.einsum("i,j,k->ijk", wg, wg, wg).ravel() * np.prod(w / 2.0)
        _, g = eval_cell(c, pts)
        K = np.einsum("q,qia,qja->ij", wt, g, g)
        s = cell_id(c) * n ** 3
        M[s:s + n ** 3, s:s + n ** 3] += K
    for c in cells:
        lo, w = geom(c)
        volK = np.prod(w)
        for a in range(3):
            for side in (0, 1):                      # the low (0) or high (1) face of c normal to axis a
                nb = list(c)
                nb[a] += 1 if side else -1
                inside = 0 <= nb[a] < nc[a]
                if inside and side == 0:
                    continue                         # each interior facet once, from its low cell
                t = [b for b in range(3) if b != a]
                area = w[t[0]] * w[t[1]]
                ft = [lo[b] + 0.5 * w[b] * (xg + 1.0) for b in t]
                P1, P2 = np.meshgrid(ft[0], ft[1], indexing="ij")
                pts = np.zeros((q * q, 3))
                pts[:, t[0]], pts[:, t[1]] = P1.ravel(), P2.ravel()
                pts[:, a] = lo[a] + (w[a] if side else 0.0)
                ws = np.einsum("i,j->ij", wg, wg).ravel() * area / 4.0
                normal = np.zeros(3)
                normal[a] = 1.0 if side else -1.0    # outward normal of c
                phi, g = eval_cell(c, pts)
                if inside:
                    nbt = tuple(nb)
                    phin, gn = eval_cell(nbt, pts)
                    volN = np.prod(geom(nbt)[1])
                    hinv = area * 0.5 * (1.0 / volK + 1.0 / volN)
                    # jumps along the normal of c: v_c n_c + v_nb (-n_c)
                    J = np.concatenate([phi, -phin], axis=1)
                    G = 0.5 * np.concatenate([g @ normal, gn @ normal], axis=1)
                    idx = np.concatenate([cell_id(c) * n ** 3 + np.arange(n ** 3),
                                          cell_id(nbt) * n ** 3 + np.arange(n ** 3)])
                else:
                    hinv = area / volK
                    J = phi
                    G = g @ normal
                    idx = cell_id(c) * n ** 3 + np.arange(n ** 3)
                F = (eta * hinv * np.einsum("q,qi,qj->ij", ws, J, J)
                     - np.einsum("q,qi,qj->ij", ws, J, G) - np.einsum("q,qi,qj->ij", ws, G, J))
                M[np.ix_(idx, idx)] += F
    return M


def q1_stiffness_hex(X, cells, q):
    """Stiffness matrix of the conforming Q1 space on a general hexahedral
    mesh (trilinear cells, corners at index a + 2b + 4c), indexed by mesh
    vertex: each entry summed over cells of the q^3-point Gauss rule of
    grad N_u . grad N_v |det J| with the physical gradients J^{-T} grad_xi."""
    X = np.asarray(X, dtype=np.float64)
    nv = X.shape[0]
    A = np.zeros((nv, nv))
    t, w = leg.leggauss(q)
    corners = [(a, b, c) for c in (0, 1) for b in (0, 1) for a in (0, 1)]

    def hat(s, k):
        return 0.5 * (1.0 + s) if k else 0.5 * (1.0 - s)

    def dhat(k):
        return 0.5 if k else -0.5

    for cell in np.asarray(cells):
        P = X[cell]
        for i, xi in enumerate(t):
            for j, eta in enumerate(t):
                for k, zeta in enumerate(t):
                    # reference gradients of the 8 trilinear functions, [8, 3]
                    g = np.array([[dhat(a) * hat(eta, b) * hat(zeta, c),
                                   hat(xi, a) * dhat(b) * hat(zeta, c),
                                   hat(xi, a) * hat(eta, b) * dhat(c)] for (a, b, c) in corners])
                    J = P.T @ g                      # J[i, d] = d x_i / d xi_d
                    phys = np.linalg.solve(J.T, g.T).T  # rows: physical gradients
                    wt = w[i] * w[j] * w[k] * abs(np.linalg.det(J))
                    A[np.ix_(cell, cell)] += wt * phys @ phys.T
    return A
