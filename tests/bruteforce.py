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
