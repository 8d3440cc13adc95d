"""Pins of the oracle's global operators, patches, coarse space and solvers.

References: dense matrices assembled from 3D basis gradients (brute force,
tests/bruteforce.py), dense direct solves, dense eigenvalues, the Q1
rediscretisation and the manufactured-solution convergence rate.
"""
import numpy as np
import pytest

from paper_2107_14758_gb300 import inputs
from tests import bruteforce as bf


def _graded(n, seed):
    return inputs.graded_vertices(n, seed)


def _affine_jac(p, nx, ny, nz, xv, yv, zv, shear):
    """Jacobian of x -> M x on every cell (an affine, non-Cartesian mesh)."""
    q = p + 1
    jac = np.zeros((nx * ny * nz, q ** 3, 9))
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                e = cx + nx * (cy + ny * cz)
                h = np.array([xv[cx + 1] - xv[cx], yv[cy + 1] - yv[cy], zv[cz + 1] - zv[cz]])
                J = shear @ np.diag(h / 2)
                jac[e, :, :] = J.ravel()
    return jac


@pytest.mark.parametrize("p", [1, 2, 3])
def test_stiffness_box_vs_dense(oracle_lib, p):
    xv, yv, zv = _graded(2, 7)
    zv = np.array([0.0, 0.3, 0.55, 1.0])
    P = oracle_lib.Problem(p, xv, yv, zv)
    A = bf.dense_matrix(p, xv, yv, zv)
    free = bf.free_mask(p, 2, 2, 3)
    u = np.random.default_rng(0).standard_normal(P.ndof)
    y = P.stiffness_apply(u)
    uf = np.where(free, u, 0.0)
    yref = np.where(free, A @ uf, 0.0)
    assert np.allclose(y, yref, atol=1e-12 * np.abs(yref).max())
    M = bf.dense_matrix(p, xv, yv, zv, mass=True)
    b = P.mass_apply(u)
    assert np.allclose(b, np.where(free, M @ uf, 0.0), atol=1e-13)


@pytest.mark.parametrize("p", [2, 3])
def test_stiffness_curved_vs_dense(oracle_lib, p):
    n = 2
    xv, yv, zv = inputs.uniform_vertices(n)
    jac, pts = inputs.deformed_jacobians(n, p)
    kap = inputs.kappa_field(pts, 3)
    P = oracle_lib.Problem(p, xv, yv, zv, jac=jac, kappa=kap)
    A = bf.dense_matrix(p, xv, yv, zv, jac=jac, kappa=kap)
    free = bf.free_mask(p, n, n, n)
    u = np.random.default_rng(1).standard_normal(P.ndof)
    y = P.stiffness_apply(u)
    yref = np.where(free, A @ np.where(free, u, 0.0), 0.0)
    assert np.allclose(y, yref, atol=1e-12 * np.abs(yref).max())


def test_box_as_curved_equals_kronecker(oracle_lib):
    # eq. (kron) is the quadrature form with Ghat = diag(mu) (Section 2.7)
    p = 3
    xv, yv, zv = _graded(3, 11)
    jac = _affine_jac(p, 3, 3, 3, xv, yv, zv, np.eye(3))
    P1 = oracle_lib.Problem(p, xv, yv, zv)
    P2 = oracle_lib.Problem(p, xv, yv, zv, jac=jac)
    u = np.random.default_rng(2).standard_normal(P1.ndof)
    assert np.allclose(P1.stiffness_apply(u), P2.stiffness_apply(u), atol=1e-12)
    assert np.allclose(P1.get_mu(), P2.get_mu(), rtol=1e-13)


def test_parallelogram_spectrum(oracle_lib):
    # Section 2.7 example: sigma(mu^-1/2 G mu^-1/2) = [1-|cos t|, 1+|cos t|]
    p = 2
    for theta in (0.3, 1.0, 2.2):
        L1, L2 = 0.7, 1.3
        M = np.array([[1.0, np.cos(theta) * L2 / L1, 0.0],
                      [0.0, np.sin(theta) * L2 / L1, 0.0],
                      [0.0, 0.0, 1.0]])
        xv = yv = zv = np.array([0.0, 1.0])
        jac = _affine_jac(p, 1, 1, 1, xv, yv, zv, M)
        P = oracle_lib.Problem(p, xv, yv, zv, jac=jac)
        mu = P.get_mu()[0]
        J = jac[0, 0].reshape(3, 3)
        G = abs(np.linalg.det(J)) * np.linalg.inv(J) @ np.linalg.inv(J).T
        s = np.sort(np.linalg.eigvalsh(np.diag(mu ** -0.5) @ G @ np.diag(mu ** -0.5)))
        c = abs(np.cos(theta))
        assert np.allclose([s[0], s[-1]], [1 - c, 1 + c], atol=1e-12)
        assert abs(s[1] - 1.0) < 1e-12


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_basis_change_roundtrip(oracle_lib, p):
    xv, yv, zv = _graded(2, 5)
    P = oracle_lib.Problem(p, xv, yv, zv)
    free = bf.free_mask(p, 2, 2, 2)
    u = np.where(free, np.random.default_rng(3).standard_normal(P.ndof), 0.0)
    # T_g is invertible; interp(restrict) pairs are transposes: <T^T r, w> = <r, T w>
    w = np.where(free, np.random.default_rng(4).standard_normal(P.ndof), 0.0)
    assert abs(P.restrict_fdm(u) @ w - u @ P.interp_fdm(w)) < 1e-12 * np.abs(u).sum()


def test_patch_structure_counts(oracle_lib):
    # Section 2.6: interior rows of A_j have d+1 = 4 nonzeros; nnz(A_j) is the
    # 7-point-stencil count on the (2p-1)^3 grid; A_II diagonal.
    for p in (3, 4):
        xv, yv, zv = inputs.uniform_vertices(2)
        P = oracle_lib.Problem(p, xv, yv, zv)
        v = 13  # the interior vertex of a 2^3 mesh
        g, nI = P.patch_dofs(v)
        m = 2 * p - 1
        assert len(g) == m ** 3 and nI == 8 * (p - 1) ** 3
        Aj = P.patch_matrix(v)
        assert np.allclose(Aj, Aj.T, atol=1e-14)
        assert np.count_nonzero(Aj) == m ** 3 + 6 * m ** 2 * (m - 1)
        Nx = 2 * p + 1
        for s, gi in enumerate(g):
            gx, gy, gz = gi % Nx, (gi // Nx) % Nx, gi // Nx ** 2
            if gx % p and gy % p and gz % p:
                assert np.count_nonzero(Aj[s]) == 4


def test_patch_equals_direct_solve_on_2cube(oracle_lib):
    # the interior star of a 2^3 mesh covers every free dof: its patch solve
    # is the global direct solve (through the FDM basis change)
    for p in (2, 3, 4):
        xv, yv, zv = _graded(2, 9)
        P = oracle_lib.Problem(p, xv, yv, zv)
        P.setup_patches([13])
        A = bf.dense_matrix(p, xv, yv, zv)
        free = bf.free_mask(p, 2, 2, 2)
        r = np.where(free, np.random.default_rng(5).standard_normal(P.ndof), 0.0)
        g, _ = P.patch_dofs(13)
        x_fdm = np.zeros(P.ndof)
        x_fdm[g] = P.patch_solve(13, P.restrict_fdm(r)[g])
        x = P.interp_fdm(x_fdm)
        xd = np.zeros(P.ndof)
        xd[free] = np.linalg.solve(A[np.ix_(free, free)], r[free])
        assert np.allclose(x, xd, atol=1e-11 * np.abs(xd).max())


@pytest.mark.parametrize("p,n", [(1, 3), (2, 3), (3, 2), (4, 2)])
def test_asm_fdm_equals_asm_gll(oracle_lib, p, n):
    # basis invariance: the FDM-basis patch spaces are the GLL-basis star spaces
    xv, yv, zv = _graded(n, 13)
    P = oracle_lib.Problem(p, xv, yv, zv)
    P.setup_patches()
    P.set_omega(1.0)
    A = bf.dense_matrix(p, xv, yv, zv)
    free = bf.free_mask(p, n, n, n)
    Af = np.where(np.outer(free, free), A, 0.0) + np.diag(~free * 1.0)
    r = np.where(free, np.random.default_rng(6).standard_normal(P.ndof), 0.0)
    z = P.asm_apply(r)
    zref = bf.asm_gll(p, xv, yv, zv, Af, r)
    assert np.allclose(z, zref, atol=1e-11 * np.abs(zref).max())


def test_schur_symmetric_and_pattern(oracle_lib):
    p = 4
    xv, yv, zv = inputs.uniform_vertices(2)
    P = oracle_lib.Problem(p, xv, yv, zv)
    S = P.patch_schur(13)
    assert S.shape == (12 * (p - 1) ** 2 + 6 * (p - 1) + 1,) * 2
    assert np.allclose(S, S.T, atol=1e-14 * np.abs(S).max())
    L = oracle_lib.cholesky(S)
    assert np.allclose(L @ L.T, S, atol=1e-12 * np.abs(S).max())
    fill = oracle_lib.symbolic_fill(S != 0)
    assert not np.any((L != 0) & ~fill)       # numeric nonzeros within the symbolic fill


def test_coarse_is_q1_rediscretisation(oracle_lib):
    # Galerkin P^T A P on box cells equals the Q1 stiffness on the same mesh
    xv, yv, zv = _graded(3, 17)
    for p in (2, 4):
        P = oracle_lib.Problem(p, xv, yv, zv)
        P.setup_coarse()
        Ac = P.coarse_matrix()
        A1 = bf.q1_dense(xv, yv, zv)
        f1 = bf.free_mask(1, 3, 3, 3)
        assert np.allclose(Ac, A1[np.ix_(f1, f1)], atol=1e-12)


def test_coarse_projection_property(oracle_lib):
    # C A P v = P v  (C = P A_c^{-1} P^T is the A-orthogonal projector onto range P)
    p = 3
    xv, yv, zv = _graded(3, 19)
    jac, pts = inputs.deformed_jacobians(3, p, vertices=(xv, yv, zv))
    P = oracle_lib.Problem(p, xv, yv, zv, jac=jac)
    P.setup_coarse()
    # P v for a random coarse v: interpolate a trilinear field to the GLL grid
    rng = np.random.default_rng(8)
    vc = np.zeros((4, 4, 4)); vc[1:3, 1:3, 1:3] = rng.standard_normal((2, 2, 2))
    xi = inputs.gll_points(p)
    def hat(v, pp):
        out = np.zeros((len(v), 3 * pp + 1, ))
        return out
    N = 3 * p + 1
    w1 = np.zeros((N, 4))
    for c in range(3):
        for i in range(p + 1):
            w1[c * p + i, c] = 0.5 * (1 - xi[i]); w1[c * p + i, c + 1] = 0.5 * (1 + xi[i])
    u = np.einsum("zc,yb,xa,cba->zyx", w1, w1, w1, vc).ravel()
    z = P.coarse_apply(P.stiffness_apply(u))
    assert np.allclose(z, u, atol=1e-11 * np.abs(u).max())


def test_pcg_matches_direct_solve(oracle_lib):
    p, n = 3, 3
    xv, yv, zv = _graded(n, 21)
    P = oracle_lib.Problem(p, xv, yv, zv)
    P.setup_patches(); P.setup_coarse()
    b0 = inputs.lanczos_start(P.ndof)
    P.lanczos_omega(b0)
    A = bf.dense_matrix(p, xv, yv, zv)
    free = bf.free_mask(p, n, n, n)
    b = np.where(free, np.random.default_rng(9).standard_normal(P.ndof), 0.0)
    xd = np.zeros(P.ndof)
    xd[free] = np.linalg.solve(A[np.ix_(free, free)], b[free])
    for pc in (0, 1, 2):
        x, it, hist, conv = P.pcg(b, rtol=1e-10, maxit=500, pc=pc)
        assert conv
        assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)


def test_pc_symmetric_positive(oracle_lib):
    p, n = 2, 3
    xv, yv, zv = _graded(n, 23)
    P = oracle_lib.Problem(p, xv, yv, zv)
    P.setup_patches(); P.setup_coarse()
    P.lanczos_omega(inputs.lanczos_start(P.ndof))
    free = bf.free_mask(p, n, n, n)
    rng = np.random.default_rng(10)
    r1 = np.where(free, rng.standard_normal(P.ndof), 0.0)
    r2 = np.where(free, rng.standard_normal(P.ndof), 0.0)
    z1, z2 = P.pc_apply(r1), P.pc_apply(r2)
    assert abs(z1 @ r2 - z2 @ r1) < 1e-11 * abs(z1 @ r1)
    assert z1 @ r1 > 0 and z2 @ r2 > 0


def test_lanczos_extremes_vs_dense_eigs(oracle_lib):
    # enough Lanczos steps on a tiny problem recover the exact extreme
    # eigenvalues of P_ASM^{-1} A (dense, GLL basis, brute force)
    p, n = 2, 2
    xv, yv, zv = _graded(n, 25)
    P = oracle_lib.Problem(p, xv, yv, zv)
    P.setup_patches()
    A = bf.dense_matrix(p, xv, yv, zv)
    free = bf.free_mask(p, n, n, n)
    Af = A[np.ix_(free, free)]
    nf = free.sum()
    Pinv = np.zeros((nf, nf))
    idx = np.flatnonzero(free)
    for v in range(27):
        s = bf.star_nodes(p, n, n, n, v)
        loc = np.searchsorted(idx, s)
        Pinv[np.ix_(loc, loc)] += np.linalg.inv(Af[np.ix_(loc, loc)])
    ev = np.sort(np.linalg.eigvals(Pinv @ Af).real)
    lo, hi, om = P.lanczos_omega(inputs.lanczos_start(P.ndof), k=nf)
    assert abs(hi - ev[-1]) < 1e-8 * ev[-1]
    assert abs(lo - ev[0]) < 1e-6 * ev[-1]
    assert abs(om - 2.0 / (1.25 * hi + 0.75 * lo)) < 1e-14


@pytest.mark.slow
def test_manufactured_convergence(oracle_lib):
    # O(h^{p+1}) L2 error for the manufactured sine solution (Section 2.8 setup)
    from numpy.polynomial import legendre as leg
    for p in (1, 2, 3):
        errs = []
        for n in (2, 4, 8):
            xv, yv, zv = inputs.uniform_vertices(n)
            P = oracle_lib.Problem(p, xv, yv, zv)
            P.setup_patches(); P.setup_coarse()
            P.lanczos_omega(inputs.lanczos_start(P.ndof))
            b = P.mass_apply(inputs.manufactured_f(xv, yv, zv, p))
            x, it, _, conv = P.pcg(b, rtol=1e-12, maxit=300)
            assert conv
            # L2 error by a (p+3)-point Gauss rule per direction and cell
            xg, wg = leg.leggauss(p + 3)
            Vq, _ = bf._basis_at(p, xg)
            N = n * p + 1
            X = x.reshape(N, N, N)
            err2 = 0.0
            h = 1.0 / n
            for cz in range(n):
                for cy in range(n):
                    for cx in range(n):
                        U = X[cz * p:cz * p + p + 1, cy * p:cy * p + p + 1, cx * p:cx * p + p + 1]
                        uq = np.einsum("ck,bj,ai,kji->cba", Vq, Vq, Vq, U)
                        pz = (cz + 0.5 * (1 + xg)) * h
                        py = (cy + 0.5 * (1 + xg)) * h
                        px = (cx + 0.5 * (1 + xg)) * h
                        ex = np.einsum("c,b,a->cba", np.sin(np.pi * pz), np.sin(np.pi * py), np.sin(np.pi * px))
                        w = np.einsum("c,b,a->cba", wg, wg, wg) * (h / 2) ** 3
                        err2 += np.sum(w * (uq - ex) ** 2)
            errs.append(np.sqrt(err2))
        rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
        assert rates[-1] > p + 1 - 0.35, (p, errs, rates)


def test_iterations_flat_in_p(oracle_lib):
    # Table 1 context: Cartesian 3D iteration counts stay flat (~12) in p
    its = []
    for p in (2, 3, 4, 5):
        xv, yv, zv = inputs.uniform_vertices(3)
        P = oracle_lib.Problem(p, xv, yv, zv)
        P.setup_patches(); P.setup_coarse()
        P.lanczos_omega(inputs.lanczos_start(P.ndof))
        b = P.mass_apply(np.ones(P.ndof))
        _, it, _, conv = P.pcg(b, rtol=1e-8, maxit=100)
        assert conv
        its.append(it)
    assert max(its) - min(its) <= 3 and max(its) <= 16, its


# ---------------------------------------------------------------- geometric multigrid on the Q1 problem
def _coarsened(v):
    return v[::2].copy()


def test_gmg_galerkin_level_equals_rediscretised_q1(oracle_lib):
    """Nested Q1 spaces: P^T A_0 P on the graded 8^3 mesh equals the Q1
    stiffness of the mesh with every other vertex (pins the interpolation
    weights in the graded coordinates and the triple product)."""
    xv, yv, zv = inputs.graded_vertices(8, 17)
    P = oracle_lib.Problem(3, xv, yv, zv)
    P.setup_coarse()
    assert P.setup_coarse_gmg(2) == 2
    A1 = P.gmg_level(1)
    Q = oracle_lib.Problem(1, _coarsened(xv), _coarsened(yv), _coarsened(zv))
    Q.setup_coarse()
    ref = Q.coarse_matrix()
    assert A1.shape == ref.shape == (27, 27)
    assert np.abs(A1 - ref).max() <= 1e-12 * np.abs(ref).max()
    A2 = P.gmg_level(2)
    assert A2.shape == (1, 1)


def test_gmg_vcycle_converges_as_iteration(oracle_lib):
    """One V-cycle (2 + 2 damped Jacobi sweeps, omega = 2/3) used as a
    stationary iteration on the Q1 problem reduces the residual by a factor
    well below one per cycle, on a graded mesh."""
    xv, yv, zv = inputs.graded_vertices(12, 18)
    P = oracle_lib.Problem(1, xv, yv, zv)
    P.setup_coarse()
    assert P.setup_coarse_gmg(5) == 2                 # 12 -> 6 -> 3 cells per axis
    A = P.coarse_matrix()
    b = np.random.default_rng(3).standard_normal(A.shape[0])
    x = np.zeros_like(b)
    r0 = np.linalg.norm(b)
    rates = []
    for _ in range(6):
        r = b - A @ x
        x = x + P.gmg_vcycle(r)
        rn = np.linalg.norm(b - A @ x)
        rates.append(rn / np.linalg.norm(r))
    assert max(rates[1:]) < 0.35, rates
    assert np.linalg.norm(b - A @ x) < 1e-3 * r0


def test_pcg_with_gmg_coarse_solve(oracle_lib):
    """The hybrid V(1,1) with one multigrid V-cycle on the Q1 problem as its
    coarse correction: PCG converges in at most two more iterations than with
    the exact coarse solve."""
    xv, yv, zv = inputs.graded_vertices(8, 19)
    P = oracle_lib.Problem(3, xv, yv, zv)
    P.setup_patches()
    P.setup_coarse()
    P.lanczos_omega(inputs.lanczos_start(P.ndof))
    free = bf.free_mask(3, 8, 8, 8)
    b = np.where(free, P.mass_apply(inputs.normal_rhs(P.ndof, 5)), 0.0)
    x0, it0, _, conv0 = P.pcg(b, 1e-8, 200)
    assert P.setup_coarse_gmg(2) == 2
    x1, it1, _, conv1 = P.pcg(b, 1e-8, 200)
    assert conv0 and conv1
    assert it0 <= it1 <= it0 + 2, (it0, it1)
    assert np.abs(x1 - x0).max() <= 1e-6 * np.abs(x0).max()


def _fdm_basis_1d(p):
    """The 1D FDM basis change T (Sec. 2.4) built independently of the
    oracle: interior eigenvectors of A_II s = lambda B_II s from scipy's
    symmetric-definite solver (ascending, B-orthonormal, first interior entry
    positive), vertex functions B-orthogonal to them."""
    import scipy.linalg as sla
    A, B = bf.ref_matrices_exact(p)
    n = p + 1
    T = np.eye(n)
    if p >= 2:
        I = np.arange(1, p)
        _, S = sla.eigh(A[np.ix_(I, I)], B[np.ix_(I, I)])
        S = S * np.where(S[0] < 0, -1.0, 1.0)
        T[np.ix_(I, I)] = S
        T[np.ix_(I, [0, p])] = -np.linalg.solve(B[np.ix_(I, I)], B[np.ix_(I, [0, p])])
    return T


def _global_fdm_basis(p, nx, ny, nz):
    """T_g = T_z (x) T_y (x) T_x over the grid slots: column s is the GLL
    expansion of the FDM function in slot s (x fastest)."""
    T = _fdm_basis_1d(p)
    mats = []
    for nc in (nx, ny, nz):
        N = nc * p + 1
        G = np.zeros((N, N))
        for c in range(nc):
            G[c * p + 1:c * p + p, c * p:c * p + p + 1] = T[1:p, :]
        for v in range(nc + 1):
            G[v * p, v * p] = 1.0
        mats.append(G)
    return np.kron(mats[2], np.kron(mats[1], mats[0]))


def _surrogate_jac(mu, q):
    """Box cells whose Kronecker stiffness has the per-axis coefficients mu
    (mu_a = L_x L_y L_z / L_a^2 for half-widths L): L = (sqrt(mu_y mu_z),
    sqrt(mu_x mu_z), sqrt(mu_x mu_y)), one diagonal Jacobian per cell."""
    mu = np.asarray(mu).reshape(-1, 3)
    L = np.stack([np.sqrt(mu[:, 1] * mu[:, 2]), np.sqrt(mu[:, 0] * mu[:, 2]), np.sqrt(mu[:, 0] * mu[:, 1])], axis=1)
    jac = np.zeros((len(mu), q ** 3, 9))
    jac[:, :, 0], jac[:, :, 4], jac[:, :, 8] = L[:, None, 0], L[:, None, 1], L[:, None, 2]
    return jac


@pytest.mark.parametrize("p,curved", [(2, False), (3, False), (4, False), (2, True), (3, True)])
def test_patch_matrix_is_basis_transform_of_gll_patch(oracle_lib, p, curved):
    """Every star's sparse FDM-basis matrix equals T_j^T A_j^GLL T_j, with
    A_j^GLL the dense GLL-basis matrix of the star's separable surrogate
    (the operator itself on box cells) assembled from 3D basis gradients and
    T_j the star's columns of the global FDM basis change (<= 1e-12).  A 3^3
    mesh has interior, face, edge and corner stars."""
    n = 3
    if curved:
        xv, yv, zv = inputs.uniform_vertices(n)
        jac, pts = inputs.deformed_jacobians(n, p)
        P = oracle_lib.Problem(p, xv, yv, zv, jac=jac, kappa=inputs.kappa_field(pts, 3))
        A = bf.dense_matrix(p, xv, yv, zv, jac=_surrogate_jac(P.get_mu(), p + 1))
    else:
        xv, yv, zv = _graded(n, 41)
        P = oracle_lib.Problem(p, xv, yv, zv)
        A = bf.dense_matrix(p, xv, yv, zv)
    free = bf.free_mask(p, n, n, n)
    A = np.where(np.outer(free, free), A, 0.0)
    Tg = _global_fdm_basis(p, n, n, n)
    classes = set()
    for v in range((n + 1) ** 3):
        g, _ = P.patch_dofs(v)
        if len(g) == 0:
            continue
        vx, vy, vz = v % (n + 1), (v // (n + 1)) % (n + 1), v // (n + 1) ** 2
        classes.add(sum(c in (0, n) for c in (vx, vy, vz)))
        Tj = Tg[:, g]
        ref = Tj.T @ A @ Tj
        Aj = P.patch_matrix(v)
        assert np.abs(Aj - ref).max() <= 1e-12 * np.abs(ref).max(), v
    assert classes == {0, 1, 2, 3}  # interior, face, edge and corner stars
