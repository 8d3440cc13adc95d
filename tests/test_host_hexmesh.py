"""CPU tests of the library's host topology for general hexahedral meshes
(fdm_hexmesh_*, through the C-ABI; no GPU) against the unstructured oracle
(oracle/unstructured.py), which numbers nodes independently by merging the
cells' GLL nodes by position and glues its star FDM bases by matching traces:

* the library's node numbering is a consistent bijection onto the oracle's
  (every cell-local node maps through it to the oracle's node);
* Dirichlet nodes and every star's node set agree;
* the star FDM functions built from the library's signed cell-to-global map
  agree on every node shared by two cells (the parity signs are right), and
  the library's structural star pattern equals the numerical pattern of the
  oracle's surrogate star matrix in that basis;
* interior rows of every star pattern have d + 1 = 4 entries and no
  interior-interior coupling (Section 2.6);
* every class's symbolic factorisation of the interface Schur complement
  (fill and elimination tree) equals the oracle's symbolic fill of the
  numerically formed Schur complement, and the numeric Cholesky factor stays
  inside it; stars are ordered canonically, so a tensor mesh has 4 classes in
  any cell orientation;
* one additive Schwarz sweep assembled from the library's tables and factors
  alone, in the steps of a GPU apply (cell-local FDM residuals, assembly per
  FDM slot, star block eliminations, sum per slot, basis change back per
  cell), equals the oracle's sweep; so do the stiffness apply from the
  library's geometry factors and node-to-cell map, the library's Q1 coarse
  operator and the hybrid V(1,1) built from them (with a coefficient kappa);
* the Schur-coupling form of every star (L_BB, S_TB, W) solves the oracle's
  interface Schur complement and stores fewer values on the large stars;
* the numeric set-up (fdm_hexmesh_factor) gives the oracle's surrogate
  coefficients (also with a coefficient at the Gauss points), interior pivots
  and interface Schur complement (L L^T), and the star solve from D and L in
  the FDM basis is the oracle's star solve;
* invalid meshes and geometry are rejected.
"""
import numpy as np
import pytest

from oracle.unstructured import HexProblem, _kron3
from paper_2107_14758_gb300 import inputs


@pytest.fixture(scope="module")
def fdmpc():
    from paper_2107_14758_gb300 import build
    build.build()
    from paper_2107_14758_gb300 import fdmpc as f
    return f


MESHES = {
    "unstructured": lambda: inputs.unstructured_hex_mesh(2, 2, 5),
    "reoriented_tensor": lambda: (lambda X, c: (X, inputs.reorient_cells(c, 11)))(
        *inputs.tensor_hex_mesh(*inputs.graded_vertices(3, 4))),
}


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("p", [1, 2, 3])
def test_topology_matches_the_oracle(fdmpc, name, p):
    X, cells = MESHES[name]()
    H = fdmpc.HexMesh(X.shape[0], cells, p)
    U = HexProblem(p, X, cells)
    n = p + 1
    cn = H.cell_nodes()
    assert H.nnode == U.ndof
    pi = -np.ones(H.nnode, dtype=np.int64)
    pi[cn.ravel()] = U.gid.ravel()
    assert np.array_equal(pi[cn], U.gid)                      # consistent
    assert np.array_equal(np.sort(pi), np.arange(U.ndof))     # bijective
    assert np.array_equal(H.dirichlet(), U.dirichlet[pi])
    stars = H.stars()
    assert len(stars) == sum(1 for v in range(X.shape[0]) if len(U.star_dofs(v)))
    cf, cs = H.cell_fdm()
    T3 = _kron3(U.T1, U.T1, U.T1)
    for (v, nodes), (rp, cols) in zip(stars, H.patterns()):
        assert np.array_equal(np.sort(pi[nodes]), U.star_dofs(v))
        pos = {int(g): i for i, g in enumerate(nodes)}
        ns = len(nodes)
        Tv = np.zeros((ns, ns))
        setm = np.zeros((ns, ns), dtype=bool)
        for e in U.vertex_cells[v]:
            rows = np.array([pos.get(int(g), -1) for g in cn[e]])
            inside = rows >= 0
            for c in range(n ** 3):
                col = pos.get(int(cf[e, c]))
                if col is None:
                    continue
                vals = cs[e, c] * T3[:, c]
                assert np.abs(vals[~inside]).max(initial=0.0) <= 1e-13
                r = rows[inside]
                prev = setm[r, col]
                assert np.abs(Tv[r[prev], col] - vals[inside][prev]).max(initial=0.0) <= 1e-12
                Tv[r, col] = vals[inside]
                setm[r, col] = True
        dofs = pi[nodes]
        Af = Tv.T @ U.As[dofs][:, dofs].toarray() @ Tv
        P = np.zeros((ns, ns), dtype=bool)
        for r in range(ns):
            P[r, cols[rp[r]:rp[r + 1]]] = True
        assert np.array_equal(np.abs(Af) > 1e-12 * np.abs(Af).max(), P)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_interior_rows_of_star_patterns(fdmpc, p):
    X, cells = inputs.unstructured_hex_mesh(2, 2, 5)
    H = fdmpc.HexMesh(X.shape[0], cells, p)
    cn = H.cell_nodes()
    interior = np.zeros(H.nnode, dtype=bool)
    n = p + 1
    idx = np.arange(n)
    I3 = np.stack(np.meshgrid(idx, idx, idx, indexing="ij"), axis=-1).reshape(-1, 3)
    cell_int = np.all((I3 > 0) & (I3 < p), axis=1)
    interior[cn[:, cell_int].ravel()] = True
    for (v, nodes), (rp, cols) in zip(H.stars(), H.patterns()):
        ni = int(interior[nodes].sum())
        assert interior[nodes[:ni]].all() and not interior[nodes[ni:]].any()  # interiors first
        for r in range(ni):
            row = cols[rp[r]:rp[r + 1]]
            assert r in row and not np.any((row < ni) & (row != r))
            # itself plus the faces of its cell that contain v (3, fewer at the boundary)
            assert len(row) <= 4


def test_invalid_meshes(fdmpc):
    X, cells = inputs.tensor_hex_mesh(*inputs.uniform_vertices(2))
    nv = X.shape[0]
    with pytest.raises(fdmpc.FdmError):
        fdmpc.HexMesh(nv, cells, 0)
    with pytest.raises(fdmpc.FdmError):
        fdmpc.HexMesh(nv, cells, 16)
    bad = cells.copy()
    bad[0, 0] = nv
    with pytest.raises(fdmpc.FdmError, match="out of range"):
        fdmpc.HexMesh(nv, bad, 2)
    bad = cells.copy()
    bad[0, 1] = bad[0, 0]
    with pytest.raises(fdmpc.FdmError, match="degenerate"):
        fdmpc.HexMesh(nv, bad, 2)
    three = np.concatenate([cells[:1], cells[:1], cells[:1]])
    with pytest.raises(fdmpc.FdmError, match="more than two cells"):
        fdmpc.HexMesh(nv, three, 2)


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("p", [2, 3, 4])
def test_class_symbolic_factorisation(fdmpc, oracle_lib, name, p):
    """Each class's fill and elimination tree equal the oracle's symbolic
    fill of the numerically formed interface Schur complement of its first
    star (in the basis of the library's signed FDM map), the numeric Cholesky
    factor stays inside the fill, and every star of a class has its pattern."""
    X, cells = MESHES[name]()
    H = fdmpc.HexMesh(X.shape[0], cells, p)
    U = HexProblem(p, X, cells)
    n = p + 1
    cn = H.cell_nodes()
    cf, cs = H.cell_fdm()
    pi = np.zeros(H.nnode, dtype=np.int64)
    pi[cn.ravel()] = U.gid.ravel()
    T3 = _kron3(U.T1, U.T1, U.T1)
    stars, pats = H.stars(), H.patterns()
    cls, nint, per = H.classes()
    assert len(cls) == len(stars) and cls.max() + 1 == len(per)
    for k in range(len(stars)):
        first = per[cls[k]][0]
        assert nint[k] == nint[first]
        assert all(np.array_equal(a, b) for a, b in zip(pats[k], pats[first]))
    for first, nnzl, (rp, cols), parent in per:
        v, nodes = stars[first]
        pos = {int(g): i for i, g in enumerate(nodes)}
        ns, ni = len(nodes), int(nint[first])
        Tv = np.zeros((ns, ns))
        for e in U.vertex_cells[v]:
            rows = np.array([pos.get(int(g), -1) for g in cn[e]])
            inside = rows >= 0
            for c in range(n ** 3):
                col = pos.get(int(cf[e, c]))
                if col is not None:
                    Tv[rows[inside], col] = cs[e, c] * T3[inside, c]
        Af = Tv.T @ U.As[pi[nodes]][:, pi[nodes]].toarray() @ Tv
        S = Af[ni:, ni:] - Af[ni:, :ni] @ (Af[:ni, ni:] / np.diag(Af)[:ni, None])
        nG = ns - ni
        if nG == 0:
            assert nnzl == 0
            continue
        Lp = np.zeros((nG, nG), dtype=bool)
        for r in range(nG):
            Lp[r, cols[rp[r]:rp[r + 1]]] = True
        assert Lp.sum() == nnzl
        assert np.array_equal(oracle_lib.symbolic_fill(np.abs(S) > 1e-12 * np.abs(S).max()), Lp)
        L = np.linalg.cholesky(S)
        assert not np.any((np.abs(L) > 1e-12 * np.abs(L).max()) & ~Lp)
        for j in range(nG):
            below = np.flatnonzero(Lp[j + 1:, j])
            assert parent[j] == (j + 1 + below[0] if len(below) else -1)


def test_canonical_star_classes(fdmpc):
    """Stars are ordered canonically (a walk over their cells from the
    smallest encoding), so equal configurations share a class whatever the
    cells' orientation: a tensor mesh has 4 classes (interior, face, edge and
    corner stars; the three face and edge kinds are the same up to axis
    labels) in lexicographic and in random orientation, with the same fill;
    the unstructured mesh has far fewer classes than stars."""
    X, cells = inputs.tensor_hex_mesh(*inputs.graded_vertices(4, 4))
    for p in (3, 4):
        ref = None
        for c in (cells, inputs.reorient_cells(cells, 3)):
            cls, nint, per = fdmpc.HexMesh(X.shape[0], c, p).classes()
            assert len(per) == 4
            got = sorted((int(nint[f]), int(nnzl)) for f, nnzl, _, _ in per)
            assert got[-1][0] == 8 * (p - 1) ** 3  # the interior star's 8 cell interiors
            assert ref is None or got == ref
            ref = got
    Xu, cu = inputs.unstructured_hex_mesh(3, 3, 7)
    cls, nint, per = fdmpc.HexMesh(Xu.shape[0], cu, 3).classes()
    assert len(per) <= 20 and len(cls) > 250


def _star_fdm_matrix(U, H, k, pi):
    """The oracle's surrogate star matrix of star k in the basis of the
    library's signed FDM map, and the star's GLL-basis nodes (oracle order)."""
    p, n = U.p, U.n
    cn = H.cell_nodes()
    cf, cs = H.cell_fdm()
    T3 = _kron3(U.T1, U.T1, U.T1)
    v, nodes = H.stars()[k]
    pos = {int(g): i for i, g in enumerate(nodes)}
    ns = len(nodes)
    Tv = np.zeros((ns, ns))
    for e in U.vertex_cells[v]:
        rows = np.array([pos.get(int(g), -1) for g in cn[e]])
        inside = rows >= 0
        for c in range(n ** 3):
            col = pos.get(int(cf[e, c]))
            if col is not None:
                Tv[rows[inside], col] = cs[e, c] * T3[inside, c]
    dofs = pi[nodes]
    return Tv, Tv.T @ U.As[dofs][:, dofs].toarray() @ Tv, v, dofs


@pytest.mark.parametrize("p", [2, 3])
def test_numeric_factorisation(fdmpc, p):
    """fdm_hexmesh_factor: the surrogate coefficients equal the oracle's, the
    interior pivots and L L^T equal the oracle's star matrix and its interface
    Schur complement, and the star solve from D and L (in the FDM basis) is
    the oracle's star solve; with a coefficient kappa at the Gauss points too."""
    X, cells = inputs.unstructured_hex_mesh(2, 2, 5)
    rng = np.random.default_rng(p)
    for kappa in (None, np.exp(rng.uniform(-1, 1, size=(cells.shape[0], (p + 1) ** 3)))):
        H = fdmpc.HexMesh(X.shape[0], cells, p)
        U = HexProblem(p, X, cells, kappa=kappa)
        mu, fac = H.factor(X, kappa)
        assert np.allclose(mu, U.mu, rtol=1e-13, atol=0)
        cn = H.cell_nodes()
        pi = np.zeros(H.nnode, dtype=np.int64)
        pi[cn.ravel()] = U.gid.ravel()
        cls, nint, per = H.classes()
        for k in range(0, len(cls), 7):
            Tv, Af, v, dofs = _star_fdm_matrix(U, H, k, pi)
            ni = int(nint[k])
            D, Lv = fac[k]
            assert np.allclose(D, np.diag(Af)[:ni], rtol=1e-13, atol=0)
            nG = len(dofs) - ni
            rp, fcols = per[cls[k]][2]
            L = np.zeros((nG, nG))
            for r in range(nG):
                L[r, fcols[rp[r]:rp[r + 1]]] = Lv[rp[r]:rp[r + 1]]
            S = Af[ni:, ni:] - Af[ni:, :ni] @ (Af[:ni, ni:] / D[:, None])
            if nG:
                assert np.abs(L @ L.T - S).max() <= 1e-12 * np.abs(S).max()
            # the star solve: y = A_v^{-1} g in the FDM basis by block elimination
            r = rng.standard_normal(U.ndof)
            g = Tv.T @ r[dofs]
            gI, gG = g[:ni], g[ni:]
            xG = np.linalg.solve(L.T, np.linalg.solve(L, gG - Af[ni:, :ni] @ (gI / D))) if nG else gG
            xI = (gI - Af[:ni, ni:] @ xG) / D
            want = U.patch_solve(v, r)[1]
            got = Tv @ np.concatenate([xI, xG])
            order = np.argsort(dofs)
            assert np.abs(got[order] - want).max() <= 1e-11 * np.abs(want).max()


def test_factor_rejects_bad_geometry(fdmpc):
    X, cells = inputs.tensor_hex_mesh(*inputs.uniform_vertices(2))
    H = fdmpc.HexMesh(X.shape[0], cells, 2)
    with pytest.raises(fdmpc.FdmError):
        H.factor(X[:-1])
    flat = X.copy()
    flat[:, 2] = 0.0
    with pytest.raises(fdmpc.FdmError, match="degenerate"):
        H.factor(flat)


def test_factor_reports_not_spd(fdmpc):
    """A negative coefficient makes the surrogate's pivots negative: the set-up
    returns FDM_ENOTSPD (a status code, nothing aborts)."""
    X, cells = inputs.unstructured_hex_mesh(2, 2, 5)
    H = fdmpc.HexMesh(X.shape[0], cells, 2)
    with pytest.raises(fdmpc.FdmError) as err:
        H.factor(X, -np.ones((cells.shape[0], 27)))
    assert err.value.code == fdmpc.FDM_ENOTSPD and "pivot" in str(err.value)
    mu, fac = H.factor(X)  # the same object sets up again afterwards
    assert np.all(mu > 0) and len(fac) == len(H.stars())


def _emulated_asm(H, r, basis, mu, fac):
    """One additive Schwarz sweep (undamped) computed from the library's
    tables and factors only, in the steps a GPU apply takes: cell-local FDM
    residuals E_e = (T^T)^{x3} (W r)_e (W = 1/multiplicity), their assembly per
    FDM slot through FDM_HQ_SLOT_CELLS with the map's signs, per star the
    block elimination with D, A_GI (from mu and the 1D A_f, B_f) and L, the
    sum of the star solutions per slot through FDM_HQ_SLOT_STARS, and the basis
    change back T^{x3} per cell with the node taken from its owner cell.
    Returns (z in library node order, largest mismatch of a node's value
    between the cells that hold it)."""
    p, n = H.p, H.n
    n3 = n ** 3
    T3 = _kron3(basis["T"], basis["T"], basis["T"])
    Af, Bf = basis["Af"], basis["Bf"]
    cn = H.cell_nodes()
    cf, cs = H.cell_fdm()
    scp, sc, ssp, ss, owner = H.inverse_maps()
    cls, nint, per = H.classes()
    dirichlet = H.dirichlet()
    mult = np.bincount(cn.ravel(), minlength=H.nnode)
    rW = np.where(dirichlet, 0.0, r) / mult
    E = rW[cn] @ T3                                   # [cell, c]
    rf = np.zeros(H.nnode)
    for g in range(H.nnode):
        for t in range(scp[g], scp[g + 1]):
            e, c = divmod(int(sc[t]), n3)
            rf[g] += cs[e, c] * E[e, c]

    def coupling(e, c1, c2):
        a = (c1 % n, (c1 // n) % n, c1 // (n * n))
        b = (c2 % n, (c2 // n) % n, c2 // (n * n))
        val = 0.0
        for d in range(3):
            t = mu[e, d] * Af[a[d], b[d]]
            for o in range(3):
                if o != d:
                    t *= Bf[a[o], b[o]]
            val += t
        return cs[e, c1] * cs[e, c2] * val

    xs = []
    for k, (v, nodes) in enumerate(H.stars()):
        ni = int(nint[k])
        nG = len(nodes) - ni
        pos = {int(g): i for i, g in enumerate(nodes)}
        D, Lv = fac[k]
        AGI = np.zeros((nG, ni))
        for i in range(ni):
            e, ci = divmod(int(sc[scp[nodes[i]]]), n3)  # an interior slot has one cell
            for c in range(n3):
                j = pos.get(int(cf[e, c]), -1)
                if j >= ni:
                    AGI[j - ni, i] = coupling(e, c, ci)
        rp, fcols = per[cls[k]][2]
        L = np.zeros((nG, nG))
        for rr in range(nG):
            L[rr, fcols[rp[rr]:rp[rr + 1]]] = Lv[rp[rr]:rp[rr + 1]]
        g = rf[nodes]
        gI, gG = g[:ni], g[ni:]
        xG = np.linalg.solve(L.T, np.linalg.solve(L, gG - AGI @ (gI / D))) if nG else gG
        xI = (gI - AGI.T @ xG) / D
        xs.append(np.concatenate([xI, xG]))
    zf = np.zeros(H.nnode)
    for g in range(H.nnode):
        for t in range(ssp[g], ssp[g + 1]):
            zf[g] += xs[ss[t, 0]][ss[t, 1]]
    Z = (cs * zf[cf]) @ T3.T                          # [cell, local node]
    z = Z.ravel()[owner]
    z[dirichlet] = 0.0
    return z, np.abs(Z - z[cn]).max()


@pytest.mark.parametrize("p", [1, 2, 3])
def test_emulated_gpu_sweep_is_the_oracle_asm(fdmpc, p):
    """The relaxation assembled from the library's tables and factors (the
    blueprint of the GPU apply for general meshes) equals the oracle's
    additive Schwarz sweep, and the glued FDM functions give every node one
    value from all its cells."""
    import oracle
    X, cells = inputs.unstructured_hex_mesh(2, 2, 5)
    H = fdmpc.HexMesh(X.shape[0], cells, p)
    U = HexProblem(p, X, cells)
    cn = H.cell_nodes()
    pi = np.zeros(H.nnode, dtype=np.int64)
    pi[cn.ravel()] = U.gid.ravel()
    r = np.random.default_rng(p).standard_normal(U.ndof)
    mu, fac = H.factor(X)
    z, mismatch = _emulated_asm(H, r[pi], oracle.basis1d(p), mu, fac)
    want = U.asm(r)[pi]
    assert np.abs(z - want).max() <= 1e-11 * np.abs(want).max()
    assert mismatch <= 1e-11 * np.abs(want).max()


def _emulated_operator(H, u, geom, ptr, nodec, p):
    """y = A u from the library's geometry factors and node-to-cell map: per
    cell sum_{d,f} D_d^T (G_df o D_f u_e) (D_d: the GLL Lagrange basis
    differentiated along axis d at the Gauss points), summed per node in the
    map's order; 0 on Dirichlet nodes."""
    import oracle
    n = p + 1
    xi = oracle.basis1d(p)["xi"]
    xq, _ = oracle.gauss(n)
    V, Dq = oracle.lagrange(p, xi, xq)
    Dm = [_kron3(V, V, Dq), _kron3(V, Dq, V), _kron3(Dq, V, V)]
    cn = H.cell_nodes()
    dirichlet = H.dirichlet()
    ue = np.where(dirichlet, 0.0, u)[cn]                       # [cell, node]
    grads = [ue @ D.T for D in Dm]                           # [cell, q]
    comp = {(0, 0): 0, (1, 1): 1, (2, 2): 2, (0, 1): 3, (1, 0): 3, (0, 2): 4, (2, 0): 4, (1, 2): 5, (2, 1): 5}
    ye = np.zeros_like(ue)
    for d in range(3):
        flux = sum(geom[:, :, comp[d, f]] * grads[f] for f in range(3))
        ye += flux @ Dm[d]
    flat = ye.ravel()
    y = np.array([flat[nodec[ptr[g]:ptr[g + 1]]].sum() for g in range(H.nnode)])
    y[dirichlet] = 0.0
    return y


@pytest.mark.parametrize("p", [1, 2, 3])
def test_emulated_operator_and_vcycle(fdmpc, p):
    """The stiffness apply from the library's geometry factors and the hybrid
    V(1,1) from the library's tables, factors and Q1 operator (the steps of
    the GPU apply) equal the oracle's, on the unstructured mesh with a
    coefficient at the Gauss points."""
    import oracle
    X, cells = inputs.unstructured_hex_mesh(2, 2, 5)
    kappa = np.exp(np.random.default_rng(p).uniform(-0.5, 0.5, size=(cells.shape[0], (p + 1) ** 3)))
    H = fdmpc.HexMesh(X.shape[0], cells, p)
    U = HexProblem(p, X, cells, kappa=kappa)
    mu, fac = H.factor(X, kappa)
    ptr, nodec, geom, cof, Ac = H.operator_tables()
    cn = H.cell_nodes()
    pi = np.zeros(H.nnode, dtype=np.int64)
    pi[cn.ravel()] = U.gid.ravel()
    rng = np.random.default_rng(10 + p)
    u = rng.standard_normal(U.ndof)
    y = _emulated_operator(H, u[pi], geom, ptr, nodec, p)
    want = U.apply(u)[pi]
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()
    # coarse space: P from the vertices' Q1 functions at each cell's GLL nodes
    U.setup_coarse()
    xi = oracle.basis1d(p)["xi"]
    hat = np.stack([0.5 * (1 - xi), 0.5 * (1 + xi)], axis=1)
    P = np.zeros((H.nnode, Ac.shape[0]))
    for e in range(cells.shape[0]):
        for c in range(8):
            k = cof[cells[e, c]]
            if k >= 0:
                P[cn[e], k] = _kron3(hat[:, c >> 2], hat[:, (c >> 1) & 1], hat[:, c & 1])
    P[H.dirichlet()] = 0.0
    assert np.abs(Ac - U.Ac).max() <= 1e-12 * np.abs(U.Ac).max()
    # V(1,1) with the oracle's omega
    U.setup_patches()
    lo, hi, om = U.lanczos_omega(inputs.lanczos_start(U.ndof))
    basis = oracle.basis1d(p)
    A = lambda x: _emulated_operator(H, x, geom, ptr, nodec, p)  # noqa: E731
    S = lambda x: _emulated_asm(H, x, basis, mu, fac)[0]  # noqa: E731
    r = rng.standard_normal(U.ndof)[pi]
    r[H.dirichlet()] = 0.0
    x1 = om * S(r)
    x1 = x1 + P @ np.linalg.solve(Ac, P.T @ (r - A(x1)))
    z = x1 + om * S(r - A(x1))
    want = U.pc_apply(r[np.argsort(pi)])[pi]
    assert np.abs(z - want).max() <= 1e-11 * np.abs(want).max()


@pytest.mark.parametrize("p", [2, 3, 4])
def test_schur_coupling_form(fdmpc, p):
    """The Schur-coupling form of every star's interface solve (y_B = S_BB^{-1}
    g_B, x_T = W (g_T - S_TB y_B), x_B = y_B - S_BB^{-1} S_BT x_T, from the
    library's L_BB, S_TB and W) solves the oracle's interface Schur
    complement, and it stores fewer values than the L form on the large stars."""
    X, cells = inputs.unstructured_hex_mesh(2, 2, 5)
    H = fdmpc.HexMesh(X.shape[0], cells, p)
    U = HexProblem(p, X, cells)
    mu, fac = H.factor(X)
    per_sc, vals = H.schur_coupling()
    cls, nint, per = H.classes()
    cn = H.cell_nodes()
    pi = np.zeros(H.nnode, dtype=np.int64)
    pi[cn.ravel()] = U.gid.ravel()
    rng = np.random.default_rng(p)
    for k in range(len(cls)):
        t, (rb, cb), (rt, ct) = per_sc[cls[k]]
        Tv, Af, v, dofs = _star_fdm_matrix(U, H, k, pi)
        ni = int(nint[k])
        nG = len(dofs) - ni
        nB = nG - t
        if nG == 0:
            assert t == 0 and len(vals[k]) == 0
            continue
        D = np.diag(Af)[:ni]
        S = Af[ni:, ni:] - Af[ni:, :ni] @ (Af[:ni, ni:] / D[:, None])
        val = vals[k]
        LB = np.zeros((nB, nB))
        for r in range(nB):
            LB[r, cb[rb[r]:rb[r + 1]]] = val[rb[r]:rb[r + 1]]
        o = rb[-1]
        STB = np.zeros((t, nB))
        for r in range(t):
            STB[r, ct[rt[r]:rt[r + 1]]] = val[o + rt[r]:o + rt[r + 1]]
        o += rt[-1]
        W = np.zeros((t, t))
        W[np.tril_indices(t)] = val[o:]
        W = W + np.tril(W, -1).T
        assert len(val) == o + t * (t + 1) // 2
        g = rng.standard_normal(nG)
        solve_B = lambda y: np.linalg.solve(LB.T, np.linalg.solve(LB, y)) if nB else y  # noqa: E731
        yB = solve_B(g[:nB])
        xT = W @ (g[nB:] - STB @ yB)
        xB = yB - solve_B(STB.T @ xT)
        x = np.concatenate([xB, xT])
        want = np.linalg.solve(S, g)
        assert np.abs(x - want).max() <= 1e-10 * np.abs(want).max()
        if nG > 100:
            assert len(val) < per[cls[k]][1]
