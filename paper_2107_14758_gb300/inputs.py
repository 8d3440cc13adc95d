"""Seeded synthetic workloads (mesh geometry, coefficients, right-hand sides).

This module holds no arithmetic of the method: it only draws random numbers
and evaluates the synthetic geometry and coefficient fields at given points.
Both the oracle-based tests and the CUDA path read the arrays it returns.

Workload families (stand-ins for the paper's Cartesian Poisson runs, Section
2.8, and for the separable / deformed / batched variants):

* uniform:   unit cube, n^3 equal cells.
* graded:    unit cube, per-axis cell widths drawn U(0.5, 1.5) (x, then y,
             then z, one generator), normalised to sum 1.
* deformed:  uniform n^3 mesh mapped by Phi(x) = x + 0.1 g(x) (1,1,1) with
             g = sin(2 pi x) sin(2 pi y) sin(2 pi z); curved cells are given by
             their Jacobian at the (p+1)^3 Gauss-Legendre points.
* kappa:     kappa = exp(G), G = sqrt(2/M) sum_m cos(2 pi k_m . x + phi_m),
             M = 8 modes, k_m uniform in {1..8}^3, phi_m ~ U(0, 2 pi)
             (unit variance in the mode average).
* rhs:       i.i.d. N(0,1) nodal values, or the manufactured
             f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) sampled at the GLL nodes.
* unstructured hexahedra: a 2D quad mesh of the unit square with vertices of
             valence 3, 4, 6 and 8 (an m x m grid of squares cut into two
             triangles along a random diagonal, each triangle cut into three
             quads through its centroid and edge midpoints, interior grid
             points jittered), extruded through graded layers in z; every
             cell's reference axes reoriented by a random symmetry of the
             cube.  A stand-in for the paper's unstructured meshes (2D base
             meshes extruded with six layers), which are not available.
* Kershaw-type: the tensor mesh with its y and z grid lines squeezed towards
             alternating sides in slabs along x (aspect ratios ~0.3 near the
             corners): an own stand-in for the paper's Kershaw meshes, whose
             coordinate field is not given.
"""
import numpy as np
from numpy.polynomial import legendre as _leg


def uniform_vertices(n):
    v = np.linspace(0.0, 1.0, n + 1)
    return v.copy(), v.copy(), v.copy()


def graded_vertices(n, seed):
    """Per-axis widths ~ U(0.5, 1.5), normalised; drawn x, y, z in order."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(3):
        w = rng.uniform(0.5, 1.5, size=n)
        w = w / w.sum()
        v = np.concatenate([[0.0], np.cumsum(w)])
        v[-1] = 1.0
        out.append(v)
    return tuple(out)


def gll_points(p):
    """GLL nodes on [-1, 1] from numpy's Legendre module (geometry only)."""
    if p == 1:
        return np.array([-1.0, 1.0])
    inner = np.sort(_leg.Legendre.basis(p).deriv().roots().real)
    return np.concatenate([[-1.0], inner, [1.0]])


def body_force_load(xv, yv, zv, p, f):
    """Load vector [3][ndof] (component-major, x fastest) of a constant body
    force f: b_a(node) = f_a int phi_node, the integral of the GLL Lagrange
    function being (GLL weight) x (half-width) per cell and axis, summed over
    the cells holding the node; the solver ignores the clamped entries."""
    xi = gll_points(p)
    w = 2.0 / (p * (p + 1) * _leg.Legendre.basis(p)(xi) ** 2)
    ints = []
    for v in (xv, yv, zv):
        v = np.asarray(v, dtype=np.float64)
        m = np.zeros((len(v) - 1) * p + 1)
        for c in range(len(v) - 1):
            m[c * p:(c + 1) * p + 1] += 0.5 * (v[c + 1] - v[c]) * w
        ints.append(m)
    mass = np.einsum("k,j,i->kji", ints[2], ints[1], ints[0]).ravel()
    return np.outer(np.asarray(f, dtype=np.float64), mass)


def node_coords(v, p):
    """Physical coordinates of the GLL nodes along one axis."""
    xi = gll_points(p)
    n = len(v) - 1
    x = np.empty(n * p + 1)
    for c in range(n):
        x[c * p:(c + 1) * p + 1] = v[c] + 0.5 * (1.0 + xi) * (v[c + 1] - v[c])
    return x


def manufactured_f(xv, yv, zv, p):
    """f = 3 pi^2 prod sin(pi x_i) at the GLL grid (x fastest)."""
    x, y, z = node_coords(xv, p), node_coords(yv, p), node_coords(zv, p)
    fz, fy, fx = np.meshgrid(np.sin(np.pi * z), np.sin(np.pi * y), np.sin(np.pi * x), indexing="ij")
    return (3.0 * np.pi ** 2 * fz * fy * fx).ravel()


def manufactured_u(xv, yv, zv, p):
    x, y, z = node_coords(xv, p), node_coords(yv, p), node_coords(zv, p)
    fz, fy, fx = np.meshgrid(np.sin(np.pi * z), np.sin(np.pi * y), np.sin(np.pi * x), indexing="ij")
    return (fz * fy * fx).ravel()


def normal_rhs(ndof, seed):
    return np.random.default_rng(seed).standard_normal(ndof)


def _deform(x, y, z, amp=0.1):
    g = np.sin(2 * np.pi * x) * np.sin(2 * np.pi * y) * np.sin(2 * np.pi * z)
    return x + amp * g, y + amp * g, z + amp * g


def _deform_grad(x, y, z, amp=0.1):
    s = np.sin
    c = np.cos
    tp = 2 * np.pi
    gx = tp * c(tp * x) * s(tp * y) * s(tp * z)
    gy = tp * s(tp * x) * c(tp * y) * s(tp * z)
    gz = tp * s(tp * x) * s(tp * y) * c(tp * z)
    return amp * gx, amp * gy, amp * gz


def deformed_jacobians(n, p, amp=0.1, vertices=None):
    """J = dPhi/dx * diag(h/2) at the (p+1)^3 Gauss points of each cell.

    Returns (jac, pts): jac[cell, q, 9] row-major dx_r/dxhat_c, pts[cell, q, 3]
    the physical coordinates of the points (for coefficient evaluation).
    Cells and points are numbered x fastest.
    """
    xv, yv, zv = vertices if vertices is not None else uniform_vertices(n)
    nx, ny, nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
    q = p + 1
    xg, _ = _leg.leggauss(q)
    jac = np.zeros((nx * ny * nz, q ** 3, 9))
    pts = np.zeros((nx * ny * nz, q ** 3, 3))
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                e = cx + nx * (cy + ny * cz)
                h = np.array([xv[cx + 1] - xv[cx], yv[cy + 1] - yv[cy], zv[cz + 1] - zv[cz]])
                X = xv[cx] + 0.5 * (1 + xg) * h[0]
                Y = yv[cy] + 0.5 * (1 + xg) * h[1]
                Z = zv[cz] + 0.5 * (1 + xg) * h[2]
                ZZ, YY, XX = np.meshgrid(Z, Y, X, indexing="ij")
                XX, YY, ZZ = XX.ravel(), YY.ravel(), ZZ.ravel()
                dgx, dgy, dgz = _deform_grad(XX, YY, ZZ, amp)
                J = np.zeros((len(XX), 3, 3))
                for r in range(3):
                    J[:, r, 0] = ((r == 0) + dgx) * 0.5 * h[0]
                    J[:, r, 1] = ((r == 1) + dgy) * 0.5 * h[1]
                    J[:, r, 2] = ((r == 2) + dgz) * 0.5 * h[2]
                jac[e] = J.reshape(-1, 9)
                px, py, pz = _deform(XX, YY, ZZ, amp)
                pts[e, :, 0], pts[e, :, 1], pts[e, :, 2] = px, py, pz
    return jac, pts


def deformed_samples27(n, seed, amp=0.1, vertices=None):
    """kappa and the Jacobian at the 3 x 3 x 3 Gauss points of every cell of the
    deformed mesh (x fastest; cells x fastest): [cell, 27, 10] = (kappa, J
    row-major).  The same map and field as deformed_jacobians / kappa_field."""
    xv, yv, zv = vertices if vertices is not None else uniform_vertices(n)
    nx, ny, nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
    xg, _ = _leg.leggauss(3)
    out = np.zeros((nx * ny * nz, 27, 10))
    allpts = np.zeros((nx * ny * nz, 27, 3))
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                e = cx + nx * (cy + ny * cz)
                h = np.array([xv[cx + 1] - xv[cx], yv[cy + 1] - yv[cy], zv[cz + 1] - zv[cz]])
                X = xv[cx] + 0.5 * (1 + xg) * h[0]
                Y = yv[cy] + 0.5 * (1 + xg) * h[1]
                Z = zv[cz] + 0.5 * (1 + xg) * h[2]
                ZZ, YY, XX = np.meshgrid(Z, Y, X, indexing="ij")
                XX, YY, ZZ = XX.ravel(), YY.ravel(), ZZ.ravel()
                dgx, dgy, dgz = _deform_grad(XX, YY, ZZ, amp)
                for r in range(3):
                    out[e, :, 1 + 3 * r + 0] = ((r == 0) + dgx) * 0.5 * h[0]
                    out[e, :, 1 + 3 * r + 1] = ((r == 1) + dgy) * 0.5 * h[1]
                    out[e, :, 1 + 3 * r + 2] = ((r == 2) + dgz) * 0.5 * h[2]
                px, py, pz = _deform(XX, YY, ZZ, amp)
                allpts[e, :, 0], allpts[e, :, 1], allpts[e, :, 2] = px, py, pz
    out[:, :, 0] = kappa_field(allpts, seed)
    return out


def kappa_field(pts, seed, modes=8, kmax=8):
    """kappa = exp(G) with G a random Fourier sum of unit variance."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, kmax + 1, size=(modes, 3))
    phi = rng.uniform(0.0, 2 * np.pi, size=modes)
    x = pts.reshape(-1, 3)
    G = np.sqrt(2.0 / modes) * np.cos(2 * np.pi * x @ k.T + phi).sum(axis=1)
    return np.exp(G).reshape(pts.shape[:-1])


def lanczos_start(ndof, seed=12345):
    return np.random.default_rng(seed).standard_normal(ndof)


# ---- the five workloads --------------------------------------------------

def workload(name, seed=None):
    """Returns a dict: p, xv, yv, zv, jac (or None), kappa (or None), rhs kind."""
    if name == "q4_uniform4":       # 4^3 uniform, Q4, manufactured sine
        xv, yv, zv = uniform_vertices(4)
        return dict(name=name, p=4, xv=xv, yv=yv, zv=zv, jac=None, kappa=None, rhs="manufactured", seed=1)
    if name == "q7_graded16":       # 16^3 graded tensor mesh, Q7, N(0,1) nodal f
        xv, yv, zv = graded_vertices(16, 2 if seed is None else seed)
        return dict(name=name, p=7, xv=xv, yv=yv, zv=zv, jac=None, kappa=None, rhs="nodal_normal", seed=2)
    if name == "q7_graded32":       # 32^3 graded tensor mesh, Q7, N(0,1) nodal f (multigrid coarse solve)
        xv, yv, zv = graded_vertices(32, 6 if seed is None else seed)
        return dict(name=name, p=7, xv=xv, yv=yv, zv=zv, jac=None, kappa=None, rhs="nodal_normal", seed=6)
    if name == "q15_uniform8":      # 8^3 uniform, Q15, manufactured sine
        xv, yv, zv = uniform_vertices(8)
        return dict(name=name, p=15, xv=xv, yv=yv, zv=zv, jac=None, kappa=None, rhs="manufactured", seed=3)
    if name == "q8_deformed12":     # 12^3 deformed, Q8, kappa = exp(G)
        p = 8
        xv, yv, zv = uniform_vertices(12)
        jac, pts = deformed_jacobians(12, p)
        sd = 4 if seed is None else seed
        kap = kappa_field(pts, sd)
        return dict(name=name, p=p, xv=xv, yv=yv, zv=zv, jac=jac, kappa=kap, samples27=deformed_samples27(12, sd),
                    rhs="normal", seed=4)
    raise KeyError(name)


def deformed_problem(n, p, seed, amp=0.1):
    """Deformed uniform n^3 mesh with kappa = exp(G) (seeded), as q8_deformed12:
    jac and kappa at the (p+1)^3 Gauss points and the 27-point samples."""
    xv, yv, zv = uniform_vertices(n)
    jac, pts = deformed_jacobians(n, p, amp)
    return dict(name="deformed%d_q%d_s%d" % (n, p, seed), p=p, xv=xv, yv=yv, zv=zv, jac=jac,
                kappa=kappa_field(pts, seed), samples27=deformed_samples27(n, seed, amp), rhs="normal", seed=seed)


def mlp_init(seed, nin=189, nh=64, nout=3):
    """Initial network weights (float32, packed W1, b1, W2, b2, W3, b3):
    W ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)), the output layer scaled by 0.1,
    biases 0."""
    rng = np.random.default_rng(seed)
    parts = []
    for fo, fi, scale in ((nh, nin, 1.0), (nh, nh, 1.0), (nout, nh, 0.1)):
        parts.append(rng.uniform(-1.0, 1.0, fo * fi) * scale / np.sqrt(fi))
        parts.append(np.zeros(fo))
    return np.concatenate(parts).astype(np.float32)


def batch_problems(count=64, seed0=1000):
    """Independent graded problems: n ~ U{2..10}, p ~ U{3..15}, N(0,1) rhs."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        n = int(rng.integers(2, 11))
        p = int(rng.integers(3, 16))
        xv, yv, zv = graded_vertices(n, seed0 + i)
        out.append(dict(name="batch%d" % i, p=p, xv=xv, yv=yv, zv=zv, jac=None, kappa=None,
                        rhs="normal", seed=seed0 + i))
    return out


def rhs_for(w, ndof):
    """Right-hand side data: ('nodal', f) to be multiplied by the mass matrix,
    or ('load', b) used as the load vector directly."""
    if w["rhs"] == "manufactured":
        return "nodal", manufactured_f(w["xv"], w["yv"], w["zv"], w["p"])
    if w["rhs"] == "nodal_normal":
        return "nodal", normal_rhs(ndof, w["seed"])
    return "load", normal_rhs(ndof, w["seed"])


# ---- general hexahedral meshes (vertex coordinates + cell-to-vertex lists) ----
#
# A cell lists its 8 vertices in the order of the reference cube's corners
# (a, b, c) in {0, 1}^3 at index a + 2 b + 4 c (reference coordinate -1 -> 0,
# +1 -> 1); the geometry is the trilinear map through them.

def tensor_hex_mesh(xv, yv, zv):
    """The tensor mesh of the vertex vectors as vertices X[nv, 3] (x fastest)
    and cells[nc, 8] (cells x fastest, reference axes along x, y, z)."""
    xv, yv, zv = (np.asarray(a, dtype=np.float64) for a in (xv, yv, zv))
    nx, ny, nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
    Z, Y, X = np.meshgrid(zv, yv, xv, indexing="ij")
    verts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    cells = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                cells.append([(i + a) + (nx + 1) * ((j + b) + (ny + 1) * (k + c))
                              for c in (0, 1) for b in (0, 1) for a in (0, 1)])
    return verts, np.array(cells, dtype=np.int64)


def reorient_cells(cells, seed):
    """Lists every cell's vertices in the frame of a random symmetry of the
    reference cube (one of the 48 axis permutations with reflections), so that
    neighbouring cells see their shared faces and edges in different
    orientations.  The cells themselves are unchanged."""
    rng = np.random.default_rng(seed)
    cells = np.asarray(cells, dtype=np.int64)
    out = np.empty_like(cells)
    for e in range(cells.shape[0]):
        perm = rng.permutation(3)
        flip = rng.integers(0, 2, size=3)
        for a in (0, 1):
            for b in (0, 1):
                for c in (0, 1):
                    r = (a, b, c)
                    old = [0, 0, 0]
                    for d in range(3):
                        old[perm[d]] = 1 - r[d] if flip[d] else r[d]
                    out[e, a + 2 * b + 4 * c] = cells[e, old[0] + 2 * old[1] + 4 * old[2]]
    return out


def unstructured_quad_mesh(m, seed, jitter=0.2):
    """2D quad mesh of the unit square: returns vertices V[nv, 2] and quads
    [nq, 4] listed counter-clockwise.  An m x m grid of squares, each cut into
    two triangles along a diagonal drawn at random, each triangle cut into
    three quads (corner, edge midpoint, centroid, edge midpoint).  Interior
    grid points move by up to jitter * h per coordinate (h = 1/m) before the
    midpoints and centroids are placed, which keeps every quad convex.
    Valences: centroids 3, edge midpoints 4 (2 on the boundary), grid points
    the number of triangles around them (4, 6 or 8 inside)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / m
    g = np.array([[i * h, j * h] for j in range(m + 1) for i in range(m + 1)])
    for j in range(1, m):
        for i in range(1, m):
            g[i + (m + 1) * j] += rng.uniform(-jitter * h, jitter * h, size=2)
    verts = [tuple(v) for v in g]
    mid = {}

    def midpoint(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            mid[key] = len(verts)
            verts.append(tuple(0.5 * (g[a] + g[b])))
        return mid[key]

    quads = []
    for j in range(m):
        for i in range(m):
            c00, c10 = i + (m + 1) * j, i + 1 + (m + 1) * j
            c01, c11 = i + (m + 1) * (j + 1), i + 1 + (m + 1) * (j + 1)
            if rng.integers(0, 2):
                tris = [(c00, c10, c11), (c00, c11, c01)]
            else:
                tris = [(c00, c10, c01), (c10, c11, c01)]
            for (a, b, c) in tris:  # counter-clockwise
                cen = len(verts)
                verts.append(tuple((g[a] + g[b] + g[c]) / 3.0))
                mab, mbc, mca = midpoint(a, b), midpoint(b, c), midpoint(c, a)
                quads += [[a, mab, cen, mca], [b, mbc, cen, mab], [c, mca, cen, mbc]]
    return np.array(verts), np.array(quads, dtype=np.int64)


def extruded_hex_mesh(V2, quads, zv):
    """Extrudes a counter-clockwise 2D quad mesh through the layers of zv:
    vertices X[nv2 * len(zv), 3] (layer-major) and cells[nq * (len(zv)-1), 8]
    with reference axes (quad edge a->b, quad edge a->d, z)."""
    V2 = np.asarray(V2, dtype=np.float64)
    zv = np.asarray(zv, dtype=np.float64)
    nv2 = V2.shape[0]
    X = np.concatenate([np.column_stack([V2, np.full(nv2, z)]) for z in zv])
    cells = []
    for layer in range(len(zv) - 1):
        for (a, b, c, d) in quads:
            lo = [a, b, d, c]
            cells.append([v + nv2 * layer for v in lo] + [v + nv2 * (layer + 1) for v in lo])
    return X, np.array(cells, dtype=np.int64)


def unstructured_hex_mesh(m, nz, seed, jitter=0.2):
    """The unstructured workload mesh: unstructured_quad_mesh(m) extruded
    through nz graded layers (widths U(0.5, 1.5), normalised), cells
    reoriented at random.  Returns X, cells."""
    V2, quads = unstructured_quad_mesh(m, seed, jitter)
    rng = np.random.default_rng(seed + 1)
    w = rng.uniform(0.5, 1.5, size=nz)
    zv = np.concatenate([[0.0], np.cumsum(w / w.sum())])
    zv[-1] = 1.0
    X, cells = extruded_hex_mesh(V2, quads, zv)
    return X, reorient_cells(cells, seed + 2)


def kershaw_like_mesh(n, eps=0.3):
    """A structured but strongly distorted hexahedral mesh of the unit cube in
    the spirit of the paper's Kershaw meshes (Section 3): n^3 cells (n a
    multiple of 2), the grid lines in y and z squeezed towards one side or the
    other of the cube in alternating slabs along x, so that cells near the
    corners have aspect ratios of about eps, with a linear blend between
    neighbouring slabs (the vertices move, the topology stays that of the
    tensor mesh).  Own construction: the paper's coordinate field is not
    given.  Returns X, cells."""
    if n % 2:
        raise ValueError("n must be even")

    def squeeze(t, left):
        # piecewise-linear map of [0, 1] onto itself sending 1/2 to eps/(1+eps)
        # (left) or 1/(1+eps) (right): the cells of one half shrink by eps
        m = eps / (1.0 + eps) if left else 1.0 / (1.0 + eps)
        return np.where(t <= 0.5, 2.0 * t * m, m + (2.0 * t - 1.0) * (1.0 - m))

    u = np.linspace(0.0, 1.0, n + 1)
    X3 = np.zeros((n + 1, n + 1, n + 1, 3))
    for i, x in enumerate(u):
        # slab index along x: 3 slabs with alternating squeeze, blended
        s = min(2.999999, 3.0 * x)
        k = int(s)
        w = s - k
        side = (k % 2 == 0)
        for j, y in enumerate(u):
            for l, z in enumerate(u):
                y0, z0 = squeeze(y, side), squeeze(z, not side)
                y1, z1 = squeeze(y, not side), squeeze(z, side)
                blend = 0.5 - 0.5 * np.cos(np.pi * w)
                X3[l, j, i] = (x, (1 - blend) * y0 + blend * y1 if k < 2 else y0,
                               (1 - blend) * z0 + blend * z1 if k < 2 else z0)
    X = X3.reshape(-1, 3)
    cells = []
    for k in range(n):
        for j in range(n):
            for i in range(n):
                cells.append([(i + a) + (n + 1) * ((j + b) + (n + 1) * (k + c))
                              for c in (0, 1) for b in (0, 1) for a in (0, 1)])
    return X, np.array(cells, dtype=np.int64)
