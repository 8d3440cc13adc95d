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
