"""GPU parity of the CUDA path (through the C-ABI) against the FP64 oracle.

Tolerances: integer/index data (orderings, sparsity patterns) bit-exact;
FP64 path <= 1e-11 relative (max norm) per operator application and for the
PCG iterates at equal iteration counts; FP32 preconditioner: <= 1e-4 relative
per application (FP32 unit roundoff 6e-8 times the growth through the patch
Schur complements, whose condition numbers stay below about 1e2 at p <= 7) and
a final true residual ||b - A x|| <= 1e-8 ||b|| (PCG declares convergence on
the true residual); PCG iteration counts within +1 of the oracle.
"""
from tests.record import record
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2107_14758_gb300 import fdmpc, inputs  # noqa: E402

DEV = "cuda:0"
FP64, FP32 = fdmpc.FDM_PREC_FP64, fdmpc.FDM_PREC_FP32


def T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def N(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()


def pair(p, xv, yv, zv, jac=None, kappa=None, precision=FP64, pc=fdmpc.FDM_PC_VCYCLE, omega=0.0,
         patches=True, coarse=True):
    nd = (len(xv) - 1) * p + 1
    ndof = nd * ((len(yv) - 1) * p + 1) * ((len(zv) - 1) * p + 1)
    start = inputs.lanczos_start(ndof)
    ctx = fdmpc.Context(p, xv, yv, zv, jac=jac, kappa=kappa, precision=precision, pc=pc, omega=omega,
                        lanczos_start=start)
    ref = oracle.Problem(p, xv, yv, zv, jac=jac, kappa=kappa)
    if patches:
        ref.setup_patches()
    if coarse:
        ref.setup_coarse()
    ref.set_omega(ctx.omega)
    return ctx, ref, start


def free_random(ref, seed):
    from tests import bruteforce as bf
    m = bf.free_mask(ref.p, ref.nx, ref.ny, ref.nz)
    return np.where(m, np.random.default_rng(seed).standard_normal(ref.ndof), 0.0)


# ---------------------------------------------------------------- set-up data
@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 11, 15])
def test_basis_parity(p):
    xv = yv = zv = np.linspace(0, 1, 3)
    ctx = fdmpc.Context(p, xv, yv, zv, precision=FP64, omega=1.0)
    n = p + 1
    got = ctx.query(fdmpc.FDM_Q_BASIS, np.float64, 5 * n * n).reshape(5, n, n)
    ref = oracle.basis1d(p)
    for k, name in enumerate(("A", "B", "T", "Af", "Bf")):
        scale = max(np.abs(ref[name]).max(), 1.0)
        assert np.abs(got[k] - ref[name]).max() <= 1e-12 * scale, name


def _oracle_gamma_perm(ref, v, gpos):
    g, nI = ref.patch_dofs(v)
    N0 = ref.N[0]
    p = ref.p
    isG = np.array([not ((gi % N0) % p and ((gi // N0) % ref.N[1]) % p and (gi // (N0 * ref.N[1])) % p)
                    for gi in g])
    rank = np.cumsum(isG) - 1
    return rank[gpos]


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_patterns_bit_exact(p):
    xv, yv, zv = inputs.graded_vertices(4, 3)
    yv = yv[:4]; yv = yv / yv[-1]
    ctx = fdmpc.Context(p, xv, yv, zv, precision=FP64, omega=1.0)
    ref = oracle.Problem(p, xv, yv, zv)
    info = ctx.class_info()
    orders = ctx.gamma_orders()
    classes = ctx.query(fdmpc.FDM_Q_PATCH_CLASS, np.int32, ctx.npatch)
    seen = 0
    for cls in range(8):
        if info[cls, 2] == 0:
            continue
        v = int(np.flatnonzero(classes == cls)[0])
        perm = _oracle_gamma_perm(ref, v, orders[cls])
        assert sorted(perm) == list(range(len(perm)))            # a permutation of the interface
        S = ref.patch_schur(v)[np.ix_(perm, perm)]
        fill = oracle.symbolic_fill(S != 0)
        lib_pat = ctx.pattern(cls)
        assert np.array_equal(np.tril(fill), np.tril(lib_pat)), "class %d" % cls
        assert int(np.tril(fill).sum()) == int(info[cls, 7])
        seen += 1
    assert seen >= 4


@pytest.mark.parametrize("p", [2, 4, 5])
def test_factor_parity(p):
    xv, yv, zv = inputs.graded_vertices(3, 5)
    ctx = fdmpc.Context(p, xv, yv, zv, precision=FP64, omega=1.0)
    ref = oracle.Problem(p, xv, yv, zv)
    orders = ctx.gamma_orders()
    classes = ctx.query(fdmpc.FDM_Q_PATCH_CLASS, np.int32, ctx.npatch)
    for cls in (7, 6, 3, 1):
        vs = np.flatnonzero(classes == cls)
        if len(vs) == 0:
            continue
        v = int(vs[-1])
        perm = _oracle_gamma_perm(ref, v, orders[cls])
        S = ref.patch_schur(v)[np.ix_(perm, perm)]
        Lref = oracle.cholesky(S)
        L = ctx.factor_dense(v)
        assert relerr(L, Lref) <= 1e-11, cls


# ---------------------------------------------------------------- operators
def test_stiffness_and_mass_box():
    xv, yv, zv = inputs.graded_vertices(4, 8)
    zv = np.array([0.0, 0.2, 0.45, 0.8, 0.9, 1.0])
    ctx, ref, _ = pair(3, xv, yv, zv, patches=False, coarse=False, omega=1.0)
    u = np.random.default_rng(1).standard_normal(ref.ndof)
    assert relerr(N(ctx.stiffness_apply(T(u))), ref.stiffness_apply(u)) <= 1e-12
    assert relerr(N(ctx.mass_apply(T(u))), ref.mass_apply(u)) <= 1e-12


@pytest.mark.parametrize("p", list(range(1, 16)))
def test_stiffness_box_every_degree(p):
    """The FP64 box stiffness (the element-eigenbasis kernel, specialised on
    n = p + 1: odd n takes its middle-node terms, even n not) against the
    oracle's Kronecker apply at every degree, on a 3 x 2 x 2 graded mesh (12
    cells: a partly filled last CTA where several cells share one)."""
    xv = np.array([0.0, 0.3, 0.55, 1.0])
    yv = np.array([0.0, 0.6, 1.0])
    zv = np.array([0.0, 0.45, 1.0])
    ctx, ref, _ = pair(p, xv, yv, zv, patches=False, coarse=False, omega=1.0)
    for seed in (3, 4):  # two calls in a row
        u = np.random.default_rng(seed).standard_normal(ref.ndof)
        assert relerr(N(ctx.stiffness_apply(T(u))), ref.stiffness_apply(u)) <= 1e-12


@pytest.mark.parametrize("p", [2, 4])
def test_stiffness_curved(p):
    n = 3
    xv, yv, zv = inputs.uniform_vertices(n)
    jac, pts = inputs.deformed_jacobians(n, p)
    kap = inputs.kappa_field(pts, 4)
    ctx, ref, _ = pair(p, xv, yv, zv, jac=jac, kappa=kap, patches=False, coarse=False, omega=1.0)
    u = np.random.default_rng(2).standard_normal(ref.ndof)
    assert relerr(N(ctx.stiffness_apply(T(u))), ref.stiffness_apply(u)) <= 1e-12
    assert relerr(N(ctx.mass_apply(T(u))), ref.mass_apply(u)) <= 1e-12
    mu = ctx.query(fdmpc.FDM_Q_MU, np.float64, 3 * ctx.ncell).reshape(-1, 3)
    assert relerr(mu, ref.get_mu()) <= 1e-13


# ---------------------------------------------------------------- relaxation
@pytest.mark.parametrize("p", [1, 2, 3, 4, 6])
def test_asm_parity_fp64(p):
    xv, yv, zv = inputs.graded_vertices(3, 12)
    yv = np.array([0.0, 0.3, 0.4, 0.75, 1.0])
    ctx, ref, _ = pair(p, xv, yv, zv, pc=fdmpc.FDM_PC_ASM, omega=1.0, coarse=False)
    ref.set_omega(1.0)
    r = np.random.default_rng(3).standard_normal(ref.ndof)
    z = N(ctx.asm_apply(T(r)))
    assert relerr(z, ref.asm_apply(r)) <= 1e-11


@pytest.mark.parametrize("p", [2, 4, 7])
def test_asm_parity_fp32(p):
    xv, yv, zv = inputs.graded_vertices(3, 13)
    ctx, ref, _ = pair(p, xv, yv, zv, precision=FP32, pc=fdmpc.FDM_PC_ASM, omega=1.0, coarse=False)
    ref.set_omega(1.0)
    r = np.random.default_rng(4).standard_normal(ref.ndof)
    assert relerr(N(ctx.asm_apply(T(r))), ref.asm_apply(r)) <= 1e-4


def test_lanczos_omega_and_vcycle_parity():
    p = 4
    xv, yv, zv = inputs.graded_vertices(3, 14)
    ctx, ref, start = pair(p, xv, yv, zv)
    lo, hi, om = ref.lanczos_omega(start, k=20)
    lam = ctx.query(fdmpc.FDM_Q_LAMBDA, np.float64, 2)
    assert abs(lam[0] - lo) <= 1e-9 * hi and abs(lam[1] - hi) <= 1e-9 * hi
    assert abs(ctx.omega - om) <= 1e-10 * om
    ref.set_omega(ctx.omega)
    r = np.random.default_rng(5).standard_normal(ref.ndof)
    assert relerr(N(ctx.pc_apply(T(r))), ref.pc_apply(r)) <= 1e-11


def test_vcycle_parity_curved():
    p = 3
    n = 3
    xv, yv, zv = inputs.uniform_vertices(n)
    jac, pts = inputs.deformed_jacobians(n, p)
    kap = inputs.kappa_field(pts, 6)
    ctx, ref, _ = pair(p, xv, yv, zv, jac=jac, kappa=kap)
    r = np.random.default_rng(6).standard_normal(ref.ndof)
    assert relerr(N(ctx.pc_apply(T(r))), ref.pc_apply(r)) <= 1e-11


# ---------------------------------------------------------------- solver
def _rhs(ctx, ref, w):
    kind, data = inputs.rhs_for(w, ref.ndof)
    return ref.mass_apply(data) if kind == "nodal" else data


def test_pcg_parity_fp64_manufactured():
    w = inputs.workload("q4_uniform4")
    ctx, ref, _ = pair(w["p"], w["xv"], w["yv"], w["zv"])
    b = _rhs(ctx, ref, w)
    x_ref, it_ref, hist, conv = ref.pcg(b, rtol=1e-8, maxit=100)
    assert conv
    x, info = ctx.pcg_solve(T(b), rtol=1e-8, maxit=100)
    assert abs(info.iterations - it_ref) <= 1
    assert info.true_rnorm <= 1e-8 * info.rnorm0
    # same number of iterations: identical iterates up to rounding
    x2, info2 = ctx.pcg_solve(T(b), rtol=0.0, maxit=it_ref, raise_on_noconv=False)
    assert info2.iterations == it_ref
    record("pcg_fp64_manufactured", x_relerr=relerr(N(x2), x_ref), true_rel=info.true_rnorm / info.rnorm0)
    assert relerr(N(x2), x_ref) <= 1e-11
    # and the discrete solution approximates the manufactured sine
    u = inputs.manufactured_u(w["xv"], w["yv"], w["zv"], w["p"])
    assert np.abs(N(x) - u).max() < 1e-4


def test_pcg_parity_fp64_curved():
    p, n = 3, 3
    xv, yv, zv = inputs.uniform_vertices(n)
    jac, pts = inputs.deformed_jacobians(n, p)
    kap = inputs.kappa_field(pts, 7)
    ctx, ref, _ = pair(p, xv, yv, zv, jac=jac, kappa=kap)
    b = free_random(ref, 8)
    x_ref, it_ref, _, conv = ref.pcg(b, rtol=1e-8, maxit=200)
    x, info = ctx.pcg_solve(T(b), rtol=1e-8, maxit=200)
    assert abs(info.iterations - it_ref) <= 1
    x2, _ = ctx.pcg_solve(T(b), rtol=0.0, maxit=it_ref, raise_on_noconv=False)
    record("pcg_fp64_curved", x_relerr=relerr(N(x2), x_ref), iterations=it_ref)
    assert relerr(N(x2), x_ref) <= 1e-11


@pytest.mark.parametrize("p", [3, 5])
def test_pcg_mixed_precision(p):
    xv, yv, zv = inputs.graded_vertices(4, 15)
    ctx, ref, _ = pair(p, xv, yv, zv, precision=FP32)
    b = ref.mass_apply(inputs.normal_rhs(ref.ndof, 16))
    x_ref, it_ref, _, _ = ref.pcg(b, rtol=1e-8, maxit=200)
    x, info = ctx.pcg_solve(T(b), rtol=1e-8, maxit=200)
    record("pcg_mixed_p%d" % p, true_rel=info.true_rnorm / info.rnorm0, x_relerr=relerr(N(x), x_ref),
           iterations=info.iterations, oracle_iterations=it_ref)
    assert info.converged and info.true_rnorm <= 1e-8 * info.rnorm0
    assert info.iterations <= it_ref + 1
    # the same discrete solution as the FP64 oracle to the solver tolerance
    assert relerr(N(x), x_ref) <= 1e-6


def test_determinism():
    xv, yv, zv = inputs.graded_vertices(3, 17)
    ctx = fdmpc.Context(4, xv, yv, zv, precision=FP32)
    r = T(np.random.default_rng(9).standard_normal(ctx.ndof))
    z1, z2 = N(ctx.pc_apply(r)), N(ctx.pc_apply(r))
    assert np.array_equal(z1, z2)
    b = ctx.mass_apply(r)
    x1, i1 = ctx.pcg_solve(b, rtol=1e-8, maxit=100)
    x2, i2 = ctx.pcg_solve(b, rtol=1e-8, maxit=100)
    assert i1.iterations == i2.iterations and np.array_equal(N(x1), N(x2))


# ---------------------------------------------------------------- edge cases
@pytest.mark.parametrize("dims,p", [((1, 1, 1), 3), ((1, 2, 3), 2), ((5, 2, 3), 1), ((2, 2, 2), 1), ((2, 3, 2), 6)])
def test_edge_meshes(dims, p):
    xv = np.linspace(0, 1.0, dims[0] + 1)
    yv = np.linspace(0, 0.7, dims[1] + 1)
    zv = np.linspace(0, 1.3, dims[2] + 1) ** 1.2
    ctx, ref, _ = pair(p, xv, yv, zv)
    r = np.random.default_rng(10).standard_normal(ref.ndof)
    assert relerr(N(ctx.pc_apply(T(r))), ref.pc_apply(r)) <= 1e-11
    b = free_random(ref, 11)
    if np.abs(b).max() == 0:
        x, info = ctx.pcg_solve(T(b), rtol=1e-8, maxit=50)
        assert info.iterations == 0 and np.abs(N(x)).max() == 0
        return
    x_ref, it_ref, _, _ = ref.pcg(b, rtol=1e-8, maxit=200)
    x, info = ctx.pcg_solve(T(b), rtol=1e-8, maxit=200)
    assert abs(info.iterations - it_ref) <= 1


def test_zero_rhs_and_errors():
    xv, yv, zv = inputs.graded_vertices(2, 1)
    ctx = fdmpc.Context(2, xv, yv, zv, precision=FP64)
    x, info = ctx.pcg_solve(torch.zeros(ctx.ndof, dtype=torch.float64, device=DEV))
    assert info.iterations == 0 and info.converged == 1
    b = T(np.random.default_rng(0).standard_normal(ctx.ndof))
    with pytest.raises(fdmpc.FdmError) as e:
        ctx.pcg_solve(b, rtol=1e-12, maxit=1)
    assert e.value.code == fdmpc.FDM_ENOCONV
    bad = b.clone()
    bad[ctx.ndof // 2] = float("nan")
    with pytest.raises(fdmpc.FdmError) as e:
        ctx.pcg_solve(bad, rtol=1e-8, maxit=5)
    assert e.value.code == fdmpc.FDM_ENAN
    with pytest.raises(fdmpc.FdmError) as e:
        ctx.surrogate_load(-np.ones(3 * ctx.ncell))
    assert e.value.code == fdmpc.FDM_EINVAL


# ---------------------------------------------------------------- full-size sampled checks
def _node_in_cell_interior(ref, cell, seed):
    rng = np.random.default_rng(seed)
    p = ref.p
    cx, cy, cz = cell % ref.nx, (cell // ref.nx) % ref.ny, cell // (ref.nx * ref.ny)
    i, j, k = rng.integers(1, p, size=3)
    return (cx * p + i) + ref.N[0] * ((cy * p + j) + ref.N[1] * (cz * p + k)), (cx, cy, cz)


@pytest.mark.parametrize("name", ["q7_graded16", "q15_uniform8", "q8_deformed12"])
def test_full_size_sampled(name):
    """At the benchmark sizes: the full stiffness apply, and the relaxation
    applied to a unit vector at a sampled cell-interior node, which only
    involves the 8 vertex stars of that cell (set up alone in the oracle).
    The deformed workload runs with its curved cells, kappa and averaged
    surrogate."""
    w = inputs.workload(name)
    p = w["p"]
    for precision in (FP64, FP32):
        ctx = fdmpc.Context(p, w["xv"], w["yv"], w["zv"], jac=w["jac"], kappa=w["kappa"], precision=precision,
                            pc=fdmpc.FDM_PC_ASM, omega=1.0)
        ref = oracle.Problem(p, w["xv"], w["yv"], w["zv"], jac=w["jac"], kappa=w["kappa"])
        if precision == FP64:
            u = np.random.default_rng(12).standard_normal(ref.ndof)
            assert relerr(N(ctx.stiffness_apply(T(u))), ref.stiffness_apply(u)) <= 1e-12
        cell = ref.ncell // 2 + ref.nx // 2
        g, (cx, cy, cz) = _node_in_cell_interior(ref, cell, 13)
        verts = [(cx + a) + (ref.nx + 1) * ((cy + b) + (ref.ny + 1) * (cz + c))
                 for c in (0, 1) for b in (0, 1) for a in (0, 1)]
        ref.setup_patches(verts)
        ref.set_omega(1.0)
        e = np.zeros(ref.ndof)
        e[g] = 1.0
        z_ref = ref.asm_apply(e)
        z = N(ctx.asm_apply(T(e)))
        tol = 1e-11 if precision == FP64 else 1e-4
        assert relerr(z, z_ref) <= tol, (name, precision)
        ctx.close()


# ---------------------------------------------------------------- kernels and failure detection
@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5])
def test_both_patch_kernels_agree(kernel):
    """The classic (one CTA per patch), streamed (bulk copies into a
    shared-memory ring) and resident (whole factor in shared memory) patch
    solves give the oracle's relaxation."""
    xv, yv, zv = inputs.graded_vertices(3, 21)
    for p in (2, 5):
        ctx = fdmpc.Context(p, xv, yv, zv, precision=FP64, pc=fdmpc.FDM_PC_ASM, omega=1.0, patch_kernel=kernel)
        ref = oracle.Problem(p, xv, yv, zv)
        ref.setup_patches()
        ref.set_omega(1.0)
        r = np.random.default_rng(22).standard_normal(ref.ndof)
        assert relerr(N(ctx.asm_apply(T(r))), ref.asm_apply(r)) <= 1e-11
        ctx.close()


@pytest.mark.parametrize("nbuf,kb", [(2, 8), (3, 16), (6, 24)])
def test_stream_ring_shapes(nbuf, kb):
    w = inputs.workload("q4_uniform4")
    ctx = fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], precision=FP32, pc=fdmpc.FDM_PC_ASM, omega=1.0,
                        stream_buffers=nbuf, stream_buffer_kb=kb, patch_kernel=2)
    ref = oracle.Problem(w["p"], w["xv"], w["yv"], w["zv"])
    ref.setup_patches()
    ref.set_omega(1.0)
    r = np.random.default_rng(23).standard_normal(ref.ndof)
    assert relerr(N(ctx.asm_apply(T(r))), ref.asm_apply(r)) <= 1e-4
    assert ctx.status() == 0


@pytest.mark.parametrize("p,precision", [(3, FP64), (4, FP32), (7, FP32)])
def test_resident_matches_classic_bitwise(p, precision):
    """The resident kernel runs the classic kernel's arithmetic on a shared-
    memory copy of the factor: with the same number of threads (which fixes
    the summation order) the results are identical, bit for bit."""
    xv, yv, zv = inputs.graded_vertices(3, 5)
    r = T(np.random.default_rng(31).standard_normal(((len(xv) - 1) * p + 1) ** 3))
    out = []
    for kernel in (1, 3):
        ctx = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7, patch_kernel=kernel,
                            patch_threads=512, patch_form=1)
        out.append(N(ctx.asm_apply(r)))
        assert ctx.status() == 0
        ctx.close()
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("kernel", [1, 2, 3, 4, 5, 6])
def test_bounded_wait_reports_timeout_kernels(kernel):
    """As below, for every patch solve with a bounded device-side wait: the
    Schur-coupling kernels (its staging copy), the streamed, resident and
    cluster kernels."""
    xv, yv, zv = inputs.graded_vertices(2, 3)
    ctx = fdmpc.Context(3, xv, yv, zv, precision=FP32, omega=0.2, inject_stall=1, wait_timeout_s=0.02,
                        patch_kernel=kernel)
    b = T(np.random.default_rng(0).standard_normal(ctx.ndof))
    with pytest.raises(fdmpc.FdmError) as e:
        ctx.pcg_solve(b, rtol=1e-8, maxit=2)
    assert e.value.code == fdmpc.FDM_ETIMEOUT
    y = ctx.stiffness_apply(b)
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()


@pytest.mark.parametrize("p,precision", [(4, FP32), (7, FP32), (3, FP64)])
def test_autotuned_context_matches(p, precision):
    """The autotuner keeps one of its candidates; the tuned context gives the
    default context's relaxation to rounding (the variants sum in different
    orders) and the same PCG solution."""
    xv, yv, zv = inputs.graded_vertices(3, 8)
    r = T(np.random.default_rng(41).standard_normal(((len(xv) - 1) * p + 1) ** 3))
    a = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7)
    b = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7, autotune=1)
    kernel, threads, rows8, us, ncand = b.tuning()
    # Schur-coupling form (default): six shapes plus the fully staged and warp-per-patch kernels where they fit
    assert kernel in (5, 6, 7, 8) and threads in (128, 256, 512, 1024) and us > 0 and 6 <= ncand <= 11
    c = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7, autotune=1, patch_form=1)
    kernel, threads, rows8, us, ncand = c.tuning()
    assert kernel in (1, 3) and threads in (256, 512, 1024) and rows8 in (0, 1) and us > 0 and ncand >= 4
    assert a.tuning()[4] == 0
    tol = 1e-12 if precision == FP64 else 1e-5
    assert relerr(N(b.asm_apply(r)), N(a.asm_apply(r))) <= tol
    assert relerr(N(c.asm_apply(r)), N(a.asm_apply(r))) <= tol
    assert b.status() == 0


@pytest.mark.parametrize("p,precision", [(3, FP64), (5, FP64), (4, FP32), (7, FP32), (8, FP32)])
def test_cluster_kernel_matches_classic(p, precision):
    """The cluster patch solve (L21 held in shared memory across a cluster)
    gives the classic kernel's relaxation to rounding."""
    xv, yv, zv = inputs.graded_vertices(3, 9)
    r = T(np.random.default_rng(51).standard_normal(((len(xv) - 1) * p + 1) ** 3))
    out = []
    for kernel in (1, 4):
        ctx = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7, patch_kernel=kernel)
        out.append(N(ctx.asm_apply(r)))
        assert ctx.status() == 0
        ctx.close()
    assert relerr(out[1], out[0]) <= (1e-12 if precision == FP64 else 1e-5)


def test_bounded_wait_reports_timeout():
    """Failure detection without a GPU fault: the streamed solve is made to
    wait on a barrier that nothing completes; the wait gives up after the
    configured limit, the kernel drains its copies and returns, and the host
    sees FDM_ETIMEOUT.  The context stays usable afterwards."""
    xv, yv, zv = inputs.graded_vertices(2, 3)
    ctx = fdmpc.Context(3, xv, yv, zv, precision=FP32, omega=0.2, inject_stall=1, wait_timeout_s=0.02,
                        patch_kernel=2)
    b = T(np.random.default_rng(0).standard_normal(ctx.ndof))
    with pytest.raises(fdmpc.FdmError) as e:
        ctx.pcg_solve(b, rtol=1e-8, maxit=2)
    assert e.value.code == fdmpc.FDM_ETIMEOUT
    y = ctx.stiffness_apply(b)  # the CUDA context is still healthy
    torch.cuda.synchronize()
    assert torch.isfinite(y).all()


@pytest.mark.parametrize("p,precision", [(1, FP64), (2, FP64), (3, FP64), (7, FP64), (11, FP64), (4, FP32), (7, FP32),
                                         (15, FP32)])
def test_patch_forms_agree(p, precision):
    """The Schur-coupling form (x_T = W (g_T - S_TB y_B), x_B = y_B - S_BB^{-1}
    S_BT x_T) and the L form (forward and backward solves with L_G) are the same
    exact patch solve: the relaxations agree to rounding, and the Schur-coupling
    form stores fewer values (no dense L21, W in place of Z)."""
    xv, yv, zv = inputs.graded_vertices(2 if p >= 11 else 3, 12)
    r = T(np.random.default_rng(61).standard_normal(((len(xv) - 1) * p + 1) ** 3))
    out, ab, lf = [], [], []
    for form in (1, 2):
        ctx = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7, patch_form=form)
        out.append(N(ctx.asm_apply(r)))
        ab.append(ctx.algo_bytes()["patch64"])
        lf.append(ctx.algo_bytes()["lform64"])
        assert ctx.status() == 0
        ctx.close()
    assert relerr(out[1], out[0]) <= (1e-12 if precision == FP64 else 2e-5)
    assert lf[0] == lf[1] == ab[0]   # the L-form count does not depend on the form in use
    if p >= 7:
        assert ab[1] < 0.6 * ab[0]
    elif p >= 3:
        assert ab[1] < ab[0]


def test_patch_form_rejects_l_kernels():
    xv = np.linspace(0, 1, 3)
    with pytest.raises(fdmpc.FdmError):
        fdmpc.Context(3, xv, xv, xv, precision=FP32, omega=1.0, patch_kernel=3, patch_form=2)


@pytest.mark.parametrize("variant", [1, 2, 3])
def test_sc_variants_agree(variant):
    """The Schur-coupling kernels (two or four rows of W per warp, what is
    staged in shared memory; 128, 256 and 512 threads) give the oracle's
    relaxation."""
    xv, yv, zv = inputs.graded_vertices(3, 13)
    for p, precision in ((3, FP64), (7, FP64), (7, FP32)):
        ref = oracle.Problem(p, xv, yv, zv)
        ref.setup_patches()
        ref.set_omega(0.7)
        r = np.random.default_rng(62).standard_normal(ref.ndof)
        for threads in (128, 256, 512):
            ctx = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7,
                                sc_variant=variant, patch_threads=threads)
            assert relerr(N(ctx.asm_apply(T(r))), ref.asm_apply(r)) <= (1e-11 if precision == FP64 else 1e-4)
            assert ctx.status() == 0
            ctx.close()


@pytest.mark.parametrize("p,precision", [(3, FP64), (7, FP64), (7, FP32), (15, FP32)])
def test_persistent_sc_matches(p, precision):
    """The persistent Schur-coupling kernel (double-buffered staging, a CTA
    walking many patches) gives the one-CTA-per-patch kernel's relaxation to
    rounding, and reports no expired wait."""
    xv, yv, zv = inputs.graded_vertices(2 if p >= 11 else 3, 14)
    r = T(np.random.default_rng(63).standard_normal(((len(xv) - 1) * p + 1) ** 3))
    out = []
    for kernel in (1, 5):
        ctx = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7, patch_kernel=kernel)
        out.append(N(ctx.asm_apply(r)))
        assert ctx.status() == 0
        ctx.close()
    assert relerr(out[1], out[0]) <= (1e-12 if precision == FP64 else 1e-5)


@pytest.mark.parametrize("p,precision", [(2, FP64), (3, FP64), (5, FP64), (4, FP32), (7, FP32)])
def test_fully_staged_sc_matches(p, precision):
    """The persistent kernel that stages each patch's whole operator (pivots,
    L10, line blocks, S_TB and W) in one of two shared-memory buffers gives the
    oracle's relaxation with 256, 512 and 1024 threads, and reports no
    expired wait; the 3^3 graded mesh has every star class."""
    xv, yv, zv = inputs.graded_vertices(3, 15)
    ref = oracle.Problem(p, xv, yv, zv)
    ref.setup_patches()
    ref.set_omega(0.7)
    r = np.random.default_rng(64).standard_normal(ref.ndof)
    zr = ref.asm_apply(r)
    for threads in (256, 512, 1024):
        ctx = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7, patch_kernel=6,
                            patch_threads=threads)
        z = N(ctx.asm_apply(T(r)))
        record("scf_p%d_t%d" % (p, threads), relerr=relerr(z, zr))
        assert relerr(z, zr) <= (1e-11 if precision == FP64 else 1e-4)
        assert ctx.status() == 0
        ctx.close()


def test_fully_staged_sc_rejects_what_does_not_fit():
    """Two FP64 patch operators at p = 8 (38,504 values each) exceed shared
    memory: the set-up refuses the kernel instead of launching it."""
    xv = np.linspace(0, 1, 3)
    with pytest.raises(fdmpc.FdmError) as e:
        fdmpc.Context(8, xv, xv, xv, precision=FP64, omega=1.0, patch_kernel=6)
    assert e.value.code == fdmpc.FDM_EINVAL


@pytest.mark.parametrize("p,precision", [(1, FP64), (2, FP64), (3, FP64), (7, FP64), (4, FP32), (7, FP32), (9, FP32),
                                         (11, FP32)])
def test_warp_per_patch_matches(p, precision):
    """The warp-per-patch Schur-coupling solve (one warp per star, 4 or 8
    stars per CTA, no CTA barrier) gives the oracle's relaxation on a mesh with
    every star class; p = 9 and 11 take its wider register column sums."""
    xv, yv, zv = inputs.graded_vertices(2 if p >= 9 else 3, 16)
    ref = oracle.Problem(p, xv, yv, zv)
    ref.setup_patches()
    ref.set_omega(0.7)
    r = np.random.default_rng(65).standard_normal(ref.ndof)
    zr = ref.asm_apply(r)
    for threads in (128, 256):
        ctx = fdmpc.Context(p, xv, yv, zv, precision=precision, pc=fdmpc.FDM_PC_ASM, omega=0.7, patch_kernel=7,
                            patch_threads=threads)
        z = N(ctx.asm_apply(T(r)))
        record("scw_p%d_t%d" % (p, threads), relerr=relerr(z, zr))
        assert relerr(z, zr) <= (1e-11 if precision == FP64 else 1e-4)
        ctx.close()


def test_warp_per_patch_rejects_large_interfaces():
    """At p = 12 the top block (529 rows) exceeds the warp kernel's register
    column sums: the set-up refuses it."""
    xv = np.linspace(0, 1, 3)
    with pytest.raises(fdmpc.FdmError) as e:
        fdmpc.Context(12, xv, xv, xv, precision=FP32, omega=1.0, patch_kernel=7)
    assert e.value.code == fdmpc.FDM_EINVAL
