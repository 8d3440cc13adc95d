"""GPU parity of the SIPG (DQ_p) Poisson path (Section 5) against the FP64
oracle, through the C-ABI.

Tolerances: operator <= 1e-12 relative (sum factorisation against the
oracle's Kronecker traces); star solves in FP64 <= 1e-10 relative (fast
diagonalisation from FP64 Jacobi eigenvectors against a dense Cholesky of the
star matrix; the 1D pencils' condition numbers are below 1e5), in FP32
<= 2e-4; relaxation, V(1,1) and Lanczos extremes <= 1e-10, omega <= 1e-9; PCG
iterations within +-1 and iterates <= 1e-9 at equal iteration counts; the
mixed-precision solve reaches the FP64 true residual 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2107_14758_gb300 import fdmpc, inputs  # noqa: E402

FP64, FP32 = fdmpc.FDM_PREC_FP64, fdmpc.FDM_PREC_FP32
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()


@pytest.fixture(scope="module")
def Sipg():
    from oracle.sipg import Sipg
    return Sipg


def T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=DEV)


def N(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


MESH = ([0, .3, .5, 1], [0, .45, 1.0], [0, .2, .7, .9, 1.1])   # 3 x 2 x 4 graded cells


@pytest.mark.parametrize("p", [1, 2, 4, 7, 10])
def test_apply_parity(Sipg, p):
    ref = Sipg(p, *MESH)
    gpu = fdmpc.Sipg(p, *MESH, precision=FP64, omega=1.0)
    u = np.random.default_rng(p).standard_normal(ref.N)
    assert relerr(N(gpu.apply(T(u))), ref.apply(u)) <= 1e-12


def test_apply_parity_benchmark_size(Sipg):
    """The 16^3 graded Q7 mesh of the SIPG workload at its full size."""
    xv, yv, zv = inputs.graded_vertices(16, 7)
    ref = Sipg(7, xv, yv, zv)
    gpu = fdmpc.Sipg(7, xv, yv, zv, precision=FP64, omega=1.0, pc=fdmpc.FDM_PC_ASM)
    u = np.random.default_rng(5).standard_normal(ref.N)
    assert relerr(N(gpu.apply(T(u))), ref.apply(u)) <= 1e-12


def test_penalty_parameter(Sipg):
    ref = Sipg(3, *MESH, eta=40.0)
    gpu = fdmpc.Sipg(3, *MESH, eta=40.0, precision=FP64, omega=1.0)
    u = np.random.default_rng(3).standard_normal(ref.N)
    assert relerr(N(gpu.apply(T(u))), ref.apply(u)) <= 1e-12


@pytest.mark.parametrize("p,prec,tol", [(1, FP64, 1e-10), (3, FP64, 1e-10), (7, FP64, 1e-10), (3, FP32, 2e-4),
                                        (7, FP32, 2e-4)])
def test_star_solve_parity(Sipg, p, prec, tol):
    ref = Sipg(p, *MESH)
    gpu = fdmpc.Sipg(p, *MESH, precision=prec, omega=1.0, pc=fdmpc.FDM_PC_ASM)
    r = np.random.default_rng(10 + p).standard_normal(ref.N)
    verts = ref.vertices()
    got = N(gpu.patch_solve(T(r), verts))
    for k, v in enumerate(verts):
        assert relerr(got[k], ref.patch_solve(v, r)) <= tol, v


def test_star_solve_rejects_boundary_vertex():
    gpu = fdmpc.Sipg(2, *MESH, precision=FP64, omega=1.0)
    r = torch.zeros(gpu.ndof, dtype=torch.float64, device=DEV)
    with pytest.raises(fdmpc.FdmError):
        gpu.patch_solve(r, [(0, 1, 1)])
    with pytest.raises(fdmpc.FdmError):
        gpu.patch_solve(r, [(1, 2, 1)])   # ny = 2: vy = 2 is on the boundary


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-10), (FP32, 2e-4)])
def test_asm_parity(Sipg, prec, tol):
    ref = Sipg(3, *MESH)
    ref.setup_patches()
    gpu = fdmpc.Sipg(3, *MESH, precision=prec, omega=0.7, pc=fdmpc.FDM_PC_ASM)
    r = np.random.default_rng(4).standard_normal(ref.N)
    assert relerr(N(gpu.asm_apply(T(r))), 0.7 * ref.asm(r)) <= tol
    assert relerr(N(gpu.pc_apply(T(r))), 0.7 * ref.asm(r)) <= tol


def test_vcycle_parity(Sipg):
    ref = Sipg(2, *MESH)
    ref.setup_patches()
    ref.setup_coarse()
    ref.omega = 0.6
    gpu = fdmpc.Sipg(2, *MESH, precision=FP64, omega=0.6)
    r = np.random.default_rng(6).standard_normal(ref.N)
    assert relerr(N(gpu.pc_apply(T(r))), ref.pc_apply(r, pc=2)) <= 1e-10


def test_lanczos_parity(Sipg):
    ref = Sipg(3, *MESH)
    ref.setup_patches()
    start = inputs.lanczos_start(ref.N)
    gpu = fdmpc.Sipg(3, *MESH, precision=FP64, lanczos_start=start)
    lo, hi = gpu.lanczos_extremes()
    lo_r, hi_r, om_r = ref.lanczos_omega(start)
    assert abs(lo - lo_r) <= 1e-10 * hi_r and abs(hi - hi_r) <= 1e-10 * hi_r
    assert gpu.omega == pytest.approx(om_r, rel=1e-9)


def test_pcg_parity_fp64(Sipg):
    xv, yv, zv = inputs.graded_vertices(4, 73)
    ref = Sipg(2, xv, yv, zv)
    ref.setup_patches()
    ref.setup_coarse()
    start = inputs.lanczos_start(ref.N)
    ref.lanczos_omega(start)
    gpu = fdmpc.Sipg(2, xv, yv, zv, precision=FP64, lanczos_start=start)
    b = np.random.default_rng(8).standard_normal(ref.N)
    x_ref, it_ref, conv = ref.pcg(b, rtol=1e-8, maxit=200)
    assert conv
    x, info = gpu.pcg_solve(T(b), rtol=1e-8, maxit=200)
    assert abs(info.iterations - it_ref) <= 1
    x2, info2 = gpu.pcg_solve(T(b), rtol=0.0, maxit=it_ref, raise_on_noconv=False)
    assert info2.iterations == it_ref
    assert relerr(N(x2), x_ref) <= 1e-9
    # the Q1 coarse problem by one multigrid V-cycle instead of the exact solve
    gmg = fdmpc.Sipg(2, xv, yv, zv, precision=FP64, lanczos_start=start, coarse_levels=1)
    _, ig = gmg.pcg_solve(T(b), rtol=1e-8, maxit=200)
    assert ig.converged and ig.iterations <= it_ref + 5


def test_mixed_precision_manufactured_solution(Sipg):
    """-lap u = 3 pi^2 sin sin sin on a graded 4^3 mesh, p = 5: the FP32
    preconditioner reaches the FP64 true residual, the iterate matches the
    oracle's FP64 solve, and both approximate the exact solution."""
    xv, yv, zv = inputs.graded_vertices(4, 11)
    p = 5
    ref = Sipg(p, xv, yv, zv)
    f = lambda x, y, z: 3 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    b = ref.load(f)
    fp64 = fdmpc.Sipg(p, xv, yv, zv, precision=FP64)
    mixed = fdmpc.Sipg(p, xv, yv, zv, precision=FP32)
    x64, i64 = fp64.pcg_solve(T(b), rtol=1e-10, maxit=300)
    x32, i32 = mixed.pcg_solve(T(b), rtol=1e-10, maxit=300)
    assert i32.converged and i32.true_rnorm <= 1e-10 * i32.rnorm0
    assert i32.iterations <= i64.iterations + 1
    assert relerr(N(x32), N(x64)) <= 1e-8
    X = ref.nodes()
    exact = np.sin(np.pi * X[0]) * np.sin(np.pi * X[1]) * np.sin(np.pi * X[2])
    assert np.abs(N(x64) - exact).max() < 1e-3
    assert np.abs(ref.apply(N(x64)) - b).max() <= 1e-9 * np.abs(b).max()


def test_full_size_sampled(Sipg):
    """16^3 graded Q7 (2.1 M values, 3375 stars) in the launch configuration
    the benchmark times: star solves on sampled vertices (corner, edge, face,
    interior) in both precisions against the oracle's dense Cholesky, and the
    V(1,1) preconditioner the benchmark runs is positive on a random vector."""
    xv, yv, zv = inputs.graded_vertices(16, 7)
    ref = Sipg(7, xv, yv, zv)
    r = np.random.default_rng(21).standard_normal(ref.N)
    verts = [(1, 1, 1), (15, 1, 1), (1, 8, 15), (7, 9, 4)]
    want = [ref.patch_solve(v, r) for v in verts]
    for prec, tol in ((FP64, 1e-10), (FP32, 2e-4)):
        # omega from Lanczos: undamped, the 8-fold overlapping sum makes V(1,1) indefinite
        gpu = fdmpc.Sipg(7, xv, yv, zv, precision=prec)
        got = N(gpu.patch_solve(T(r), verts))
        for k in range(len(verts)):
            assert relerr(got[k], want[k]) <= tol, (prec, verts[k])
        z = N(gpu.pc_apply(T(r)))
        assert np.all(np.isfinite(z)) and float(z @ r) > 0


def test_zero_rhs_and_invalid():
    gpu = fdmpc.Sipg(2, *MESH)
    x, info = gpu.pcg_solve(torch.zeros(gpu.ndof, dtype=torch.float64, device=DEV))
    assert info.converged and info.iterations == 0 and float(x.abs().max()) == 0.0
    with pytest.raises(fdmpc.FdmError):
        fdmpc.Sipg(11, *MESH)
    with pytest.raises(fdmpc.FdmError):
        fdmpc.Sipg(2, [0, 1], [0, .5, 1], [0, .5, 1])
    with pytest.raises(fdmpc.FdmError):
        fdmpc.Sipg(2, [0, .5, .4], [0, .5, 1], [0, .5, 1])


# ---------------------------------------------------------------- tensor-core star solves (DQ_7)
# TF32 inputs rounded to nearest carry a relative error of at most u = 2^-11;
# each of the six passes rounds its input line and its matrix (2u per product
# term), and the eigenvector matrices are B-orthonormal rather than orthogonal
# (a growth factor of a few through the passes): 12 u x 3 ~ 2e-2 bounds the
# relative error of one star solve and of one relaxation sweep.
TC_TOL = 2e-2


def test_tensor_core_star_solves(Sipg):
    """The tcgen05 (TF32, FP32 accumulation) star solves against the oracle's
    dense Cholesky of the star matrix, on a graded 3^3 DQ_7 mesh (all 8
    interior stars)."""
    from tests.record import record
    xv, yv, zv = inputs.graded_vertices(3, 23)
    ref = Sipg(7, xv, yv, zv)
    r = np.random.default_rng(24).standard_normal(ref.N)
    verts = [(a, b, c) for c in (1, 2) for b in (1, 2) for a in (1, 2)]
    gpu = fdmpc.Sipg(7, xv, yv, zv, precision=FP32, tensor_core=1)
    got = N(gpu.patch_solve(T(r), verts))
    errs = [relerr(got[k], ref.patch_solve(v, r)) for k, v in enumerate(verts)]
    record("sipg_tc_star", worst=max(errs))
    assert max(errs) <= TC_TOL
    assert gpu.status() == 0


def test_tensor_core_sweep_and_pcg():
    """A relaxation sweep with the tensor-core star solves against the FP32
    CUDA-core sweep (TF32 tolerance), and the mixed-precision PCG with it:
    the FP64 true residual 1e-8 with at most one more iteration than with the
    CUDA-core star solves."""
    from tests.record import record
    xv, yv, zv = inputs.graded_vertices(4, 25)
    b = torch.randn(4 ** 3 * 512, dtype=torch.float64, device=DEV, generator=torch.Generator(device=DEV).manual_seed(3))
    start = inputs.lanczos_start(4 ** 3 * 512)
    cc = fdmpc.Sipg(7, xv, yv, zv, precision=FP32, lanczos_start=start)
    tc = fdmpc.Sipg(7, xv, yv, zv, precision=FP32, lanczos_start=start, tensor_core=1)
    z0, z1 = N(cc.asm_apply(b)), N(tc.asm_apply(b))
    _, i0 = cc.pcg_solve(b, rtol=1e-8, maxit=500)
    _, i1 = tc.pcg_solve(b, rtol=1e-8, maxit=500)
    record("sipg_tc_sweep", relerr=relerr(z1, z0), its_cuda_core=i0.iterations, its_tensor_core=i1.iterations,
           omega_rel=abs(tc.omega - cc.omega) / cc.omega)
    assert relerr(z1, z0) <= TC_TOL
    assert i1.converged and i1.true_rnorm <= 1e-8 * i1.rnorm0
    assert i1.iterations <= i0.iterations + 1
    assert tc.status() == 0


def test_tensor_core_only_at_dq7():
    with pytest.raises(fdmpc.FdmError) as e:
        fdmpc.Sipg(3, *MESH, precision=FP32, tensor_core=1)
    assert e.value.code == fdmpc.FDM_EINVAL
