"""GPU parity of primal linear elasticity with the SDC/FDM/sparse relaxation
(Section 4.1) against the FP64 oracle, through the C-ABI.

Tolerances: operator <= 1e-12 relative (sum factorisation on Gauss points
against the oracle's Kronecker products); FP64 relaxation and V(1,1)
<= 1e-11; Lanczos extremes <= 1e-9, omega <= 1e-10; PCG iterations within +1
and iterates <= 1e-10 at equal iteration counts; the mixed-precision solve
reaches the FP64 true residual 1e-8.
"""
import numpy as np
import pytest

from tests.record import record  # noqa: E402

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
def el():
    import oracle
    oracle.build()
    from oracle import elasticity
    return elasticity


def T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64).ravel(), device=DEV)


def N(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def rand_free(E, seed):
    return np.where(np.tile(E.free, 3), np.random.default_rng(seed).standard_normal(3 * E.N), 0.0)


@pytest.mark.parametrize("p", [1, 2, 4, 7])
def test_apply_parity(el, p):
    xv, yv, zv = np.array([0, 0.3, 1.0]), np.array([0, 0.45, 0.8, 1.0]), np.array([0, 0.2, 0.7, 1.1])
    ref = el.Elasticity(p, xv, yv, zv, 0.8, 3.7)
    gpu = fdmpc.Elasticity(p, xv, yv, zv, 0.8, 3.7, precision=FP64, omega=1.0)
    u = np.random.default_rng(p).standard_normal(3 * ref.N)       # Dirichlet entries are ignored
    got = N(gpu.apply(T(u)))
    want = ref.apply(u).ravel()
    assert relerr(got, want) <= 1e-12


@pytest.mark.parametrize("p", [7, 15])
def test_apply_parity_benchmark_size(el, p):
    """The 8^3 uniform mesh of the elasticity workload at its full size."""
    xv = np.linspace(0, 1, 9)
    ref = el.Elasticity(p, xv, xv, xv, 1.0, 100.0)
    gpu = fdmpc.Elasticity(p, xv, xv, xv, 1.0, 100.0, precision=FP64, omega=1.0, pc=fdmpc.FDM_PC_ASM)
    u = rand_free(ref, 10 + p)
    assert relerr(N(gpu.apply(T(u))), ref.apply(u).ravel()) <= 1e-12


def _pair(el, p, xv, yv, zv, mu, lam, precision=FP64, pc=fdmpc.FDM_PC_VCYCLE, omega=0.0):
    ref = el.Elasticity(p, xv, yv, zv, mu, lam)
    ref.setup_sdc()
    ref.setup_coarse()
    start = inputs.lanczos_start(3 * ref.N)
    gpu = fdmpc.Elasticity(p, xv, yv, zv, mu, lam, precision=precision, pc=pc, omega=omega, lanczos_start=start)
    if omega > 0:
        ref.omega = omega
    else:
        ref.lanczos_omega(start)
    return ref, gpu


def test_lanczos_parity(el):
    xv, yv, zv = inputs.graded_vertices(3, 71)
    ref, gpu = _pair(el, 3, xv, yv, zv, 1.0, 10.0)
    lo, hi = gpu.lanczos_extremes()
    start = inputs.lanczos_start(3 * ref.N)
    lo_r, hi_r, om_r = ref.lanczos_omega(start)
    assert abs(lo - lo_r) <= 1e-9 * hi_r and abs(hi - hi_r) <= 1e-9 * hi_r
    assert gpu.omega == pytest.approx(om_r, rel=1e-10)


@pytest.mark.parametrize("pc", [fdmpc.FDM_PC_ASM, fdmpc.FDM_PC_VCYCLE])
def test_pc_apply_parity(el, pc):
    xv, yv, zv = inputs.graded_vertices(3, 72)
    ref, gpu = _pair(el, 3, xv, yv, zv, 1.3, 7.0, pc=pc, omega=0.7)
    r = rand_free(ref, 3)
    z = N(gpu.pc_apply(T(r)))
    zr = ref.pc_apply(r, pc=1 if pc == fdmpc.FDM_PC_ASM else 2).ravel()
    assert relerr(z, zr) <= 1e-11


def test_pcg_parity_fp64(el):
    xv, yv, zv = inputs.graded_vertices(4, 73)
    ref, gpu = _pair(el, 2, xv, yv, zv, 1.0, 10.0)
    b = ref.body_force([0.0, -0.02, 0.0]).ravel()
    x_ref, it_ref, conv = ref.pcg(b, rtol=1e-8, maxit=400)
    assert conv
    x, info = gpu.pcg_solve(T(b), rtol=1e-8, maxit=400)
    assert abs(info.iterations - it_ref) <= 1
    x2, info2 = gpu.pcg_solve(T(b), rtol=0.0, maxit=it_ref, raise_on_noconv=False)
    assert info2.iterations == it_ref
    record("elast_pcg_fp64", x_relerr=relerr(N(x2), x_ref.ravel()), iterations=it_ref)
    assert relerr(N(x2), x_ref.ravel()) <= 1e-11


@pytest.mark.parametrize("lam", [0.0, 1.0, 10.0, 100.0])
def test_iterations_follow_the_oracle(el, lam):
    """4^3 uniform, p = 3, body force -0.02 e_2: the FP64 GPU solve takes the
    oracle's iteration count (+-1) at every lambda, and the mixed-precision
    solve at most one more."""
    xv = np.linspace(0, 1, 5)
    ref, gpu = _pair(el, 3, xv, xv, xv, 1.0, lam)
    b = ref.body_force([0.0, -0.02, 0.0]).ravel()
    _, it_ref, conv = ref.pcg(b, rtol=1e-8, maxit=500)
    assert conv
    _, info = gpu.pcg_solve(T(b), rtol=1e-8, maxit=500)
    assert abs(info.iterations - it_ref) <= 1
    mixed = fdmpc.Elasticity(3, xv, xv, xv, 1.0, lam, precision=FP32,
                             lanczos_start=inputs.lanczos_start(3 * ref.N))
    _, im = mixed.pcg_solve(T(b), rtol=1e-8, maxit=500)
    record("elast_mixed_lam%g" % lam, true_rel=im.true_rnorm / im.rnorm0, iterations=im.iterations)
    assert im.converged and im.true_rnorm <= 1e-8 * im.rnorm0
    assert im.iterations <= info.iterations + 1


def test_mixed_precision_solution(el):
    xv, yv, zv = inputs.graded_vertices(3, 74)
    ref = el.Elasticity(4, xv, yv, zv, 1.0, 5.0)
    ref.setup_sdc()
    ref.setup_coarse()
    ref.lanczos_omega(inputs.lanczos_start(3 * ref.N))
    b = rand_free(ref, 9)
    x_ref, _, conv = ref.pcg(b, rtol=1e-10, maxit=500)
    gpu = fdmpc.Elasticity(4, xv, yv, zv, 1.0, 5.0, precision=FP32)
    x, info = gpu.pcg_solve(T(b), rtol=1e-10, maxit=500)
    assert info.converged and info.true_rnorm <= 1e-10 * info.rnorm0
    assert relerr(N(x), x_ref.ravel()) <= 1e-7


def test_zero_rhs_and_invalid():
    xv = np.linspace(0, 1, 3)
    gpu = fdmpc.Elasticity(2, xv, xv, xv, 1.0, 1.0)
    x, info = gpu.pcg_solve(torch.zeros(3 * gpu.ndof, dtype=torch.float64, device=DEV))
    assert info.converged and info.iterations == 0 and float(x.abs().max()) == 0.0
    with pytest.raises(fdmpc.FdmError):
        fdmpc.Elasticity(2, xv, xv, xv, -1.0, 1.0)


# ---------------------------------------------------------------- traction-free faces (Sec. 4.1's setting)
STAR = fdmpc.FDM_SDC_STAR_FDM
MASKS = {"x0": 1, "x0_z1": 1 | 32, "y0_y1": 4 | 8}


def _pair_bc(el, p, xv, yv, zv, mu, lam, mask, precision=FP64, pc=fdmpc.FDM_PC_VCYCLE, omega=0.0):
    ref = el.Elasticity(p, xv, yv, zv, mu, lam, dirichlet_faces=mask)
    ref.setup_sdc()
    ref.setup_coarse()
    start = inputs.lanczos_start(3 * ref.N)
    gpu = fdmpc.Elasticity(p, xv, yv, zv, mu, lam, precision=precision, pc=pc, omega=omega, lanczos_start=start,
                           dirichlet_faces=mask)
    if omega > 0:
        ref.omega = omega
    else:
        ref.lanczos_omega(start)
    return ref, gpu


@pytest.mark.parametrize("mask", sorted(MASKS))
@pytest.mark.parametrize("p", [1, 2, 4])
def test_traction_free_apply_parity(el, p, mask):
    xv, yv, zv = np.array([0, 0.3, 1.0]), np.array([0, 0.45, 0.8, 1.0]), np.array([0, 0.2, 0.7, 1.1])
    ref = el.Elasticity(p, xv, yv, zv, 0.8, 3.7, dirichlet_faces=MASKS[mask])
    gpu = fdmpc.Elasticity(p, xv, yv, zv, 0.8, 3.7, precision=FP64, omega=1.0, dirichlet_faces=MASKS[mask])
    u = np.random.default_rng(p).standard_normal(3 * ref.N)
    got = N(gpu.apply(T(u)))
    want = ref.apply(u).ravel()
    record("elast_tf_apply_%s_p%d" % (mask, p), relerr=relerr(got, want))
    assert relerr(got, want) <= 1e-12


@pytest.mark.parametrize("p", [2, 5])
def test_star_fdm_equals_fdm_sparse_when_clamped(p):
    """Every face clamped: the star-local FDM and the FDM/sparse relaxation
    invert the same star matrices (FP64 <= 1e-11, FP32 <= 1e-4)."""
    xv, yv, zv = inputs.graded_vertices(3, 75)
    r = T(np.random.default_rng(p).standard_normal(3 * (3 * p + 1) ** 3))
    for prec, tol in ((FP64, 1e-11), (FP32, 1e-4)):
        z = []
        for form in (fdmpc.FDM_SDC_FDM_SPARSE, STAR):
            e = fdmpc.Elasticity(p, xv, yv, zv, 1.0, 10.0, precision=prec, pc=fdmpc.FDM_PC_ASM, omega=0.6,
                                 sdc_form=form)
            z.append(N(e.pc_apply(r)))
            e.close()
        record("elast_star_vs_sparse_p%d_%s" % (p, "fp64" if prec == FP64 else "fp32"), relerr=relerr(z[1], z[0]))
        assert relerr(z[1], z[0]) <= tol


def test_star_fdm_widest_star_when_clamped():
    """p = 15 on 2^3 cells: one star of 29^3 nodes (the FP64 kernel's largest
    shared-memory footprint) against the FDM/sparse relaxation."""
    xv = np.array([0.0, 0.4, 1.0])
    r = T(np.random.default_rng(15).standard_normal(3 * 31 ** 3))
    z = []
    for form in (fdmpc.FDM_SDC_FDM_SPARSE, STAR):
        e = fdmpc.Elasticity(15, xv, xv, xv, 1.0, 3.0, precision=FP64, pc=fdmpc.FDM_PC_ASM, omega=1.0, sdc_form=form)
        z.append(N(e.pc_apply(r)))
        e.close()
    record("elast_star_vs_sparse_p15", relerr=relerr(z[1], z[0]))
    assert relerr(z[1], z[0]) <= 1e-11


@pytest.mark.parametrize("mask", sorted(MASKS))
@pytest.mark.parametrize("pc", [fdmpc.FDM_PC_ASM, fdmpc.FDM_PC_VCYCLE])
def test_traction_free_pc_parity(el, pc, mask):
    xv, yv, zv = inputs.graded_vertices(3, 76)
    ref, gpu = _pair_bc(el, 3, xv, yv, zv, 1.3, 7.0, MASKS[mask], pc=pc, omega=0.7)
    r = rand_free(ref, 4)
    zr = ref.pc_apply(r, pc=1 if pc == fdmpc.FDM_PC_ASM else 2).ravel()
    z = N(gpu.pc_apply(T(r)))
    record("elast_tf_pc%d_%s" % (pc, mask), relerr=relerr(z, zr))
    assert relerr(z, zr) <= 1e-11
    g32 = fdmpc.Elasticity(3, xv, yv, zv, 1.3, 7.0, precision=FP32, pc=pc, omega=0.7, dirichlet_faces=MASKS[mask])
    assert relerr(N(g32.pc_apply(T(r))), zr) <= 1e-4


def test_traction_free_star_p15(el):
    """p = 15 with natural faces: 1 x 1 x 2 cells clamped at x = 0, so the
    stars are 15 x 15 x 15 (traction-free ends) and 15 x 15 x 29 (an interior
    vertex along z), FP64 relaxation against the oracle's dense star solves."""
    xv, yv, zv = np.array([0.0, 1.0]), np.array([0.0, 0.8]), np.array([0.0, 0.5, 1.2])
    ref, gpu = _pair_bc(el, 15, xv, yv, zv, 1.0, 2.0, 1, pc=fdmpc.FDM_PC_ASM, omega=1.0)
    r = rand_free(ref, 5)
    zr = ref.pc_apply(r, pc=1).ravel()
    z = N(gpu.pc_apply(T(r)))
    record("elast_tf_asm_p15", relerr=relerr(z, zr))
    assert relerr(z, zr) <= 1e-11


def test_traction_free_lanczos_and_pcg(el):
    xv, yv, zv = inputs.graded_vertices(3, 77)
    ref, gpu = _pair_bc(el, 2, xv, yv, zv, 1.0, 10.0, 1)
    lo, hi = gpu.lanczos_extremes()
    lo_r, hi_r, om_r = ref.lanczos_omega(inputs.lanczos_start(3 * ref.N))
    assert abs(lo - lo_r) <= 1e-9 * hi_r and abs(hi - hi_r) <= 1e-9 * hi_r
    assert gpu.omega == pytest.approx(om_r, rel=1e-10)
    b = ref.body_force([0.0, -0.02, 0.0]).ravel()
    x_ref, it_ref, conv = ref.pcg(b, rtol=1e-8, maxit=400)
    assert conv
    x, info = gpu.pcg_solve(T(b), rtol=1e-8, maxit=400)
    assert abs(info.iterations - it_ref) <= 1 and info.true_rnorm <= 1e-8 * info.rnorm0
    x2, info2 = gpu.pcg_solve(T(b), rtol=0.0, maxit=it_ref, raise_on_noconv=False)
    assert info2.iterations == it_ref
    record("elast_tf_pcg_fp64", x_relerr=relerr(N(x2), x_ref.ravel()), iterations=it_ref)
    assert relerr(N(x2), x_ref.ravel()) <= 1e-11


@pytest.mark.parametrize("lam", [0.0, 1.0, 10.0, 100.0])
def test_table3_setting_iterations(el, lam):
    """The unit cube clamped at x_1 = 0, traction-free elsewhere, mu = 1, body
    force -0.02 e_2, 4^3 uniform, p = 3: the FP64 GPU solve takes the oracle's
    iteration count (+-1), which reproduces Table 3's printed row; the
    mixed-precision solve at most one more, to a true residual 1e-8."""
    xv = np.linspace(0, 1, 5)
    ref, gpu = _pair_bc(el, 3, xv, xv, xv, 1.0, lam, 1)
    b = ref.body_force([0.0, -0.02, 0.0]).ravel()
    _, it_ref, conv = ref.pcg(b, rtol=1e-8, maxit=800)
    assert conv
    _, info = gpu.pcg_solve(T(b), rtol=1e-8, maxit=800)
    assert abs(info.iterations - it_ref) <= 1
    rec, misses = gpu.recursive_iterations()  # the recursive residual's first 1e-8 comes no later
    assert 0 < rec <= info.iterations and misses >= 0
    mixed = fdmpc.Elasticity(3, xv, xv, xv, 1.0, lam, precision=FP32, dirichlet_faces=1,
                             lanczos_start=inputs.lanczos_start(3 * ref.N))
    _, im = mixed.pcg_solve(T(b), rtol=1e-8, maxit=800)
    record("elast_tf_table3_lam%g" % lam, iterations_fp64=info.iterations, iterations_oracle=it_ref,
           iterations_mixed=im.iterations, true_rel=im.true_rnorm / im.rnorm0)
    assert im.converged and im.true_rnorm <= 1e-8 * im.rnorm0
    assert im.iterations <= info.iterations + 1


def test_traction_free_invalid():
    xv = np.linspace(0, 1, 3)
    for kw in ({"dirichlet_faces": 0}, {"dirichlet_faces": 64},
               {"dirichlet_faces": 1, "sdc_form": fdmpc.FDM_SDC_FDM_SPARSE}, {"sdc_form": 3}):
        with pytest.raises(fdmpc.FdmError) as e:
            fdmpc.Elasticity(2, xv, xv, xv, 1.0, 1.0, **kw)
        assert e.value.code == fdmpc.FDM_EINVAL
