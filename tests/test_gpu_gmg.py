"""GPU parity of the geometric multigrid for the Q1 coarse problem (Section 3:
the p-coarse problem is solved by multigrid) against the FP64 oracle, through
the C-ABI.

Tolerances: level operators <= 1e-12 relative (Galerkin products summed in a
different order); FP64 preconditioner applications <= 1e-11 relative; PCG
iterations within +1 of the oracle and iterates <= 1e-10 at equal iteration
counts; the mixed-precision solve reaches the FP64 true residual 1e-8.
"""
import numpy as np
import pytest

from tests.record import record  # noqa: E402

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2107_14758_gb300 import fdmpc, inputs  # noqa: E402
from tests import bruteforce as bf  # noqa: E402

FP64, FP32 = fdmpc.FDM_PREC_FP64, fdmpc.FDM_PREC_FP32
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()


def T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def N(t):
    return t.detach().cpu().numpy()


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def pair(p, xv, yv, zv, levels, jac=None, kappa=None, precision=FP64, nu=2, omega=2.0 / 3.0):
    nd = [(len(v) - 1) * p + 1 for v in (xv, yv, zv)]
    start = inputs.lanczos_start(nd[0] * nd[1] * nd[2])
    ctx = fdmpc.Context(p, xv, yv, zv, jac=jac, kappa=kappa, precision=precision, lanczos_start=start,
                        coarse_levels=levels, gmg_nu=nu, gmg_omega=omega)
    ref = oracle.Problem(p, xv, yv, zv, jac=jac, kappa=kappa)
    ref.setup_patches()
    ref.setup_coarse()
    built = ref.setup_coarse_gmg(levels, nu, omega)
    ref.set_omega(ctx.omega)
    return ctx, ref, built


def free_random(ref, seed):
    m = bf.free_mask(ref.p, ref.nx, ref.ny, ref.nz)
    return np.where(m, np.random.default_rng(seed).standard_normal(ref.ndof), 0.0)


def dense_to_stencil(A, m):
    """[27, nf] stencil of a dense level matrix over m[0] x m[1] x m[2] vertices."""
    nf = m[0] * m[1] * m[2]
    S = np.zeros((27, nf))
    for i in range(nf):
        ix, iy, iz = i % m[0], (i // m[0]) % m[1], i // (m[0] * m[1])
        for k in range(27):
            jx, jy, jz = ix + k % 3 - 1, iy + (k // 3) % 3 - 1, iz + k // 9 - 1
            if 0 <= jx < m[0] and 0 <= jy < m[1] and 0 <= jz < m[2]:
                S[k, i] = A[i, jx + m[0] * (jy + m[1] * jz)]
    return S


def check_levels(ctx, ref, built):
    lev = ctx.gmg_levels()
    assert len(lev) == built + 1
    sts = ctx.gmg_stencils()
    for l, (nx, ny, nz, nf) in enumerate(lev):
        A = ref.gmg_level(l)
        assert A.shape == (nf, nf)
        S = dense_to_stencil(A, (nx - 1, ny - 1, nz - 1))
        assert np.abs(sts[l] - S).max() <= 1e-12 * np.abs(S).max()
        # nothing of the dense matrix lies outside the 27-point stencil
        assert abs(np.abs(A).sum() - np.abs(S).sum()) <= 1e-12 * np.abs(A).sum()


def test_levels_graded():
    xv, yv, zv = inputs.graded_vertices(8, 51)
    ctx, ref, built = pair(3, xv, yv, zv, 5)
    assert built == 2
    assert ctx.gmg_levels() == [(8, 8, 8, 343), (4, 4, 4, 27), (2, 2, 2, 1)]
    check_levels(ctx, ref, built)


def test_levels_anisotropic_box_and_limit():
    # 8 x 4 x 12 cells: 8 -> 4 -> 2 would need 4 -> 2 on y too, 12 -> 6 -> 3 stops all
    xv = np.linspace(0, 1, 9) ** 1.3
    yv = np.linspace(0, 0.5, 5)
    zv = np.linspace(0, 2, 13) ** 1.1
    ctx, ref, built = pair(2, xv, yv, zv, 1)
    assert built == 1 and ctx.gmg_levels()[1][:3] == (4, 2, 6)
    check_levels(ctx, ref, built)


def test_levels_curved_kappa():
    w = inputs.deformed_problem(8, 2, 52)
    ctx, ref, built = pair(w["p"], w["xv"], w["yv"], w["zv"], 3, jac=w["jac"], kappa=w["kappa"])
    assert built == 2
    check_levels(ctx, ref, built)


@pytest.mark.parametrize("nu", [1, 2, 3])
def test_pc_apply_parity(nu):
    xv, yv, zv = inputs.graded_vertices(8, 53)
    ctx, ref, built = pair(3, xv, yv, zv, 2, nu=nu)
    assert built == 2
    r = free_random(ref, 4)
    z = N(ctx.pc_apply(T(r)))
    zr = ref.pc_apply(r)
    assert relerr(z, zr) <= 1e-11


def test_pc_apply_curved_parity():
    w = inputs.deformed_problem(8, 2, 54)
    ctx, ref, built = pair(w["p"], w["xv"], w["yv"], w["zv"], 2, jac=w["jac"], kappa=w["kappa"])
    r = free_random(ref, 5)
    assert relerr(N(ctx.pc_apply(T(r))), ref.pc_apply(r)) <= 1e-11


def test_pcg_parity_fp64():
    xv, yv, zv = inputs.graded_vertices(8, 55)
    ctx, ref, built = pair(4, xv, yv, zv, 2)
    b = free_random(ref, 6)
    x_ref, it_ref, _, conv = ref.pcg(b, rtol=1e-8, maxit=200)
    assert conv
    x, info = ctx.pcg_solve(T(b), rtol=1e-8, maxit=200)
    assert abs(info.iterations - it_ref) <= 1
    x2, info2 = ctx.pcg_solve(T(b), rtol=0.0, maxit=it_ref, raise_on_noconv=False)
    record("gmg_pcg_fp64", x_relerr=relerr(N(x2), x_ref), iterations=it_ref)
    assert relerr(N(x2), x_ref) <= 1e-11


def test_pcg_mixed_precision_and_exact_coarse():
    """FP32 preconditioner with the multigrid coarse solve: converges to the
    FP64 true residual and needs at most two more iterations than the exact
    coarse solve of the same problem."""
    xv, yv, zv = inputs.graded_vertices(8, 56)
    p = 5
    start = inputs.lanczos_start((8 * p + 1) ** 3)
    exact = fdmpc.Context(p, xv, yv, zv, precision=FP32, lanczos_start=start, coarse_levels=0)
    mg = fdmpc.Context(p, xv, yv, zv, precision=FP32, lanczos_start=start, coarse_levels=3)
    assert len(exact.gmg_levels()) == 1 and len(mg.gmg_levels()) == 3
    b = exact.mass_apply(T(inputs.normal_rhs(exact.ndof, 7)))
    _, i0 = exact.pcg_solve(b, rtol=1e-8, maxit=300)
    _, i1 = mg.pcg_solve(b, rtol=1e-8, maxit=300)
    assert i0.converged and i1.converged
    assert i1.true_rnorm <= 1e-8 * i1.rnorm0
    assert i1.iterations <= i0.iterations + 2


def test_auto_rule():
    """Default coarse_levels = -1: exact up to 4096 Q1 unknowns, multigrid above."""
    xv = np.linspace(0, 1, 17)
    small = fdmpc.Context(1, xv, xv, xv, precision=FP64, omega=1.0)           # 15^3 = 3375 unknowns
    assert len(small.gmg_levels()) == 1
    xv = np.linspace(0, 1, 19)
    big = fdmpc.Context(1, xv, xv, xv, precision=FP64, omega=1.0)             # 17^3 = 4913 unknowns
    assert big.gmg_levels() == [(18, 18, 18, 4913), (9, 9, 9, 512)]


def test_mesh_independence_32():
    """32^3 Q3 graded mesh (the exact coarse solve would hold a 29791^2 dense
    inverse): the multigrid coarse solve keeps the PCG iteration count of the
    16^3 problem with the exact coarse solve (within 25 %), mixed precision to
    the FP64 true residual 1e-8."""
    its = []
    for n, levels in ((16, 0), (32, -1)):
        xv, yv, zv = inputs.graded_vertices(n, 57)
        ctx = fdmpc.Context(3, xv, yv, zv, precision=FP32)
        assert (len(ctx.gmg_levels()) > 1) == (levels != 0)
        b = ctx.mass_apply(T(inputs.normal_rhs(ctx.ndof, 8)))
        _, info = ctx.pcg_solve(b, rtol=1e-8, maxit=300)
        assert info.converged and info.true_rnorm <= 1e-8 * info.rnorm0
        its.append(info.iterations)
        del ctx
    assert its[1] <= 1.25 * its[0] + 1, its
