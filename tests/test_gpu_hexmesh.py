"""GPU parity of the general hexahedral mesh path (fdm_hex_*, through the
C-ABI) against the unstructured oracle (oracle/unstructured.py), which numbers
nodes by position and glues its star FDM bases by matching traces, on the
extruded unstructured mesh (vertex valences 3 to 16, randomly oriented cells)
and on the Kershaw-type distorted mesh, with a coefficient at the Gauss
points:

* the stiffness apply <= 1e-12 relative (max norm);
* one FP64 relaxation sweep and the hybrid V(1,1) <= 1e-11; the FP32 sweep
  <= 1e-4 (the FP32 tolerance of the structured path's derivation);
* omega from the device Lanczos against the oracle's with the same start
  vector (<= 1e-10 relative; the extreme eigenvalues <= 1e-9);
* FP64 PCG: iterations within +1 of the oracle's, iterates at equal iteration
  counts <= 1e-11; mixed precision: the true residual <= 1e-8 ||b|| with at
  most one more iteration than FP64;
* a mesh without its numeric set-up is refused (FDM_EINVAL).
Vectors map between the numberings through the cell-local nodes.
"""
import numpy as np
import pytest

from tests.record import record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle.unstructured import HexProblem  # noqa: E402
from paper_2107_14758_gb300 import inputs  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module")
def fdmpc():
    import __graft_entry__ as g
    g.build()
    from paper_2107_14758_gb300 import fdmpc as f
    assert torch.cuda.is_available()
    return f


MESHES = {"unstructured": lambda: inputs.unstructured_hex_mesh(2, 2, 5),
          "kershaw": lambda: inputs.kershaw_like_mesh(4, 0.3)}


def _relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _T(a):
    return torch.tensor(np.ascontiguousarray(a, dtype=np.float64), device=DEV)


def _N(t):
    return t.detach().cpu().numpy()


def _setup(fdmpc, name, p, kappa_seed=None, **kw):
    """(library mesh, oracle problem, node map pi: library node -> oracle dof, kappa)."""
    X, cells = MESHES[name]()
    kappa = None
    if kappa_seed is not None:
        kappa = np.exp(np.random.default_rng(kappa_seed).uniform(-0.5, 0.5, size=(cells.shape[0], (p + 1) ** 3)))
    H = fdmpc.HexMesh(X.shape[0], cells, p)
    H.factor(X, kappa)
    U = HexProblem(p, X, cells, kappa=kappa)
    cn = H.cell_nodes()
    pi = np.zeros(H.nnode, dtype=np.int64)
    pi[cn.ravel()] = U.gid.ravel()
    return H, U, pi


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_stiffness_apply(fdmpc, name, p):
    H, U, pi = _setup(fdmpc, name, p, kappa_seed=p)
    G = fdmpc.HexGpu(H, omega=1.0, pc=fdmpc.FDM_PC_NONE)
    u = np.random.default_rng(10 + p).standard_normal(U.ndof)
    y = _N(G.stiffness_apply(_T(u[pi])))
    want = U.apply(u)[pi]
    record("hex_op_%s_p%d" % (name, p), relerr=_relerr(y, want))
    assert _relerr(y, want) <= 1e-12
    G.close()


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("form", [0, 2])
def test_relaxation_sweep(fdmpc, name, p, form):
    """Both interface-solve forms: the dense inverse of the star's interface
    Schur complement (form 0) and the Schur-coupling form with level-scheduled
    sparse solves (form 2)."""
    H, U, pi = _setup(fdmpc, name, p, kappa_seed=20 + p)
    r = np.random.default_rng(p).standard_normal(U.ndof)
    want = 0.7 * U.asm(r)[pi]
    for prec, tol in ((fdmpc.FDM_PREC_FP64, 1e-11), (fdmpc.FDM_PREC_FP32, 1e-4)):
        G = fdmpc.HexGpu(H, precision=prec, omega=0.7, pc=fdmpc.FDM_PC_ASM, patch_form=form)
        z = _N(G.asm_apply(_T(r[pi])))
        record("hex_asm_%s_p%d_%s_form%d" % (name, p, "fp64" if prec == fdmpc.FDM_PREC_FP64 else "fp32", form),
               relerr=_relerr(z, want))
        assert _relerr(z, want) <= tol
        G.close()


def test_dense_form_on_the_largest_stars(fdmpc):
    """The dense form's widest register column sums (interfaces above 512):
    p = 6 on the m = 3 unstructured mesh (largest interface 571) against the
    Schur-coupling form's sweep (both exact star solves, each pinned to the
    oracle on the meshes above), FP64."""
    X, cells = inputs.unstructured_hex_mesh(3, 2, 5)
    H = fdmpc.HexMesh(X.shape[0], cells, 6)
    H.factor(X)
    r = _T(np.random.default_rng(77).standard_normal(H.nnode))
    out = []
    for form in (0, 2):
        G = fdmpc.HexGpu(H, omega=1.0, pc=fdmpc.FDM_PC_ASM, patch_form=form)
        assert G.sizes()[5] > 512
        out.append(_N(G.asm_apply(r)))
        G.close()
    record("hex_asm_dense_vs_sc_p6", relerr=_relerr(out[0], out[1]))
    assert _relerr(out[0], out[1]) <= 1e-11


@pytest.mark.parametrize("name", sorted(MESHES))
@pytest.mark.parametrize("p", [2, 3])
def test_lanczos_and_vcycle(fdmpc, name, p):
    H, U, pi = _setup(fdmpc, name, p, kappa_seed=30 + p)
    start = inputs.lanczos_start(U.ndof)
    U.setup_patches()
    U.setup_coarse()
    lo, hi, om = U.lanczos_omega(start)
    G = fdmpc.HexGpu(H, lanczos_start=start[pi])
    glo, ghi = G.lanczos_extremes()
    assert abs(G.omega - om) <= 1e-10 * om
    assert abs(glo - lo) <= 1e-9 * hi and abs(ghi - hi) <= 1e-9 * hi
    r = np.random.default_rng(40 + p).standard_normal(U.ndof)
    z = _N(G.pc_apply(_T(r[pi])))
    want = U.pc_apply(r)[pi]
    record("hex_vcycle_%s_p%d" % (name, p), relerr=_relerr(z, want), omega_relerr=abs(G.omega - om) / om)
    assert _relerr(z, want) <= 1e-11
    G.close()


@pytest.mark.parametrize("name", sorted(MESHES))
def test_pcg(fdmpc, name):
    p = 3
    H, U, pi = _setup(fdmpc, name, p)
    start = inputs.lanczos_start(U.ndof)
    U.setup_patches()
    U.setup_coarse()
    U.lanczos_omega(start)
    b = U.mass_apply(np.ones(U.ndof))
    x_ref, it_ref, conv = U.pcg(b, rtol=1e-8, maxit=500)
    assert conv
    G = fdmpc.HexGpu(H, lanczos_start=start[pi])
    x, info = G.pcg_solve(_T(b[pi]), rtol=1e-8, maxit=500)
    assert abs(info.iterations - it_ref) <= 1 and info.true_rnorm <= 1e-8 * info.rnorm0
    x2, info2 = G.pcg_solve(_T(b[pi]), rtol=0.0, maxit=it_ref, raise_on_noconv=False)
    assert info2.iterations == it_ref
    record("hex_pcg_%s" % name, x_relerr=_relerr(_N(x2), x_ref[pi]), iterations=it_ref)
    assert _relerr(_N(x2), x_ref[pi]) <= 1e-11
    M = fdmpc.HexGpu(H, precision=fdmpc.FDM_PREC_FP32, lanczos_start=start[pi])
    xm, im = M.pcg_solve(_T(b[pi]), rtol=1e-8, maxit=500)
    record("hex_pcg_mixed_%s" % name, true_rel=im.true_rnorm / im.rnorm0, iterations=im.iterations)
    assert im.converged and im.true_rnorm <= 1e-8 * im.rnorm0
    assert im.iterations <= info.iterations + 1
    assert _relerr(_N(xm), x_ref[pi]) <= 1e-6
    G.close()
    M.close()


def test_unfactored_mesh_is_refused(fdmpc):
    X, cells = MESHES["unstructured"]()
    H = fdmpc.HexMesh(X.shape[0], cells, 2)
    with pytest.raises(fdmpc.FdmError) as e:
        fdmpc.HexGpu(H)
    assert e.value.code == fdmpc.FDM_EINVAL
