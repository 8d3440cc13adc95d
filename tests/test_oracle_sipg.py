"""Pins of the SIPG oracle (Section 5) against what the weak form and the
mathematics fix, independently of the oracle's own formulas:

* the matrix equals explicit 3D quadrature of the weak form in physical
  coordinates (tests/bruteforce.py: physical normals, |e| and |K|);
* symmetric positive definite with eta = p(p+1), also on strongly graded meshes;
* consistency: the discrete solution of a manufactured problem converges
  spectrally in p;
* a star's matrix is the principal submatrix of A on its 8 cells;
* the Q1 functions vanishing on the boundary have no jumps, so P^T A P is the
  conforming Q1 stiffness (the C oracle's coarse matrix and the brute-force Q1
  matrix);
* on a 2 x 2 x 2 mesh the single star covers everything: ASM = A^{-1};
* PCG with the hybrid V(1,1) reaches the dense solution.
"""
import numpy as np
import pytest

from tests import bruteforce as bf
from oracle.sipg import Sipg


MESHES = [
    (1, [0, .4, 1], [0, 1], [0, .3, 1]),
    (2, [0, .3, 1], [0, .6, 1], [0, 1]),
    (3, [0, .2, .5, 1], [0, .45, 1], [0, .7, 1.1]),
]


@pytest.mark.parametrize("p,xv,yv,zv", MESHES)
def test_matrix_is_the_weak_form(p, xv, yv, zv):
    S = Sipg(p, xv, yv, zv)
    A = S.matrix()
    B = bf.dense_sipg(p, xv, yv, zv, S.eta)
    assert np.abs(A - B).max() <= 1e-13 * np.abs(B).max()


def test_penalty_parameter_enters_linearly():
    p, xv, yv, zv = MESHES[1]
    A1 = Sipg(p, xv, yv, zv, eta=3.0).matrix()
    A2 = Sipg(p, xv, yv, zv, eta=7.0).matrix()
    B1 = bf.dense_sipg(p, xv, yv, zv, 3.0)
    B2 = bf.dense_sipg(p, xv, yv, zv, 7.0)
    assert np.abs((A2 - A1) - (B2 - B1)).max() <= 1e-13 * np.abs(B2).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6])
def test_spd_on_graded_mesh(p):
    S = Sipg(p, [0, 0.05, 1], [0, 1], [0, 0.5, 1])
    A = S.matrix()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def _mms(p):
    f = lambda x, y, z: 3 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    S = Sipg(p, [0, .45, 1], [0, .55, 1], [0, .5, 1])
    x = np.linalg.solve(S.matrix(), S.load(f))
    X = S.nodes()
    return np.abs(x - np.sin(np.pi * X[0]) * np.sin(np.pi * X[1]) * np.sin(np.pi * X[2])).max()


def test_manufactured_solution_converges_spectrally():
    err = [_mms(p) for p in (2, 3, 4, 5, 6)]
    for a, b in zip(err, err[1:]):
        assert b < a / 4
    assert err[-1] < 2e-5


def test_load_of_one_is_the_volume():
    S = Sipg(3, [0, .2, 1], [0, .7, 1.5], [0, 2])
    assert S.load(lambda x, y, z: 1.0 + 0 * x).sum() == pytest.approx(3.0, rel=1e-13)


def test_star_matrix_is_principal_submatrix():
    S = Sipg(2, [0, .3, .5, 1], [0, .2, .6, 1.0], [0, .4, .7, 1])
    A = S.matrix()
    for v in S.vertices():
        d = S.patch_dofs(v)
        assert np.abs(S.patch_matrix(v) - A[np.ix_(d, d)]).max() <= 1e-14 * np.abs(A).max()


def test_galerkin_coarse_is_q1_stiffness(oracle_lib):
    import oracle
    xv, yv, zv = [0, .3, .5, 1], [0, .2, .6, 1.0], [0, .4, .7, .9, 1]
    S = Sipg(3, xv, yv, zv)
    S.setup_coarse()
    P = oracle.Problem(1, xv, yv, zv)
    P.setup_coarse()
    Aq = P.coarse_matrix()
    assert np.abs(S.Ac - Aq).max() <= 1e-13 * np.abs(Aq).max()
    free = bf.free_mask(1, 3, 3, 4)
    Q = bf.q1_dense(xv, yv, zv)[np.ix_(free, free)]
    assert np.abs(S.Ac - Q).max() <= 1e-13 * np.abs(Q).max()


def test_prolongation_is_trilinear_interpolation():
    xv, yv, zv = [0, .3, .5, 1], [0, .2, .6, 1.0], [0, .4, .7, 1]
    S = Sipg(2, xv, yv, zv)
    rng = np.random.default_rng(4)
    xc = rng.standard_normal(8)
    u = S.prolong(xc)
    # direct evaluation of the Q1 function at the nodes
    X = np.zeros((4, 4, 4))
    X[1:-1, 1:-1, 1:-1] = xc.reshape(2, 2, 2)
    from scipy.interpolate import RegularGridInterpolator
    f = RegularGridInterpolator((zv, yv, xv), X)
    P = S.nodes()
    assert np.abs(u - f(np.stack([P[2], P[1], P[0]], axis=1))).max() <= 1e-14
    r = rng.standard_normal(S.N)
    assert S.restrict(r) @ xc == pytest.approx(r @ u, rel=1e-13)


def test_single_star_asm_is_the_inverse():
    S = Sipg(3, [0, .4, 1], [0, .55, 1.2], [0, .3, 1])
    A = S.matrix()
    x = np.random.default_rng(1).standard_normal(S.N)
    assert np.abs(S.asm(A @ x) - x).max() <= 1e-10 * np.abs(x).max()


def test_pcg_reaches_the_dense_solution():
    S = Sipg(2, [0, .3, .5, 1], [0, .2, .6, 1.0], [0, .4, .7, 1])
    S.setup_patches()
    S.setup_coarse()
    rng = np.random.default_rng(2)
    lo, hi, om = S.lanczos_omega(rng.standard_normal(S.N))
    assert 0 < lo <= hi and 0 < om < 2 / hi
    b = rng.standard_normal(S.N)
    x, it, conv = S.pcg(b, rtol=1e-10, maxit=100)
    assert conv and it < 40
    xd = np.linalg.solve(S.matrix(), b)
    assert np.abs(x - xd).max() <= 1e-8 * np.abs(xd).max()
