"""Pins of the oracle's patch-condition-number labels (oracle/patch_kappa.py):
the learned surrogate's training labels scored by the Lanczos estimate of
kappa(A~_P^{-1} A_P) on each cell's interior patch (Section 2.7, Theorem 1).

Each check compares against something other than the module itself: the C
oracle's sum-factorised stiffness of a one-cell problem, dense generalised
eigenvalues, Theorem 1's bound (computed by the C oracle), the box-cell closed
form and invariances of the definitions.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from oracle import patch_kappa as pk
from paper_2107_14758_gb300 import inputs


def _cell_jac(J, p):
    nq = (p + 1) ** 3
    return np.tile(np.asarray(J, dtype=np.float64).ravel(), (1, nq, 1)).reshape(1, nq, 9)


def _random_cell(p, seed, amp=0.15, kamp=0.8):
    rng = np.random.default_rng(seed)
    nq = (p + 1) ** 3
    jac = (np.eye(3) * 0.5 + amp * rng.standard_normal((nq, 3, 3))).reshape(1, nq, 9)
    kap = np.exp(kamp * rng.standard_normal((1, nq)))
    return jac, kap


def _patches(p, jac, kap=None):
    G, mubar = oracle.surr_cell_ghat(p, jac, kap)
    return pk.CellPatches(p, G, mubar)


@pytest.mark.parametrize("p", [2, 3, 4])
def test_true_matrix_is_the_c_oracle_cell_stiffness(p):
    """A_P equals the one-cell problem's stiffness (the C oracle's sum
    factorisation on its own Gauss rule) on the interior functions."""
    jac, kap = _random_cell(p, 11 + p)
    P = _patches(p, jac, kap)
    prob = oracle.Problem(p, [0.0, 1.0], [0.0, 1.0], [0.0, 1.0], jac=jac, kappa=kap)
    n = p + 1
    inner = [i + n * (j + n * k) for k in range(1, p) for j in range(1, p) for i in range(1, p)]
    A = np.zeros((len(inner), len(inner)))
    for c, g in enumerate(inner):
        u = np.zeros(n ** 3)
        u[g] = 1.0
        A[:, c] = prob.stiffness_apply(u)[inner]
    At = P.true_matrix(0)
    assert np.abs(At - A).max() <= 1e-12 * np.abs(A).max()


def test_box_cell_is_exact():
    """Box cell, constant kappa: the averaged surrogate is the stiffness, so
    kappa = 1 at mubar and the label is 0."""
    p = 3
    P = _patches(p, _cell_jac(np.diag([0.3, 0.7, 1.1]), p), 2.5 * np.ones((1, (p + 1) ** 3)))
    f, lo, hi = P.log_kappa(0, np.zeros(3))
    assert abs(f) < 1e-12 and abs(lo - 1.0) < 1e-12 and abs(hi - 1.0) < 1e-12
    c, f0, f1, _ = P.label(0)
    assert np.abs(c).max() < 1e-12 and abs(f1) < 1e-12


@pytest.mark.parametrize("p,seed", [(2, 1), (3, 2), (4, 3)])
def test_lanczos_extremes_against_dense_eigenvalues(p, seed):
    """Ritz values of the Lanczos matrix lie inside the spectrum of
    A~^{-1} A (Cauchy interlacing) and equal its extremes once the Krylov space
    is the whole patch space."""
    jac, kap = _random_cell(p, seed)
    P = _patches(p, jac, kap)
    A = P.true_matrix(0)
    mu = P.mubar[0] * np.exp(np.array([0.1, -0.3, 0.2]))
    At = P.surrogate_matrix(mu)
    ev = sl.eigh(A, At, eigvals_only=True)
    C = P.symmetric_form(A, mu)  # similar to At^{-1} A: the same spectrum
    assert np.abs(np.linalg.eigvalsh(C) - ev).max() <= 1e-11 * ev[-1]
    lo, hi = P.lanczos(A, mu, steps=8)
    assert ev[0] * (1 - 1e-12) <= lo <= hi <= ev[-1] * (1 + 1e-12)
    lo_f, hi_f = P.lanczos(A, mu, steps=P.m)
    assert lo_f == pytest.approx(ev[0], rel=1e-10) and hi_f == pytest.approx(ev[-1], rel=1e-10)


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_patch_kappa_within_theorem1_bound(seed):
    """Theorem 1 (Section 2.7): lo a~ <= a <= hi a~ on the cell's space, so on
    its interior patch kappa(A~^{-1} A) <= hi / lo (the C oracle's bound), for
    any scalings mu."""
    p = 3
    jac, kap = _random_cell(p, seed)
    P = _patches(p, jac, kap)
    A = P.true_matrix(0)
    G, _ = oracle.surr_cell_ghat(p, jac, kap)
    rng = np.random.default_rng(seed)
    for _ in range(4):
        mu = P.mubar[0] * np.exp(0.4 * rng.standard_normal(3))
        ev = sl.eigh(A, P.surrogate_matrix(mu), eigvals_only=True)
        F, lo, hi = oracle.surr_bound(G[0], mu)
        assert lo * (1 - 1e-12) <= ev[0] and ev[-1] <= hi * (1 + 1e-12)
        assert np.log(ev[-1] / ev[0]) <= F + 1e-12


@pytest.mark.parametrize("p,seed", [(2, 7), (3, 8)])
def test_label_is_a_local_minimum_and_centred(p, seed):
    """The compass search never increases log kappa, ends where no move of the
    smallest step improves it, and the centred label has lambda_min
    lambda_max = 1."""
    jac, kap = _random_cell(p, seed)
    P = _patches(p, jac, kap)
    c, f0, f1, evals = P.label(0)
    assert f1 <= f0 + 1e-15 and evals > 1
    t = c[1:] - c[0]
    s = pk.SEARCH_SMIN
    for dt in ((s, 0.0), (-s, 0.0), (0.0, s), (0.0, -s)):
        f, _, _ = P.log_kappa(0, np.array([0.0, t[0] + dt[0], t[1] + dt[1]]))
        assert f >= f1 - pk.IMPROVE - 1e-12
    f, lo, hi = P.log_kappa(0, c)
    assert f == pytest.approx(f1, abs=1e-12) and lo * hi == pytest.approx(1.0, rel=1e-12)


def test_label_invariant_to_a_constant_coefficient_factor():
    p = 3
    jac, kap = _random_cell(p, 9)
    c1 = _patches(p, jac, kap).label(0)[0]
    c2 = _patches(p, jac, 7.0 * kap).label(0)[0]
    assert np.abs(c1 - c2).max() <= 1e-10


def test_labels_on_deformed_family():
    """On the deformed workload family the labels lower the patch condition
    number of every cell against mubar."""
    w = inputs.deformed_problem(2, 3, 4)
    G, mubar = oracle.surr_cell_ghat(3, w["jac"], w["kappa"])
    c, f0, f1 = _patches(3, w["jac"], w["kappa"]).labels()
    assert c.shape == (8, 3)
    assert np.all(f1 <= f0 + 1e-15) and np.any(f1 < f0 - 1e-3)
