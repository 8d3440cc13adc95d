"""Pins of the oracle's learned-surrogate functions (Section 2.7, Theorem 1).

Each check compares against something other than the oracle itself: finite
differences, closed forms (box and parallelogram cells, the first Adam step),
brute-force grid searches and invariances of the definitions.
"""
import numpy as np
import pytest

import oracle
from paper_2107_14758_gb300 import inputs

NP = oracle.MLP_NPARAM
OFF_B1 = 64 * 189
OFF_W2 = OFF_B1 + 64
OFF_B2 = OFF_W2 + 64 * 64
OFF_W3 = OFF_B2 + 64
OFF_B3 = OFF_W3 + 3 * 64


def test_parameter_count():
    assert NP == 189 * 64 + 64 + 64 * 64 + 64 + 64 * 3 + 3 == 16515


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(7)
    P = rng.standard_normal(NP) * 0.15
    f = rng.standard_normal((7, 189))
    lab = rng.standard_normal((7, 3))
    _, g = oracle.mlp_loss_grad(P, f, lab)
    idx = np.concatenate([rng.choice(OFF_B1, 25, replace=False), OFF_B1 + rng.choice(64, 5, replace=False),
                          OFF_W2 + rng.choice(4096, 15, replace=False), OFF_B2 + rng.choice(64, 5, replace=False),
                          OFF_W3 + rng.choice(192, 10, replace=False), OFF_B3 + np.arange(3)])
    gmax = np.abs(g).max()
    for i in idx:
        h = 1e-6
        Pp = P.copy(); Pp[i] += h
        Pm = P.copy(); Pm[i] -= h
        fd = (oracle.mlp_loss_grad(Pp, f, lab, False)[0] - oracle.mlp_loss_grad(Pm, f, lab, False)[0]) / (2 * h)
        assert abs(g[i] - fd) <= 1e-6 * max(abs(fd), 1e-3 * gmax), (i, g[i], fd)


def test_loss_is_half_mean_square():
    rng = np.random.default_rng(3)
    P = np.zeros(NP)
    P[OFF_B3:] = [0.3, -0.2, 0.1]          # constant output c = b3
    f = rng.standard_normal((5, 189))
    lab = rng.standard_normal((5, 3))
    loss, g = oracle.mlp_loss_grad(P, f, lab)
    r = np.array([0.3, -0.2, 0.1]) - lab
    assert loss == pytest.approx(0.5 * (r ** 2).sum() / 5, rel=1e-14)
    assert np.allclose(g[OFF_B3:], r.mean(axis=0), rtol=1e-13)


def test_forward_closed_form():
    """W1 routes feature k to unit 0, W2 unit 0 to unit 0, W3 unit 0 to output 1."""
    P = np.zeros(NP)
    k = 17
    P[0 * 189 + k] = 1.3
    P[OFF_B1 + 0] = -0.2
    P[OFF_W2 + 0 * 64 + 0] = 0.7
    P[OFF_W3 + 1 * 64 + 0] = 2.0
    P[OFF_B3:] = [0.5, 0.25, -1.0]
    f = np.random.default_rng(1).standard_normal((4, 189))
    c = oracle.mlp_forward(P, f)
    # hidden units other than 0 are tanh(0) = 0
    expect1 = 2.0 * np.tanh(0.7 * np.tanh(1.3 * f[:, k] - 0.2)) + 0.25
    assert np.allclose(c[:, 0], 0.5, rtol=0, atol=0)
    assert np.allclose(c[:, 1], expect1, rtol=1e-15)
    assert np.allclose(c[:, 2], -1.0, rtol=0, atol=0)


def test_adam_steps_closed_form():
    """With a constant gradient the bias-corrected moments are g and g^2 at
    every step, so each step moves a parameter by -lr g / (|g| + eps)."""
    rng = np.random.default_rng(2)
    P = rng.standard_normal(50)
    g = rng.standard_normal(50) * np.logspace(-6, 1, 50)
    m = np.zeros(50); v = np.zeros(50)
    P0 = P.copy()
    for t in range(1, 6):
        oracle.mlp_adam(P, g, m, v, t, 1e-2)
        step = -1e-2 * g / (np.abs(g) + 1e-8)
        assert np.allclose(P - P0, t * step, rtol=1e-10, atol=1e-15)


def test_apply_fallback():
    mubar = np.array([[1.0, 2.0, 3.0]] * 5)
    c = np.array([[0.1, -0.2, 0.3], [np.nan, 0, 0], [0, np.inf, 0], [2.5, 0, 0], [0, 0, -2.0]])
    mu, nf = oracle.surr_apply(mubar, c)
    assert nf == 3
    assert np.allclose(mu[0], mubar[0] * np.exp(c[0]), rtol=1e-15)
    assert np.array_equal(mu[1:4], mubar[1:4])
    assert np.allclose(mu[4], mubar[4] * np.exp(c[4]), rtol=1e-15)   # |c| = 2 is allowed


def _cell_jac(J, p):
    nq = (p + 1) ** 3
    return np.tile(np.asarray(J, dtype=float).reshape(1, 1, 9), (1, nq, 1))


def test_box_cell_surrogate_is_exact():
    """Section 2.2: on a box cell with constant kappa the averaged surrogate is
    the true stiffness: bound ratio 1 (log 0), label c* = 0."""
    p = 3
    J = np.diag([0.3, 0.7, 1.1])
    mubar, cs, F0, F1 = oracle.surr_label(p, _cell_jac(J, p), 2.5 * np.ones((1, (p + 1) ** 3)))
    L = np.diag(J)
    assert np.allclose(mubar[0], 2.5 * L.prod() / L ** 2, rtol=1e-13)
    assert abs(F0[0]) < 1e-13 and abs(F1[0]) < 1e-13
    assert np.allclose(cs, 0.0, atol=1e-13)


@pytest.mark.parametrize("shear", [0.2, 0.6, -0.9])
def test_parallelogram_cell_bound(shear):
    """Sheared (affine) cell: diag(M)^{-1/2} M diag(M)^{-1/2} has the 2x2 block
    [[1, r], [r, 1]] plus 1, so the bound's spectrum is [1 - |r|, 1 + |r|]
    with r the cosine of the angle between the cell's edges' duals (the
    Section 2.7 parallelogram example).  For a 2x2 block diagonal scaling is
    optimal, so the search stays at mu_avg and centring gives
    c* = log(1 - r^2) / 2 in every direction."""
    p = 2
    J = np.array([[1.0, shear, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]]) * 0.5
    Jinv = np.linalg.inv(J)
    M = abs(np.linalg.det(J)) * Jinv @ Jinv.T
    r = M[0, 1] / np.sqrt(M[0, 0] * M[1, 1])
    assert abs(abs(r) - abs(shear) / np.sqrt(1 + shear ** 2)) < 1e-14   # |cos| of the edge angle
    mubar, cs, F0, F1 = oracle.surr_label(p, _cell_jac(J, p))
    expect = np.log((1 + abs(r)) / (1 - abs(r)))
    assert F0[0] == pytest.approx(expect, rel=1e-12)
    assert F1[0] == pytest.approx(expect, rel=1e-12)
    assert np.allclose(cs[0], 0.5 * np.log(1 - r * r), rtol=1e-12)


def _random_cell(p, seed):
    rng = np.random.default_rng(seed)
    nq = (p + 1) ** 3
    jac = (np.eye(3) * 0.5 + 0.15 * rng.standard_normal((nq, 3, 3))).reshape(1, nq, 9)
    kap = np.exp(0.8 * rng.standard_normal((1, nq)))
    return jac, kap


@pytest.mark.parametrize("p,seed", [(1, 1), (1, 2), (1, 4), (2, 6)])
def test_label_matches_grid_search(p, seed):
    """Brute force on tiny cells: the label's bound ratio is no larger than the
    minimum over a grid in (u_y, u_z) (u_x = 0: the ratio is invariant to a
    common scaling) refined around its best point, no larger than every point
    of fine grids around the label itself (local = global minimum for the
    convex ratio), and the centred label has lo * hi = 1."""
    jac, kap = _random_cell(p, seed)
    mubar, cs, F0, F1 = oracle.surr_label(p, jac, kap)
    G, mb2 = oracle.surr_cell_ghat(p, jac, kap)
    assert np.allclose(mb2, mubar, rtol=1e-15)

    def F(u1, u2):
        return oracle.surr_bound(G[0], mubar[0] * np.exp([0.0, u1, u2]))[0]

    best, arg = np.inf, None
    for u1 in np.linspace(-2, 2, 41):
        for u2 in np.linspace(-2, 2, 41):
            f = F(u1, u2)
            if f < best:
                best, arg = f, (u1, u2)
    for h in (0.05, 0.01, 0.002, 0.0004):      # refine around the grid optimum
        c1, c2 = arg
        for u1 in c1 + h * np.arange(-5, 6):
            for u2 in c2 + h * np.arange(-5, 6):
                f = F(u1, u2)
                if f < best:
                    best, arg = f, (u1, u2)
    assert F1[0] <= F0[0] + 1e-15
    assert F1[0] <= best + 1e-9
    u = cs[0] - cs[0][0]
    for h in (1e-3, 1e-5, 1e-7):
        for d1 in h * np.arange(-3, 4):
            for d2 in h * np.arange(-3, 4):
                assert F1[0] <= F(u[1] + d1, u[2] + d2) + 1e-10
    Fc, lo, hi = oracle.surr_bound(G[0], mubar[0] * np.exp(cs[0]))
    assert Fc == pytest.approx(F1[0], abs=1e-12)
    assert lo * hi == pytest.approx(1.0, rel=1e-12)


def test_bound_matches_dense_eigenvalues():
    """lo/hi are the extreme eigenvalues of D^{-1/2} M_q D^{-1/2} over q
    (checked with numpy's symmetric eigensolver)."""
    p = 2
    jac, kap = _random_cell(p, 5)
    G, mubar = oracle.surr_cell_ghat(p, jac, kap)
    mu = mubar[0] * np.array([1.3, 0.8, 1.1])
    lo = np.inf; hi = -np.inf
    for g in G[0]:
        M = np.array([[g[0], g[3], g[4]], [g[3], g[1], g[5]], [g[4], g[5], g[2]]])
        ev = np.linalg.eigvalsh(M / np.sqrt(np.outer(mu, mu)))
        lo, hi = min(lo, ev[0]), max(hi, ev[-1])
    F, l2, h2 = oracle.surr_bound(G[0], mu)
    assert l2 == pytest.approx(lo, rel=1e-13) and h2 == pytest.approx(hi, rel=1e-13)
    assert F == pytest.approx(np.log(hi / lo), rel=1e-13)


def test_ghat_against_quadrature_mass_volume():
    """mubar of a box cell from the general (Jacobian) route equals the box
    formula prod L / L_j^2 (Section 2.2)."""
    p = 4
    L = np.array([0.2, 0.45, 0.7])
    G, mubar = oracle.surr_cell_ghat(p, _cell_jac(np.diag(L), p))
    assert np.allclose(mubar[0], L.prod() / L ** 2, rtol=1e-13)


def test_features_box_cell_and_invariances():
    s27 = inputs.deformed_samples27(3, 4)
    f = oracle.surr_features(s27)
    assert f.shape == (27, 189)
    # a box cell with constant kappa has all-zero inputs
    box = np.zeros((1, 27, 10))
    box[0, :, 0] = 3.0
    box[0, :, 1:] = np.diag([0.1, 0.2, 0.3]).reshape(9)
    assert np.allclose(oracle.surr_features(box), 0.0, atol=1e-14)
    # scaling kappa by a constant and the cell uniformly leaves the inputs unchanged
    s2 = s27.copy()
    s2[:, :, 0] *= 7.5
    s2[:, :, 1:] *= 0.37
    assert np.allclose(oracle.surr_features(s2), f, atol=1e-12)
    # a rigid rotation of the physical coordinates (J -> R J) leaves Ghat unchanged
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1.0]])
    s3 = s27.copy()
    J = s27[:, :, 1:].reshape(-1, 3, 3)
    s3[:, :, 1:] = (R[None] @ J).reshape(27, 27, 9)
    assert np.allclose(oracle.surr_features(s3), f, atol=1e-12)
    # the log-kappa inputs have zero Gauss-weighted mean per cell
    _, w = oracle.gauss(3)
    w27 = np.einsum("k,j,i->kji", w, w, w).reshape(27)
    assert np.allclose(f[:, 0::7] @ w27, 0.0, atol=1e-13)


def test_labels_on_deformed_family():
    """On the deformed workload family the search never increases the bound,
    and the centred labels have lo * hi = 1."""
    w = inputs.deformed_problem(3, 3, 4)
    mubar, cs, F0, F1 = oracle.surr_label(3, w["jac"], w["kappa"])
    assert np.all(F1 <= F0 + 1e-15)
    G, _ = oracle.surr_cell_ghat(3, w["jac"], w["kappa"])
    for e in range(0, 27, 5):
        F, lo, hi = oracle.surr_bound(G[e], mubar[e] * np.exp(cs[e]))
        assert F == pytest.approx(F1[e], abs=1e-12)
        assert lo * hi == pytest.approx(1.0, rel=1e-12)
