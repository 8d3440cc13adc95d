"""Pins of the oracle's 1D building blocks (Sections 2.1, 2.3, 2.4).

Closed forms, exact polynomial integration and the continuous eigenvalue
limit pin the GLL rule, A_hat/B_hat, the interior eigenproblem and the FDM
basis change independently of the oracle's own arithmetic.
"""
import numpy as np
import pytest

from tests import bruteforce as bf


def test_gauss_closed_forms(oracle_lib):
    x, w = oracle_lib.gauss(2)
    assert np.allclose(x, [-1 / np.sqrt(3), 1 / np.sqrt(3)], atol=1e-15)
    assert np.allclose(w, [1, 1], atol=1e-15)
    x, w = oracle_lib.gauss(3)
    assert np.allclose(x, [-np.sqrt(0.6), 0, np.sqrt(0.6)], atol=1e-15)
    assert np.allclose(w, [5 / 9, 8 / 9, 5 / 9], atol=1e-15)


@pytest.mark.parametrize("p,nodes", [
    (1, [-1, 1]),
    (2, [-1, 0, 1]),
    (3, [-1, -1 / np.sqrt(5), 1 / np.sqrt(5), 1]),
    (4, [-1, -np.sqrt(3 / 7), 0, np.sqrt(3 / 7), 1]),
])
def test_gll_closed_forms(oracle_lib, p, nodes):
    # Section 2.1: roots of (1 - x^2) P_p'(x)
    xi, w = oracle_lib.gll(p)
    assert np.allclose(xi, nodes, atol=1e-15)
    assert abs(w.sum() - 2.0) < 1e-14
    if p == 2:
        assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)


def test_reference_matrices_closed_forms(oracle_lib):
    b = oracle_lib.basis1d(1)
    assert np.allclose(b["A"], 0.5 * np.array([[1, -1], [-1, 1]]), atol=1e-15)
    assert np.allclose(b["B"], np.array([[2, 1], [1, 2]]) / 3, atol=1e-15)
    b = oracle_lib.basis1d(2)
    A2 = np.array([[7, -8, 1], [-8, 16, -8], [1, -8, 7]]) / 6
    B2 = np.array([[4, 2, -1], [2, 16, 2], [-1, 2, 4]]) / 15
    assert np.allclose(b["A"], A2, atol=1e-14)
    assert np.allclose(b["B"], B2, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3, 5, 8, 12])
def test_reference_matrices_vs_exact_integration(oracle_lib, p):
    # exact polynomial integration (well conditioned for small p) and a
    # higher-order Gauss rule on the product-form basis (all p)
    A, B = bf.ref_matrices_quad(p)
    if p <= 5:
        Ae, Be = bf.ref_matrices_exact(p)
        assert np.allclose(A, Ae, atol=1e-12) and np.allclose(B, Be, atol=1e-13)
    b = oracle_lib.basis1d(p)
    assert np.allclose(b["A"], A, rtol=0, atol=1e-11 * np.abs(A).max())
    assert np.allclose(b["B"], B, rtol=0, atol=1e-12)
    assert np.allclose(b["A"].sum(axis=1), 0, atol=1e-11 * np.abs(A).max())   # constants in kernel
    assert abs(b["B"].sum() - 2.0) < 1e-13                                   # int 1 = 2


def test_interior_eigenvalues_closed_forms(oracle_lib):
    # p=2: single bubble 1-x^2: lambda = (8/3)/(16/15) = 5/2
    assert abs(oracle_lib.basis1d(2)["lam"][0] - 2.5) < 1e-13
    # p=3: bubbles (1-x^2) and x(1-x^2): 5/2 and 21/2
    assert np.allclose(oracle_lib.basis1d(3)["lam"], [2.5, 10.5], atol=1e-12)
    # p=4: even pair from the exact 2x2 pencil on {1-x^2, x^2(1-x^2)}, odd 21/2
    K = np.array([[8 / 3, 8 / 15], [8 / 15, 88 / 105]])
    M = np.array([[16 / 15, 16 / 105], [16 / 105, 16 / 315]])
    ev = np.sort(np.linalg.eigvals(np.linalg.solve(M, K)).real)
    assert np.allclose(oracle_lib.basis1d(4)["lam"], np.sort([ev[0], 10.5, ev[1]]), rtol=1e-12)


def test_continuous_limit(oracle_lib):
    # Section 2.3: lambda_j -> j^2 pi^2 / 4 and s_j -> sin(j pi (1+x)/2)
    errs = []
    for p in (7, 11, 15):
        b = oracle_lib.basis1d(p)
        errs.append(abs(b["lam"][0] - np.pi ** 2 / 4))
        xi_int = b["xi"][1:-1]
        for j in (1, 2):
            s = np.sin(j * np.pi * (1 + xi_int) / 2)
            assert np.max(np.abs(b["S"][:, j - 1] - s)) < (1e-3 if p == 7 else 1e-6)
    assert errs[0] < 1e-8 and errs[1] < errs[0] and errs[2] < 1e-12
    lam = oracle_lib.basis1d(15)["lam"]
    assert np.allclose(lam[:4], (np.arange(1, 5) * np.pi / 2) ** 2, rtol=1e-9)


@pytest.mark.parametrize("p", [2, 4, 7, 15])
def test_fdm_basis_properties(oracle_lib, p):
    b = oracle_lib.basis1d(p)
    A, B = bf.ref_matrices_quad(p)
    S, lam, T = b["S"], b["lam"], b["T"]
    I = slice(1, p)
    # eq:eigenproblem: S^T A_II S = Lambda, S^T B_II S = I  (<= 1e-12 relative)
    assert np.allclose(S.T @ B[I, I] @ S, np.eye(p - 1), atol=1e-12)
    assert np.allclose(S.T @ A[I, I] @ S, np.diag(lam), atol=1e-12 * lam.max())
    # Section 2.4: dual basis = vertex evaluation + moments against s_j
    assert T[0, 0] == 1 and T[p, p] == 1 and np.all(T[0, 1:] == 0) and np.all(T[p, :p] == 0)
    Bf = T.T @ B @ T
    Af = T.T @ A @ T
    scale = np.abs(Bf).max()
    assert np.max(np.abs(Bf[I, 0])) < 1e-12 * scale and np.max(np.abs(Bf[I, p])) < 1e-12 * scale
    off = Af[I, I] - np.diag(np.diag(Af[I, I]))
    assert np.max(np.abs(off)) < 1e-12 * np.abs(Af).max()
    # oracle's cleaned matrices agree with these and have exact zeros
    assert np.allclose(b["Af"], Af, atol=1e-11 * np.abs(Af).max())
    assert np.allclose(b["Bf"], Bf, atol=1e-12)
    assert np.all(b["Bf"][I, 0] == 0) and np.all(b["Bf"][I, p] == 0)
    assert np.count_nonzero(b["Af"][I, I] - np.diag(np.diag(b["Af"][I, I]))) == 0
    # the 1D FDM pattern: interior rows of Af have 3 nonzeros (self + 2 vertices)
    for i in range(1, p):
        assert np.count_nonzero(b["Af"][i]) == 3
        assert np.count_nonzero(b["Bf"][i]) == 1


def test_eigenvector_sign_and_order(oracle_lib):
    b = oracle_lib.basis1d(9)
    assert np.all(np.diff(b["lam"]) > 0)
    assert np.all(b["S"][0, :] > 0)


def test_lagrange_cardinality(oracle_lib):
    xi, _ = oracle_lib.gll(6)
    V, D = oracle_lib.lagrange(6, xi, xi)
    assert np.allclose(V, np.eye(7), atol=1e-14)
    Vr, Dr = bf._basis_at(6, np.linspace(-1, 1, 11))
    V2, D2 = oracle_lib.lagrange(6, xi, np.linspace(-1, 1, 11))
    assert np.allclose(V2, Vr, atol=1e-12) and np.allclose(D2, Dr, atol=1e-10)
