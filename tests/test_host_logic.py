"""Host logic of the library checked without a GPU (compiled with g++ from
the package's own host sources): the patch-class tables of the L and the
Schur-coupling factor forms for p = 1..15, and the multigrid Galerkin
coarsening against the Q1 stiffness assembled directly on each coarsened
graded mesh (nested Q1 spaces make them equal), and the SIPG star pencils
(Section 5): their generalized eigendecompositions, and the Kronecker sum of
the three pencils of a star against the oracle's star matrix."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2107_14758_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("host") / "check_host")
    cuda_inc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "include")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", cuda_inc, "-o", out, os.path.join(HERE, "host", "check_host.cpp"),
                    os.path.join(CSRC, "topology.cpp"), os.path.join(CSRC, "gmg.cpp"),
                    os.path.join(CSRC, "basis1d.cpp"), os.path.join(CSRC, "sipg_host.cpp")], check=True)
    return out


def run(checker, what):
    r = subprocess.run([checker, what], capture_output=True, text=True)
    return r.returncode, r.stdout.splitlines()


def test_patch_class_tables(checker):
    rc, lines = run(checker, "topology")
    assert rc == 0, "\n".join(l for l in lines if "ok=0" in l or "FAIL" in l)
    rows = [dict(kv.split("=") for kv in l.split()[1:]) for l in lines if l.startswith("topology")]
    assert len(rows) > 100
    # the interior class (7): the Schur-coupling form stores fewer values from p = 3 on
    for p in range(3, 16):
        sc = [r for r in rows if r["p"] == str(p) and r["sc"] == "1" and r["cls"] == "7"][0]
        lf = [r for r in rows if r["p"] == str(p) and r["sc"] == "0" and r["cls"] == "7"][0]
        assert int(sc["nnzSC"]) < int(lf["nnzL"]) and int(sc["nval"]) < int(lf["nval"])
        assert sc["nG"] == lf["nG"] and sc["n2"] == lf["n2"]
        assert int(sc["nG"]) == 3 * (2 * p - 1) ** 2 - 3 * (2 * p - 1) + 1   # three vertex planes of the star


def test_gmg_galerkin_levels(checker):
    rc, lines = run(checker, "gmg")
    assert rc == 0, "\n".join(lines)
    assert any("levels=2" in l for l in lines)


def sipg_pencil(checker, p, eta, h0, h1, hl, hr):
    r = subprocess.run([checker, "sipg", str(p)] + ["%.17g" % float(x) for x in (eta, h0, h1, hl, hr)],
                       capture_output=True, text=True, check=True)
    import numpy as np
    out = {}
    for line in r.stdout.splitlines():
        k, *v = line.split()
        out[k] = np.array([float(x) for x in v])
    m = 2 * (p + 1)
    for k in ("A", "M", "S"):
        out[k] = out[k].reshape(m, m)
    return out


@pytest.mark.parametrize("p", [1, 3, 7, 10])
def test_sipg_pencil_eigendecomposition(checker, p):
    import numpy as np
    from tests import bruteforce as bf
    P = sipg_pencil(checker, p, p * (p + 1.0), 0.3, 0.07, 0.2, -1.0)
    L = bf.lagrange_polys(bf.gll_nodes(p))
    assert np.allclose(P["dm"], [q.deriv()(-1.0) for q in L], rtol=1e-11, atol=1e-11 * p * p)
    assert np.allclose(P["dp"], [q.deriv()(1.0) for q in L], rtol=1e-11, atol=1e-11 * p * p)
    S, A, M, lam = P["S"], P["A"], P["M"], P["lam"]
    assert np.all(lam > 0)
    assert np.abs(S.T @ M @ S - np.eye(len(lam))).max() <= 1e-11
    assert np.abs(S.T @ A @ S - np.diag(lam)).max() <= 1e-11 * lam.max()


def test_sipg_star_is_kronecker_sum_of_pencils(checker):
    """The star matrix of every vertex of a graded 4 x 3 x 3 mesh (the oracle's
    principal submatrix of A) is Ax (x) My (x) Mz + Mx (x) Ay (x) Mz + Mx (x) My
    (x) Az of the host's pencils, and the fast-diagonalisation inverse built
    from their eigendecompositions inverts it."""
    import numpy as np
    from oracle.sipg import Sipg
    p = 2
    S = Sipg(p, [0, .3, .5, 1, 1.2], [0, .2, .6, 1.0], [0, .4, .7, 1])
    for v in S.vertices():
        pen = []
        for a in range(3):
            k, h = v[a], S.h[a]
            hl = h[k - 2] if k >= 2 else -1.0
            hr = h[k + 1] if k + 1 < S.nc[a] else -1.0
            pen.append(sipg_pencil(checker, p, S.eta, h[k - 1], h[k], hl, hr))
        X, Y, Z = pen
        K = (np.kron(Z["A"], np.kron(Y["M"], X["M"])) + np.kron(Z["M"], np.kron(Y["A"], X["M"])) +
             np.kron(Z["M"], np.kron(Y["M"], X["A"])))
        Av = S.patch_matrix(v)
        assert np.abs(K - Av).max() <= 1e-13 * np.abs(Av).max()
        Sk = np.kron(Z["S"], np.kron(Y["S"], X["S"]))
        D = (Z["lam"][:, None, None] + Y["lam"][None, :, None] + X["lam"][None, None, :]).ravel()
        inv = Sk @ np.diag(1.0 / D) @ Sk.T
        assert np.abs(inv @ Av - np.eye(len(D))).max() <= 1e-10


def _modes_apply(V, lam, mu, U):
    """The pass order of the element-mode box stiffness, in numpy: forward along
    z and y, along x forward, D, backward, then backward along y and z.  U is
    indexed [z, y, x]; V holds the modes by rows (even modes first), of which
    the passes use only the first half of each row, as the kernel does."""
    n = len(lam)
    H, NE = n // 2, (n + 1) // 2

    def fwd(x):
        sp = np.array([x[j] + x[n - 1 - j] for j in range(H)] + ([x[H]] if n % 2 else []))
        dm = np.array([x[j] - x[n - 1 - j] for j in range(H)])
        return np.array([V[k, :NE] @ sp for k in range(NE)] + [V[k, :H] @ dm for k in range(NE, n)])

    def bwd(w):
        x = np.zeros(n)
        for i in range(H):
            e, o = V[:NE, i] @ w[:NE], V[NE:, i] @ w[NE:]
            x[i], x[n - 1 - i] = e + o, e - o
        if n % 2:
            x[H] = V[:NE, H] @ w[:NE]
        return x

    W = U.copy()
    W = np.apply_along_axis(fwd, 0, W)  # z
    W = np.apply_along_axis(fwd, 1, W)  # y
    W = np.apply_along_axis(fwd, 2, W)  # x
    W = W * (mu[0] * lam[None, None, :] + mu[1] * lam[None, :, None] + mu[2] * lam[:, None, None])
    W = np.apply_along_axis(bwd, 2, W)
    W = np.apply_along_axis(bwd, 1, W)
    return np.apply_along_axis(bwd, 0, W)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 10, 15])
def test_library_element_modes(checker, p):
    """The element modes of the FP64 box stiffness (V = S^T B by rows, even
    modes first, with S^T B S = I and A S = B S diag(lam)): V^T diag(lam) V
    reproduces A_hat and V^T V reproduces B_hat, every row is exactly even or
    odd about the element centre, and the kernel's pass order (forward along
    z, y, x, the diagonal mu1 lam_i + mu2 lam_j + mu3 lam_k, backward along x,
    y, z, half rows only) gives the Kronecker form of the box-cell stiffness."""
    r = subprocess.run([checker, "basis", str(p)], capture_output=True, text=True, check=True)
    lib = {}
    for line in r.stdout.splitlines():
        k, *v = line.split()
        lib[k] = np.array([float(x) for x in v])
    n = p + 1
    A, B, V, lam = lib["A"].reshape(n, n), lib["B"].reshape(n, n), lib["Ve"].reshape(n, n), lib["lame"]
    NE = (n + 1) // 2
    assert np.abs(V.T @ np.diag(lam) @ V - A).max() <= 1e-13 * np.abs(A).max()
    assert np.abs(V.T @ V - B).max() <= 1e-14 * np.abs(B).max()
    assert np.array_equal(V[:NE], V[:NE, ::-1]) and np.array_equal(V[NE:], -V[NE:, ::-1])
    assert np.all(np.diff(lam[:NE]) > 0) and np.all(np.diff(lam[NE:]) > 0) and abs(lam[0]) <= 1e-12 * lam.max()
    rng = np.random.default_rng(p)
    U = rng.standard_normal((n, n, n))
    mu = rng.uniform(0.2, 3.0, 3)
    K = (mu[0] * np.kron(B, np.kron(B, A)) + mu[1] * np.kron(B, np.kron(A, B)) + mu[2] * np.kron(A, np.kron(B, B)))
    y = (K @ U.ravel()).reshape(n, n, n)
    assert np.abs(_modes_apply(V, lam, mu, U) - y).max() <= 1e-13 * np.abs(y).max()


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 10, 15])
def test_library_basis_matches_the_oracle(checker, oracle_lib, p):
    """The library's 1D basis (host code, make_basis) against the oracle's:
    GLL rule, exact A_hat and B_hat, the interior eigenbasis (same order and
    sign convention), T, and A_f, B_f with the same exact structural zeros."""
    import numpy as np
    r = subprocess.run([checker, "basis", str(p)], capture_output=True, text=True, check=True)
    lib = {}
    for line in r.stdout.splitlines():
        k, *v = line.split()
        lib[k] = np.array([float(x) for x in v])
    ref = oracle_lib.basis1d(p)
    n, m = p + 1, p - 1
    assert np.abs(lib["xi"] - ref["xi"]).max() <= 1e-14
    for k in ("A", "B", "T", "Af", "Bf"):
        a, b = lib[k].reshape(n, n), ref[k]
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), k
        assert np.array_equal(a == 0.0, b == 0.0), k  # identical exact zeros
    if m > 0:
        assert np.abs(lib["S"].reshape(m, m) - ref["S"]).max() <= 1e-11
        assert np.abs(lib["lam"] - ref["lam"]).max() <= 1e-11 * ref["lam"].max()
