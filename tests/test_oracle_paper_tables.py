"""The oracle against the iteration counts and condition numbers the paper
prints (Tables 1 and 2, Section 3; tests/golden/table1_cartesian_3d.txt and
table2_cartesian_3d.txt): on a Cartesian mesh of the unit cube with f = 1 and
the hybrid V(1,1) with the vertex-star relaxation, PCG reaches a 1e8
reduction in about the same number of iterations for every p, and
kappa(P^{-1} A) is about the same for every p.  The
paper's coarse solver and base mesh differ (the Q1 problem is solved exactly
here), so the check is the trend in p and the size of the count (within two
of the paper's), not the exact number."""
import os

import numpy as np
import pytest

from paper_2107_14758_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_cartesian_3d.txt")


def table1():
    rows = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if line:
            rows[int(line[0])] = [None if v == "-" else int(v) for v in line[1:]]
    return rows


def test_golden_table_is_the_papers():
    t = table1()
    assert t[3] == [12, 12, 12] and t[7] == [12, 12, 12] and t[15] == [12, 13, None]


def test_iterations_flat_in_p_like_table1(oracle_lib):
    paper = table1()
    its = {}
    for p in (3, 7):
        xv, yv, zv = inputs.uniform_vertices(4)
        P = oracle_lib.Problem(p, xv, yv, zv)
        P.setup_patches()
        P.setup_coarse()
        P.lanczos_omega(inputs.lanczos_start(P.ndof))
        b = P.mass_apply(np.ones(P.ndof))
        x, it, _, conv = P.pcg(b, rtol=1e-8, maxit=100)
        assert conv
        its[p] = it
        assert abs(it - paper[p][0]) <= 2, (p, it, paper[p][0])
    assert abs(its[7] - its[3]) <= 1


def table2():
    rows = {}
    for line in open(GOLDEN.replace("table1", "table2")):
        line = line.split("#")[0].split()
        if line:
            rows[int(line[0])] = [None if v == "-" else float(v) for v in line[1:]]
    return rows


def lanczos_extremes(apply_A, apply_P, b, k=40):
    """Extreme eigenvalues of P^{-1} A from k steps of CG-Lanczos started at b
    (the CG coefficients give the Lanczos tridiagonal matrix)."""
    r = b.copy()
    z = apply_P(r)
    d = z.copy()
    rz = r @ z
    al, be = [], []
    for _ in range(k):
        q = apply_A(d)
        a = rz / (d @ q)
        r = r - a * q
        z = apply_P(r)
        rz1 = r @ z
        al.append(a)
        be.append(rz1 / rz)
        rz = rz1
        d = z + be[-1] * d
        if abs(rz) < 1e-28:
            break
    m = len(al)
    T = np.zeros((m, m))
    for j in range(m):
        T[j, j] = 1.0 / al[j] + (be[j - 1] / al[j - 1] if j > 0 else 0.0)
        if j + 1 < m:
            T[j, j + 1] = T[j + 1, j] = np.sqrt(be[j]) / al[j]
    ev = np.linalg.eigvalsh(T)
    return ev[0], ev[-1]


def test_condition_number_flat_in_p_like_table2(oracle_lib):
    """kappa(P^{-1} A) of the hybrid V(1,1) on a uniform 4^3 mesh: of the size
    of Table 2's (2.8 at l = 0; within 1.5 of it here, where the Q1 coarse
    problem is solved exactly) and flat in p (within 20 %)."""
    paper = table2()
    kap = {}
    for p in (3, 7):
        xv, yv, zv = inputs.uniform_vertices(4)
        P = oracle_lib.Problem(p, xv, yv, zv)
        P.setup_patches()
        P.setup_coarse()
        P.lanczos_omega(inputs.lanczos_start(P.ndof))
        b = P.mass_apply(np.ones(P.ndof))
        lo, hi = lanczos_extremes(P.stiffness_apply, P.pc_apply, b)
        kap[p] = hi / lo
        assert lo > 0 and abs(kap[p] - paper[p][0]) <= 1.5, (p, kap[p], paper[p][0])
    assert max(kap.values()) <= 1.2 * min(kap.values())
