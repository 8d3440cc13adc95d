"""The oracle against the iteration counts the paper prints (Table 1, Section
3; tests/golden/table1_cartesian_3d.txt): on a Cartesian mesh of the unit cube
with f = 1 and the hybrid V(1,1) with the vertex-star relaxation, PCG reaches
a 1e8 reduction in about the same number of iterations for every p.  The
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
