"""Host logic of the library checked without a GPU (compiled with g++ from
the package's own host sources): the patch-class tables of the L and the
Schur-coupling factor forms for p = 1..15, and the multigrid Galerkin
coarsening against the Q1 stiffness assembled directly on each coarsened
graded mesh (nested Q1 spaces make them equal)."""
import os
import shutil
import subprocess

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
                    os.path.join(CSRC, "topology.cpp"), os.path.join(CSRC, "gmg.cpp")], check=True)
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
