"""Build of the CUDA library libfdmpc.so for sm_103a (in-tree, no cmake)."""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfdmpc.so")
SOURCES = ["api.cu", "k_asm.cu", "k_stream.cu", "k_ops.cu", "k_factor.cu", "k_surr.cu", "k_cell_op.cu", "k_cell_ri.cu", "k_cluster.cu", "k_gmg.cu", "k_elast.cu", "elast.cu", "k_sipg.cu", "sipg.cu", "noalloc.cu", "k_patch_warp.cu", "basis1d.cpp", "topology.cpp", "gmg.cpp", "sipg_host.cpp", "hexmesh.cpp", "partition.cpp", "k_hex.cu", "hexgpu.cu", "k_sipg_tc.cu", "k_star_fdm.cu", "k_surr_kappa.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, ptxas_info=False):
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "fdmpc.h"))
    nvcc = _nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            extra = ["-Xptxas", "-v"] if (ptxas_info and s.endswith(".cu")) else []
            jobs.append([nvcc] + ARCH + FLAGS + extra + ["-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4) or 1) as ex:
        outs = list(ex.map(run, jobs))
    if verbose:
        for o in outs:
            sys.stdout.write(o)
    if jobs or not os.path.exists(LIB):
        tmp = LIB + ".tmp%d" % os.getpid()
        run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
