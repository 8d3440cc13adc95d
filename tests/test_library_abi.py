"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, and exports every function that include/fdmpc.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                             src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2107_14758_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("fdm_setup", "stiffness_apply", "pc_apply", "asm_apply", "pcg_solve", "fdm_query",
                     "fdm_destroy", "fdm_last_error", "fdm_batch_setup", "pcg_solve_batched",
                     "fdm_surrogate_load", "fdm_surrogate_train", "fdm_surrogate_grad", "fdm_surrogate_apply",
                     "fdm_elast_setup", "elast_apply", "elast_pc_apply", "elast_pcg_solve", "fdm_elast_query",
                     "fdm_elast_destroy", "fdm_sipg_setup", "sipg_apply", "sipg_asm_apply", "sipg_pc_apply",
                     "sipg_patch_solve", "sipg_pcg_solve", "fdm_sipg_query", "fdm_sipg_last_error",
                     "fdm_sipg_destroy", "stiffness_apply_noalloc", "fdm_hexmesh_create", "fdm_hexmesh_query",
                     "fdm_hexmesh_last_error", "fdm_hexmesh_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_invalid_arguments_rejected_without_gpu(lib):
    from paper_2107_14758_gb300 import fdmpc
    L = fdmpc.load()
    # null mesh and out-of-range degree are rejected on the host before any CUDA call
    h = ctypes.c_void_p()
    assert L.fdm_setup(None, 3, None, None, ctypes.byref(h), None) == fdmpc.FDM_EINVAL
    mesh = fdmpc.fdm_mesh()
    import numpy as np
    v = np.linspace(0, 1, 3)
    mesh.nx = mesh.ny = mesh.nz = 2
    mesh.xv = mesh.yv = mesh.zv = v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.fdm_setup(ctypes.byref(mesh), 16, None, None, ctypes.byref(h), None) == fdmpc.FDM_EINVAL
    assert "p <= 15" in fdmpc.fdm_last_error(None)
    assert L.stiffness_apply(None, None, None, None) == fdmpc.FDM_EINVAL
    w = np.zeros(fdmpc.FDM_MLP_NPARAM, dtype=np.float32)
    wp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    assert L.fdm_surrogate_train(0, None, wp, 10, 1e-3, 0.0, wp, None, None) == fdmpc.FDM_EINVAL
    assert L.fdm_surrogate_apply(None, wp, 1, None, None, None) == fdmpc.FDM_EINVAL
    assert L.fdm_surrogate_grad(None, wp, wp, None, None) == fdmpc.FDM_EINVAL
    o = fdmpc.fdm_default_options()
    assert o.precision == fdmpc.FDM_PREC_FP32 and o.pc == fdmpc.FDM_PC_VCYCLE and o.lanczos_steps == 20
    # elasticity: Lame parameters, degree and curved cells are checked on the host
    for mu, lam, p in ((0.0, 1.0, 3), (1.0, -1.0, 3), (1.0, 1.0, 16), (float("nan"), 1.0, 3)):
        assert L.fdm_elast_setup(ctypes.byref(mesh), p, mu, lam, ctypes.byref(o), ctypes.byref(h), None) == \
            fdmpc.FDM_EINVAL
    jac = np.zeros(9 * 8 * 4 ** 3)
    mesh.jac = jac.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert L.fdm_elast_setup(ctypes.byref(mesh), 3, 1.0, 1.0, ctypes.byref(o), ctypes.byref(h), None) == \
        fdmpc.FDM_EINVAL
    assert "box cells" in L.fdm_elast_last_error(None).decode()
    mesh.jac = None
    # boundary mask and SDC form: no face clamped, bits beyond the six faces, the
    # FDM/sparse form with a traction-free face, an unknown form
    for mask, form in ((0, 0), (64, 0), (1, fdmpc.FDM_SDC_FDM_SPARSE), (63, 3)):
        assert L.fdm_elast_setup_bc(ctypes.byref(mesh), 3, 1.0, 1.0, mask, form, ctypes.byref(o), ctypes.byref(h),
                                    None) == fdmpc.FDM_EINVAL
    assert L.elast_apply(None, None, None, None) == fdmpc.FDM_EINVAL
    assert L.fdm_surrogate_labels(None, fdmpc.FDM_LABEL_PATCH_KAPPA, None, None, None) == fdmpc.FDM_EINVAL
    assert L.fdm_batch_setup_mode(0, None, 7, ctypes.byref(h)) == fdmpc.FDM_EINVAL  # unknown schedule


def test_sipg_and_noalloc_arguments_rejected_without_gpu(lib):
    """SIPG set-up checks the mesh (at least 2 cells per axis, strictly
    increasing vertices, box cells), the degree (1..10) and the penalty on the
    host; every SIPG entry point and the fixed-scratch stiffness apply reject
    a null context or null vectors before any CUDA call."""
    import numpy as np
    from paper_2107_14758_gb300 import fdmpc
    L = fdmpc.load()
    h = ctypes.c_void_p()
    o = fdmpc.fdm_default_options()
    dbl = ctypes.POINTER(ctypes.c_double)

    def mesh_of(xv, yv, zv):
        m = fdmpc.fdm_mesh()
        m.nx, m.ny, m.nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
        m.xv, m.yv, m.zv = (a.ctypes.data_as(dbl) for a in (xv, yv, zv))
        return m

    v3 = np.array([0.0, 0.4, 1.0])
    ok = mesh_of(v3, v3, v3)
    for p, eta in ((0, -1.0), (11, -1.0), (3, float("nan")), (3, float("inf"))):
        assert L.fdm_sipg_setup(ctypes.byref(ok), p, eta, ctypes.byref(o), ctypes.byref(h), None) == \
            fdmpc.FDM_EINVAL
    assert "degree (1..10)" in L.fdm_sipg_last_error(None).decode()
    one = np.array([0.0, 1.0])
    thin = mesh_of(v3, one, v3)  # one cell along y: no interior vertex line
    assert L.fdm_sipg_setup(ctypes.byref(thin), 3, -1.0, ctypes.byref(o), ctypes.byref(h), None) == fdmpc.FDM_EINVAL
    bad = np.array([0.0, 0.6, 0.5])
    dec = mesh_of(v3, bad, v3)
    assert L.fdm_sipg_setup(ctypes.byref(dec), 3, -1.0, ctypes.byref(o), ctypes.byref(h), None) == fdmpc.FDM_EINVAL
    assert "increase strictly" in L.fdm_sipg_last_error(None).decode()
    jac = np.zeros(9 * 8 * 4 ** 3)
    ok.jac = jac.ctypes.data_as(dbl)
    assert L.fdm_sipg_setup(ctypes.byref(ok), 3, -1.0, ctypes.byref(o), ctypes.byref(h), None) == fdmpc.FDM_EINVAL
    assert "box cells" in L.fdm_sipg_last_error(None).decode()
    assert L.fdm_sipg_setup(ctypes.byref(ok), 3, -1.0, ctypes.byref(o), None, None) == fdmpc.FDM_EINVAL
    assert L.sipg_apply(None, None, None, None) == fdmpc.FDM_EINVAL
    assert L.sipg_asm_apply(None, None, None, None) == fdmpc.FDM_EINVAL
    assert L.sipg_pc_apply(None, None, None, None) == fdmpc.FDM_EINVAL
    assert L.sipg_patch_solve(None, None, 0, None, None, None) == fdmpc.FDM_EINVAL
    assert L.sipg_pcg_solve(None, None, None, ctypes.c_double(1e-8), 10, None, None) == fdmpc.FDM_EINVAL
    n = ctypes.c_size_t(8)
    assert L.fdm_sipg_query(None, fdmpc.FDM_Q_NDOF, ctypes.byref(ctypes.c_int64()), ctypes.byref(n)) == \
        fdmpc.FDM_EINVAL
    assert L.stiffness_apply_noalloc(None, None, None, None) == fdmpc.FDM_EINVAL


def test_default_options_match_header(lib):
    """The Python struct mirrors the C layout: the defaults written by the
    library land in the fields of the same names."""
    from paper_2107_14758_gb300 import fdmpc
    o = fdmpc.fdm_default_options()
    assert o.precision == fdmpc.FDM_PREC_FP32 and o.pc == fdmpc.FDM_PC_VCYCLE
    assert o.lanczos_steps == 20 and o.lanczos_seed == 12345 and o.wait_timeout_s == 1.0
    assert o.pcg_graph == 1 and o.autotune == 0 and o.patch_rows_per_warp == 0
    assert o.coarse_levels == -1 and o.gmg_nu == 2 and o.gmg_omega == pytest.approx(2.0 / 3.0, rel=1e-15)


def test_allocation_limit_reports_enomem_without_gpu(lib, monkeypatch):
    """FDM_ALLOC_LIMIT_BYTES caps a context's device memory: a set-up that
    would exceed it returns FDM_ENOMEM before any device call (so the error
    path runs without a GPU), for the scalar, elasticity and SIPG contexts;
    unset, empty, negative or non-numeric values set no limit (the set-up then
    reaches cudaMalloc, which fails here only because there is no GPU)."""
    import numpy as np
    from paper_2107_14758_gb300 import fdmpc
    L = fdmpc.load()
    mesh = fdmpc.fdm_mesh()
    v = np.linspace(0, 1, 3)
    mesh.nx = mesh.ny = mesh.nz = 2
    mesh.xv = mesh.yv = mesh.zv = v.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    o = fdmpc.fdm_default_options()
    for limit in ("0", "100"):
        monkeypatch.setenv("FDM_ALLOC_LIMIT_BYTES", limit)
        assert L.fdm_setup(ctypes.byref(mesh), 2, None, ctypes.byref(o), ctypes.byref(h), None) == fdmpc.FDM_ENOMEM
        assert "FDM_ALLOC_LIMIT_BYTES = %s" % limit in fdmpc.fdm_last_error(None)
        assert L.fdm_elast_setup(ctypes.byref(mesh), 2, 1.0, 1.0, ctypes.byref(o), ctypes.byref(h),
                                 None) == fdmpc.FDM_ENOMEM
        assert "FDM_ALLOC_LIMIT_BYTES" in L.fdm_elast_last_error(None).decode()
        assert L.fdm_sipg_setup(ctypes.byref(mesh), 2, -1.0, ctypes.byref(o), ctypes.byref(h),
                                None) == fdmpc.FDM_ENOMEM
        assert "FDM_ALLOC_LIMIT_BYTES" in L.fdm_sipg_last_error(None).decode()
    import torch
    if torch.cuda.is_available():
        return  # the no-limit case below needs cudaMalloc to fail
    for value in (None, "", "abc", "-5"):
        if value is None:
            monkeypatch.delenv("FDM_ALLOC_LIMIT_BYTES", raising=False)
        else:
            monkeypatch.setenv("FDM_ALLOC_LIMIT_BYTES", value)
        assert L.fdm_setup(ctypes.byref(mesh), 2, None, ctypes.byref(o), ctypes.byref(h), None) == fdmpc.FDM_ENOMEM
        assert "FDM_ALLOC_LIMIT_BYTES" not in fdmpc.fdm_last_error(None)


def test_header_is_plain_c(tmp_path):
    """include/fdmpc.h is a C header: it compiles as pedantic C99 (no torch or
    C++ types in the boundary)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    src = tmp_path / "use_header.c"
    src.write_text('#include "fdmpc.h"\nint main(void) { fdm_options o; fdm_default_options(&o); return o.pc; }\n')
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
