"""Thin ctypes binding of libfdmpc.so (C-ABI declared in include/fdmpc.h).

Functions carry the C names and only marshal arguments; every step of the
computation runs in the library's CUDA kernels.  Device vectors are passed as
torch CUDA tensors (float64, contiguous) whose data pointers go straight to
the library.  There is no CPU fallback: if the library cannot be loaded or no
GPU is present the calls raise.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdmpc.so")

FDM_OK, FDM_EINVAL, FDM_ENOMEM, FDM_ENOTSPD, FDM_ENOCONV, FDM_ENAN, FDM_ETIMEOUT, FDM_ECUDA = (
    0, -1, -2, -3, -4, -5, -6, -7)
FDM_PREC_FP64, FDM_PREC_FP32 = 0, 1
FDM_PC_NONE, FDM_PC_ASM, FDM_PC_VCYCLE = 0, 1, 2
FDM_SDC_AUTO, FDM_SDC_FDM_SPARSE, FDM_SDC_STAR_FDM = 0, 1, 2
FDM_LABEL_THEOREM1, FDM_LABEL_PATCH_KAPPA = 0, 1
FDM_BATCH_BRANCHES, FDM_BATCH_LOCKSTEP = 0, 1
FDM_SURR_AVERAGED, FDM_SURR_EXTERNAL = 0, 1
(FDM_Q_NDOF, FDM_Q_OMEGA, FDM_Q_LAMBDA, FDM_Q_MU, FDM_Q_NPATCH, FDM_Q_PATCH_CLASS, FDM_Q_CLASS_INFO,
 FDM_Q_GAMMA_ORDER, FDM_Q_FACTOR_NNZ, FDM_Q_PATTERN, FDM_Q_FACTOR, FDM_Q_BASIS, FDM_Q_FACTOR_BYTES,
 FDM_Q_SETUP_SECONDS, FDM_Q_KERNEL_TIMES, FDM_Q_LAUNCHES, FDM_Q_ALGO_BYTES, FDM_Q_STATUS,
 FDM_Q_SURR_FEATURES, FDM_Q_SURR_LABELS, FDM_Q_SURR_BOUNDS, FDM_Q_MUBAR, FDM_Q_SURR_OUTPUT, FDM_Q_TUNING,
 FDM_Q_GMG_LEVELS, FDM_Q_GMG_STENCIL, FDM_Q_ALGO_BYTES_LFORM, FDM_Q_RECURSIVE_ITS) = range(1, 29)
(FDM_HQ_NNODE, FDM_HQ_CELL_NODES, FDM_HQ_CELL_FDM, FDM_HQ_CELL_SIGN, FDM_HQ_DIRICHLET, FDM_HQ_NSTAR,
 FDM_HQ_STAR_VERTEX, FDM_HQ_STAR_PTR, FDM_HQ_STAR_NODES, FDM_HQ_PATTERN_PTR, FDM_HQ_PATTERN_ROWPTR,
 FDM_HQ_PATTERN_COLPTR, FDM_HQ_PATTERN_COLS, FDM_HQ_STAR_NINT, FDM_HQ_STAR_CLASS, FDM_HQ_NCLASS,
 FDM_HQ_CLASS_STAR, FDM_HQ_CLASS_NNZL, FDM_HQ_FILL_PTR, FDM_HQ_FILL_ROWPTR, FDM_HQ_FILL_COLPTR, FDM_HQ_FILL_COLS,
 FDM_HQ_ETREE_PTR, FDM_HQ_ETREE, FDM_HQ_MU, FDM_HQ_DIAG_PTR, FDM_HQ_DIAG, FDM_HQ_FACTOR_PTR,
 FDM_HQ_FACTOR, FDM_HQ_SLOT_CELLS_PTR, FDM_HQ_SLOT_CELLS, FDM_HQ_SLOT_STARS_PTR, FDM_HQ_SLOT_STARS,
 FDM_HQ_NODE_OWNER, FDM_HQ_NODE_CELLS_PTR, FDM_HQ_NODE_CELLS, FDM_HQ_GEOM, FDM_HQ_COARSE_OF,
 FDM_HQ_COARSE, FDM_HQ_SC_SPLIT, FDM_HQ_SC_PTR, FDM_HQ_SC_ROWPTR, FDM_HQ_SC_COLPTR, FDM_HQ_SC_COLS,
 FDM_HQ_SC_VALUES_PTR, FDM_HQ_SC_VALUES) = range(1, 47)
FDM_XQ_NNODE, FDM_XQ_OMEGA, FDM_XQ_LAMBDA, FDM_XQ_LAUNCHES, FDM_XQ_SIZES, FDM_XQ_ALGO_BYTES = range(1, 7)
(FDM_PQ_CELL_BOX, FDM_PQ_NODE_BOX, FDM_PQ_HALO_BOX, FDM_PQ_NNEIGH, FDM_PQ_NEIGHBORS, FDM_PQ_SEND_PTR, FDM_PQ_SEND,
 FDM_PQ_RECV_PTR, FDM_PQ_SUM_PTR, FDM_PQ_SUM, FDM_PQ_OWNED, FDM_PQ_STARS) = range(1, 13)
FDM_MLP_NPARAM = 16515
TIMERS = ("restrict", "patch", "interp", "op64", "op32", "coarse", "vec")


class fdm_mesh(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("xv", C.POINTER(C.c_double)), ("yv", C.POINTER(C.c_double)), ("zv", C.POINTER(C.c_double)),
                ("jac", C.POINTER(C.c_double))]


class fdm_coeff(C.Structure):
    _fields_ = [("kappa_q", C.POINTER(C.c_double)), ("samples27", C.POINTER(C.c_double)),
                ("mu", C.POINTER(C.c_double))]


class fdm_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("pc", C.c_int), ("surrogate", C.c_int), ("lanczos_steps", C.c_int),
                ("omega", C.c_double), ("lanczos_seed", C.c_uint64), ("flexible_beta", C.c_int),
                ("wait_timeout_s", C.c_double), ("lanczos_start", C.POINTER(C.c_double)),
                ("kernel_timing", C.c_int), ("patch_ctas_per_sm", C.c_int), ("patch_threads", C.c_int),
                ("patch_kernel", C.c_int), ("stream_buffers", C.c_int), ("stream_buffer_kb", C.c_int),
                ("inject_stall", C.c_int), ("patch_prefetch", C.c_int), ("pcg_graph", C.c_int),
                ("patch_l2_hints", C.c_int), ("autotune", C.c_int), ("patch_rows_per_warp", C.c_int),
                ("patch_form", C.c_int), ("coarse_levels", C.c_int), ("gmg_nu", C.c_int),
                ("gmg_omega", C.c_double), ("sc_variant", C.c_int), ("tensor_core", C.c_int)]


class fdm_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("rnorm0", C.c_double), ("rnorm", C.c_double),
                ("true_rnorm", C.c_double), ("seconds", C.c_double)]


class FdmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("fdmpc error %d: %s" % (code, msg))
        self.code = code


_lib = None


def load():
    """Load libfdmpc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfdmpc.so is not built; run __graft_entry__.build()")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int)
    L.fdm_default_options.argtypes = [C.POINTER(fdm_options)]
    L.fdm_setup.argtypes = [C.POINTER(fdm_mesh), C.c_int, C.POINTER(fdm_coeff), C.POINTER(fdm_options),
                            C.POINTER(vp), vp]
    for f in ("stiffness_apply", "stiffness_apply_noalloc", "mass_apply", "asm_apply", "pc_apply"):
        getattr(L, f).argtypes = [vp, vp, vp, vp]
    L.pcg_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.POINTER(fdm_solve_info), vp]
    L.fdm_batch_setup.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(vp)]
    L.fdm_batch_setup_mode.argtypes = [C.c_int, C.POINTER(vp), C.c_int, C.POINTER(vp)]
    L.pcg_solve_batched.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.c_double, C.c_int,
                                    C.POINTER(fdm_solve_info), vp]
    L.fdm_batch_destroy.argtypes = [vp]
    L.fdm_batch_destroy.restype = None
    L.fdm_surrogate_load.argtypes = [vp, dp, vp]
    fp = C.POINTER(C.c_float)
    L.fdm_surrogate_grad.argtypes = [vp, fp, fp, dp, vp]
    L.fdm_surrogate_train.argtypes = [C.c_int, C.POINTER(vp), fp, C.c_int, C.c_double, C.c_double, fp, dp, vp]
    L.fdm_surrogate_labels.argtypes = [vp, C.c_int, dp, dp, vp]
    L.fdm_surrogate_apply.argtypes = [vp, fp, C.c_int, ip, ip, vp]
    L.fdm_query.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_size_t)]
    L.fdm_last_error.argtypes = [vp]
    L.fdm_last_error.restype = C.c_char_p
    L.fdm_destroy.argtypes = [vp]
    L.fdm_destroy.restype = None
    L.fdm_elast_setup.argtypes = [C.POINTER(fdm_mesh), C.c_int, C.c_double, C.c_double, C.POINTER(fdm_options),
                                  C.POINTER(vp), vp]
    L.fdm_elast_setup_bc.argtypes = [C.POINTER(fdm_mesh), C.c_int, C.c_double, C.c_double, C.c_int, C.c_int,
                                     C.POINTER(fdm_options), C.POINTER(vp), vp]
    for f in ("elast_apply", "elast_pc_apply"):
        getattr(L, f).argtypes = [vp, vp, vp, vp]
    L.elast_pcg_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.POINTER(fdm_solve_info), vp]
    L.fdm_elast_query.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_size_t)]
    L.fdm_elast_last_error.argtypes = [vp]
    L.fdm_elast_last_error.restype = C.c_char_p
    L.fdm_elast_destroy.argtypes = [vp]
    L.fdm_elast_destroy.restype = None
    L.fdm_sipg_setup.argtypes = [C.POINTER(fdm_mesh), C.c_int, C.c_double, C.POINTER(fdm_options), C.POINTER(vp), vp]
    for f in ("sipg_apply", "sipg_asm_apply", "sipg_pc_apply"):
        getattr(L, f).argtypes = [vp, vp, vp, vp]
    L.sipg_patch_solve.argtypes = [vp, vp, C.c_int, ip, vp, vp]
    L.sipg_pcg_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.POINTER(fdm_solve_info), vp]
    L.fdm_sipg_query.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_size_t)]
    L.fdm_sipg_last_error.argtypes = [vp]
    L.fdm_sipg_last_error.restype = C.c_char_p
    L.fdm_sipg_destroy.argtypes = [vp]
    L.fdm_sipg_destroy.restype = None
    L.fdm_hexmesh_create.argtypes = [C.c_int, C.c_int, ip, C.c_int, C.POINTER(vp)]
    L.fdm_hexmesh_create_bc.argtypes = [C.c_int, C.c_int, ip, C.c_int, vp, C.POINTER(vp)]
    L.fdm_hexmesh_factor_axes.argtypes = [vp, C.c_int, dp, dp, dp]
    L.fdm_hexmesh_query.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_size_t)]
    L.fdm_hexmesh_factor.argtypes = [vp, C.c_int, dp, dp]
    L.fdm_hexmesh_last_error.argtypes = [vp]
    L.fdm_hexmesh_last_error.restype = C.c_char_p
    L.fdm_hexmesh_destroy.argtypes = [vp]
    L.fdm_hexmesh_destroy.restype = None
    L.fdm_hex_setup.argtypes = [vp, C.POINTER(fdm_options), C.POINTER(vp), vp]
    for f in ("hex_stiffness_apply", "hex_asm_apply", "hex_pc_apply"):
        getattr(L, f).argtypes = [vp, vp, vp, vp]
    L.hex_pcg_solve.argtypes = [vp, vp, vp, C.c_double, C.c_int, C.POINTER(fdm_solve_info), vp]
    L.fdm_hex_query.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_size_t)]
    L.fdm_hex_last_error.argtypes = [vp]
    L.fdm_hex_last_error.restype = C.c_char_p
    L.fdm_hex_destroy.argtypes = [vp]
    L.fdm_hex_destroy.restype = None
    L.fdm_partition_create.argtypes = [C.c_int] * 8 + [C.POINTER(vp)]
    L.fdm_partition_query.argtypes = [vp, C.c_int, vp, C.POINTER(C.c_size_t)]
    L.fdm_partition_last_error.argtypes = []
    L.fdm_partition_last_error.restype = C.c_char_p
    L.fdm_partition_destroy.argtypes = [vp]
    L.fdm_partition_destroy.restype = None
    _lib = L
    return L


def _check(rc, ctx=None):
    if rc < 0:
        raise FdmError(rc, load().fdm_last_error(ctx).decode())
    return rc


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _tptr(t):
    import torch
    assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous(), "need a contiguous CUDA float64 tensor"
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream)


# ---- C-ABI functions under their own names -------------------------------

def fdm_default_options():
    o = fdm_options()
    _check(load().fdm_default_options(C.byref(o)))
    return o


def fdm_setup(mesh, p, coeff, opt, stream=None):
    h = C.c_void_p()
    _check(load().fdm_setup(C.byref(mesh), p, C.byref(coeff) if coeff is not None else None,
                            C.byref(opt) if opt is not None else None, C.byref(h), _stream(stream)))
    return h


def stiffness_apply(ctx, u, y, stream=None):
    _check(load().stiffness_apply(ctx, _tptr(u), _tptr(y), _stream(stream)), ctx)


def stiffness_apply_noalloc(ctx, u, y, stream=None):
    _check(load().stiffness_apply_noalloc(ctx, _tptr(u), _tptr(y), _stream(stream)), ctx)


def mass_apply(ctx, f, b, stream=None):
    _check(load().mass_apply(ctx, _tptr(f), _tptr(b), _stream(stream)), ctx)


def asm_apply(ctx, r, z, stream=None):
    _check(load().asm_apply(ctx, _tptr(r), _tptr(z), _stream(stream)), ctx)


def pc_apply(ctx, r, z, stream=None):
    _check(load().pc_apply(ctx, _tptr(r), _tptr(z), _stream(stream)), ctx)


def pcg_solve(ctx, b, x, rtol, maxit, stream=None, raise_on_noconv=True):
    info = fdm_solve_info()
    rc = load().pcg_solve(ctx, _tptr(b), _tptr(x), rtol, maxit, C.byref(info), _stream(stream))
    if rc == FDM_ENOCONV and not raise_on_noconv:
        return info
    _check(rc, ctx)
    return info


def _check_elast(rc, e=None):
    if rc < 0:
        raise FdmError(rc, load().fdm_elast_last_error(e).decode())
    return rc


def fdm_elast_setup(mesh, p, mu, lam, opt, stream=None):
    h = C.c_void_p()
    _check_elast(load().fdm_elast_setup(C.byref(mesh), p, mu, lam, C.byref(opt), C.byref(h), _stream(stream)))
    return h


def fdm_elast_setup_bc(mesh, p, mu, lam, dirichlet_faces, sdc_form, opt, stream=None):
    h = C.c_void_p()
    _check_elast(load().fdm_elast_setup_bc(C.byref(mesh), p, mu, lam, dirichlet_faces, sdc_form, C.byref(opt),
                                           C.byref(h), _stream(stream)))
    return h


def elast_apply(e, u, y, stream=None):
    _check_elast(load().elast_apply(e, _tptr(u), _tptr(y), _stream(stream)), e)


def elast_pc_apply(e, r, z, stream=None):
    _check_elast(load().elast_pc_apply(e, _tptr(r), _tptr(z), _stream(stream)), e)


def elast_pcg_solve(e, b, x, rtol, maxit, stream=None, raise_on_noconv=True):
    info = fdm_solve_info()
    rc = load().elast_pcg_solve(e, _tptr(b), _tptr(x), rtol, maxit, C.byref(info), _stream(stream))
    if rc == FDM_ENOCONV and not raise_on_noconv:
        return info
    _check_elast(rc, e)
    return info


def fdm_elast_query(e, what, out):
    n = C.c_size_t(out.nbytes)
    _check_elast(load().fdm_elast_query(e, what, out.ctypes.data_as(C.c_void_p), C.byref(n)), e)
    return n.value


def fdm_elast_destroy(e):
    load().fdm_elast_destroy(e)


def _check_sipg(rc, s=None):
    if rc < 0:
        raise FdmError(rc, load().fdm_sipg_last_error(s).decode())
    return rc


def fdm_sipg_setup(mesh, p, eta, opt, stream=None):
    h = C.c_void_p()
    _check_sipg(load().fdm_sipg_setup(C.byref(mesh), p, eta, C.byref(opt), C.byref(h), _stream(stream)))
    return h


def sipg_apply(s, u, y, stream=None):
    _check_sipg(load().sipg_apply(s, _tptr(u), _tptr(y), _stream(stream)), s)


def sipg_asm_apply(s, r, z, stream=None):
    _check_sipg(load().sipg_asm_apply(s, _tptr(r), _tptr(z), _stream(stream)), s)


def sipg_pc_apply(s, r, z, stream=None):
    _check_sipg(load().sipg_pc_apply(s, _tptr(r), _tptr(z), _stream(stream)), s)


def sipg_patch_solve(s, r, vertices, out, stream=None):
    v = np.ascontiguousarray(vertices, dtype=np.int32)
    _check_sipg(load().sipg_patch_solve(s, _tptr(r), len(v), v.ctypes.data_as(C.POINTER(C.c_int)), _tptr(out),
                                        _stream(stream)), s)


def sipg_pcg_solve(s, b, x, rtol, maxit, stream=None, raise_on_noconv=True):
    info = fdm_solve_info()
    rc = load().sipg_pcg_solve(s, _tptr(b), _tptr(x), rtol, maxit, C.byref(info), _stream(stream))
    if rc == FDM_ENOCONV and not raise_on_noconv:
        return info
    _check_sipg(rc, s)
    return info


def fdm_sipg_query(s, what, out):
    n = C.c_size_t(out.nbytes)
    _check_sipg(load().fdm_sipg_query(s, what, out.ctypes.data_as(C.c_void_p), C.byref(n)), s)
    return n.value


def fdm_sipg_destroy(s):
    load().fdm_sipg_destroy(s)


def fdm_batch_setup(ctxs, mode=None):
    """A batch of the contexts; mode FDM_BATCH_BRANCHES (default) or FDM_BATCH_LOCKSTEP."""
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    h = C.c_void_p()
    if mode is None:
        _check(load().fdm_batch_setup(len(ctxs), arr, C.byref(h)))
    else:
        _check(load().fdm_batch_setup_mode(len(ctxs), arr, mode, C.byref(h)))
    return h


def pcg_solve_batched(batch, bs, xs, rtol, maxit, stream=None, check=True):
    """Solves the batch's problems (one CUDA graph); returns the infos, or
    (return code, infos) with check=False."""
    k = len(bs)
    for t in list(bs) + list(xs):
        _tptr(t)
    barr = (C.c_void_p * k)(*[b.data_ptr() for b in bs])
    xarr = (C.c_void_p * k)(*[x.data_ptr() for x in xs])
    infos = (fdm_solve_info * k)()
    rc = load().pcg_solve_batched(batch, barr, xarr, rtol, maxit, infos, _stream(stream))
    if not check:
        return rc, list(infos)
    _check(rc)
    return list(infos)


def fdm_batch_destroy(batch):
    load().fdm_batch_destroy(batch)


def fdm_surrogate_load(ctx, mu, stream=None):
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    _check(load().fdm_surrogate_load(ctx, _dptr(mu), _stream(stream)), ctx)


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _weights(w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    assert w.size == FDM_MLP_NPARAM, "network weights: %d floats" % FDM_MLP_NPARAM
    return w


def fdm_surrogate_grad(ctx, w, stream=None):
    """(gradient float32[FDM_MLP_NPARAM], loss) of the surrogate network."""
    w = _weights(w)
    g = np.zeros(FDM_MLP_NPARAM, dtype=np.float32)
    loss = C.c_double()
    _check(load().fdm_surrogate_grad(ctx, _fptr(w), _fptr(g), C.byref(loss), _stream(stream)), ctx)
    return g, loss.value


def fdm_surrogate_labels(ctx, ncell, kind, stream=None):
    """(labels [ncell][3], score [2][ncell]) of the label kind FDM_LABEL_*,
    which becomes the context's training labels."""
    lab = np.zeros((ncell, 3))
    score = np.zeros((2, ncell))
    _check(load().fdm_surrogate_labels(ctx, kind, _dptr(lab), _dptr(score), _stream(stream)), ctx)
    return lab, score


def fdm_surrogate_train(ctxs, w_init, steps, lr, weight_decay=0.0, stream=None):
    """Trains on every cell of the contexts; returns (weights, loss history)."""
    w = _weights(w_init)
    out = np.zeros(FDM_MLP_NPARAM, dtype=np.float32)
    hist = np.zeros(steps + 1)
    arr = (C.c_void_p * len(ctxs))(*[c.value for c in ctxs])
    _check(load().fdm_surrogate_train(len(ctxs), arr, _fptr(w), steps, lr, weight_decay, _fptr(out), _dptr(hist),
                                      _stream(stream)), ctxs[0])
    return out, hist


def fdm_surrogate_apply(ctx, w, judge=1, stream=None):
    """Inference + refactorisation; returns (fallback cells, kept)."""
    w = _weights(w)
    nf = C.c_int(); kept = C.c_int()
    _check(load().fdm_surrogate_apply(ctx, _fptr(w), judge, C.byref(nf), C.byref(kept), _stream(stream)), ctx)
    return nf.value, bool(kept.value)


def fdm_query(ctx, what, out, arg=None):
    """Copies quantity `what` into the numpy array `out` (HOST); returns bytes."""
    if arg is not None:
        assert out.nbytes >= 4
        out.reshape(-1).view(np.uint8)[:4] = np.frombuffer(np.int32(arg).tobytes(), dtype=np.uint8)
    n = C.c_size_t(out.nbytes)
    _check(load().fdm_query(ctx, what, out.ctypes.data_as(C.c_void_p), C.byref(n)), ctx)
    return n.value


def fdm_last_error(ctx=None):
    return load().fdm_last_error(ctx).decode()


def fdm_destroy(ctx):
    load().fdm_destroy(ctx)


# ---- convenience wrapper ---------------------------------------------------

class Context:
    """Owns one set-up problem (a fdm_ctx) and its host inputs."""

    def __init__(self, p, xv, yv, zv, jac=None, kappa=None, samples27=None, precision=FDM_PREC_FP32, pc=FDM_PC_VCYCLE,
                 omega=0.0, lanczos_start=None, lanczos_steps=20, flexible_beta=-1, kernel_timing=0,
                 patch_ctas_per_sm=0, patch_threads=0, patch_kernel=0, stream_buffers=0, stream_buffer_kb=0,
                 inject_stall=0, wait_timeout_s=1.0, patch_prefetch=0, pcg_graph=1, patch_l2_hints=0, autotune=0, patch_rows_per_warp=0,
                 coarse_levels=-1, gmg_nu=2, gmg_omega=2.0 / 3.0, patch_form=0, sc_variant=0, stream=None):
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (xv, yv, zv)]
        mesh = fdm_mesh()
        mesh.nx, mesh.ny, mesh.nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
        mesh.xv, mesh.yv, mesh.zv = [_dptr(a) for a in self._keep]
        coeff = fdm_coeff()
        if jac is not None:
            j = np.ascontiguousarray(jac, dtype=np.float64)
            self._keep.append(j)
            mesh.jac = _dptr(j)
        if kappa is not None:
            k = np.ascontiguousarray(kappa, dtype=np.float64)
            self._keep.append(k)
            coeff.kappa_q = _dptr(k)
        if samples27 is not None:
            s27 = np.ascontiguousarray(samples27, dtype=np.float64)
            self._keep.append(s27)
            coeff.samples27 = _dptr(s27)
        opt = fdm_default_options()
        opt.precision, opt.pc, opt.omega, opt.lanczos_steps = precision, pc, omega, lanczos_steps
        opt.flexible_beta = flexible_beta
        opt.kernel_timing = kernel_timing
        opt.patch_ctas_per_sm = patch_ctas_per_sm
        opt.patch_threads = patch_threads
        opt.patch_kernel = patch_kernel
        opt.stream_buffers = stream_buffers
        opt.stream_buffer_kb = stream_buffer_kb
        opt.inject_stall = inject_stall
        opt.patch_prefetch = patch_prefetch
        opt.pcg_graph = pcg_graph
        opt.patch_l2_hints = patch_l2_hints
        opt.autotune = autotune
        opt.patch_rows_per_warp = patch_rows_per_warp
        opt.coarse_levels, opt.gmg_nu, opt.gmg_omega = coarse_levels, gmg_nu, gmg_omega
        opt.patch_form = patch_form
        opt.sc_variant = sc_variant
        opt.wait_timeout_s = wait_timeout_s
        if lanczos_start is not None:
            s = np.ascontiguousarray(lanczos_start, dtype=np.float64)
            self._keep.append(s)
            opt.lanczos_start = _dptr(s)
        self.p = p
        self.nx, self.ny, self.nz = mesh.nx, mesh.ny, mesh.nz
        self.N = (mesh.nx * p + 1, mesh.ny * p + 1, mesh.nz * p + 1)
        self.ndof = self.N[0] * self.N[1] * self.N[2]
        self.ncell = mesh.nx * mesh.ny * mesh.nz
        self.h = fdm_setup(mesh, p, coeff, opt, stream)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            fdm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, like):
        import torch
        return torch.empty(self.ndof, dtype=torch.float64, device=like.device)

    def stiffness_apply(self, u, y=None):
        y = self._out(u) if y is None else y
        stiffness_apply(self.h, u, y)
        return y

    def mass_apply(self, f, b=None):
        b = self._out(f) if b is None else b
        mass_apply(self.h, f, b)
        return b

    def asm_apply(self, r, z=None):
        z = self._out(r) if z is None else z
        asm_apply(self.h, r, z)
        return z

    def pc_apply(self, r, z=None):
        z = self._out(r) if z is None else z
        pc_apply(self.h, r, z)
        return z

    def pcg_solve(self, b, x=None, rtol=1e-8, maxit=200, raise_on_noconv=True):
        x = self._out(b) if x is None else x
        info = pcg_solve(self.h, b, x, rtol, maxit, raise_on_noconv=raise_on_noconv)
        return x, info

    def surrogate_load(self, mu):
        fdm_surrogate_load(self.h, mu)

    def surrogate_grad(self, w):
        return fdm_surrogate_grad(self.h, w)

    def surrogate_apply(self, w, judge=1):
        return fdm_surrogate_apply(self.h, w, judge)

    def surrogate_features(self):
        return self.query(FDM_Q_SURR_FEATURES, np.float32, 189 * self.ncell).reshape(self.ncell, 189)

    def surrogate_labels(self):
        return self.query(FDM_Q_SURR_LABELS, np.float64, 3 * self.ncell).reshape(self.ncell, 3)

    def select_labels(self, kind):
        """Computes and selects the training labels of kind FDM_LABEL_*:
        (labels [ncell][3], score [2][ncell] at mu_avg and at the label)."""
        return fdm_surrogate_labels(self.h, self.ncell, kind)

    def surrogate_bounds(self):
        """(F at mu_avg, F at the label, F at the current mu), F = log(hi/lo) per cell."""
        return self.query(FDM_Q_SURR_BOUNDS, np.float64, 3 * self.ncell).reshape(3, self.ncell)

    def mubar(self):
        return self.query(FDM_Q_MUBAR, np.float64, 3 * self.ncell).reshape(self.ncell, 3)

    def mu(self):
        return self.query(FDM_Q_MU, np.float64, 3 * self.ncell).reshape(self.ncell, 3)

    def surrogate_output(self):
        return self.query(FDM_Q_SURR_OUTPUT, np.float32, 3 * self.ncell).reshape(self.ncell, 3)

    def tuning(self):
        """(kernel, threads, rows8, sweep us, candidates) chosen by the autotuner."""
        t = self.query(FDM_Q_TUNING, np.float64, 8)
        return int(t[0]), int(t[1]), int(t[2]), float(t[3]), int(t[4])

    def gmg_levels(self):
        """[(nx, ny, nz, nf)] of the Q1 multigrid levels (one entry: exact coarse solve)."""
        v = self.query(FDM_Q_GMG_LEVELS, np.int32, 1 + 4 * 32)
        L = int(v[0])
        v = v[1:1 + 4 * (L + 1)].reshape(L + 1, 4)
        return [tuple(int(a) for a in r) for r in v]

    def gmg_stencils(self):
        """Each level's 27-point operator as an array [27, nf]."""
        lev = self.gmg_levels()
        v = self.query(FDM_Q_GMG_STENCIL, np.float64, 27 * sum(r[3] for r in lev))
        out, o = [], 0
        for r in lev:
            out.append(v[o:o + 27 * r[3]].reshape(27, r[3]))
            o += 27 * r[3]
        return out

    def lanczos_extremes(self):
        return tuple(self.query(FDM_Q_LAMBDA, np.float64, 2))

    def query(self, what, dtype, count, arg=None):
        out = np.zeros(count, dtype=dtype)
        fdm_query(self.h, what, out, arg)
        return out

    @property
    def omega(self):
        return float(self.query(FDM_Q_OMEGA, np.float64, 1)[0])

    def class_info(self):
        return self.query(FDM_Q_CLASS_INFO, np.int32, 64).reshape(8, 8)

    def gamma_orders(self):
        info = self.class_info()
        flat = self.query(FDM_Q_GAMMA_ORDER, np.int32, int(info[:, 2].sum()))
        out, off = [], 0
        for c in range(8):
            nG = int(info[c, 2])
            out.append(flat[off:off + nG])
            off += nG
        return out

    def pattern(self, cls):
        nG = int(self.class_info()[cls, 2])
        out = np.zeros(max(nG * nG, 4), dtype=np.uint8)
        fdm_query(self.h, FDM_Q_PATTERN, out, cls)
        return out[:nG * nG].reshape(nG, nG).astype(bool)

    def factor_dense(self, patch):
        cls = int(self.query(FDM_Q_PATCH_CLASS, np.int32, self.npatch)[patch])
        nG = int(self.class_info()[cls, 2])
        out = np.zeros(max(nG * nG, 1), dtype=np.float64)
        fdm_query(self.h, FDM_Q_FACTOR, out, patch)
        return out[:nG * nG].reshape(nG, nG)

    def kernel_times(self):
        """{timer: (launches, total ms)} since the last call (needs kernel_timing=1)."""
        h = self.query(FDM_Q_KERNEL_TIMES, np.float64, 2 * len(TIMERS)).reshape(-1, 2)
        return {name: (int(h[i, 0]), float(h[i, 1])) for i, name in enumerate(TIMERS)}

    def status(self):
        return int(self.query(FDM_Q_STATUS, np.int32, 1)[0])

    def launches(self):
        return int(self.query(FDM_Q_LAUNCHES, np.int64, 1)[0])

    def algo_bytes(self):
        v = self.query(FDM_Q_ALGO_BYTES, np.float64, 4)
        lf = self.query(FDM_Q_ALGO_BYTES_LFORM, np.float64, 2)
        return dict(patch64=v[0], patch32=v[1], asm64=v[2], asm32=v[3], lform64=lf[0], lform32=lf[1])

    def setup_seconds(self):
        return self.query(FDM_Q_SETUP_SECONDS, np.float64, 4)

    @property
    def npatch(self):
        return int(self.query(FDM_Q_NPATCH, np.int32, 1)[0])


class Elasticity:
    """Owns one primal linear-elasticity problem (fdm_elast): box cells,
    clamped on the faces of dirichlet_faces (bit 2a: lower end of axis a, 2a+1:
    upper; 63 = all) and traction-free on the others, vectors [3 * ndof]
    component-major on the device; sdc_form one of FDM_SDC_*."""

    def __init__(self, p, xv, yv, zv, mu, lam, precision=FDM_PREC_FP32, pc=FDM_PC_VCYCLE, omega=0.0,
                 lanczos_start=None, lanczos_steps=20, flexible_beta=-1, patch_threads=0, stream=None,
                 dirichlet_faces=63, sdc_form=0):
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (xv, yv, zv)]
        mesh = fdm_mesh()
        mesh.nx, mesh.ny, mesh.nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
        mesh.xv, mesh.yv, mesh.zv = [_dptr(a) for a in self._keep]
        opt = fdm_default_options()
        opt.precision, opt.pc, opt.omega, opt.lanczos_steps = precision, pc, omega, lanczos_steps
        opt.flexible_beta = flexible_beta
        opt.patch_threads = patch_threads
        if lanczos_start is not None:
            s = np.ascontiguousarray(lanczos_start, dtype=np.float64)
            self._keep.append(s)
            opt.lanczos_start = _dptr(s)
        self.p = p
        self.N = (mesh.nx * p + 1, mesh.ny * p + 1, mesh.nz * p + 1)
        self.ndof = self.N[0] * self.N[1] * self.N[2]
        self.dirichlet_faces = dirichlet_faces
        self.h = fdm_elast_setup_bc(mesh, p, mu, lam, dirichlet_faces, sdc_form, opt, stream)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            fdm_elast_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, like):
        import torch
        return torch.empty(3 * self.ndof, dtype=torch.float64, device=like.device)

    def apply(self, u, y=None):
        y = self._out(u) if y is None else y
        elast_apply(self.h, u, y)
        return y

    def pc_apply(self, r, z=None):
        z = self._out(r) if z is None else z
        elast_pc_apply(self.h, r, z)
        return z

    def pcg_solve(self, b, x=None, rtol=1e-8, maxit=500, raise_on_noconv=True):
        x = self._out(b) if x is None else x
        return x, elast_pcg_solve(self.h, b, x, rtol, maxit, raise_on_noconv=raise_on_noconv)

    @property
    def omega(self):
        out = np.zeros(1)
        fdm_elast_query(self.h, FDM_Q_OMEGA, out)
        return float(out[0])

    def recursive_iterations(self):
        """(iteration at which the last solve's recursive residual first met
        the test or -1, true-residual checks that did not)."""
        out = np.zeros(2, dtype=np.int32)
        fdm_elast_query(self.h, FDM_Q_RECURSIVE_ITS, out)
        return int(out[0]), int(out[1])

    def lanczos_extremes(self):
        out = np.zeros(2)
        fdm_elast_query(self.h, FDM_Q_LAMBDA, out)
        return float(out[0]), float(out[1])

    def launches(self):
        out = np.zeros(1, dtype=np.int64)
        fdm_elast_query(self.h, FDM_Q_LAUNCHES, out)
        return int(out[0])


class Sipg:
    """Owns one SIPG DQ_p Poisson problem (fdm_sipg): box cells, weak
    Dirichlet condition on the boundary, cell-major vectors [ndof] on the
    device (ndof = cells * (p+1)^3)."""

    def __init__(self, p, xv, yv, zv, eta=0.0, precision=FDM_PREC_FP32, pc=FDM_PC_VCYCLE, omega=0.0,
                 lanczos_start=None, lanczos_steps=20, flexible_beta=-1, coarse_levels=-1, tensor_core=0,
                 wait_timeout_s=1.0, stream=None):
        self._keep = [np.ascontiguousarray(a, dtype=np.float64) for a in (xv, yv, zv)]
        mesh = fdm_mesh()
        mesh.nx, mesh.ny, mesh.nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
        mesh.xv, mesh.yv, mesh.zv = [_dptr(a) for a in self._keep]
        opt = fdm_default_options()
        opt.precision, opt.pc, opt.omega, opt.lanczos_steps = precision, pc, omega, lanczos_steps
        opt.flexible_beta = flexible_beta
        opt.coarse_levels = coarse_levels
        opt.tensor_core = tensor_core
        opt.wait_timeout_s = wait_timeout_s
        if lanczos_start is not None:
            s = np.ascontiguousarray(lanczos_start, dtype=np.float64)
            self._keep.append(s)
            opt.lanczos_start = _dptr(s)
        self.p = p
        self.nc = (mesh.nx, mesh.ny, mesh.nz)
        self.ndof = mesh.nx * mesh.ny * mesh.nz * (p + 1) ** 3
        self.h = fdm_sipg_setup(mesh, p, eta, opt, stream)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            fdm_sipg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, like, n=None):
        import torch
        return torch.empty(self.ndof if n is None else n, dtype=torch.float64, device=like.device)

    def apply(self, u, y=None):
        y = self._out(u) if y is None else y
        sipg_apply(self.h, u, y)
        return y

    def asm_apply(self, r, z=None):
        z = self._out(r) if z is None else z
        sipg_asm_apply(self.h, r, z)
        return z

    def pc_apply(self, r, z=None):
        z = self._out(r) if z is None else z
        sipg_pc_apply(self.h, r, z)
        return z

    def vertex_index(self, vx, vy, vz):
        return vx + (self.nc[0] + 1) * (vy + (self.nc[1] + 1) * vz)

    def patch_solve(self, r, vertices):
        """A_v^{-1} R_v r for (vx, vy, vz) interior vertices: [len, (2p+2)^3] in star order."""
        idx = [self.vertex_index(*v) for v in vertices]
        m3 = (2 * self.p + 2) ** 3
        out = self._out(r, len(idx) * m3)
        sipg_patch_solve(self.h, r, idx, out)
        return out.view(len(idx), m3)

    def pcg_solve(self, b, x=None, rtol=1e-8, maxit=500, raise_on_noconv=True):
        x = self._out(b) if x is None else x
        return x, sipg_pcg_solve(self.h, b, x, rtol, maxit, raise_on_noconv=raise_on_noconv)

    @property
    def omega(self):
        out = np.zeros(1)
        fdm_sipg_query(self.h, FDM_Q_OMEGA, out)
        return float(out[0])

    def lanczos_extremes(self):
        out = np.zeros(2)
        fdm_sipg_query(self.h, FDM_Q_LAMBDA, out)
        return float(out[0]), float(out[1])

    def launches(self):
        out = np.zeros(1, dtype=np.int64)
        fdm_sipg_query(self.h, FDM_Q_LAUNCHES, out)
        return int(out[0])

    def status(self):
        """The tensor-core star solve's status word (1: a bounded wait ran out); reading clears it."""
        out = np.zeros(1, dtype=np.int32)
        fdm_sipg_query(self.h, FDM_Q_STATUS, out)
        return int(out[0])


class HexMesh:
    """Host topology of a conforming hexahedral mesh (fdm_hexmesh_create):
    node numbering, Dirichlet nodes, vertex stars in FDM order, the signed
    cell-to-global FDM map and the stars' surrogate patterns.  Host arrays
    only; needs no GPU."""

    def __init__(self, nv, cells, p, dirichlet_vertex=None):
        """dirichlet_vertex: None (every boundary face Dirichlet) or a bool array
        over the vertices; a boundary face is Dirichlet when its 4 vertices are
        marked, the other boundary faces are natural."""
        L = load()
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        self.p, self.n, self.nc = p, p + 1, cells.shape[0]
        h = C.c_void_p()
        dv = None if dirichlet_vertex is None else np.ascontiguousarray(dirichlet_vertex, dtype=np.uint8)
        self._dv = dv
        rc = L.fdm_hexmesh_create_bc(int(nv), self.nc, cells.ctypes.data_as(C.POINTER(C.c_int)), p,
                                     None if dv is None else dv.ctypes.data_as(C.c_void_p), C.byref(h))
        if rc < 0:
            raise FdmError(rc, L.fdm_hexmesh_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            load().fdm_hexmesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def query(self, what, dtype):
        L = load()
        n = C.c_size_t(0)
        rc = L.fdm_hexmesh_query(self.h, what, None, C.byref(n))
        if rc < 0:
            raise FdmError(rc, L.fdm_hexmesh_last_error(self.h).decode())
        out = np.zeros(n.value // np.dtype(dtype).itemsize, dtype=dtype)
        rc = L.fdm_hexmesh_query(self.h, what, out.ctypes.data_as(C.c_void_p), C.byref(n))
        if rc < 0:
            raise FdmError(rc, L.fdm_hexmesh_last_error(self.h).decode())
        return out

    @property
    def nnode(self):
        return int(self.query(FDM_HQ_NNODE, np.int64)[0])

    def cell_nodes(self):
        return self.query(FDM_HQ_CELL_NODES, np.int32).reshape(self.nc, self.n ** 3)

    def cell_fdm(self):
        return (self.query(FDM_HQ_CELL_FDM, np.int32).reshape(self.nc, self.n ** 3),
                self.query(FDM_HQ_CELL_SIGN, np.int8).reshape(self.nc, self.n ** 3))

    def dirichlet(self):
        return self.query(FDM_HQ_DIRICHLET, np.uint8).astype(bool)

    def stars(self):
        """[(vertex, nodes in FDM order)] for every star."""
        vert = self.query(FDM_HQ_STAR_VERTEX, np.int32)
        ptr = self.query(FDM_HQ_STAR_PTR, np.int64)
        nodes = self.query(FDM_HQ_STAR_NODES, np.int32)
        return [(int(vert[k]), nodes[ptr[k]:ptr[k + 1]]) for k in range(len(vert))]

    def patterns(self):
        """Per star, (rowptr, cols) of its surrogate pattern over star positions."""
        pp = self.query(FDM_HQ_PATTERN_PTR, np.int64)
        rp = self.query(FDM_HQ_PATTERN_ROWPTR, np.int64)
        cp = self.query(FDM_HQ_PATTERN_COLPTR, np.int64)
        cols = self.query(FDM_HQ_PATTERN_COLS, np.int32)
        return [(rp[pp[k]:pp[k + 1]], cols[cp[k]:cp[k + 1]]) for k in range(len(pp) - 1)]

    def classes(self):
        """Per star its class and interior count; per class (first star,
        nnz(L), rows of L as (rowptr, cols), elimination-tree parents)."""
        cls = self.query(FDM_HQ_STAR_CLASS, np.int32)
        nint = self.query(FDM_HQ_STAR_NINT, np.int32)
        first = self.query(FDM_HQ_CLASS_STAR, np.int32)
        nnzl = self.query(FDM_HQ_CLASS_NNZL, np.int64)
        fp = self.query(FDM_HQ_FILL_PTR, np.int64)
        fr = self.query(FDM_HQ_FILL_ROWPTR, np.int64)
        fc = self.query(FDM_HQ_FILL_COLPTR, np.int64)
        cols = self.query(FDM_HQ_FILL_COLS, np.int32)
        ep = self.query(FDM_HQ_ETREE_PTR, np.int64)
        et = self.query(FDM_HQ_ETREE, np.int32)
        per = [(int(first[k]), int(nnzl[k]), (fr[fp[k]:fp[k + 1]], cols[fc[k]:fc[k + 1]]), et[ep[k]:ep[k + 1]])
               for k in range(len(first))]
        return cls, nint, per

    def factor(self, X, kappa_q=None, kaxes=None):
        """Numeric set-up (fdm_hexmesh_factor, or fdm_hexmesh_factor_axes with
        the diagonal coefficient kaxes); returns (mu[nc,3], per star (D, L
        values in its class's fill pattern))."""
        L = load()
        X = np.ascontiguousarray(X, dtype=np.float64)
        kq = None if kappa_q is None else np.ascontiguousarray(kappa_q, dtype=np.float64)
        ka = None if kaxes is None else np.ascontiguousarray(kaxes, dtype=np.float64)
        rc = L.fdm_hexmesh_factor_axes(self.h, X.shape[0], _dptr(X), None if kq is None else _dptr(kq),
                                       None if ka is None else _dptr(ka))
        if rc < 0:
            raise FdmError(rc, L.fdm_hexmesh_last_error(self.h).decode())
        mu = self.query(FDM_HQ_MU, np.float64).reshape(self.nc, 3)
        dp_, d = self.query(FDM_HQ_DIAG_PTR, np.int64), self.query(FDM_HQ_DIAG, np.float64)
        fp_, f = self.query(FDM_HQ_FACTOR_PTR, np.int64), self.query(FDM_HQ_FACTOR, np.float64)
        return mu, [(d[dp_[k]:dp_[k + 1]], f[fp_[k]:fp_[k + 1]]) for k in range(len(dp_) - 1)]

    def inverse_maps(self):
        """(slot_cells_ptr, slot_cells, slot_stars_ptr, slot_stars[:, 2], node_owner)."""
        return (self.query(FDM_HQ_SLOT_CELLS_PTR, np.int64), self.query(FDM_HQ_SLOT_CELLS, np.int32),
                self.query(FDM_HQ_SLOT_STARS_PTR, np.int64), self.query(FDM_HQ_SLOT_STARS, np.int32).reshape(-1, 2),
                self.query(FDM_HQ_NODE_OWNER, np.int32))

    def operator_tables(self):
        """(node_cells_ptr, node_cells, geom[nc, q^3, 6], coarse_of[nv], coarse[nco, nco]);
        geom and coarse after factor()."""
        ptr = self.query(FDM_HQ_NODE_CELLS_PTR, np.int64)
        nodec = self.query(FDM_HQ_NODE_CELLS, np.int32)
        geom = self.query(FDM_HQ_GEOM, np.float64).reshape(self.nc, self.n ** 3, 6)
        cof = self.query(FDM_HQ_COARSE_OF, np.int32)
        co = self.query(FDM_HQ_COARSE, np.float64)
        m = int(round(np.sqrt(co.size)))
        return ptr, nodec, geom, cof, co.reshape(m, m)

    def schur_coupling(self):
        """Per class (t, (L_BB rowptr, cols), (S_TB rowptr, cols)); per star its
        values (L_BB, S_TB, lower triangle of W) after factor()."""
        t = self.query(FDM_HQ_SC_SPLIT, np.int32)
        sp = self.query(FDM_HQ_SC_PTR, np.int64)
        rp = self.query(FDM_HQ_SC_ROWPTR, np.int64)
        cp = self.query(FDM_HQ_SC_COLPTR, np.int64)
        cols = self.query(FDM_HQ_SC_COLS, np.int32)
        per = []
        for k in range(len(t)):
            r = rp[sp[k]:sp[k + 1]]
            nB = len(r) - int(t[k]) - 2
            rb, rt = r[:nB + 1], r[nB + 1:]
            c = cols[cp[k]:cp[k + 1]]
            per.append((int(t[k]), (rb, c[:rb[-1]]), (rt, c[rb[-1]:])))
        vp = self.query(FDM_HQ_SC_VALUES_PTR, np.int64)
        v = self.query(FDM_HQ_SC_VALUES, np.float64)
        return per, [v[vp[k]:vp[k + 1]] for k in range(len(vp) - 1)]


class Partition:
    """Box partition of an nx x ny x nz cell mesh at degree p over a
    px x py x pz rank grid, seen from one rank (fdm_partition_create): host
    index lists only (cell and node boxes, neighbours, send lists, the
    per-node sum plans, node ownership, owned stars)."""

    def __init__(self, ncell, p, nrank, rank):
        L = load()
        h = C.c_void_p()
        rc = L.fdm_partition_create(int(ncell[0]), int(ncell[1]), int(ncell[2]), int(p), int(nrank[0]),
                                    int(nrank[1]), int(nrank[2]), int(rank), C.byref(h))
        if rc < 0:
            raise FdmError(rc, L.fdm_partition_last_error().decode())
        self.h = h
        self.p, self.rank = p, rank

    def query(self, what, dtype, count=None):
        """The quantity `what` as a numpy array (size found from the library when count is None)."""
        L = load()
        if count is None:
            n = C.c_size_t(0)
            probe = np.zeros(1, dtype=np.uint8)
            L.fdm_partition_query(self.h, what, probe.ctypes.data_as(C.c_void_p), C.byref(n))
            count = n.value // np.dtype(dtype).itemsize
        out = np.zeros(max(count, 1), dtype=dtype)
        n = C.c_size_t(out.nbytes)
        rc = L.fdm_partition_query(self.h, what, out.ctypes.data_as(C.c_void_p), C.byref(n))
        if rc < 0:
            raise FdmError(rc, L.fdm_partition_last_error().decode())
        return out[:count]

    def cell_box(self):
        return self.query(FDM_PQ_CELL_BOX, np.int32, 6)

    def node_box(self):
        return self.query(FDM_PQ_NODE_BOX, np.int32, 6)

    def halo_box(self):
        return self.query(FDM_PQ_HALO_BOX, np.int32, 6)

    def neighbors(self):
        k = int(self.query(FDM_PQ_NNEIGH, np.int32, 1)[0])
        return self.query(FDM_PQ_NEIGHBORS, np.int32, k) if k else np.zeros(0, np.int32)

    def lists(self):
        """(send_ptr, send, recv_ptr, sum_ptr, sum, owned) as numpy arrays."""
        k = len(self.neighbors())
        send_ptr = self.query(FDM_PQ_SEND_PTR, np.int64, k + 1)
        recv_ptr = self.query(FDM_PQ_RECV_PTR, np.int64, k + 1)
        nb = self.node_box()
        nodes = int(np.prod(nb[1::2] - nb[0::2] + 1))
        sum_ptr = self.query(FDM_PQ_SUM_PTR, np.int64, nodes + 1)
        send = self.query(FDM_PQ_SEND, np.int64, int(send_ptr[-1]))
        summ = self.query(FDM_PQ_SUM, np.int64, int(sum_ptr[-1]))
        owned = self.query(FDM_PQ_OWNED, np.uint8, nodes)
        return send_ptr, send, recv_ptr, sum_ptr, summ, owned

    def stars(self):
        return self.query(FDM_PQ_STARS, np.int64)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().fdm_partition_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class HexGpu:
    """Owns one GPU context on a general hexahedral mesh (fdm_hex_setup) built
    from a HexMesh after its numeric set-up; vectors are CUDA float64 tensors
    of HexMesh.nnode values in the mesh's node numbering."""

    def __init__(self, mesh, precision=FDM_PREC_FP64, pc=FDM_PC_VCYCLE, omega=0.0, lanczos_start=None,
                 lanczos_steps=20, flexible_beta=-1, patch_form=0, stream=None):
        opt = fdm_default_options()
        opt.precision, opt.pc, opt.omega, opt.lanczos_steps = precision, pc, omega, lanczos_steps
        opt.flexible_beta = flexible_beta
        opt.patch_form = patch_form
        self._keep = []
        if lanczos_start is not None:
            st = np.ascontiguousarray(lanczos_start, dtype=np.float64)
            self._keep.append(st)
            opt.lanczos_start = _dptr(st)
        L = load()
        h = C.c_void_p()
        rc = L.fdm_hex_setup(mesh.h, C.byref(opt), C.byref(h), _stream(stream))
        if rc < 0:
            raise FdmError(rc, L.fdm_hex_last_error(None).decode())
        self.h = h
        self.nnode = mesh.nnode

    def _check(self, rc):
        if rc < 0:
            raise FdmError(rc, load().fdm_hex_last_error(self.h).decode())
        return rc

    def _out(self, like):
        import torch
        return torch.empty_like(like)

    def stiffness_apply(self, u, y=None, stream=None):
        y = self._out(u) if y is None else y
        self._check(load().hex_stiffness_apply(self.h, _tptr(u), _tptr(y), _stream(stream)))
        return y

    def asm_apply(self, r, z=None, stream=None):
        z = self._out(r) if z is None else z
        self._check(load().hex_asm_apply(self.h, _tptr(r), _tptr(z), _stream(stream)))
        return z

    def pc_apply(self, r, z=None, stream=None):
        z = self._out(r) if z is None else z
        self._check(load().hex_pc_apply(self.h, _tptr(r), _tptr(z), _stream(stream)))
        return z

    def pcg_solve(self, b, x=None, rtol=1e-8, maxit=500, raise_on_noconv=True, stream=None):
        x = self._out(b) if x is None else x
        info = fdm_solve_info()
        rc = load().hex_pcg_solve(self.h, _tptr(b), _tptr(x), rtol, maxit, C.byref(info), _stream(stream))
        if not (rc == FDM_ENOCONV and not raise_on_noconv):
            self._check(rc)
        return x, info

    def query(self, what, dtype, count):
        out = np.zeros(count, dtype=dtype)
        n = C.c_size_t(out.nbytes)
        self._check(load().fdm_hex_query(self.h, what, out.ctypes.data_as(C.c_void_p), C.byref(n)))
        return out

    @property
    def omega(self):
        return float(self.query(FDM_XQ_OMEGA, np.float64, 1)[0])

    def lanczos_extremes(self):
        v = self.query(FDM_XQ_LAMBDA, np.float64, 2)
        return float(v[0]), float(v[1])

    def launches(self):
        return int(self.query(FDM_XQ_LAUNCHES, np.int64, 1)[0])

    def sizes(self):
        """(cells, stars, star interface values, stored factor values, coarse unknowns, largest interface)."""
        return tuple(int(v) for v in self.query(FDM_XQ_SIZES, np.int64, 6))

    def algo_bytes(self):
        v = self.query(FDM_XQ_ALGO_BYTES, np.float64, 2)
        return dict(sweep64=float(v[0]), sweep32=float(v[1]))

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            load().fdm_hex_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
