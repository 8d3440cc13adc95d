"""ctypes binding of the FP64 CPU oracle (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never does.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force=False):
    """Compile oracle.c and surrogate.c into liboracle.so with gcc (OpenMP
    over patches and cells)."""
    srcs = [os.path.join(_HERE, f) for f in ("oracle.c", "surrogate.c")]
    if (not force and os.path.exists(_LIB_PATH)
            and all(os.path.getmtime(_LIB_PATH) >= os.path.getmtime(f)
                    for f in srcs + [os.path.join(_HERE, "oracle.h")])):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-fopenmp",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lp = C.POINTER(C.c_long)
        L.or_gauss.argtypes = [C.c_int, dp, dp]
        L.or_gll.argtypes = [C.c_int, dp, dp]
        L.or_lagrange.argtypes = [C.c_int, dp, C.c_int, dp, dp, dp]
        L.or_lagrange.restype = None
        L.or_basis1d.argtypes = [C.c_int] + [dp] * 8
        L.or_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, dp, dp, dp, dp, dp]
        L.or_create.restype = C.c_void_p
        L.or_free.argtypes = [C.c_void_p]
        L.or_free.restype = None
        L.or_last_error.restype = C.c_char_p
        L.or_ndof.argtypes = [C.c_void_p]
        L.or_ndof.restype = C.c_long
        L.or_npatch.argtypes = [C.c_void_p]
        L.or_get_mu.argtypes = [C.c_void_p, dp]
        L.or_get_mu.restype = None
        L.or_set_mu.argtypes = [C.c_void_p, dp]
        L.or_set_mu.restype = None
        for f in ("or_stiffness_apply", "or_mass_apply", "or_restrict_fdm", "or_interp_fdm"):
            getattr(L, f).argtypes = [C.c_void_p, dp, dp]
            getattr(L, f).restype = None
        L.or_setup_patches.argtypes = [C.c_void_p, ip, C.c_int, C.c_int]
        L.or_patch_dofs.argtypes = [C.c_void_p, C.c_int, ip, ip, lp]
        L.or_patch_matrix.argtypes = [C.c_void_p, C.c_int, dp]
        L.or_patch_schur.argtypes = [C.c_void_p, C.c_int, dp]
        L.or_patch_solve.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.or_cholesky.argtypes = [C.c_int, dp]
        L.or_symbolic_fill.argtypes = [C.c_int, C.POINTER(C.c_ubyte)]
        L.or_symbolic_fill.restype = None
        L.or_asm_apply.argtypes = [C.c_void_p, dp, dp]
        L.or_set_omega.argtypes = [C.c_void_p, C.c_double]
        L.or_set_omega.restype = None
        L.or_get_omega.argtypes = [C.c_void_p]
        L.or_get_omega.restype = C.c_double
        L.or_setup_coarse.argtypes = [C.c_void_p]
        L.or_coarse_apply.argtypes = [C.c_void_p, dp, dp]
        L.or_coarse_matrix.argtypes = [C.c_void_p, ip, dp]
        L.or_pc_apply.argtypes = [C.c_void_p, dp, dp]
        L.or_setup_coarse_gmg.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_double]
        L.or_gmg_level.argtypes = [C.c_void_p, C.c_int, ip, dp]
        L.or_gmg_vcycle.argtypes = [C.c_void_p, dp, dp]
        L.or_lanczos_omega.argtypes = [C.c_void_p, dp, C.c_int, dp, dp, dp]
        L.or_pcg.argtypes = [C.c_void_p, dp, dp, C.c_double, C.c_int, C.c_int, ip, dp]
        L.or_surr_bound.argtypes = [C.c_int, dp, dp, dp, dp]
        L.or_surr_bound.restype = C.c_double
        L.or_surr_cell_ghat.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp]
        L.or_surr_label.argtypes = [C.c_int, C.c_int, dp, dp, dp, dp, dp, dp]
        L.or_surr_features.argtypes = [C.c_int, dp, dp]
        L.or_mlp_forward.argtypes = [C.c_int, dp, dp, dp]
        L.or_mlp_forward.restype = None
        L.or_mlp_loss_grad.argtypes = [C.c_int, dp, dp, dp, dp]
        L.or_mlp_loss_grad.restype = C.c_double
        L.or_mlp_adam.argtypes = [C.c_int, dp, dp, dp, dp, C.c_int, C.c_double]
        L.or_mlp_adam.restype = None
        L.or_surr_apply.argtypes = [C.c_int, dp, dp, dp]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc < 0:
        raise OracleError(lib().or_last_error().decode())
    return rc


def gauss(q):
    x = np.zeros(q); w = np.zeros(q)
    _check(lib().or_gauss(q, _p(x), _p(w)))
    return x, w


def gll(p):
    x = np.zeros(p + 1); w = np.zeros(p + 1)
    _check(lib().or_gll(p, _p(x), _p(w)))
    return x, w


def lagrange(p, xi, x):
    xi = _f64(xi); x = _f64(x)
    V = np.zeros((len(x), p + 1)); D = np.zeros((len(x), p + 1))
    lib().or_lagrange(p, _p(xi), len(x), _p(x), _p(V), _p(D))
    return V, D


def basis1d(p):
    """Returns dict with xi, A, B, S, lam, T, Af, Bf (Sections 2.1-2.4)."""
    n, m = p + 1, max(p - 1, 0)
    out = {k: np.zeros(s) for k, s in
           dict(xi=n, A=(n, n), B=(n, n), S=(max(m, 1), max(m, 1)), lam=max(m, 1),
                T=(n, n), Af=(n, n), Bf=(n, n)).items()}
    _check(lib().or_basis1d(p, *[_p(out[k]) for k in ("xi", "A", "B", "S", "lam", "T", "Af", "Bf")]))
    if m == 0:
        out["S"] = np.zeros((0, 0)); out["lam"] = np.zeros(0)
    return out


def cholesky(S):
    S = _f64(S).copy()
    _check(lib().or_cholesky(S.shape[0], _p(S)))
    return S


def symbolic_fill(pattern):
    pat = np.ascontiguousarray(pattern, dtype=np.uint8).copy()
    lib().or_symbolic_fill(pat.shape[0], pat.ctypes.data_as(C.POINTER(C.c_ubyte)))
    return pat.astype(bool)


# ---- learned separable surrogate (Section 2.7, Theorem 1) ----------------
MLP_NIN, MLP_NH, MLP_NOUT = 189, 64, 3
MLP_NPARAM = MLP_NH * MLP_NIN + MLP_NH + MLP_NH * MLP_NH + MLP_NH + MLP_NOUT * MLP_NH + MLP_NOUT
SURR_CMAX = 2.0


def surr_bound(G, mu):
    """(log(hi/lo), lo, hi) of the Theorem 1 bound over points G[q][6]."""
    G = _f64(G).reshape(-1, 6); mu = _f64(mu)
    lo = C.c_double(); hi = C.c_double()
    F = lib().or_surr_bound(G.shape[0], _p(G), _p(mu), C.byref(lo), C.byref(hi))
    return F, lo.value, hi.value


def surr_cell_ghat(p, jac, kappa=None):
    """kappa*Ghat per cell and Gauss point (unweighted) and the averaged mu."""
    jac = _f64(jac); ncell = jac.shape[0]
    nq = (p + 1) ** 3
    G = np.zeros((ncell, nq, 6)); mubar = np.zeros((ncell, 3))
    kp = _p(_f64(kappa)) if kappa is not None else None
    kap = _f64(kappa) if kappa is not None else None
    _check(lib().or_surr_cell_ghat(p, ncell, _p(jac), _p(kap) if kap is not None else kp, _p(G), _p(mubar)))
    return G, mubar


def surr_label(p, jac, kappa=None):
    """Returns mubar[cell,3], cstar[cell,3], F0[cell], F1[cell]."""
    jac = _f64(jac); ncell = jac.shape[0]
    kap = _f64(kappa) if kappa is not None else None
    mubar = np.zeros((ncell, 3)); cs = np.zeros((ncell, 3)); F0 = np.zeros(ncell); F1 = np.zeros(ncell)
    _check(lib().or_surr_label(p, ncell, _p(jac), _p(kap) if kap is not None else None,
                               _p(mubar), _p(cs), _p(F0), _p(F1)))
    return mubar, cs, F0, F1


def surr_features(s27):
    s27 = _f64(s27); ncell = s27.shape[0]
    f = np.zeros((ncell, MLP_NIN))
    _check(lib().or_surr_features(ncell, _p(s27), _p(f)))
    return f


def mlp_forward(params, feat):
    params = _f64(params); feat = _f64(feat)
    c = np.zeros((feat.shape[0], MLP_NOUT))
    lib().or_mlp_forward(feat.shape[0], _p(params), _p(feat), _p(c))
    return c


def mlp_loss_grad(params, feat, label, grad=True):
    params = _f64(params); feat = _f64(feat); label = _f64(label)
    g = np.zeros(MLP_NPARAM) if grad else None
    loss = lib().or_mlp_loss_grad(feat.shape[0], _p(params), _p(feat), _p(label),
                                  _p(g) if grad else None)
    return loss, g


def mlp_adam(params, grad, m, v, t, lr):
    """One Adam step in place on params, m, v (all float64 arrays)."""
    for a in (params, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(grad)
    lib().or_mlp_adam(params.size, _p(params), _p(g), _p(m), _p(v), int(t), float(lr))


def surr_apply(mubar, c):
    mubar = _f64(mubar); c = _f64(c)
    mu = np.zeros_like(mubar)
    nf = lib().or_surr_apply(mubar.shape[0], _p(mubar), _p(c), _p(mu))
    return mu, nf


class Problem:
    """One Poisson problem on a structured hex mesh (oracle side)."""

    def __init__(self, p, xv, yv, zv, jac=None, kappa=None):
        self.p = p
        self.xv, self.yv, self.zv = _f64(xv), _f64(yv), _f64(zv)
        self.nx, self.ny, self.nz = len(xv) - 1, len(yv) - 1, len(zv) - 1
        self._keep = []
        jp = kp = None
        if jac is not None:
            jac = _f64(jac); self._keep.append(jac); jp = _p(jac)
        if kappa is not None:
            kappa = _f64(kappa); self._keep.append(kappa); kp = _p(kappa)
        h = lib().or_create(p, self.nx, self.ny, self.nz, _p(self.xv), _p(self.yv), _p(self.zv), jp, kp)
        if not h:
            raise OracleError(lib().or_last_error().decode())
        self.h = h
        self.N = (self.nx * p + 1, self.ny * p + 1, self.nz * p + 1)
        self.ndof = lib().or_ndof(h)
        self.npatch = lib().or_npatch(h)
        self.ncell = self.nx * self.ny * self.nz

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_free(self.h)
            self.h = None

    def _vecop(self, fname, u):
        u = _f64(u).ravel()
        assert u.size == self.ndof
        y = np.zeros(self.ndof)
        getattr(lib(), fname)(self.h, _p(u), _p(y))
        return y

    def stiffness_apply(self, u):
        return self._vecop("or_stiffness_apply", u)

    def mass_apply(self, f):
        return self._vecop("or_mass_apply", f)

    def restrict_fdm(self, r):
        return self._vecop("or_restrict_fdm", r)

    def interp_fdm(self, u):
        return self._vecop("or_interp_fdm", u)

    def get_mu(self):
        mu = np.zeros((self.ncell, 3))
        lib().or_get_mu(self.h, _p(mu))
        return mu

    def set_mu(self, mu):
        mu = _f64(mu)
        lib().or_set_mu(self.h, _p(mu))

    def setup_patches(self, vertices=None, nthreads=0):
        if vertices is None:
            _check(lib().or_setup_patches(self.h, None, 0, nthreads))
        else:
            v = np.ascontiguousarray(vertices, dtype=np.int32)
            _check(lib().or_setup_patches(self.h, v.ctypes.data_as(C.POINTER(C.c_int)), len(v), nthreads))

    def patch_dofs(self, v):
        nd = C.c_int(); nI = C.c_int()
        _check(lib().or_patch_dofs(self.h, v, C.byref(nd), C.byref(nI), None))
        g = np.zeros(nd.value, dtype=np.int64)
        _check(lib().or_patch_dofs(self.h, v, C.byref(nd), C.byref(nI),
                                   g.ctypes.data_as(C.POINTER(C.c_long))))
        return g, nI.value

    def patch_matrix(self, v):
        g, _ = self.patch_dofs(v)
        A = np.zeros((len(g), len(g)))
        _check(lib().or_patch_matrix(self.h, v, _p(A)))
        return A

    def patch_schur(self, v):
        g, nI = self.patch_dofs(v)
        nG = len(g) - nI
        S = np.zeros((nG, nG))
        _check(lib().or_patch_schur(self.h, v, _p(S)))
        return S

    def patch_solve(self, v, r):
        r = _f64(r)
        x = np.zeros_like(r)
        _check(lib().or_patch_solve(self.h, v, _p(r), _p(x)))
        return x

    def set_omega(self, w):
        lib().or_set_omega(self.h, float(w))

    def get_omega(self):
        return lib().or_get_omega(self.h)

    def asm_apply(self, r):
        r = _f64(r); z = np.zeros(self.ndof)
        _check(lib().or_asm_apply(self.h, _p(r), _p(z)))
        return z

    def setup_coarse(self):
        _check(lib().or_setup_coarse(self.h))

    def coarse_apply(self, r):
        r = _f64(r); z = np.zeros(self.ndof)
        _check(lib().or_coarse_apply(self.h, _p(r), _p(z)))
        return z

    def coarse_matrix(self):
        nc = C.c_int()
        _check(lib().or_coarse_matrix(self.h, C.byref(nc), None))
        A = np.zeros((nc.value, nc.value))
        _check(lib().or_coarse_matrix(self.h, C.byref(nc), _p(A)))
        return A

    def setup_coarse_gmg(self, levels, nu=2, omega=2.0 / 3.0):
        """Geometric multigrid V-cycle for the Q1 problem; returns the levels built."""
        return _check(lib().or_setup_coarse_gmg(self.h, levels, nu, omega))

    def gmg_level(self, l):
        nf = C.c_int()
        _check(lib().or_gmg_level(self.h, l, C.byref(nf), None))
        A = np.zeros((nf.value, nf.value))
        _check(lib().or_gmg_level(self.h, l, C.byref(nf), _p(A)))
        return A

    def gmg_vcycle(self, b):
        b = _f64(b)
        x = np.zeros_like(b)
        _check(lib().or_gmg_vcycle(self.h, _p(b), _p(x)))
        return x

    def pc_apply(self, r):
        r = _f64(r); z = np.zeros(self.ndof)
        _check(lib().or_pc_apply(self.h, _p(r), _p(z)))
        return z

    def lanczos_omega(self, b0, k=20):
        b0 = _f64(b0)
        lo = C.c_double(); hi = C.c_double(); om = C.c_double()
        _check(lib().or_lanczos_omega(self.h, _p(b0), k, C.byref(lo), C.byref(hi), C.byref(om)))
        return lo.value, hi.value, om.value

    def pcg(self, b, rtol=1e-8, maxit=200, pc=2):
        """pc: 0 none, 1 omega*ASM, 2 hybrid V(1,1). Returns (x, iters, hist, converged)."""
        b = _f64(b); x = np.zeros(self.ndof)
        hist = np.zeros(maxit + 1)
        it = C.c_int()
        rc = _check(lib().or_pcg(self.h, _p(b), _p(x), rtol, maxit, pc, C.byref(it), _p(hist)))
        return x, it.value, hist[: it.value + 1], rc == 0
