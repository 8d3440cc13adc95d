"""stiffness_apply_noalloc, the stiffness apply for callers that must not
allocate device memory when they call (its cell-local scratch is a fixed
device array of the library instead of the context's buffer).

Checked through the C-ABI against stiffness_apply, on two calls in a row (the
shared array keeps the previous call's contents, which must not leak into the
next result), on box cells (the Kronecker form) and on curved cells with a
coefficient (the Gauss-point form), the two cell kernels that write the
fixed scratch, and for the rejection of problems beyond it.  This file is collected last so that a run stopping
at its first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib_and_ctx(p, xv, yv, zv, **kw):
    import __graft_entry__ as g
    g.build()
    from paper_2107_14758_gb300 import fdmpc
    ctx = fdmpc.Context(p, xv, yv, zv, precision=fdmpc.FDM_PREC_FP64, omega=1.0, **kw)
    return fdmpc, fdmpc.load(), ctx


def _twice(fdmpc, L, ctx, seed):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gen = torch.Generator(device="cuda:0").manual_seed(seed)
    for call in range(2):  # two calls in a row, different inputs
        u = torch.randn(ctx.ndof, dtype=torch.float64, device="cuda:0", generator=gen)
        ref = ctx.stiffness_apply(u)
        y = torch.full_like(u, float("nan"))
        rc = L.stiffness_apply_noalloc(ctx.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()), stream)
        assert rc == 0, fdmpc.fdm_last_error(ctx.h)
        torch.cuda.synchronize()
        a, b = y.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), call


def test_noalloc_matches_stiffness_apply_twice():
    from paper_2107_14758_gb300 import inputs
    xv, yv, zv = inputs.graded_vertices(4, 31)
    fdmpc, L, ctx = _lib_and_ctx(5, xv, yv, zv)
    _twice(fdmpc, L, ctx, 7)
    ctx.close()


def test_noalloc_curved_cells_with_coefficient():
    from paper_2107_14758_gb300 import inputs
    p, n = 3, 3
    xv, yv, zv = inputs.uniform_vertices(n)
    jac, pts = inputs.deformed_jacobians(n, p)
    kap = inputs.kappa_field(pts, 5)
    fdmpc, L, ctx = _lib_and_ctx(p, xv, yv, zv, jac=jac, kappa=kap)
    _twice(fdmpc, L, ctx, 8)
    ctx.close()


def test_noalloc_rejects_problems_beyond_its_scratch():
    from paper_2107_14758_gb300 import inputs
    xv, yv, zv = inputs.graded_vertices(16, 2)
    xv = np.concatenate([xv * 16 / 17, [1.0]])  # 17 x 16 x 16 cells at p = 7: 4352 * 512 > 2^21
    fdmpc, L, ctx = _lib_and_ctx(7, xv, yv, zv)
    u = torch.zeros(ctx.ndof, dtype=torch.float64, device="cuda:0")
    y = torch.zeros_like(u)
    rc = L.stiffness_apply_noalloc(ctx.h, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                   ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == fdmpc.FDM_EINVAL
    assert "exceeds the fixed scratch" in fdmpc.fdm_last_error(ctx.h)
    ctx.close()
