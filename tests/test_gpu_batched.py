"""Batched solves of independent problems in one CUDA graph (a device-driven
PCG loop per problem, conditional WHILE nodes): parity with the one-problem
solve and with the FP64 oracle, edge cases (b = 0, maxit reached, repeated
and changed calls)."""
import numpy as np
import pytest

from tests.record import record  # noqa: E402

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from paper_2107_14758_gb300 import fdmpc, inputs  # noqa: E402

FP64, FP32 = fdmpc.FDM_PREC_FP64, fdmpc.FDM_PREC_FP32
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__ as g
    g.build()
    assert torch.cuda.is_available()


def problems(precision, specs):
    out = []
    for n, p, seed in specs:
        xv, yv, zv = inputs.graded_vertices(n, seed)
        nd = (n * p + 1) ** 3
        ctx = fdmpc.Context(p, xv, yv, zv, precision=precision, lanczos_start=inputs.lanczos_start(nd))
        b = torch.tensor(inputs.normal_rhs(nd, seed), device=DEV)
        out.append((ctx, b, (xv, yv, zv)))
    return out


SPECS = [(2, 3, 1), (3, 5, 2), (4, 2, 3), (2, 9, 4), (3, 1, 5), (5, 4, 6)]


@pytest.mark.parametrize("precision", [FP64, FP32])
def test_batched_matches_single_solves(precision):
    probs = problems(precision, SPECS)
    batch = fdmpc.fdm_batch_setup([c.h for c, _, _ in probs])
    try:
        xs = [torch.zeros_like(b) for _, b, _ in probs]
        infos = fdmpc.pcg_solve_batched(batch, [b for _, b, _ in probs], xs, 1e-8, 200)
        for (ctx, b, _), x, info in zip(probs, xs, infos):
            x1, i1 = ctx.pcg_solve(b, rtol=1e-8, maxit=200)
            assert info.converged and info.iterations == i1.iterations
            assert info.rnorm <= 1e-8 * info.rnorm0
            assert info.rnorm0 == pytest.approx(i1.rnorm0, rel=1e-14)
            assert info.true_rnorm <= 1e-7 * info.rnorm0
            assert info.seconds > 0.0
            tol = 1e-12 if precision == FP64 else 1e-6
            assert (x - x1).abs().max().item() <= tol * x1.abs().max().item()
        # the same call again reuses the graph and gives the same result
        xs2 = [torch.full_like(b, 3.0) for _, b, _ in probs]
        infos2 = fdmpc.pcg_solve_batched(batch, [b for _, b, _ in probs], xs2, 1e-8, 200)
        infos3 = fdmpc.pcg_solve_batched(batch, [b for _, b, _ in probs], xs2, 1e-8, 200)
        for a, c, i in zip(xs, xs2, infos3):
            assert torch.equal(a, c) or precision == FP32
        assert [i.iterations for i in infos2] == [i.iterations for i in infos]
    finally:
        fdmpc.fdm_batch_destroy(batch)


def test_batched_fp64_matches_oracle():
    probs = problems(FP64, [(3, 4, 11), (2, 6, 12)])
    batch = fdmpc.fdm_batch_setup([c.h for c, _, _ in probs])
    try:
        xs = [torch.zeros_like(b) for _, b, _ in probs]
        infos = fdmpc.pcg_solve_batched(batch, [b for _, b, _ in probs], xs, 1e-8, 200)
        for (ctx, b, (xv, yv, zv)), x, info in zip(probs, xs, infos):
            ref = oracle.Problem(ctx.p, xv, yv, zv)
            ref.setup_patches()
            ref.setup_coarse()
            ref.set_omega(ctx.omega)
            xr, it, _, _ = ref.pcg(b.cpu().numpy(), 1e-8, 200)
            assert abs(info.iterations - it) <= 1
            if info.iterations == it:
                record("batched_fp64", x_relerr=np.abs(x.cpu().numpy() - xr).max() / np.abs(xr).max())
                assert np.abs(x.cpu().numpy() - xr).max() <= 1e-11 * np.abs(xr).max()
    finally:
        fdmpc.fdm_batch_destroy(batch)


def test_batched_edge_cases():
    probs = problems(FP32, [(2, 3, 21), (3, 4, 22), (2, 5, 23)])
    batch = fdmpc.fdm_batch_setup([c.h for c, _, _ in probs])
    try:
        bs = [b for _, b, _ in probs]
        bs[1] = torch.zeros_like(bs[1])                  # b = 0: converged at once, x = 0
        xs = [torch.full_like(b, 7.0) for b in bs]
        infos = fdmpc.pcg_solve_batched(batch, bs, xs, 1e-8, 200)
        assert infos[1].converged and infos[1].iterations == 0 and torch.count_nonzero(xs[1]).item() == 0
        assert infos[0].converged and infos[2].converged
        # maxit reached for every problem: ENOCONV, iterations == maxit
        rc, infos = fdmpc.pcg_solve_batched(batch, bs, xs, 1e-14, 2, check=False)
        assert rc == fdmpc.FDM_ENOCONV
        assert infos[0].iterations == 2 and not infos[0].converged
        assert infos[1].iterations == 0 and infos[1].converged
        # a changed rtol rebuilds the graph and converges again
        infos = fdmpc.pcg_solve_batched(batch, bs, xs, 1e-6, 200)
        assert all(i.converged for i in infos)
        assert infos[0].rnorm <= 1e-6 * infos[0].rnorm0
    finally:
        fdmpc.fdm_batch_destroy(batch)


def _free(ctx):
    return (ctx.N[0] - 2) * (ctx.N[1] - 2) * (ctx.N[2] - 2)


def test_full_batch_workload():
    """The 64-problem workload as the benchmark runs it (n in 2..10, p in
    3..15, mixed precision, autotuned patch solves, one graph): every solve
    reaches the FP64 true residual 1e-8, and the smallest problems match the
    FP64 oracle's solution to the solver tolerance."""
    probs = inputs.batch_problems(64, 1000)
    ctxs, bs = [], []
    for w in probs:
        n, p = len(w["xv"]) - 1, w["p"]
        nd = (n * p + 1) ** 3
        ctxs.append(fdmpc.Context(p, w["xv"], w["yv"], w["zv"], precision=FP32, lanczos_start=inputs.lanczos_start(nd),
                                  autotune=1))
        bs.append(torch.tensor(inputs.normal_rhs(nd, w["seed"]), device=DEV))
    batch = fdmpc.fdm_batch_setup([c.h for c in ctxs])
    try:
        xs = [torch.empty_like(b) for b in bs]
        infos = fdmpc.pcg_solve_batched(batch, bs, xs, 1e-8, 300)
        record("batched_full_worst", true_rel=max(i.true_rnorm / i.rnorm0 for i in infos))
        for info in infos:
            assert info.converged and info.true_rnorm <= 1e-8 * info.rnorm0
        # the smaller problems run at higher kernel priority: the smallest quarter is done
        # before the largest quarter
        lat = np.array([i.seconds for i in infos])
        size = np.array([_free(c) for c in ctxs])
        order = np.argsort(size)
        assert np.median(lat[order[:16]]) < np.median(lat[order[-16:]])
        small = sorted(range(64), key=lambda i: (len(probs[i]["xv"]) - 1) ** 3 * probs[i]["p"] ** 3)[:4]
        for i in small:
            w = probs[i]
            ref = oracle.Problem(w["p"], w["xv"], w["yv"], w["zv"])
            ref.setup_patches()
            ref.setup_coarse()
            ref.set_omega(ctxs[i].omega)
            b = bs[i].cpu().numpy()
            from tests import bruteforce as bf
            n = len(w["xv"]) - 1
            b = np.where(bf.free_mask(w["p"], n, n, n), b, 0.0)
            x_ref, _, _, conv = ref.pcg(b, 1e-10, 400)
            assert conv
            x = xs[i].cpu().numpy()
            assert np.abs(x - x_ref).max() <= 1e-6 * np.abs(x_ref).max()
    finally:
        fdmpc.fdm_batch_destroy(batch)
        for c in ctxs:
            c.close()


# ---------------------------------------------------------------- lockstep schedule
def test_lockstep_matches_branches():
    """The lockstep schedule (one loop for all problems, the star solves of all
    active problems in one launch over the global patch list) against the
    branch schedule: every problem converges to the FP64 true residual 1e-8,
    within one iteration of the branch schedule's count, and the iterates agree
    to the FP32 preconditioner's precision; a problem that stops earlier is
    done earlier."""
    probs = problems(FP32, SPECS)
    hs = [c.h for c, _, _ in probs]
    bs = [b for _, b, _ in probs]
    br = fdmpc.fdm_batch_setup(hs)
    ls = fdmpc.fdm_batch_setup(hs, mode=fdmpc.FDM_BATCH_LOCKSTEP)
    try:
        x0 = [torch.zeros_like(b) for b in bs]
        x1 = [torch.zeros_like(b) for b in bs]
        i0 = fdmpc.pcg_solve_batched(br, bs, x0, 1e-8, 200)
        i1 = fdmpc.pcg_solve_batched(ls, bs, x1, 1e-8, 200)
        for a, b, xa, xb in zip(i0, i1, x0, x1):
            assert b.converged and b.true_rnorm <= 1e-8 * b.rnorm0
            assert abs(a.iterations - b.iterations) <= 1
            assert (xa - xb).abs().max().item() <= 1e-6 * xa.abs().max().item()
        its = [i.iterations for i in i1]
        lo, hi = int(np.argmin(its)), int(np.argmax(its))
        if its[lo] < its[hi]:
            assert i1[lo].seconds < i1[hi].seconds
        record("lockstep_small", iterations=sum(its), worst=max(i.true_rnorm / i.rnorm0 for i in i1))
        # the same call again reuses the graph
        i2 = fdmpc.pcg_solve_batched(ls, bs, x1, 1e-8, 200)
        assert [i.iterations for i in i2] == its
    finally:
        fdmpc.fdm_batch_destroy(br)
        fdmpc.fdm_batch_destroy(ls)


def test_lockstep_edge_cases():
    """b = 0 converges at once and drops out; maxit stops a problem with
    FDM_ENOCONV while the others converge; FP64 preconditioners are refused."""
    probs = problems(FP32, [(2, 3, 11), (3, 4, 12)])
    ls = fdmpc.fdm_batch_setup([c.h for c, _, _ in probs], mode=fdmpc.FDM_BATCH_LOCKSTEP)
    try:
        bs = [torch.zeros_like(probs[0][1]), probs[1][1]]
        xs = [torch.full_like(b, 7.0) for b in bs]
        infos = fdmpc.pcg_solve_batched(ls, bs, xs, 1e-8, 200)
        assert infos[0].converged and infos[0].iterations == 0 and float(xs[0].abs().max()) == 0.0
        assert infos[1].converged and infos[1].true_rnorm <= 1e-8 * infos[1].rnorm0
        bs2 = [probs[0][1], probs[1][1]]
        with pytest.raises(fdmpc.FdmError) as e:
            fdmpc.pcg_solve_batched(ls, bs2, xs, 1e-14, 3)
        assert e.value.code == fdmpc.FDM_ENOCONV
    finally:
        fdmpc.fdm_batch_destroy(ls)
    p64 = problems(FP64, [(2, 3, 13)])
    with pytest.raises(fdmpc.FdmError) as e:
        fdmpc.fdm_batch_setup([p64[0][0].h], mode=fdmpc.FDM_BATCH_LOCKSTEP)
    assert e.value.code == fdmpc.FDM_EINVAL
