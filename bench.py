"""Benchmark: PCG solve throughput (free DoF/s to a 1e-8 relative residual).

Default workload (N=1): Poisson on a 16^3 graded tensor hex mesh (per-axis
widths U(0.5, 1.5), normalised), Q7 on GLL nodes (113^3 = 1,442,897 nodes,
1,367,631 free dofs), f = seeded N(0,1) nodal values, b = M f; PCG with the
hybrid V(1,1) vertex-star FDM/sparse relaxation, FP32 preconditioner inside
FP64 PCG, rtol 1e-8 from x0 = 0.  A step is one full PCG solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank solves its own instance (different right-hand
side) of the same problem: independent problems, weak scaling, no
collective on the data path (the barrier and the max over ranks of the
timing are the only collectives).
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "q7_graded16"
WORKLOAD_TEXT = ("q7_graded16: 16^3 graded hex mesh, Q7, 1,367,631 free dofs, N(0,1) nodal f, "
                 "FP32 V(1,1) preconditioner in FP64 PCG, rtol 1e-8")
RTOL = 1e-8
MAXIT = 200
CPU_SAMPLE_N = 16  # CPU baseline: the oracle on the benchmark workload itself (16^3 graded, Q7)
FALLBACK_HBM_GBS = 6800.0
# DRAM traffic of one launch of the FP32 Schur-coupling patch solve at 16^3
# graded Q7 (dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture,
# summarised in profiles/patch_solve_q7_graded16.md), valid while the kernel
# source k_asm.cu has the recorded sha256; null otherwise.
PROFILED_TRAFFIC = {"kernel_source_sha256": "2b4aaf171d58b34b08b3b44559a3cc2774f39bf782c7ce6d48e9bd638376db3e",
                    "dram_bytes_per_launch": 0.34421e9,
                    "source": "profiles/patch_solve_q7_graded16.md (one ncu capture, same kernel source)"}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(value, device=None):
    """Maximum over the ranks of a per-rank number (identity without a process
    group): the slowest rank's time is the job's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world_size, units_per_rank, steps, ms_max):
    """Whole-job units per second: every rank processes units_per_rank per step
    (independent problems, weak scaling) and the job takes the slowest rank's time."""
    return world_size * units_per_rank * steps / (ms_max * 1e-3)


def rank_rhs_seed(base_seed, rank):
    """Seed of a rank's right-hand side: every rank solves its own instance."""
    return base_seed + 1000 * rank


def _peak_bf16():
    """Dense bf16 tensor peak in TFLOP/s: the measured burst figure, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:
        return 1900.0


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _traffic_from_profile(kernel_src):
    """Per-launch DRAM bytes of the patch-solve kernel from the recorded ncu
    capture, if it was taken on the current kernel source (else None)."""
    if PROFILED_TRAFFIC["dram_bytes_per_launch"] is None:
        return None
    sha = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()
    return PROFILED_TRAFFIC["dram_bytes_per_launch"] if sha == PROFILED_TRAFFIC["kernel_source_sha256"] else None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "fdmpc_clocks_%d.csv" % os.getpid())

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
            return
        # wait for the first sample so that the timed region is covered, and keep
        # only the samples taken after it (the GPU may idle at lower clocks before)
        t0 = time.time()
        self.skip = 0
        while time.time() - t0 < 5.0:
            self.f.flush()
            try:
                with open(self.path) as g:
                    n = sum(1 for _ in g)
            except OSError:
                n = 0
            if n > 0:
                break
            time.sleep(0.01)
        # let the sampler settle (its first queries can stall the GPU briefly), then
        # keep only the samples taken from here on
        time.sleep(0.5)
        self.f.flush()
        try:
            with open(self.path) as g:
                self.skip = sum(1 for _ in g)
        except OSError:
            self.skip = 0

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln, line in enumerate(open(self.path)):
            if ln < getattr(self, "skip", 0):
                continue
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nme, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nme)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _free_dofs(N):
    return (N[0] - 2) * (N[1] - 2) * (N[2] - 2)


def cpu_sample_problem():
    from paper_2107_14758_gb300 import inputs
    xv, yv, zv = inputs.graded_vertices(CPU_SAMPLE_N, 2)
    return 7, xv, yv, zv


def run_oracle_solve(P, b):
    t0 = time.perf_counter()
    x, it, _, conv = P.pcg(b, rtol=RTOL, maxit=MAXIT)
    return time.perf_counter() - t0, it, conv


def oracle_problem():
    """The CPU sample problem set up by the oracle; returns (problem, b, set-up seconds)."""
    import oracle
    from paper_2107_14758_gb300 import inputs
    oracle.build()
    p, xv, yv, zv = cpu_sample_problem()
    t0 = time.perf_counter()
    P = oracle.Problem(p, xv, yv, zv)
    P.setup_patches()
    P.setup_coarse()
    P.lanczos_omega(inputs.lanczos_start(P.ndof))
    setup_s = time.perf_counter() - t0
    b = P.mass_apply(inputs.normal_rhs(P.ndof, 2))
    return P, b, setup_s


def cpu_cores():
    """Threads the oracle's OpenMP loops use: OMP_NUM_THREADS, else the CPUs this process may run on."""
    if os.environ.get("OMP_NUM_THREADS", "").strip().isdigit():
        return int(os.environ["OMP_NUM_THREADS"])
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_single_core(n=6):
    """The oracle's PCG solve of the same family on an n^3 mesh with one
    OpenMP thread, in a fresh interpreter (the thread count is fixed when the
    OpenMP runtime starts).  Returns {"value": DoF/s, ...} or None."""
    code = ("import json, sys, time; sys.path.insert(0, %r)\n"
            "import oracle\n"
            "from paper_2107_14758_gb300 import inputs\n"
            "xv, yv, zv = inputs.graded_vertices(%d, 2)\n"
            "t0 = time.perf_counter()\n"
            "P = oracle.Problem(7, xv, yv, zv); P.setup_patches(); P.setup_coarse()\n"
            "P.lanczos_omega(inputs.lanczos_start(P.ndof))\n"
            "t1 = time.perf_counter()\n"
            "b = P.mass_apply(inputs.normal_rhs(P.ndof, 2))\n"
            "t2 = time.perf_counter()\n"
            "x, it, _, conv = P.pcg(b, rtol=%r, maxit=%d)\n"
            "t3 = time.perf_counter()\n"
            "print(json.dumps({'free': (%d * 7 - 1) ** 3, 'setup_s': t1 - t0, 'solve_s': t3 - t2, 'iterations': it}))\n"
            % (ROOT, n, RTOL, MAXIT, n))
    env = dict(os.environ, OMP_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=300)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return None
    return {"value": d["free"] / d["solve_s"], "unit": "DoF/s", "cores": 1, "setup_s": d["setup_s"],
            "iterations": d["iterations"],
            "sample": "the same family on a %d^3 mesh (Q7, %d free dofs), one OpenMP thread" % (n, d["free"])}


def oracle_secondary():
    """The FP64 oracle on bounded samples of the secondary workloads' families
    (all host cores): per family its PCG solve rate and the sample."""
    import oracle
    from oracle import elasticity as oel, sipg as osg, unstructured as oun
    from paper_2107_14758_gb300 import inputs
    oracle.build()
    out = {}

    def timed(setup, solve):
        t0 = time.perf_counter()
        setup()
        t1 = time.perf_counter()
        it = solve()
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1, it

    xv = np.linspace(0, 1, 5)
    E = oel.Elasticity(3, xv, xv, xv, 1.0, 1.0, dirichlet_faces=1)
    bE = E.body_force([0.0, -0.02, 0.0]).ravel()
    su, so, it = timed(lambda: (E.setup_sdc(), E.setup_coarse(), E.lanczos_omega(inputs.lanczos_start(3 * E.N))),
                       lambda: E.pcg(bE, rtol=RTOL, maxit=MAXIT)[1])
    free = 3 * int(E.free.sum())
    out["elasticity"] = {"value": free / so, "unit": "DoF/s", "solve_s": so, "setup_s": su, "iterations": it,
                         "sample": "4^3 uniform, p = 3, lambda = 1, x_1 = 0 clamped, %d free dofs" % free}
    sv = inputs.graded_vertices(4, 7)
    S = osg.Sipg(3, *sv)
    bS = np.random.default_rng(8).standard_normal(S.N)
    su, so, it = timed(lambda: (S.setup_patches(), S.setup_coarse(), S.lanczos_omega(inputs.lanczos_start(S.N))),
                       lambda: S.pcg(bS, rtol=RTOL, maxit=MAXIT)[1])
    out["sipg"] = {"value": S.N / so, "unit": "DoF/s", "solve_s": so, "setup_s": su, "iterations": it,
                   "sample": "DQ_3 on 4^3 graded cells, %d values" % S.N}
    X, cells = inputs.unstructured_hex_mesh(3, 2, 5)
    U = oun.HexProblem(5, X, cells)
    bU = U.mass_apply(np.ones(U.ndof))
    su, so, it = timed(lambda: (U.setup_patches(), U.setup_coarse(), U.lanczos_omega(inputs.lanczos_start(U.ndof))),
                       lambda: U.pcg(bU, rtol=RTOL, maxit=MAXIT)[1])
    free = int(U.free.sum())
    out["unstructured"] = {"value": free / so, "unit": "DoF/s", "solve_s": so, "setup_s": su, "iterations": it,
                           "sample": "extruded unstructured mesh m = 3, 2 layers (%d cells), Q5, %d free dofs"
                                     % (cells.shape[0], free)}
    w = inputs.deformed_problem(4, 8, 4)
    P = oracle.Problem(8, w["xv"], w["yv"], w["zv"], jac=w["jac"], kappa=w["kappa"])
    bP = P.mass_apply(inputs.normal_rhs(P.ndof, 4))
    su, so, it = timed(lambda: (P.setup_patches(), P.setup_coarse(), P.lanczos_omega(inputs.lanczos_start(P.ndof))),
                       lambda: P.pcg(bP, rtol=RTOL, maxit=DEFORMED_MAXIT)[1])
    free = _free_dofs(P.N)
    out["deformed"] = {"value": free / so, "unit": "DoF/s", "solve_s": so, "setup_s": su, "iterations": it,
                       "sample": "4^3 deformed mesh, kappa = exp(G), Q8, %d free dofs" % free}
    return out


SAMPLE_TEXT = ("the benchmark workload itself (16^3 graded mesh, Q7, 1,367,631 free dofs, the same b, PCG + "
               "V(1,1), rtol 1e-8) in the FP64 oracle on all host cores; one step = one full PCG solve; "
               "DoF/s = free dofs / solve wall time, set-up excluded (reported as setup_s)")


def bench_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    P, b, setup_s = oracle_problem()
    free = _free_dofs(P.N)
    for _ in range(args.warmup):
        run_oracle_solve(P, b)
    times, its = [], []
    for _ in range(args.steps):
        t, it, conv = run_oracle_solve(P, b)
        times.append(t)
        its.append(it)
    tot = sum(times)
    value = free * args.steps / tot
    line = {"impl": "reference", "metric": "pcg_solve_dofs_per_s", "value": value, "unit": "DoF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT, "sample": SAMPLE_TEXT, "same_config": True,
                       "iterations": int(np.median(its))},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": SAMPLE_TEXT, "same_config": True, "setup_s": setup_s,
                             "single_core": oracle_single_core()},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_gpu(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)

    import __graft_entry__ as ge
    if rank == 0 or ws == 1:
        ge.build()
    if ws > 1:
        dist.barrier()
    from paper_2107_14758_gb300 import fdmpc, inputs

    w = inputs.workload(WORKLOAD)
    # the timed solves: the device-driven PCG loop (captured graph), no per-kernel events
    ctx = fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], precision=fdmpc.FDM_PREC_FP32, autotune=1,
                        pcg_graph=0 if args.pcg_host_loop else 1)
    setup_s = list(ctx.setup_seconds())
    tuning = ctx.tuning()
    free = _free_dofs(ctx.N)
    f = torch.tensor(inputs.normal_rhs(ctx.ndof, rank_rhs_seed(w["seed"], rank)), device=dev)
    b = ctx.mass_apply(f)
    x = torch.empty_like(b)

    def step():
        return ctx.pcg_solve(b, x, rtol=RTOL, maxit=MAXIT)[1]

    args.warmup = max(args.warmup, 3)  # at least 3 untimed warm-up solves
    for _ in range(args.warmup):
        info = step()
    ctx.launches()
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(dev.index)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    torch.cuda.nvtx.range_push("timed_solves")
    iters = []
    for _ in range(args.steps):
        info = step()
        iters.append(info.iterations)
    torch.cuda.nvtx.range_pop()
    e1.record(stream)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    launches = ctx.launches()
    ms_max = reduce_max(ms, dev)
    value = job_throughput(ws, free, args.steps, ms_max)
    rel = info.true_rnorm / info.rnorm0

    # ---- end to end through the C-ABI with host buffers (copies timed)
    hb = torch.empty(ctx.ndof, dtype=torch.float64, pin_memory=True)
    hb.copy_(b.cpu())
    hx = torch.empty(ctx.ndof, dtype=torch.float64, pin_memory=True)
    db = torch.empty_like(b)
    torch.cuda.synchronize()
    if ws > 1:
        dist.barrier()
    db.copy_(hb, non_blocking=True)
    fdmpc.pcg_solve(ctx.h, db, x, RTOL, MAXIT)  # untimed: captures the graph for these buffers
    torch.cuda.synchronize()
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        db.copy_(hb, non_blocking=True)
        fdmpc.pcg_solve(ctx.h, db, x, RTOL, MAXIT)
        hx.copy_(x, non_blocking=True)
    e3.record(stream)
    torch.cuda.synchronize()
    e2e_value = job_throughput(ws, free, args.steps, reduce_max(e2.elapsed_time(e3), dev))

    # ---- roofline of the dominant kernel (patch solve), FP32 factors: the same
    # solves through the host loop with CUDA events around every kernel group
    ctx_kt = fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], precision=fdmpc.FDM_PREC_FP32, kernel_timing=1,
                           patch_kernel={3: 3, 6: 5, 7: 6, 8: 7}.get(tuning[0], 1), patch_threads=tuning[1],
                           patch_rows_per_warp=8 if tuning[2] else 4, sc_variant=tuning[2] + 1)
    for _ in range(args.warmup):
        ctx_kt.pcg_solve(b, x, rtol=RTOL, maxit=MAXIT)
    ctx_kt.kernel_times()
    torch.cuda.synchronize()
    e8 = torch.cuda.Event(enable_timing=True)
    e9 = torch.cuda.Event(enable_timing=True)
    e8.record(stream)
    torch.cuda.nvtx.range_push("roofline_solves")
    for _ in range(args.steps):
        ctx_kt.pcg_solve(b, x, rtol=RTOL, maxit=MAXIT)
    torch.cuda.nvtx.range_pop()
    e9.record(stream)
    torch.cuda.synchronize()
    kt = ctx_kt.kernel_times()
    ms_kt = e8.elapsed_time(e9) / args.steps
    ab = ctx_kt.algo_bytes()
    ctx_kt.close()
    pcount, pms = kt["patch"]
    patch_ms = pms / max(pcount, 1)
    peak, peak_kind = _peak_hbm()
    achieved = ab["patch32"] / (patch_ms * 1e-3) / 1e9
    traffic = _traffic_from_profile(os.path.join(ROOT, "paper_2107_14758_gb300", "csrc", "k_asm.cu"))

    # ---- secondary numbers (same workload): pc_apply throughput and the FP64 form
    r = torch.randn(ctx.ndof, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)
    for _ in range(3):
        ctx.pc_apply(r, z)
    torch.cuda.synchronize()
    e4 = torch.cuda.Event(enable_timing=True)
    e5 = torch.cuda.Event(enable_timing=True)
    e4.record(stream)
    for _ in range(20):
        ctx.pc_apply(r, z)
    e5.record(stream)
    torch.cuda.synchronize()
    pc_ms = e4.elapsed_time(e5) / 20
    ctx.kernel_times()
    ctx.launches()
    secondary = {"pc_apply_gdofs": free / (pc_ms * 1e-3) / 1e9, "pc_apply_ms": pc_ms}
    try:  # one damped additive Schwarz sweep (asm_apply), the relaxation alone
        for _ in range(3):
            ctx.asm_apply(r, z)
        torch.cuda.synchronize()
        e4.record(stream)
        for _ in range(20):
            ctx.asm_apply(r, z)
        e5.record(stream)
        torch.cuda.synchronize()
        asm_ms = e4.elapsed_time(e5) / 20
        secondary["asm_apply_gdofs"] = free / (asm_ms * 1e-3) / 1e9
        secondary["asm_apply_ms"] = asm_ms
    except Exception as exc:  # noqa: BLE001
        secondary["asm_apply_error"] = "%s: %s" % (type(exc).__name__, exc)
    if not args.no_fp64:
        ctx64 = fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], precision=fdmpc.FDM_PREC_FP64)
        for _ in range(2):
            ctx64.pcg_solve(b, x, rtol=RTOL, maxit=MAXIT)
        torch.cuda.synchronize()
        e6 = torch.cuda.Event(enable_timing=True)
        e7 = torch.cuda.Event(enable_timing=True)
        e6.record(stream)
        k64 = max(2, args.steps // 2)
        for _ in range(k64):
            info64 = ctx64.pcg_solve(b, x, rtol=RTOL, maxit=MAXIT)[1]
        e7.record(stream)
        torch.cuda.synchronize()
        ms64 = e6.elapsed_time(e7) / k64
        secondary["fp64_pc_solve_dofs_per_s"] = free / (ms64 * 1e-3)
        secondary["fp64_pc_iterations"] = info64.iterations
        secondary["mixed_over_fp64"] = (free / (ms_max * 1e-3 / args.steps)) / secondary["fp64_pc_solve_dofs_per_s"]
        ctx64.close()

    if rank == 0 and ws == 1 and not args.no_extra:
        extra = {"p15": lambda: bench_p15(dev, fdmpc, inputs, peak),
                 "deformed": lambda: bench_deformed(dev, fdmpc, inputs),
                 "batched": lambda: bench_batched(dev, fdmpc, inputs),
                 "gmg": lambda: bench_gmg(dev, fdmpc, inputs),
                 "elasticity": lambda: bench_elasticity(dev, fdmpc, inputs),
                 "sipg": lambda: bench_sipg(dev, fdmpc, inputs),
                 "unstructured": lambda: bench_unstructured(dev, fdmpc, inputs, peak)}
        for name in (args.extra.split(",") if args.extra else extra):
            # a failing secondary workload is reported in the line, not allowed to lose it
            try:
                secondary[name] = extra[name]()
            except Exception as exc:  # noqa: BLE001
                secondary[name] = {"error": "%s: %s" % (type(exc).__name__, exc)}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        P, bc, setup_cpu = oracle_problem()
        t, it, conv = run_oracle_solve(P, bc)
        cpu = {"value": _free_dofs(P.N) / t, "unit": "DoF/s", "cores": cpu_cores(), "kind": "oracle",
               "sample": SAMPLE_TEXT, "same_config": True, "solve_s": t, "setup_s": setup_cpu,
               "iterations": it, "single_core": oracle_single_core()}
        del P
        if not args.no_extra:
            try:
                cpu["secondary"] = oracle_secondary()
            except Exception as exc:  # reported, not fatal
                cpu["secondary"] = {"error": "%s: %s" % (type(exc).__name__, exc)}

    if rank == 0:
        line = {"metric": "pcg_solve_dofs_per_s", "value": value, "unit": "DoF/s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32+f64", "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT,
                           "global_batch": ws, "parallelism": "independent problems per GPU" if ws > 1 else "1 GPU",
                           "l2": "inputs larger than L2 (%.0f MB of FP32 patch factors per solve sweep)" %
                                 (ab["patch32"] / 1e6),
                           "iterations": int(np.median(iters)), "true_rel_residual": rel,
                           "setup_seconds": sum(setup_s),
                           "pcg_loop": "host" if args.pcg_host_loop else "device (CUDA graph)",
                           "autotuned_patch_solve": {"kernel": {3: "resident", 5: "one CTA per patch, Schur-coupling form",
                                                                6: "persistent, Schur-coupling form",
                                                                7: "persistent, whole patch staged, Schur-coupling form",
                                                                8: "one warp per patch, Schur-coupling form"}.get(
                                                         tuning[0], "one CTA per patch"),
                                                     "threads": tuning[1], "variant": tuning[2],
                                                     "sweep_us": tuning[3], "candidates": tuning[4]}},
                "clocks": clocks,
                "e2e": {"value": e2e_value, "unit": "DoF/s", "h2d_bytes_per_step": 8 * ctx.ndof,
                        "d2h_bytes_per_step": 8 * ctx.ndof},
                "gpu_launches": int(launches),
                "roofline": {"kernel": {3: "k_patch_resident<float>", 5: "k_patch_solve_sc<float>",
                                        6: "k_patch_solve_scp<float>", 7: "k_patch_solve_scf<float>",
                                        8: "k_patch_solve_scw<float>"}.get(
                                 tuning[0], "k_patch_solve<float>"),
                             "bound": "hbm", "achieved": achieved, "peak": peak,
                             "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                             "traffic_source": PROFILED_TRAFFIC["source"] if traffic is not None else
                                               "none: no ncu capture of the current kernel source",
                             "algorithmic_bytes_per_launch": ab["patch32"], "avg_launch_ms": patch_ms,
                             # the same launch time against the bytes the L form of the patch solve
                             # would have to move (the dense L21 block and Z): what the form change bought
                             "l_form_bytes_per_launch": ab["lform32"],
                             "l_form_equivalent_frac": ab["lform32"] / (patch_ms * 1e-3) / 1e9 / peak,
                             "launches": pcount},
                "kernel_ms_per_step": {k: v[1] / args.steps for k, v in kt.items()},
                "kernel_timed_solve_ms": ms_kt,
                "secondary": secondary,
                "cpu_baseline": cpu}
        # the figures the targets rest on, last in the line (kept by a tail of the output)
        p15 = secondary.get("p15", {})
        line["targets"] = {
            "q7": {"mixed_dofs_per_s": value, "fp64_pc_dofs_per_s": secondary.get("fp64_pc_solve_dofs_per_s"),
                   "mixed_over_fp64": secondary.get("mixed_over_fp64"), "true_rel_residual": rel,
                   "pc_apply_ms": secondary.get("pc_apply_ms"), "asm_apply_ms": secondary.get("asm_apply_ms"),
                   "patch_solve_ms": patch_ms, "patch_solve_hbm_frac": achieved / peak},
            "p15": {k: p15.get(k) for k in ("mixed_solve_dofs_per_s", "fp64_solve_dofs_per_s", "mixed_over_fp64",
                                              "mixed_true_rel_residual", "pc_apply_ms", "sweep_ms",
                                              "sweep_hbm_frac_of_measured", "sweep_lform_equivalent_frac")},
            "p15_sweep_target": "<= 450 us per FP32 sweep, >= 0.5 of measured HBM",
            "unstructured_q7": {k: (secondary.get("unstructured", {}).get("mixed", {}) or {}).get(k)
                                for k in ("solve_dofs_per_s", "iterations", "true_rel_residual")},
            "deformed_q8": {"averaged_mixed_dofs_per_s": secondary.get("deformed", {}).get("mixed_solve_dofs_per_s"),
                            "learned_judged_dofs_per_s": (secondary.get("deformed", {}).get("learned") or {}).get(
                                "judged_solve_dofs_per_s"),
                            "fp64_dofs_per_s": secondary.get("deformed", {}).get("fp64_solve_dofs_per_s"),
                            "iterations_averaged_learned": [
                                secondary.get("deformed", {}).get("mixed_iterations"),
                                (secondary.get("deformed", {}).get("learned") or {}).get("judged_iterations")]},
            "elasticity_table3_setting_p15": (secondary.get("elasticity", {}).get("iterations_traction_free_x0") or
                                              {}).get("p=15"),
            "batched": {k: secondary.get("batched", {}).get(k)
                        for k in ("aggregate_dofs_per_s", "one_after_another_dofs_per_s", "fp64_aggregate_dofs_per_s",
                                  "latency_ms_p50", "latency_ms_p99")},
            "cpu_oracle_same_config_dofs_per_s": cpu["value"] if cpu else None}
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


def _timed_solves(ctx, b, x, k, maxit=None):
    """(ms per solve, last info) of k PCG solves after 2 untimed ones (CUDA events)."""
    import torch
    maxit = maxit or MAXIT
    for _ in range(2):
        ctx.pcg_solve(b, x, rtol=RTOL, maxit=maxit)
    torch.cuda.synchronize()
    s0 = torch.cuda.Event(enable_timing=True)
    s1 = torch.cuda.Event(enable_timing=True)
    s0.record(torch.cuda.current_stream())
    for _ in range(k):
        info = ctx.pcg_solve(b, x, rtol=RTOL, maxit=maxit)[1]
    s1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    return s0.elapsed_time(s1) / k, info


def bench_p15(dev, fdmpc, inputs, peak):
    """High-order Poisson at p = 15 (8^3 uniform, manufactured sine): mixed and
    FP64 solves, pc_apply throughput and its HBM fraction."""
    import torch
    w = inputs.workload("q15_uniform8")
    ctx = fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], precision=fdmpc.FDM_PREC_FP32, autotune=1)
    free = _free_dofs(ctx.N)
    b = ctx.mass_apply(torch.tensor(inputs.manufactured_f(w["xv"], w["yv"], w["zv"], w["p"]), device=dev))
    x = torch.empty_like(b)
    ms, info = _timed_solves(ctx, b, x, 3)
    r = torch.randn(ctx.ndof, dtype=torch.float64, device=dev)
    z = torch.empty_like(r)
    for _ in range(3):
        ctx.pc_apply(r, z)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(torch.cuda.current_stream())
    for _ in range(10):
        ctx.pc_apply(r, z)
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    pc_ms = e0.elapsed_time(e1) / 10
    for _ in range(3):
        ctx.asm_apply(r, z)
    torch.cuda.synchronize()
    e0.record(torch.cuda.current_stream())
    for _ in range(10):
        ctx.asm_apply(r, z)
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    sweep_ms = e0.elapsed_time(e1) / 10
    ab = ctx.algo_bytes()
    # the L form's bytes of one sweep: sum nnz(L_Gamma) plus the same vector and cell terms
    lform_sweep = ab["lform32"] + (ab["asm32"] - ab["patch32"])
    out = {"workload": "q15_uniform8: 8^3 uniform hex mesh, Q15, %d free dofs, manufactured sine" % free,
           "sweep_ms": sweep_ms, "sweep_bytes": ab["asm32"], "sweep_lform_bytes": lform_sweep,
           "sweep_hbm_frac_of_measured": ab["asm32"] / (sweep_ms * 1e-3) / 1e9 / peak,
           "sweep_lform_equivalent_frac": lform_sweep / (sweep_ms * 1e-3) / 1e9 / peak,
           "mixed_solve_dofs_per_s": free / (ms * 1e-3), "mixed_iterations": info.iterations,
           "mixed_true_rel_residual": info.true_rnorm / info.rnorm0,
           "pc_apply_ms": pc_ms, "pc_apply_gdofs": free / (pc_ms * 1e-3) / 1e9,
           # two FP32 relaxation sweeps' algorithmic bytes (a lower bound of pc_apply's)
           "pc_apply_sweep_bytes": 2 * ab["asm32"],
           "pc_apply_hbm_frac_of_measured": 2 * ab["asm32"] / (pc_ms * 1e-3) / 1e9 / peak}
    ctx.close()
    ctx64 = fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], precision=fdmpc.FDM_PREC_FP64)
    ms64, info64 = _timed_solves(ctx64, b, x, 2)
    out["fp64_solve_dofs_per_s"] = free / (ms64 * 1e-3)
    out["fp64_iterations"] = info64.iterations
    out["mixed_over_fp64"] = ms64 / ms
    ctx64.close()
    return out


def bench_gmg(dev, fdmpc, inputs):
    """32^3 graded Q7 (11 M free dofs): the Q1 coarse problem (29,791 unknowns)
    is solved by one geometric multigrid V-cycle per preconditioner application
    (levels 32^3 -> 16^3 -> 8^3 -> 4^3 -> 2^3 cells, exact solve on the last);
    the exact coarse solve would stream a 29,791^2 dense inverse every V-cycle."""
    import numpy as np
    import torch
    w = inputs.workload("q7_graded32")
    ctx = fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], precision=fdmpc.FDM_PREC_FP32, autotune=1)
    free = _free_dofs(ctx.N)
    f = torch.randn(ctx.ndof, dtype=torch.float64, device=dev,
                    generator=torch.Generator(device=dev).manual_seed(w["seed"]))
    b = ctx.mass_apply(f)
    x = torch.empty_like(b)
    ms, info = _timed_solves(ctx, b, x, 3)
    setup = ctx.query(fdmpc.FDM_Q_SETUP_SECONDS, np.float64, 4)
    out = {"workload": "q7_graded32: 32^3 graded hex mesh, Q7, %d free dofs, N(0,1) nodal f" % free,
           "coarse": "geometric multigrid V(2,2), damped Jacobi 2/3, levels %s" % [l[:3] for l in ctx.gmg_levels()],
           "mixed_solve_dofs_per_s": free / (ms * 1e-3), "ms_per_solve": ms, "mixed_iterations": info.iterations,
           "mixed_true_rel_residual": info.true_rnorm / info.rnorm0,
           "setup_seconds": {"symbolic": setup[0], "factor": setup[1], "coarse": setup[2], "lanczos": setup[3]}}
    ctx.close()
    return out


# FP32 CUDA-core FMA peak from the unit counts and the maximum SM clock
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 * 1e-12


def bench_sipg(dev, fdmpc, inputs):
    """SIPG on DQ_7 (Section 5), 16^3 graded cells, 2.1 M values, eta = p(p+1):
    PCG to 1e-8 with the hybrid V(1,1) (vertex-star Schwarz with exact star
    solves, Q1 coarse space) in mixed precision and in FP64, and the FP32
    relaxation sweep (3375 stars of 16^3 values, 8 launches) with its FLOP
    rate: 6 line passes of 16^4 multiply-adds per star."""
    import torch
    p = 7
    xv, yv, zv = inputs.graded_vertices(16, 7)
    ndof = 16 ** 3 * (p + 1) ** 3
    m = 2 * (p + 1)
    stars = 15 ** 3
    out = {"workload": "SIPG DQ_7, 16^3 graded cells (widths U(0.5, 1.5), seed 7), %d values, b ~ N(0,1)" % ndof}
    b = torch.randn(ndof, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(7))
    for name, prec, tcore in (("mixed", fdmpc.FDM_PREC_FP32, 0), ("mixed_tensor_core", fdmpc.FDM_PREC_FP32, 1),
                              ("fp64", fdmpc.FDM_PREC_FP64, 0)):
        s = fdmpc.Sipg(p, xv, yv, zv, precision=prec, lanczos_start=inputs.lanczos_start(ndof), tensor_core=tcore)
        x = torch.empty_like(b)
        info = s.pcg_solve(b, x, rtol=RTOL, maxit=1000)[1]
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        for _ in range(3):
            info = s.pcg_solve(b, x, rtol=RTOL, maxit=1000)[1]
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        out[name] = {"ms_per_solve": ms, "solve_dofs_per_s": ndof / (ms * 1e-3), "iterations": info.iterations,
                     "true_rel_residual": info.true_rnorm / info.rnorm0, "omega": s.omega}
        if name.startswith("mixed"):
            z = torch.empty_like(b)
            for _ in range(3):
                s.asm_apply(b, z)
            torch.cuda.synchronize()
            e0.record(torch.cuda.current_stream())
            for _ in range(20):
                s.asm_apply(b, z)
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            ms_sweep = e0.elapsed_time(e1) / 20
            flops = 2.0 * 6 * m ** 4 * stars
            tflops = flops / (ms_sweep * 1e-3) * 1e-12
            if tcore:  # the contractions on the tensor cores: against the TF32 tensor peak
                tf32_peak = _peak_bf16() * 0.5
                out["tf32_sweep"] = {"ms": ms_sweep, "gflop": flops * 1e-9, "tflops": tflops,
                                     "roofline": {"bound": "tensor", "achieved": tflops, "peak": tf32_peak,
                                                  "unit": "TFLOP/s", "frac": tflops / tf32_peak,
                                                  "peak_kind": "measured dense bf16 x 0.5 (nominal TF32/BF16 "
                                                               "ratio 1.1/2.25 PFLOP/s)"}}
            else:
                out["fp32_sweep"] = {"ms": ms_sweep, "gflop": flops * 1e-9, "tflops": tflops,
                                     "roofline": {"bound": "alu", "achieved": tflops, "peak": FP32_ALU_TFLOPS,
                                                  "unit": "TFLOP/s", "frac": tflops / FP32_ALU_TFLOPS,
                                                  "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2 flops x "
                                                               "2.07 GHz"}}
        s.close()
    out["mixed_over_fp64"] = out["mixed"]["solve_dofs_per_s"] / out["fp64"]["solve_dofs_per_s"]
    out["tensor_core_over_cuda_core_sweep"] = out["fp32_sweep"]["ms"] / out["tf32_sweep"]["ms"]
    return out


ELAST_LAMBDAS = (0.0, 1.0, 10.0, 100.0, 1000.0)


TABLE3_ITERATIONS = {3: [20, 22, 39, 114, 362], 7: [25, 28, 48, 123, 381], 15: [27, 29, 51, 125, 373]}
ELAST_MAXIT = 1000  # the iteration tables count PCG steps to the recursive residual's 1e-8


def bench_elasticity(dev, fdmpc, inputs):
    """Primal linear elasticity (Section 4.1) on the 8^3 uniform mesh of the
    unit cube, mu = 1, body force -0.02 e_2, in Table 3's boundary setting
    (clamped at x_1 = 0, traction-free elsewhere; star-local FDM star solves)
    and clamped on every face (FDM/sparse): PCG iterations with the SDC
    relaxation in the hybrid V(1,1) for p = 3, 7, 15 and lambda = 0 .. 1000
    (mixed precision) to the recursive residual's 1e-8 (the count Table 3
    prints, beside it), with the iterations the true residual needs (None:
    not within ELAST_MAXIT) and the true residual reached, and the solve
    throughput at p = 7, lambda = 1."""
    import torch
    xv = [i / 8.0 for i in range(9)]
    out = {"workload": "elasticity 8^3 uniform unit cube, mu = 1, body force -0.02 e_2, SDC relaxation, "
                       "mixed precision",
           "table3_paper": {"lambda": list(ELAST_LAMBDAS), **{"p=%d" % p: v for p, v in TABLE3_ITERATIONS.items()}}}
    for name, mask, degrees in (("traction_free_x0", 1, (3, 7, 15)), ("clamped", 63, (3, 7, 15))):
        table, true_its, true_rel = {}, {}, {}
        for p in degrees:
            its, tits, trel = [], [], []
            n1 = 8 * p + 1
            b = torch.tensor(inputs.body_force_load(xv, xv, xv, p, [0.0, -0.02, 0.0]).ravel(), device=dev)
            x = torch.empty_like(b)
            for lam in ELAST_LAMBDAS:
                e = fdmpc.Elasticity(p, xv, xv, xv, 1.0, lam, precision=fdmpc.FDM_PREC_FP32, dirichlet_faces=mask)
                info = e.pcg_solve(b, x, rtol=RTOL, maxit=ELAST_MAXIT, raise_on_noconv=False)[1]
                its.append(e.recursive_iterations()[0])
                tits.append(info.iterations if info.converged else None)
                trel.append(info.true_rnorm / info.rnorm0)
                if p == 7 and lam == 1.0:
                    free = 3 * (n1 - 2) ** 3 if mask == 63 else 3 * (n1 - 1) * n1 * n1
                    torch.cuda.synchronize()
                    s0 = torch.cuda.Event(enable_timing=True)
                    s1 = torch.cuda.Event(enable_timing=True)
                    s0.record(torch.cuda.current_stream())
                    for _ in range(3):
                        info = e.pcg_solve(b, x, rtol=RTOL, maxit=3000)[1]
                    s1.record(torch.cuda.current_stream())
                    torch.cuda.synchronize()
                    ms = s0.elapsed_time(s1) / 3
                    out["q7_lambda1_" + name] = {"free_dofs": free, "ms_per_solve": ms,
                                                 "solve_dofs_per_s": free / (ms * 1e-3),
                                                 "iterations": info.iterations,
                                                 "true_rel_residual": info.true_rnorm / info.rnorm0}
                e.close()
            table["p=%d" % p] = its
            true_its["p=%d" % p] = tits
            true_rel["p=%d" % p] = trel
        out["iterations_" + name] = {"lambda": list(ELAST_LAMBDAS), **table}
        out["true_residual_iterations_" + name] = true_its
        out["true_residual_reached_" + name] = true_rel
    return out


DEFORMED_MAXIT = 2000  # kappa = exp(G) needs far more iterations than the Poisson cases


def bench_deformed(dev, fdmpc, inputs):
    """Non-separable Poisson (12^3 deformed mesh, kappa = exp(G), Q8): averaged
    surrogate (mixed and FP64) and the learned surrogate judged by it."""
    import torch
    w = inputs.workload("q8_deformed12")
    nd = (12 * 8 + 1) ** 3

    def make(precision):
        return fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], jac=w["jac"], kappa=w["kappa"],
                             samples27=w["samples27"], precision=precision, lanczos_start=inputs.lanczos_start(nd))
    ctx = make(fdmpc.FDM_PREC_FP32)
    free = _free_dofs(ctx.N)
    b = torch.tensor(inputs.normal_rhs(ctx.ndof, w["seed"]), device=dev)
    x = torch.empty_like(b)
    ms, info = _timed_solves(ctx, b, x, 3, DEFORMED_MAXIT)
    lo, hi = ctx.lanczos_extremes()
    out = {"workload": "q8_deformed12: 12^3 deformed hex mesh, kappa = exp(G), Q8, %d free dofs, N(0,1) load" % free,
           "mixed_solve_dofs_per_s": free / (ms * 1e-3), "mixed_iterations": info.iterations,
           "lanczos_cond_averaged": hi / lo}
    # the two label kinds applied directly here (mu = mu_avg exp(c)): what each target is worth
    direct = {}
    for name, kind in (("theorem1", fdmpc.FDM_LABEL_THEOREM1), ("patch_kappa", fdmpc.FDM_LABEL_PATCH_KAPPA)):
        c = make(fdmpc.FDM_PREC_FP32)
        torch.cuda.synchronize()
        t0 = time.time()
        lab, score = c.select_labels(kind)
        torch.cuda.synchronize()
        label_s = time.time() - t0
        c.surrogate_load(c.mubar() * np.exp(lab))
        lo_k, hi_k = c.lanczos_extremes()
        _, info_k = _timed_solves(c, b, x, 1, DEFORMED_MAXIT)
        direct[name] = {"iterations": info_k.iterations, "lanczos_cond": hi_k / lo_k, "label_seconds": label_s,
                        "mean_criterion_avg_label": [float(score[0].mean()), float(score[1].mean())]}
        c.close()
    # learned surrogate: training problems of the family (12^3 Q8, seeds 101-103: the workload's cell
    # size against the coefficient's wavelengths); each label kind is scored by PCG iterations with its
    # labels applied to them, and the better kind is the target
    tw = [inputs.deformed_problem(12, 8, s) for s in (101, 102, 103)]
    train = [fdmpc.Context(8, t["xv"], t["yv"], t["zv"], jac=t["jac"], kappa=t["kappa"], samples27=t["samples27"],
                           omega=1.0) for t in tw]
    score_its = {}
    for name, kind in (("theorem1", fdmpc.FDM_LABEL_THEOREM1), ("patch_kappa", fdmpc.FDM_LABEL_PATCH_KAPPA)):
        its = 0
        for t, ctx_t in zip(tw, train):
            lab, _ = ctx_t.select_labels(kind)
            s_ = fdmpc.Context(8, t["xv"], t["yv"], t["zv"], jac=t["jac"], kappa=t["kappa"],
                               samples27=t["samples27"], precision=fdmpc.FDM_PREC_FP32,
                               lanczos_start=inputs.lanczos_start((12 * 8 + 1) ** 3))
            s_.surrogate_load(s_.mubar() * np.exp(lab))
            bt = torch.tensor(inputs.normal_rhs(s_.ndof, 5), device=dev)
            its += s_.pcg_solve(bt, torch.empty_like(bt), rtol=RTOL, maxit=DEFORMED_MAXIT,
                                raise_on_noconv=False)[1].iterations
            s_.close()
        score_its[name] = its
    best = min(score_its, key=score_its.get)
    for ctx_t in train:
        ctx_t.select_labels(fdmpc.FDM_LABEL_THEOREM1 if best == "theorem1" else fdmpc.FDM_LABEL_PATCH_KAPPA)
    torch.cuda.synchronize()
    t0 = time.time()
    wts, hist = fdmpc.fdm_surrogate_train([t.h for t in train], inputs.mlp_init(7), 1000, 2e-3, 1e-4)
    torch.cuda.synchronize()
    train_s = time.time() - t0
    for t in train:
        t.close()
    raw = make(fdmpc.FDM_PREC_FP32)
    nf, _ = raw.surrogate_apply(wts, judge=0)
    lo1, hi1 = raw.lanczos_extremes()
    F = raw.surrogate_bounds()
    _, info_raw = _timed_solves(raw, b, x, 1, DEFORMED_MAXIT)
    raw.close()
    nf2, kept = ctx.surrogate_apply(wts, judge=1)
    ms2, info2 = _timed_solves(ctx, b, x, 3, DEFORMED_MAXIT)
    out.update({"labels_applied_directly": direct,
                "learned": {"label_kind_pcg_score_on_training_problems": score_its, "trained_on": best,
                            "train_cells": 3 * 1728, "train_steps": 1000, "train_seconds": train_s,
                            "train_loss_first_last": [hist[0], hist[-1]],
                            "mean_cell_bound_log_ratio": {"averaged": float(F[0].mean()), "label": float(F[1].mean()),
                                                          "network": float(F[2].mean())},
                            "lanczos_cond_network": hi1 / lo1, "network_iterations": info_raw.iterations,
                            "fallback_cells": nf, "kept_by_judge": bool(kept),
                            "judged_iterations": info2.iterations,
                            "judged_solve_dofs_per_s": free / (ms2 * 1e-3)}})
    ctx.close()
    ctx64 = make(fdmpc.FDM_PREC_FP64)
    ms64, info64 = _timed_solves(ctx64, b, x, 2, DEFORMED_MAXIT)
    out["fp64_solve_dofs_per_s"] = free / (ms64 * 1e-3)
    out["fp64_iterations"] = info64.iterations
    out["mixed_over_fp64"] = ms64 / ms
    ctx64.close()
    return out


def bench_unstructured(dev, fdmpc, inputs, peak):
    """General hexahedral mesh (the setting of the paper's unstructured
    experiments, Sec. 3): the extruded split-triangle mesh with m = 8 and six
    graded layers (2,304 cells of every orientation, vertex valences 3 to 16),
    Q7, b ~ N(0,1) on the free nodes; PCG with the hybrid V(1,1) of the
    vertex-star relaxation (averaged surrogate, glued FDM basis) and the Q1
    coarse space, mixed precision and FP64, and the FP32 sweep against HBM."""
    import torch
    X, cells = inputs.unstructured_hex_mesh(8, 6, 1)
    t0 = time.time()
    H = fdmpc.HexMesh(X.shape[0], cells, 7)
    H.factor(X)
    host_s = time.time() - t0
    free = int((~H.dirichlet()).sum())
    b = torch.randn(H.nnode, dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(8))
    start = inputs.lanczos_start(H.nnode)
    out = {"workload": "unstructured: extruded split-triangle hex mesh m = 8, 6 layers (%d cells), Q7, %d free dofs, "
                       "b ~ N(0,1)" % (cells.shape[0], free), "host_setup_seconds": host_s}
    for name, prec in (("mixed", fdmpc.FDM_PREC_FP32), ("fp64", fdmpc.FDM_PREC_FP64)):
        t1 = time.time()
        G = fdmpc.HexGpu(H, precision=prec, lanczos_start=start)
        torch.cuda.synchronize()
        gpu_setup = time.time() - t1
        x = torch.empty_like(b)
        ms, info = _timed_solves(G, b, x, 3, 500)
        res = {"ms_per_solve": ms, "solve_dofs_per_s": free / (ms * 1e-3), "iterations": info.iterations,
               "true_rel_residual": info.true_rnorm / info.rnorm0, "omega": G.omega, "gpu_setup_seconds": gpu_setup}
        if name == "mixed":
            z = torch.empty_like(b)
            for _ in range(3):
                G.asm_apply(b, z)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(torch.cuda.current_stream())
            for _ in range(10):
                G.asm_apply(b, z)
            e1.record(torch.cuda.current_stream())
            torch.cuda.synchronize()
            sweep_ms = e0.elapsed_time(e1) / 10
            ab = G.algo_bytes()
            nc, nstar, nx, nval, nco, maxg = G.sizes()
            res["sweep"] = {"ms": sweep_ms, "bytes": ab["sweep32"], "stars": nstar, "factor_values": nval,
                            "coarse_unknowns": nco, "largest_interface": maxg,
                            "hbm_frac_of_measured": ab["sweep32"] / (sweep_ms * 1e-3) / 1e9 / peak}
        out[name] = res
        G.close()
    out["mixed_over_fp64"] = out["mixed"]["solve_dofs_per_s"] / out["fp64"]["solve_dofs_per_s"]
    H.close()
    return out


def bench_batched(dev, fdmpc, inputs, reps=3):
    """64 independent graded problems (n in 2..10, p in 3..15) solved in one CUDA
    graph (smaller problems at higher kernel priority): aggregate DoF/s and
    per-solve latency (device timer); then the same problems one after another."""
    import torch
    probs = inputs.batch_problems(64, 1000)
    ctxs, bs = [], []
    t0 = time.time()
    for w in probs:
        n, p = len(w["xv"]) - 1, w["p"]
        nd = (n * p + 1) ** 3
        ctxs.append(fdmpc.Context(p, w["xv"], w["yv"], w["zv"], precision=fdmpc.FDM_PREC_FP32,
                                  lanczos_start=inputs.lanczos_start(nd), autotune=1))
        bs.append(torch.tensor(inputs.normal_rhs(nd, w["seed"]), device=dev))
    setup_s = time.time() - t0
    free = sum(_free_dofs(c.N) for c in ctxs)
    batch = fdmpc.fdm_batch_setup([c.h for c in ctxs])
    xs = [torch.empty_like(b) for b in bs]
    fdmpc.pcg_solve_batched(batch, bs, xs, RTOL, MAXIT)  # capture + first run
    times, lat = [], []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        infos = fdmpc.pcg_solve_batched(batch, bs, xs, RTOL, MAXIT)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        lat += [i.seconds * 1e3 for i in infos]
    ms = float(np.median(times))
    worst = max(i.true_rnorm / i.rnorm0 for i in infos)
    fdmpc.fdm_batch_destroy(batch)
    # the lockstep schedule: one loop, the star solves of all active problems in one launch
    lock = fdmpc.fdm_batch_setup([c.h for c in ctxs], mode=fdmpc.FDM_BATCH_LOCKSTEP)
    fdmpc.pcg_solve_batched(lock, bs, xs, RTOL, MAXIT)
    ltimes, llat = [], []
    for _ in range(reps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        linfos = fdmpc.pcg_solve_batched(lock, bs, xs, RTOL, MAXIT)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        ltimes.append(e0.elapsed_time(e1))
        llat += [i.seconds * 1e3 for i in linfos]
    lms = float(np.median(ltimes))
    lockstep = {"batch_ms": lms, "aggregate_dofs_per_s": free / (lms * 1e-3),
                "latency_ms_p50": float(np.percentile(llat, 50)), "latency_ms_p99": float(np.percentile(llat, 99)),
                "iterations_min_max": [min(i.iterations for i in linfos), max(i.iterations for i in linfos)],
                "worst_true_rel_residual": max(i.true_rnorm / i.rnorm0 for i in linfos)}
    fdmpc.fdm_batch_destroy(lock)
    # the same problems one after another (each its own device-driven solve): the time the batch
    # would take without sharing the GPU, and the throughput by degree
    seq_ms, by_p = 0.0, {}
    for c, b, x, w in zip(ctxs, bs, xs, probs):
        c.pcg_solve(b, x, rtol=RTOL, maxit=MAXIT)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(torch.cuda.current_stream())
        c.pcg_solve(b, x, rtol=RTOL, maxit=MAXIT)
        e1.record(torch.cuda.current_stream())
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        seq_ms += t
        d = by_p.setdefault(w["p"], [0, 0.0])
        d[0] += _free_dofs(c.N)
        d[1] += t
    for c in ctxs:
        c.close()
    # the same batch with the FP64 preconditioner (the plain FP64 form, same rtol on the true residual)
    c64 = [fdmpc.Context(w["p"], w["xv"], w["yv"], w["zv"], precision=fdmpc.FDM_PREC_FP64,
                         lanczos_start=inputs.lanczos_start(((len(w["xv"]) - 1) * w["p"] + 1) ** 3), autotune=1)
           for w in probs]
    b64 = fdmpc.fdm_batch_setup([c.h for c in c64])
    fdmpc.pcg_solve_batched(b64, bs, xs, RTOL, MAXIT)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(torch.cuda.current_stream())
    inf64 = fdmpc.pcg_solve_batched(b64, bs, xs, RTOL, MAXIT)
    e1.record(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1)
    worst64 = max(i.true_rnorm / i.rnorm0 for i in inf64)
    fdmpc.fdm_batch_destroy(b64)
    for c in c64:
        c.close()
    return {"workload": "64 graded problems, n^3 cells n in 2..10, Q_p p in 3..15 (seeds 1000..1063), "
                        "%d free dofs in total, mixed precision, one CUDA graph" % free,
            "lockstep": lockstep,
            "fp64_batch_ms": ms64, "fp64_aggregate_dofs_per_s": free / (ms64 * 1e-3),
            "fp64_worst_true_rel_residual": worst64, "mixed_over_fp64": ms64 / ms,
            "aggregate_dofs_per_s": free / (ms * 1e-3), "batch_ms": ms,
            "one_after_another_ms": seq_ms, "one_after_another_dofs_per_s": free / (seq_ms * 1e-3),
            "one_after_another_dofs_per_s_by_degree": {str(p): v[0] / (v[1] * 1e-3) for p, v in sorted(by_p.items())},
            "latency_ms_p50": float(np.percentile(lat, 50)), "latency_ms_p99": float(np.percentile(lat, 99)),
            "iterations_min_max": [min(i.iterations for i in infos), max(i.iterations for i in infos)],
            "worst_true_rel_residual": worst, "setup_seconds": setup_s}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 40 solves on the GPU, 5 oracle solves for --impl reference)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-preconditioner comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--pcg-host-loop", action="store_true",
                    help="timed solves through the host PCG loop instead of the captured CUDA graph "
                         "(for kernel profilers that replay launches one at a time)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the secondary workloads (p = 15, deformed, batched, multigrid, elasticity, SIPG, "
                         "unstructured)")
    ap.add_argument("--extra", default=None,
                    help="comma-separated subset of the secondary workloads to run "
                         "(p15, deformed, batched, gmg, elasticity, sipg, unstructured); default: all")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.steps is None:
            args.steps = 5
        return bench_reference(args)
    if args.steps is None:
        args.steps = 40
    return bench_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
