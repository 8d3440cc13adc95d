"""The N > 1 path of bench.py on the CPU: two ranks over gloo.  Each rank
reports its own time; both must take the maximum (the slowest rank is the
job's time) and compute the same whole-job throughput; every rank solves its
own right-hand side; the reference arm runs on rank 0 only, and its JSON line
carries the contract's keys."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = 10.0 + 5.0 * rank                       # rank 1 is the slower one
    ms_max = bench.reduce_max(local_ms)
    value = bench.job_throughput(ws, 1000, 4, ms_max)
    seed = bench.rank_rhs_seed(2, rank)
    # the reference arm: only rank 0 works
    class A:
        gpus, steps, warmup = ws, 1, 0
    if rank != 0:
        bench.oracle_problem = lambda: (_ for _ in ()).throw(RuntimeError("rank != 0 must not run the oracle"))
        rc = bench.bench_reference(A())
    else:
        rc = 0
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms_max, value, seed, rc))


def test_two_rank_gloo_reduction():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [15.0, 15.0]
    assert out[0][2] == out[1][2] == pytest.approx(2 * 1000 * 4 / 15e-3)
    assert out[0][3] != out[1][3]
    assert [o[4] for o in out] == [0, 0]


def test_single_process_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.job_throughput(1, 10, 2, 1000.0) == pytest.approx(20.0)


def test_reference_arm_line():
    """`bench.py --impl reference` prints one JSON line with the contract's
    keys: the oracle's DoF/s on the host cores, its sample, a one-thread
    measurement, and an e2e block without host-device copies."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["metric"] == "pcg_solve_dofs_per_s" and d["unit"] == "DoF/s"
    assert d["value"] > 0 and d["higher_is_better"] is True and d["steps"] == 1
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert cb["single_core"]["cores"] == 1 and cb["single_core"]["value"] > 0
    assert d["e2e"] == {"value": d["value"], "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["iterations"] <= 20
