"""Box partition of the structured mesh over ranks (fdm_partition_*), on the
CPU: the send lists and per-node sum plans reproduce the single-domain node
sums (the direct stiffness summation of per-cell contributions, ascending
global cell index, as the node gather forms them) bit for bit on every node
of every rank's node box, the shared face, edge and corner nodes included;
node ownership and star ownership partition the nodes and vertices; every
star's cells lie in its owner's cells plus the one-cell halo.  The exchange
runs in one process over all ranks of several rank grids, and over two gloo
ranks with torch.distributed."""
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    import __graft_entry__ as g
    from paper_2107_14758_gb300 import build, fdmpc
    build.build()
    del g
    return fdmpc


def _cell_contrib(ncell, p, seed):
    """Seeded per-cell contributions E[cell][(p+1)^3] over the whole mesh (cells and nodes x fastest)."""
    n = p + 1
    return np.random.default_rng(seed).standard_normal((int(np.prod(ncell)), n ** 3))


def _reference_sums(E, ncell, p):
    """Single-domain node sums: for every grid node, the contributions of the
    cells containing it added one by one from 0 in ascending global cell index."""
    nx, ny, nz = ncell
    n = p + 1
    N = (nx * p + 1, ny * p + 1, nz * p + 1)
    terms = [[] for _ in range(N[0] * N[1] * N[2])]
    for cz in range(nz):
        for cy in range(ny):
            for cx in range(nx):
                c = cx + nx * (cy + ny * cz)
                for k in range(n):
                    for j in range(n):
                        for i in range(n):
                            g = (cx * p + i) + N[0] * ((cy * p + j) + N[1] * (cz * p + k))
                            terms[g].append(E[c, i + n * (j + n * k)])
    out = np.zeros(len(terms))
    for g, t in enumerate(terms):  # cells were visited in ascending index
        s = 0.0
        for v in t:
            s = s + v
        out[g] = s
    return out, N


def _local_E(E, ncell, p, cb):
    nx, ny, _ = ncell
    rows = []
    for cz in range(cb[4], cb[5]):
        for cy in range(cb[2], cb[3]):
            for cx in range(cb[0], cb[1]):
                rows.append(E[cx + nx * (cy + ny * cz)])
    return np.concatenate(rows)


def _sum_plan(local, recv, sum_ptr, summ):
    out = np.zeros(len(sum_ptr) - 1)
    for i in range(len(out)):
        s = 0.0
        for q in summ[sum_ptr[i]:sum_ptr[i + 1]]:
            s = s + (local[q] if q >= 0 else recv[-1 - q])
        out[i] = s
    return out


def _box_nodes(nb, N):
    gx = np.arange(nb[0], nb[1] + 1)
    gy = np.arange(nb[2], nb[3] + 1)
    gz = np.arange(nb[4], nb[5] + 1)
    return (gx[None, None, :] + N[0] * (gy[None, :, None] + N[1] * gz[:, None, None])).ravel()


@pytest.mark.parametrize("ncell,p,nrank", [((5, 4, 3), 3, (2, 1, 1)), ((4, 5, 3), 2, (1, 2, 1)),
                                           ((4, 4, 4), 2, (2, 2, 2)), ((6, 3, 4), 1, (3, 1, 2)),
                                           ((3, 3, 3), 4, (1, 1, 3))])
def test_exchange_reproduces_single_domain_sums(ncell, p, nrank):
    fdmpc = _lib()
    E = _cell_contrib(ncell, p, 11)
    ref, N = _reference_sums(E, ncell, p)
    nr = int(np.prod(nrank))
    parts = [fdmpc.Partition(ncell, p, nrank, r) for r in range(nr)]
    info = []
    for P in parts:
        cb, nb = P.cell_box(), P.node_box()
        send_ptr, send, recv_ptr, sum_ptr, summ, owned = P.lists()
        info.append(dict(cb=cb, nb=nb, neigh=list(P.neighbors()), send_ptr=send_ptr, send=send, recv_ptr=recv_ptr,
                         sum_ptr=sum_ptr, sum=summ, owned=owned, local=_local_E(E, ncell, p, cb)))
    owners = np.zeros(N[0] * N[1] * N[2], dtype=int)
    for r, d in enumerate(info):
        msgs = []
        for R in d["neigh"]:  # the message neighbour R sent to r
            e = info[R]
            k = e["neigh"].index(r)
            msgs.append(e["local"][e["send"][e["send_ptr"][k]:e["send_ptr"][k + 1]]])
        for k, m in enumerate(msgs):
            assert len(m) == d["recv_ptr"][k + 1] - d["recv_ptr"][k]
        recv = np.concatenate(msgs) if msgs else np.zeros(0)
        got = _sum_plan(d["local"], recv, d["sum_ptr"], d["sum"])
        nodes = _box_nodes(d["nb"], N)
        assert np.array_equal(got, ref[nodes]), r   # bit for bit
        owners[nodes[d["owned"] == 1]] += 1
    assert np.all(owners == 1)          # every node has exactly one owner
    # with more than one rank, every rank's box has shared nodes that take received contributions
    assert sum(1 for d in info if (d["sum"] < 0).any()) == (nr if nr > 1 else 0)
    # stars: every vertex owned once; its cells within the owner's halo box
    V = (ncell[0] + 1, ncell[1] + 1, ncell[2] + 1)
    seen = np.zeros(V[0] * V[1] * V[2], dtype=int)
    for P in parts:
        hb = P.halo_box()
        for v in P.stars():
            seen[v] += 1
            vx, vy, vz = v % V[0], (v // V[0]) % V[1], v // (V[0] * V[1])
            for c, lo, hi, nc in ((vx, hb[0], hb[1], ncell[0]), (vy, hb[2], hb[3], ncell[1]),
                                  (vz, hb[4], hb[5], ncell[2])):
                for cc in (c - 1, c):  # the star's cells along this axis
                    if 0 <= cc < nc:
                        assert lo <= cc < hi
    assert np.all(seen == 1)
    for P in parts:
        P.close()


def test_invalid_partitions():
    fdmpc = _lib()
    for args in [((2, 2, 2), 3, (3, 1, 1), 0), ((2, 2, 2), 3, (1, 1, 1), 1), ((2, 2, 2), 0, (1, 1, 1), 0),
                 ((2, 2, 2), 16, (1, 1, 1), 0)]:
        with pytest.raises(fdmpc.FdmError) as e:
            fdmpc.Partition(*args)
        assert e.value.code == fdmpc.FDM_EINVAL


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _gloo_rank(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from paper_2107_14758_gb300 import fdmpc
        ncell, p, nrank = (5, 3, 4), 3, (2, 1, 1)
        E = _cell_contrib(ncell, p, 12)
        P = fdmpc.Partition(ncell, p, nrank, rank)
        cb, nb = P.cell_box(), P.node_box()
        neigh = list(P.neighbors())
        send_ptr, send, recv_ptr, sum_ptr, summ, owned = P.lists()
        local = _local_E(E, ncell, p, cb)
        reqs, bufs = [], []
        for k, R in enumerate(neigh):  # one neighbour-sum exchange per apply
            out = torch.from_numpy(np.ascontiguousarray(local[send[send_ptr[k]:send_ptr[k + 1]]]))
            inc = torch.empty(int(recv_ptr[k + 1] - recv_ptr[k]), dtype=torch.float64)
            reqs.append(dist.isend(out, R))
            reqs.append(dist.irecv(inc, R))
            bufs.append(inc)
        for rq in reqs:
            rq.wait()
        recv = torch.cat(bufs).numpy() if bufs else np.zeros(0)
        got = _sum_plan(local, recv, sum_ptr, summ)
        ref, N = _reference_sums(E, ncell, p)
        ok = bool(np.array_equal(got, ref[_box_nodes(nb, N)]))
        # the owned nodes' sum over the ranks covers every node once
        cnt = torch.tensor([float(owned.sum())], dtype=torch.float64)
        dist.all_reduce(cnt)
        q.put((rank, ok, int(cnt.item()), N[0] * N[1] * N[2], len(neigh)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_exchange():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    _lib()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=180) for _ in range(2))
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    for rank, ok, owned_total, nodes, nneigh in out:
        assert ok, rank
        assert owned_total == nodes and nneigh == 1
    del torch
