"""Sharding of the batched form across ranks (world size 2, gloo, CPU).

The per-rank computation is injected (the oracle stands in for the GPU call),
so this covers the host logic: the shards partition the clouds, balance them,
and the gathered pairs equal those of one process computing everything."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2502_05063_b300 import parallel, synth


def _oracle_compute(pts, offs, dmax, thr):
    import oracle
    out = []
    for i in range(len(offs) - 1):
        c = pts[offs[i]:offs[i + 1]]
        n = c.shape[0]
        D = oracle.distances_f32(c).astype(np.float64)
        t = oracle.enclosing_radius(D, n) if not np.isfinite(thr) else thr
        pairs, _ = oracle.cohom(D, n, dmax, t, clearing=True)
        dg = oracle.diagram(pairs, dmax)
        out.append([[(float(r["birth"]), float(r["death"]), int(r["birth_cidx"])) for r in dg[p]]
                    for p in range(dmax + 1)])
    return out


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, pts, offs, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = parallel.sharded_batched(pts, offs, dmax=1, compute=_oracle_compute)
    if rank == 0:
        q.put(res)
    dist.barrier()
    dist.destroy_process_group()


def test_shards_partition_and_balance():
    rng = np.random.default_rng(0)
    sizes = rng.integers(32, 257, size=101)
    shards = [parallel.shard_clouds(sizes, 4, r) for r in range(4)]
    flat = sorted(i for s in shards for i in s)
    assert flat == list(range(101))
    work = [sum(int(sizes[i]) ** 2 for i in s) for s in shards]
    assert max(work) / min(work) < 1.1


def test_gloo_world2_equals_single_process():
    clouds = [synth.circle(int(n), 1.0, 0.1, 2, seed=int(n)) for n in (12, 30, 7, 25, 18, 9, 22)]
    pts, offs = synth.pack(clouds)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, pts, offs, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    want = _oracle_compute(pts, offs, 1, float("inf"))
    assert res == want
