"""The multi-GPU path (replicas, no data-path collective) on CPU: two gloo ranks.

Each rank runs its own instances (weak scaling); the benchmark takes the slowest rank's time and
the sum of all ranks' work.  Here two processes check that their shards are disjoint and that
the rank reductions bench.py uses give the maximum and the sum on every rank.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    insts = bench.workload(1, rank)          # one instance per density on each rank
    sig = [int(np.asarray(i.W).sum()) * 1000003 + int(np.asarray(i.b).sum()) for i in insts]
    mx = bench.over_ranks(10.0 * (rank + 1), dist, "cpu", "max")
    sm = bench.over_ranks(3.0 + rank, dist, "cpu", "sum")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, sig, mx, sm))


def test_two_replicas_shard_and_reduce():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(world))
    sig0, sig1 = set(res[0][1]), set(res[1][1])
    assert len(sig0) == 4 and not (sig0 & sig1), "ranks must run different instances"
    for _, _, mx, sm in res:
        assert mx == 20.0 and sm == 7.0


def test_single_process_reduction_is_identity():
    import bench
    assert bench.over_ranks(5.5, None, "cpu", "max") == 5.5
    assert bench.over_ranks(5.5, None, "cpu", "sum") == 5.5
