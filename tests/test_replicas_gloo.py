"""Multi-GPU path = independent replicas: per-rank seeded workloads and the timing reduction.

Runs two gloo ranks on the CPU (no GPU): each rank builds its replica of the
workload and reduces (time, units) the way bench.py does under torchrun.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w = bench.make_workload("large", rank, 4)
    ms, units = bench.reduce_over_ranks(10.0 + rank, 1000 * (rank + 1), world)
    q.put((rank, ms, units, w.info_words[:8].tolist(), w.cbs["Z"].tolist()))
    dist.destroy_process_group()


def test_two_gloo_replicas_reduce_like_the_bench():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, units, words, zs in res:
        assert ms == 11.0            # slowest rank
        assert units == 3000         # all ranks' work
    # replicas: same shapes (weak scaling), different seeded payloads
    assert res[0][4] == res[1][4]
    assert not np.array_equal(res[0][3], res[1][3])
