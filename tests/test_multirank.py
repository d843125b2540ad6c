"""The N > 1 path of bench.py on CPU: two gloo ranks get disjoint seed
ranges (samples are independent, so no data-path collective is needed) and
agree on the slowest rank's time; their oracle results concatenate to the
single-rank results for the union of seeds."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    seeds = bench.shard_seeds(rank, n)
    nj, nc = oracle.samples(16, 2, [int(s) for s in seeds])
    slowest = bench.max_over_ranks(1.0 + rank, dist)
    q.put((rank, seeds.tolist(), nj.tolist(), nc.tolist(), slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_samples():
    import oracle
    oracle.build()
    world, n = 2, 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, n, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seeds = out[0][1] + out[1][1]
    assert seeds == list(range(1, world * n + 1))          # disjoint, contiguous
    assert all(o[4] == float(world) for o in out)           # both see the max
    wj, wc = oracle.samples(16, 2, seeds)
    assert out[0][2] + out[1][2] == wj.tolist()
    assert out[0][3] + out[1][3] == wc.tolist()
