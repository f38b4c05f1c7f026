"""The N > 1 path of bench.py on CPU: two gloo ranks (world size 2).

The method shards as independent products (replicas, no data-path
collective): each rank draws its own operands, the ranks meet at a barrier
around the timed region, and rank 0 reports all ranks' units over the slowest
rank's seconds.  The CPU oracle stands in for the GPU product so that the
ranks do real, different work.
"""
import multiprocessing as mp
import os
import socket

import numpy as np


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import time
    import bench
    import synth
    from oracle import clmul as O
    w, r, _ = bench.dist_setup(world, backend="gloo")
    na = nb = 1 << 12
    seed = bench.replica_seed(2, r)
    a, b = synth.operand(seed, na), synth.operand(seed + 1, nb)
    bench.dist_barrier(w)
    t0 = time.perf_counter()
    c = O.mul(a, na, b, nb)
    time.sleep(0.05 * (r + 1))                 # ranks of unequal speed
    secs = time.perf_counter() - t0
    bench.dist_barrier(w)
    worst = bench.dist_max(secs, w, device="cpu")
    value = bench.whole_job_value(na + nb, worst, w)
    q.put((r, w, seed, secs, worst, value, int(c[0]), int(c.sum() % (1 << 62))))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas():
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
    (r0, w0, s0, t0, m0, v0, c0, h0), (r1, w1, s1, t1, m1, v1, c1, h1) = res
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert s0 != s1 and (c0, h0) != (c1, h1)            # independent products
    assert m0 == m1 == max(t0, t1)                      # max over ranks, the same on both
    assert v0 == v1 and np.isclose(v0, 2 * ((1 << 12) + (1 << 12)) / max(t0, t1) / 1e9)
