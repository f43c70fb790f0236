"""The N > 1 replica path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Blocks are independent, so ranks are independent replicas: the only
cross-rank steps are the timing barrier and the max-over-ranks of the timed
interval, which rank 0 turns into the whole-job throughput."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import bench
    r, w, local = bench._dist_env()
    dist = bench._init_pg(w)
    bench._barrier(dist)
    # each rank "timed" a different interval; every rank must see the maximum
    mx = bench._max_over_ranks(dist, 1.0 + rank)
    q.put((r, w, local, mx))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_max_interval():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, 2, 0, 2.0), (1, 2, 1, 2.0)]


def test_single_process_needs_no_group():
    import bench
    assert bench._init_pg(1) is None
    assert bench._max_over_ranks(None, 3.5) == 3.5
