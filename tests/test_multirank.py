"""Host-side logic of bench.py's multi-rank run (one replica per rank, weak scaling): two
processes on the CPU with the gloo backend."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks(1.0 + rank)  # rank 1 is the slow one
        out.put((rank, t, bench.job_updates(64, 10, world)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_updates():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]
    assert all(r[2] == 2 * 64 * 64 * 10 for r in res)


def test_replicas_get_different_seeds():
    import numpy as np
    import bench
    a, b = bench.workload_rho(32, seed=5), bench.workload_rho(32, seed=6)
    assert not np.array_equal(a, b)
    assert np.allclose(a.mean(), 0.5 * (bench.RHO_L + bench.RHO_G), rtol=1e-3)
