"""The bench's multi-rank logic on CPU: two gloo ranks, each with its own
independent system (weak scaling, no exchange on the data path), the job's
time taken as the slowest rank's and the throughput as all ranks' steps over
that time."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as d

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    d.init_process_group("gloo", rank=rank, world_size=world)
    try:
        system = bench.rank_system(rank)
        digest = float(np.abs(system.coef).sum() + system.var.sum())
        # each rank reports a different local time; the job time is the max
        t_local = 1.0 + 0.5 * rank
        t_max = bench.max_over_ranks(t_local, d, "cpu")
        digests = [None] * world
        d.all_gather_object(digests, digest)
        q.put((rank, t_max, bench.job_throughput(world, 20, t_max), digests, system.N, system.n))
    finally:
        d.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t_max, thr, digests, N, n in res:
        assert t_max == 1.5  # the slowest rank's time
        assert thr == pytest.approx(2 * 20 / 1.5)
        assert N == n == 256
        # the two ranks hold different systems (different seeds)
        assert digests[0] != digests[1]


def test_single_rank_helpers():
    import bench

    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.job_throughput(1, 10, 0.5) == 20.0
