"""The N > 1 host path of the bench (one process per GPU, independent seeded
ensembles, no data-path exchange, timings reduced to the slowest rank) with
world size 2 over the gloo backend on CPU."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_1501_03450_b300.replicas import aggregate_rate, max_over_ranks, rank_seed


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z, _ = W.gaussian_particles(64, 45.5, seed=rank_seed(3450, rank))
        t_local = 1.0 + 0.5 * rank                      # the slower rank decides
        t_max = max_over_ranks(t_local, dist, "cpu")
        rate = aggregate_rate(1000.0, world, t_max)
        checksum = torch.tensor([float(z.sum())], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, checksum)
        out.put((rank, t_max, rate, [float(g.item()) for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_two_replicas_over_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t_max, rate, sums in res:
        assert t_max == pytest.approx(1.5)
        assert rate == pytest.approx(1000.0 * 2 / 1.5)
        assert sums[0] != sums[1]                       # independent ensembles per rank
    assert res[0][3] == res[1][3]


def test_single_process_identities():
    assert max_over_ranks(2.5) == 2.5
    assert aggregate_rate(10.0, 1, 2.0) == 5.0
    assert rank_seed(7, 3) == 10
    with pytest.raises(ValueError):
        aggregate_rate(1.0, 1, 0.0)
