"""Sharding the filters over ranks (CPU, gloo, world size 2 and 3).

* partition: contiguous ranges covering all filters, balanced by particles to
  within the largest filter.
* ensemble_mean over ranks equals the single-process value bit for bit (FP64
  correctly rounded sums), for ragged filter counts and several statistics.
"""
import math
import os
import socket

import numpy as np
import pytest

from paper_1407_8071_gb300 import shard, workloads as W


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_partition_balances_particles(world):
    N = W.ragged_counts(256, 64, 4096)
    ranges = shard.partition(N, world)
    assert ranges[0][0] == 0 and ranges[-1][1] == len(N)
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c and a < b
    loads = [int(N[a:b].sum()) for a, b in ranges]
    assert max(loads) - min(loads) <= 2 * int(N.max())
    assert sum(loads) == int(N.sum())


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, N, est, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b, e = shard.partition(N, world)[rank]
        out.put((rank, shard.ensemble_mean(est[b:e], b, len(N))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_ensemble_mean_over_ranks_is_bit_identical(world):
    import torch.multiprocessing as mp
    N = W.ragged_counts(37, 16, 512, seed=4)
    rng = np.random.default_rng(11)
    est = rng.normal(0.0, 1.0, (len(N), 5)) * 10.0 ** rng.integers(-6, 6, (len(N), 1))
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, N, est, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ref = np.array([math.fsum(est[:, s]) / len(N) for s in range(est.shape[1])])
    for r in range(world):
        assert np.array_equal(got[r], ref)
    assert np.allclose(ref, est.mean(axis=0), rtol=1e-12, atol=0)
