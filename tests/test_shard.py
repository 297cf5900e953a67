"""Sharding the filters over ranks (CPU, gloo, world size 2 and 3).

* partition: contiguous ranges covering all filters, balanced by particles to
  within the largest filter.
* ensemble_mean over ranks equals the single-process value bit for bit (FP64
  correctly rounded sums), for ragged filter counts and several statistics.
* the library's Definition 1 average (pf_ensemble_average, host code, no GPU)
  is the exact sum rounded once: it equals the exact rational sum (Python's
  fractions) rounded to a double, divided by M, on hard cases -- cancellation across the
  whole exponent range, subnormals, ties -- and does not depend on the order.
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


def _fsum_mean(est):
    """Exact rational sum (fractions.Fraction), rounded once by Python's correctly
    rounded int / int division, then divided by M."""
    from fractions import Fraction
    est = np.asarray(est, dtype=np.float64).reshape(len(est), -1)
    out = []
    for s in range(est.shape[1]):
        tot = sum((Fraction(float(v)) for v in est[:, s]), Fraction(0))
        out.append(float(tot) / est.shape[0])
    return np.array(out)


def test_library_average_is_the_exact_sum_rounded_once():
    from paper_1407_8071_gb300 import pf
    rng = np.random.default_rng(5)
    cases = [
        rng.normal(0.0, 1.0, (1000, 3)),
        rng.normal(0.0, 1.0, (257, 4)) * 10.0 ** rng.integers(-300, 300, (257, 4)),
        np.array([[1e308], [1e308], [-1e308], [-1e308], [1e-308], [3.0]]),   # cancellation, no overflow
        np.array([[2.0 ** 53], [1.0], [1.0]]),                                 # 2^53 + 2: exact only if summed exactly
        np.array([[1.0], [2.0 ** -53], [2.0 ** -106]]),                        # just above a tie: rounds up
        np.array([[1.0], [2.0 ** -53]]),                                       # an exact tie: to even (down)
        np.array([[5e-324], [5e-324], [-1e-323], [4e-323]]),                   # subnormals
        np.array([[0.1]] * 10),
        np.array([[-0.0], [-0.0]]),
    ]
    for est in cases:
        got = pf.pf_ensemble_average(est)
        ref = _fsum_mean(est)
        assert np.array_equal(got, ref), (est.ravel()[:6], got, ref)
        for _ in range(3):  # any order of the filters gives the same bits
            assert np.array_equal(pf.pf_ensemble_average(est[rng.permutation(len(est))]), got)
    assert pf.pf_ensemble_average(np.array([[2.0 ** 53], [1.0], [1.0]]))[0] * 3 == 2.0 ** 53 + 2
    assert np.isnan(pf.pf_ensemble_average(np.array([[1.0], [np.nan]]))[0])
    assert np.isnan(pf.pf_ensemble_average(np.array([[np.inf], [-np.inf]]))[0])
    assert pf.pf_ensemble_average(np.array([[np.inf], [1.0]]))[0] == np.inf
