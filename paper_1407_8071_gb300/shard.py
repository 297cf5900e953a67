"""Sharding the M independent filters over several GPUs, one process per GPU.

The filters share nothing (Sec. 3.1: the ensemble is M independent filters),
so ranks exchange no particle and no weight: each rank runs a contiguous range
of filters, balanced by particle count, through its own context, and the only
collective is the gather of per-filter estimates for the M-average of
Definition 1.  The average is formed by the library (pf_ensemble_average): the
exact sum over all filters rounded once to FP64, divided by M, so it does not
depend on how the filters were split or in which order they arrive: any number
of ranks gives the number one process gives, bit for bit.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import numpy as np


def partition(N: Sequence[int], world: int) -> List[Tuple[int, int]]:
    """Contiguous filter ranges [begin, end) per rank, cut where the running
    particle count crosses r / world of the total (every rank gets at least one
    filter when M >= world)."""
    N = np.asarray(N, dtype=np.int64)
    M = len(N)
    if world < 1 or M < 1:
        raise ValueError("need world >= 1 and at least one filter")
    csum = np.concatenate([[0], np.cumsum(N)])
    total = csum[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        c = int(np.searchsorted(csum, target, side="left"))
        # the nearer of the two neighbouring cut points, kept increasing and leaving room
        if c > 0 and abs(csum[c - 1] - target) <= abs(csum[min(c, M)] - target):
            c -= 1
        c = max(c, cuts[-1] + (1 if M >= world else 0))
        c = min(c, M - (world - r) if M >= world else M)
        cuts.append(c)
    cuts.append(M)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def ensemble_mean(local_est: np.ndarray, begin: int, M: int, group=None) -> np.ndarray:
    """Definition 1's average over all M filters from each rank's per-filter
    estimates (local_est: rows for filters begin, begin + 1, ...).  Gathers
    every rank's rows (torch.distributed, any backend) in filter order; the
    library forms the average."""
    import torch
    import torch.distributed as dist
    local_est = np.ascontiguousarray(local_est, dtype=np.float64)
    if local_est.ndim == 1:
        local_est = local_est[:, None]
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    if world == 1:
        rows = local_est
    else:
        meta = torch.tensor([begin, local_est.shape[0]], dtype=torch.int64)
        metas = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(metas, meta, group=group)
        width = local_est.shape[1]
        most = max(int(m[1]) for m in metas)
        pad = np.zeros((most, width))
        pad[:local_est.shape[0]] = local_est
        parts = [torch.zeros((most, width), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(parts, torch.from_numpy(pad), group=group)
        rows = np.empty((M, width))
        seen = np.zeros(M, dtype=bool)
        for m, part in zip(metas, parts):
            b, n = int(m[0]), int(m[1])
            rows[b:b + n] = part.numpy()[:n]
            seen[b:b + n] = True
        if not seen.all():
            raise ValueError("the ranks' filter ranges do not cover all M filters")
    from . import pf
    return pf.pf_ensemble_average(rows)
