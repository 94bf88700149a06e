"""Box sharding across ranks (one process per GPU).

Boxes are independent units of the method, so a batch splits across ranks
with no exchange during propagation; the only communication is gathering the
per-box results at the end (and, for timing, a max over ranks).  This module
holds that host-side logic; it works with any torch.distributed backend
(NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np


def box_cost(boxes: np.ndarray) -> np.ndarray:
    """Work estimate per box: wider boxes have more unstable neurons, hence
    more composition work; use the sum of side lengths plus a floor."""
    w = (boxes[..., 1].astype(np.float64) - boxes[..., 0].astype(np.float64)).sum(-1)
    return 1.0 + w / max(1e-30, float(w.max()) if len(w) else 1.0)


def shard_ranges(costs: Sequence[float], world: int) -> List[tuple]:
    """Split [0, n) into `world` contiguous ranges of near-equal total cost
    (contiguous ranges keep the gathered results in input order)."""
    costs = np.asarray(costs, np.float64)
    n = len(costs)
    if world < 1:
        raise ValueError("world must be >= 1")
    if n == 0:
        return [(0, 0)] * world
    cum = np.concatenate([[0.0], np.cumsum(costs)])
    total = cum[-1]
    cuts = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(cum, target, side="left"))
        k = min(max(k, cuts[-1]), n)
        cuts.append(k)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard_boxes(boxes: np.ndarray, rank: int, world: int) -> tuple:
    """(start, stop) of this rank's slice of the batch."""
    return shard_ranges(box_cost(boxes), world)[rank]


def gather_results(local: dict, rank: int, world: int, dist=None) -> dict:
    """Concatenate every rank's per-box result arrays in rank order (one
    all_gather_object); identity when world == 1."""
    if world == 1 or dist is None:
        return local
    parts = [None] * world
    dist.all_gather_object(parts, {k: np.asarray(v) for k, v in local.items()})
    return {k: np.concatenate([p[k] for p in parts], 0) for k in local}


def max_over_ranks(value: float, world: int, dist=None, device=None) -> float:
    """Max of a scalar over ranks (the timing rule of the benchmark)."""
    if world == 1 or dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
