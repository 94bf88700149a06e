"""Box sharding across ranks (one process per GPU).

Boxes are independent units of the method, so a batch splits across ranks
with no exchange during propagation; the only communication is gathering the
per-box results at the end (and, for timing, a max over ranks).

* ``interval_cost``: a per-box work estimate from the network itself: interval
  arithmetic over the box counts, layer by layer, the neurons whose
  pre-activation interval straddles 0 (the ones that need the composition),
  each weighted by the number of term pairs its square takes at that layer's
  degree, plus the layer step's products.  Boxes whose neurons are all
  decided cost little; wide boxes cost the most.
* ``shard_ranges``: contiguous ranges of near-equal total cost (contiguous, so
  the gathered results come back in input order).
* ``gather_tensors``: the per-box result tensors of every rank concatenated
  in rank order, one ``all_gather`` per tensor of equal-size (padded) slices;
  with NCCL these are device-side collectives on the GPU tensors themselves.
* ``propagate_sharded``: the whole thing around ``Context.propagate``.

It works with any torch.distributed backend (NCCL on GPUs, gloo in the CPU
tests).
"""
from __future__ import annotations

from typing import Callable, Dict, List, Optional, Sequence

import numpy as np


def _num_monomials(n: int, D: int) -> int:
    r = 1
    for i in range(1, n + 1):
        r = r * (D + i) // i
    return r


def interval_cost(widths: Sequence[int], W, b, boxes: np.ndarray, degree=2,
                  cap: int = 16) -> np.ndarray:
    """Work estimate per box (arbitrary units): sum over hidden layers of
    (neurons whose interval pre-activation straddles 0) x (term pairs of the
    square at that layer's input degree), plus h_out x h_in x M per layer step.

    Interval arithmetic (float64, midpoint-radius) propagates each box through
    the network; a neuron is counted unstable when its interval contains 0 in
    its interior, dead or active otherwise (the interval is wider than the
    Bernstein enclosure, so this over-counts, uniformly across boxes)."""
    widths = [int(x) for x in widths]
    n, H = widths[0], len(widths) - 1
    boxes = np.asarray(boxes, np.float64)
    B = boxes.shape[0]
    if B == 0:
        return np.zeros(0)
    degs = [int(degree)] * (H - 1) if np.ndim(degree) == 0 else [int(x) for x in degree]
    c = 0.5 * (boxes[:, :, 0] + boxes[:, :, 1])
    r = 0.5 * (boxes[:, :, 1] - boxes[:, :, 0])
    cost = np.zeros(B)
    D = 1
    for i in range(H):
        Wi = np.asarray(W[i], np.float64)
        bi = np.asarray(b[i], np.float64)
        M = _num_monomials(n, D)
        cost += widths[i + 1] * widths[i] * M
        zc = c @ Wi.T + bi
        zr = r @ np.abs(Wi).T
        if i == H - 1:
            break
        lo, hi = zc - zr, zc + zr
        unstable = (lo < 0) & (hi > 0)
        cost += unstable.sum(1) * (M * (M + 1) / 2.0)
        # ReLU of the interval
        plo, phi = np.maximum(lo, 0.0), np.maximum(hi, 0.0)
        c, r = 0.5 * (plo + phi), 0.5 * (phi - plo)
        D = min(D * degs[i], cap)
    return cost


def box_cost(boxes: np.ndarray) -> np.ndarray:
    """Network-free fallback estimate: the sum of side lengths plus a floor."""
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
        # the cut nearer to the target of the two around it
        if 0 < k <= n and abs(cum[k - 1] - target) < abs(cum[k] - target):
            k -= 1
        k = min(max(k, cuts[-1]), n)
        cuts.append(k)
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def shard_boxes(boxes: np.ndarray, rank: int, world: int, costs=None) -> tuple:
    """(start, stop) of this rank's slice of the batch."""
    return shard_ranges(box_cost(boxes) if costs is None else costs, world)[rank]


def gather_tensors(local: Dict[str, "object"], count: int, counts: Sequence[int],
                   dist=None) -> Dict[str, "object"]:
    """Concatenate every rank's per-box torch tensors (leading dimension =
    boxes) in rank order.  Each rank pads its slice to the largest count, one
    all_gather per tensor moves the padded slices (device tensors with NCCL),
    and the padding is cut off again; identity when there is one rank."""
    if dist is None or len(counts) == 1:
        return dict(local)
    import torch
    cmax = max(int(x) for x in counts)
    out = {}
    for k, t in local.items():
        if t is None:
            out[k] = None
            continue
        pad = torch.zeros((cmax,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
        if count:
            pad[:count] = t[:count]
        parts = [torch.empty_like(pad) for _ in counts]
        dist.all_gather(parts, pad)
        out[k] = torch.cat([p[: int(c)] for p, c in zip(parts, counts)], 0)
    return out


def gather_results(local: dict, rank: int, world: int, dist=None) -> dict:
    """Concatenate every rank's per-box numpy arrays in rank order (one
    all_gather_object; for small host-side records); identity when world == 1."""
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


def propagate_sharded(propagate: Callable, widths, W_host, b_host, boxes: np.ndarray, rank: int,
                      world: int, dist=None, degree=2, cap: int = 16,
                      costs: Optional[np.ndarray] = None, gather: bool = True, **kw):
    """Bound a batch of boxes on `world` ranks: every rank takes its
    cost-balanced contiguous slice (``interval_cost`` of the network unless
    `costs` is given), runs ``propagate(boxes_slice, degree=..., cap=...,
    **kw)`` (normally ``Context.propagate`` bound to this rank's GPU and the
    network's device tensors), and, with `gather`, the result tensors of all
    ranks are concatenated in box order on every rank.  Returns (result,
    (start, stop), counts)."""
    if costs is None:
        costs = interval_cost(widths, W_host, b_host, boxes, degree, cap)
    ranges = shard_ranges(costs, world)
    a, z = ranges[rank]
    counts = [r1 - r0 for r0, r1 in ranges]
    local = propagate(np.ascontiguousarray(boxes[a:z]), degree=degree, cap=cap, **kw)
    if not gather:
        return local, (a, z), counts
    return gather_tensors(local, z - a, counts, dist), (a, z), counts
