"""Batched branch-and-bound refinement of an input box (the refinement loop
around the bound propagation): leaves are sub-boxes of the root with sound
output bounds from the plain method; every round the leaves with the largest
upper bound of the chosen output are split in two along a proposed input
dimension and their children are bounded in one batched propagation.

Objective: bound max_x NN_j(x) over the root box.  U = max over leaves of hi
is a sound upper bound of that maximum; L = max over leaves of lo is a sound
lower bound, so a leaf with hi < L cannot hold the maximum and is dropped.

Split dimension: the learned split head (a BF16 MLP over the features of
bern_split_features, one class per input dimension) or, as the fallback,
the widest side relative to the root box.  Whatever dimension is proposed,
the children cover the parent exactly (they share the float32 midpoint), so
the bounds stay sound.

Multi-GPU: every rank refines its own leaves (no collective in the data
path); every `rebalance_every` rounds the ranks exchange a summary (their
leaf counts and best upper bounds) and move leaves so that the leaves that
will be split next are spread evenly (rebalance()).
"""
from __future__ import annotations

from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

BoundFn = Callable[[np.ndarray], Tuple[np.ndarray, np.ndarray, np.ndarray]]
SplitFn = Callable[[np.ndarray, np.ndarray], np.ndarray]


def split_boxes(boxes: np.ndarray, dims: np.ndarray) -> np.ndarray:
    """Children [2B, n, 2] of boxes [B, n, 2] halved along dims [B]: child 2i
    keeps the lower half, 2i+1 the upper half; they share the float32
    midpoint, so their union is the parent."""
    boxes = np.asarray(boxes, np.float32)
    B = boxes.shape[0]
    dims = np.asarray(dims, np.int64)
    lo = boxes[np.arange(B), dims, 0].astype(np.float64)
    hi = boxes[np.arange(B), dims, 1].astype(np.float64)
    mid = (lo + 0.5 * (hi - lo)).astype(np.float32)
    mid = np.minimum(np.maximum(mid, boxes[np.arange(B), dims, 0]), boxes[np.arange(B), dims, 1])
    out = np.repeat(boxes, 2, axis=0)
    out[2 * np.arange(B), dims, 1] = mid
    out[2 * np.arange(B) + 1, dims, 0] = mid
    return out


def widest_split(boxes: np.ndarray, root: np.ndarray) -> np.ndarray:
    """Fallback split rule: the side that is widest relative to the root."""
    side = boxes[:, :, 1].astype(np.float64) - boxes[:, :, 0]
    rside = np.maximum(root[:, 1].astype(np.float64) - root[:, 0], 1e-300)
    return np.argmax(side / rside[None, :], axis=1)


class BranchAndBound:
    """State and rounds of one rank's refinement."""

    def __init__(self, bound_fn: BoundFn, root: np.ndarray, split_fn: Optional[SplitFn] = None,
                 batch: int = 1024, max_leaves: int = 65536, boxes: Optional[np.ndarray] = None):
        self.bound_fn = bound_fn
        self.root = np.asarray(root, np.float32)
        self.n = self.root.shape[0]
        self.split_fn = split_fn
        self.batch = int(batch)
        self.max_leaves = int(max_leaves)
        start = self.root[None] if boxes is None else np.asarray(boxes, np.float32)
        self.boxes = start.copy()
        if len(start):
            self.lo, self.hi, self.feats = bound_fn(self.boxes)
        else:
            self.lo, self.hi, self.feats = np.zeros(0), np.zeros(0), np.zeros((0, 0), np.float32)
        self.propagated = len(start)
        self.history: List[Dict] = []

    # ---- queries
    def upper(self) -> float:
        return float(np.max(self.hi)) if len(self.hi) else -np.inf

    def lower(self) -> float:
        return float(np.max(self.lo)) if len(self.lo) else -np.inf

    def count(self) -> int:
        return int(len(self.boxes))

    # ---- one round
    def prune(self, incumbent: Optional[float] = None):
        """Drop leaves that cannot hold the maximum (hi < the best lower bound)."""
        L = self.lower() if incumbent is None else max(self.lower(), incumbent)
        keep = self.hi >= L
        if not np.all(keep):
            self._take(keep)

    def _take(self, keep):
        self.boxes, self.lo, self.hi = self.boxes[keep], self.lo[keep], self.hi[keep]
        self.feats = self.feats[keep]

    def step(self, incumbent: Optional[float] = None) -> int:
        """Split up to `batch` leaves with the largest upper bounds (as many
        as the leaf budget allows); returns the number of parents split."""
        self.prune(incumbent)
        room = self.max_leaves - self.count()
        K = min(self.batch, room, self.count())
        if K <= 0:
            return 0
        order = np.argsort(-self.hi, kind="stable")
        sel, rest = order[:K], order[K:]
        parents = self.boxes[sel]
        if self.split_fn is not None:
            dims = np.asarray(self.split_fn(parents, self.feats[sel]), np.int64)
        else:
            dims = widest_split(parents, self.root)
        dims = np.clip(dims, 0, self.n - 1)
        kids = split_boxes(parents, dims)
        lo, hi, feats = self.bound_fn(kids)
        self.propagated += len(kids)
        self.boxes = np.concatenate([self.boxes[rest], kids], 0)
        self.lo = np.concatenate([self.lo[rest], lo])
        self.hi = np.concatenate([self.hi[rest], hi])
        self.feats = np.concatenate([self.feats[rest], feats], 0)
        self.history.append({"leaves": self.count(), "U": self.upper(), "L": self.lower(),
                             "split": int(K), "propagated": int(self.propagated)})
        return K

    def run(self, rounds: int, incumbent_fn=None) -> List[Dict]:
        for _ in range(rounds):
            inc = incumbent_fn() if incumbent_fn else None
            if self.step(inc) == 0:
                break
        return self.history


# ---------------------------------------------------------------- multi-rank
def plan_moves(counts: List[int], active: List[int]) -> List[Tuple[int, int, int]]:
    """Deterministic leaf moves (src, dst, how many) that even out the
    `active` leaves (those above the global split threshold) across ranks:
    every rank ends with floor or ceil of their mean, the surplus of the
    richest ranks going to the poorest, in rank order."""
    world = len(active)
    total = int(sum(active))
    target = [total // world + (1 if r < total % world else 0) for r in range(world)]
    # give the larger targets to the ranks that already hold the most
    order = sorted(range(world), key=lambda r: (-active[r], r))
    tgt = [0] * world
    for k, r in enumerate(order):
        tgt[r] = target[k]
    surplus = [(r, active[r] - tgt[r]) for r in range(world) if active[r] > tgt[r]]
    deficit = [(r, tgt[r] - active[r]) for r in range(world) if active[r] < tgt[r]]
    moves = []
    i = j = 0
    while i < len(surplus) and j < len(deficit):
        s, a = surplus[i]
        d, b = deficit[j]
        k = min(a, b)
        moves.append((s, d, k))
        surplus[i] = (s, a - k)
        deficit[j] = (d, b - k)
        if surplus[i][1] == 0:
            i += 1
        if deficit[j][1] == 0:
            j += 1
    return moves


def rebalance(bb: BranchAndBound, dist, batch_total: Optional[int] = None) -> Dict:
    """Exchange summaries (leaf count and the `batch` largest upper bounds of
    every rank), pick the global split threshold (the batch_total-th largest
    upper bound), and move active leaves from ranks with more than their
    share to ranks with fewer.  Every rank computes the same plan."""
    world = dist.get_world_size()
    rank = dist.get_rank()
    top = np.sort(bb.hi)[::-1][:bb.batch].astype(np.float64)
    summaries = [None] * world
    dist.all_gather_object(summaries, (bb.count(), top.tolist()))
    allv = np.sort(np.concatenate([np.asarray(s[1]) for s in summaries]))[::-1]
    K = batch_total if batch_total is not None else bb.batch * world
    thr = allv[min(K, len(allv)) - 1] if len(allv) else np.inf
    active = [int(np.sum(np.asarray(s[1]) >= thr)) for s in summaries]
    counts = [s[0] for s in summaries]
    moves = plan_moves(counts, active)
    # pack what this rank sends: its active leaves with the smallest upper bounds first
    outgoing = {}
    act_idx = np.nonzero(bb.hi >= thr)[0]
    act_idx = act_idx[np.argsort(bb.hi[act_idx], kind="stable")]
    used = 0
    send_mask = np.zeros(bb.count(), bool)
    for (s, d, k) in moves:
        if s != rank:
            continue
        idx = act_idx[used:used + k]
        used += k
        send_mask[idx] = True
        outgoing[d] = (bb.boxes[idx], bb.lo[idx], bb.hi[idx], bb.feats[idx])
    parcels = [None] * world
    dist.all_gather_object(parcels, outgoing)
    if send_mask.any():
        bb._take(~send_mask)
    for src in range(world):
        got = parcels[src].get(rank) if parcels[src] else None
        if got is None:
            continue
        bx, lo, hi, ft = got
        bb.boxes = np.concatenate([bb.boxes, bx], 0)
        bb.lo = np.concatenate([bb.lo, lo])
        bb.hi = np.concatenate([bb.hi, hi])
        bb.feats = np.concatenate([bb.feats, ft], 0) if len(bb.feats) else ft
    return {"threshold": float(thr), "active": active, "moves": moves}


def global_bounds(bb: BranchAndBound, dist) -> Tuple[float, float, int]:
    """(U, L, total leaves) over all ranks."""
    vals = [None] * dist.get_world_size()
    dist.all_gather_object(vals, (bb.upper(), bb.lower(), bb.count()))
    return max(v[0] for v in vals), max(v[1] for v in vals), sum(v[2] for v in vals)


# ---------------------------------------------------------------- GPU bounds and the split head
def gpu_bound_fn(ctx, widths, W, b, root, degree=2, cap=16, tau=0.0, output=0) -> BoundFn:
    """Bounds of output `output` and the split features of every box, by one
    batched bern_propagate (plus bern_split_features) per call."""
    import torch
    from . import bern
    Wd = [torch.as_tensor(np.asarray(w, np.float32)).cuda() for w in W]
    bd = [torch.as_tensor(np.asarray(x, np.float32)).cuda() for x in b]
    n = int(widths[0])
    root_d = torch.as_tensor(np.asarray(root, np.float32)).cuda()

    def fn(boxes: np.ndarray):
        bx = torch.as_tensor(np.ascontiguousarray(boxes, np.float32)).cuda()
        out = ctx.propagate(widths, Wd, bd, bx, degree=degree, cap=cap, tau=tau)
        x = torch.empty(bx.shape[0], 2 * n + 2, device="cuda")
        ctx.split_features(n, bx, root_d, out, output, x)
        ctx.check("split_features")
        return (out["lo"][:, output].double().cpu().numpy(),
                out["hi"][:, output].double().cpu().numpy(), x.cpu().numpy())

    return fn


def split_labels(bound_fn: BoundFn, boxes: np.ndarray, chunk: int = 4096) -> np.ndarray:
    """Label of each box: the input dimension whose halving gives the
    smallest larger child upper bound (ties: the smaller mean child width),
    computed by the plain method on all 2n children."""
    B, n = boxes.shape[0], boxes.shape[1]
    score = np.zeros((B, n))
    for k in range(n):
        kids = split_boxes(boxes, np.full(B, k))
        his, wid = [], []
        for s in range(0, len(kids), chunk):
            lo, hi, _ = bound_fn(kids[s:s + chunk])
            his.append(hi)
            wid.append(hi - lo)
        hi = np.concatenate(his).reshape(B, 2)
        w = np.concatenate(wid).reshape(B, 2)
        score[:, k] = hi.max(axis=1) + 1e-9 * w.mean(axis=1)
    return np.argmin(score, axis=1)


def train_split_head(ctx, feats: np.ndarray, labels: np.ndarray, n: int, steps=500, lr=3e-3,
                     seed=0):
    """The split head: an Mlp over the 2n+2 split features with n classes,
    trained on the GPU with the library's kernels."""
    import torch
    from . import bern
    F = feats.shape[1]
    P = int(bern.load().bern_mlp_num_params(F, n))
    H = bern.BERN_MLP_HIDDEN
    rng = np.random.default_rng(seed)
    theta = np.zeros(P, np.float32)
    theta[:H * F] = rng.normal(0, np.sqrt(2.0 / F), H * F)
    o = H * F + H
    theta[o:o + n * H] = rng.normal(0, np.sqrt(1.0 / H), n * H)
    m = bern.Mlp(torch, F, n, theta)
    X = torch.as_tensor(np.ascontiguousarray(feats, np.float32)).cuda()
    y = torch.as_tensor(np.asarray(labels, np.int32)).cuda()
    g = torch.empty(P, device="cuda")
    loss = torch.empty(1, device="cuda")
    for _ in range(steps):
        ctx.mlp_backward(m, X, y, None, g, loss)
        ctx.mlp_adam(m, g, lr)
    ctx.check("split head training")
    return m, float(loss.item())


def mlp_split_fn(ctx, mlp, root: np.ndarray, min_ratio: float = 0.5) -> SplitFn:
    """Split rule of a trained split head: the most probable dimension, unless
    its side (relative to the root) is below min_ratio times the widest
    relative side, in which case the widest side is split (the fallback)."""
    import torch
    root = np.asarray(root, np.float32)

    def fn(boxes: np.ndarray, feats: np.ndarray) -> np.ndarray:
        X = torch.as_tensor(np.ascontiguousarray(feats, np.float32)).cuda()
        z = torch.empty(X.shape[0], mlp.C, device="cuda")
        ctx.mlp_forward(mlp, X, z)
        dims = z.argmax(1).cpu().numpy()
        side = boxes[:, :, 1].astype(np.float64) - boxes[:, :, 0]
        rel = side / np.maximum(root[:, 1].astype(np.float64) - root[:, 0], 1e-300)[None, :]
        wide = np.argmax(rel, axis=1)
        r = np.arange(len(dims))
        return np.where(rel[r, dims] >= min_ratio * rel[r, wide], dims, wide)

    return fn


def split_training_boxes(bound_fn: BoundFn, root: np.ndarray, rounds: int = 10, batch: int = 64,
                         seed: int = 0):
    """Boxes (and their split features) for training the split head: the
    leaves of a widest-side search and of a random-dimension search from the
    root, so that the head sees both balanced and elongated boxes."""
    rng = np.random.default_rng(seed)
    n = np.asarray(root).shape[0]
    a = BranchAndBound(bound_fn, root, batch=batch, max_leaves=1 << 30)
    a.run(rounds)
    b = BranchAndBound(bound_fn, root, split_fn=lambda bx, ft: rng.integers(0, n, len(bx)),
                       batch=batch, max_leaves=1 << 30)
    b.run(rounds)
    return np.concatenate([a.boxes, b.boxes], 0), np.concatenate([a.feats, b.feats], 0)
