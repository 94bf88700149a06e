"""Host logic of the batched branch-and-bound refinement (CPU, no GPU):
children cover their parent exactly, the bounds of the search stay sound and
improve, the leaf budget holds, and the multi-rank rebalancing (two gloo
ranks on CPU) conserves leaves and evens out the leaves to be split next.

The bounding function here is a stand-in with the same contract as the GPU
propagation: natural interval arithmetic of a known function."""
import os

import numpy as np
import pytest

from paper_2211_14438_gb300 import bnb

C0 = np.array([0.3, -0.2, 0.55])


def f(x):
    return -np.sum((x - C0) ** 2 * np.array([1.0, 2.0, 0.5]), axis=-1)


def interval_bound(boxes):
    """Sound bounds of f on each box (each term's square ranges over the box)."""
    lo = boxes[:, :, 0].astype(np.float64) - C0
    hi = boxes[:, :, 1].astype(np.float64) - C0
    sq_hi = np.maximum(lo * lo, hi * hi)
    sq_lo = np.where((lo <= 0) & (hi >= 0), 0.0, np.minimum(lo * lo, hi * hi))
    wts = np.array([1.0, 2.0, 0.5])
    return -(sq_hi * wts).sum(1), -(sq_lo * wts).sum(1), np.zeros((len(boxes), 1), np.float32)


def test_children_cover_parent_exactly():
    rng = np.random.default_rng(0)
    lo = rng.uniform(-1, 1, (200, 4)).astype(np.float32)
    hi = (lo + rng.uniform(0, 1e-3, (200, 4)).astype(np.float32)).astype(np.float32)
    hi[:5] = lo[:5]                       # degenerate sides
    boxes = np.stack([lo, hi], -1)
    dims = rng.integers(0, 4, 200)
    kids = bnb.split_boxes(boxes, dims)
    a, b = kids[0::2], kids[1::2]
    r = np.arange(200)
    assert np.array_equal(a[r, dims, 0], boxes[r, dims, 0])
    assert np.array_equal(b[r, dims, 1], boxes[r, dims, 1])
    assert np.array_equal(a[r, dims, 1], b[r, dims, 0])          # shared midpoint
    assert np.all(a[r, dims, 1] >= boxes[r, dims, 0]) and np.all(a[r, dims, 1] <= boxes[r, dims, 1])
    other = np.ones((200, 4), bool)
    other[r, dims] = False
    assert np.array_equal(a[other], boxes[other]) and np.array_equal(b[other], boxes[other])


def test_search_is_sound_and_improves():
    root = np.array([[-1, 1], [-1, 1], [-1, 1]], np.float32)
    bb = bnb.BranchAndBound(interval_bound, root, batch=16, max_leaves=600)
    U0 = bb.upper()
    hist = bb.run(100)
    assert bb.count() <= 600
    Us = [h["U"] for h in hist]
    assert all(u2 <= u1 + 1e-15 for u1, u2 in zip([U0] + Us, Us))
    # the true maximum (0, at C0 inside the root) lies between L and U
    assert bb.lower() <= 0.0 <= bb.upper()
    assert bb.upper() < 0.05 * (U0 - bb.lower()) + 1e-9 or bb.upper() - bb.lower() < 0.1
    # every leaf that was dropped could not hold the maximum: the leaf holding C0 survives
    inside = np.all((bb.boxes[:, :, 0] <= C0) & (C0 <= bb.boxes[:, :, 1]), axis=1)
    assert inside.any()


def test_custom_split_rule_is_used_and_clipped():
    root = np.array([[-1, 1], [-1, 1], [-1, 1]], np.float32)
    calls = []

    def always_last(boxes, feats):
        calls.append(len(boxes))
        return np.full(len(boxes), 7)      # out of range: clipped to n-1
    bb = bnb.BranchAndBound(interval_bound, root, split_fn=always_last, batch=4, max_leaves=20)
    bb.run(3)
    assert calls and np.allclose(bb.boxes[:, :2, :], root[None, :2, :])


def test_widest_split_is_relative_to_the_root():
    # the fallback split takes the side widest relative to the root's side,
    # not the widest in absolute terms; ties go to the lowest dimension
    root = np.array([[-1, 1], [0, 10], [0, 0.5]], np.float32)
    boxes = np.array([
        [[0, 1], [0, 4], [0, 0.1]],      # relative sides 0.5, 0.4, 0.2
        [[0, 0.2], [0, 9], [0, 0.25]],   # 0.1, 0.9, 0.5
        [[0, 0.2], [0, 1], [0, 0.45]],   # 0.1, 0.1, 0.9
        [[0, 1], [0, 5], [0, 0.25]],     # 0.5, 0.5, 0.5: a tie
    ], np.float32)
    assert bnb.widest_split(boxes, root).tolist() == [0, 1, 2, 0]
    # a degenerate root side never divides by zero and is never chosen over
    # a side that is actually wide
    root0 = np.array([[0, 0], [0, 1]], np.float32)
    b0 = np.array([[[0, 0], [0, 0.5]]], np.float32)
    assert bnb.widest_split(b0, root0).tolist() == [1]


@pytest.mark.parametrize("active", [[10, 0], [3, 3], [7, 2, 0, 9], [0, 0, 5]])
def test_plan_moves_balances(active):
    moves = bnb.plan_moves([a + 5 for a in active], active)
    after = list(active)
    for s, d, k in moves:
        assert k > 0 and s != d
        after[s] -= k
        after[d] += k
    assert sum(after) == sum(active)
    assert max(after) - min(after) <= 1


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    root = np.array([[-1, 1], [-1, 1], [-1, 1]], np.float32)
    # rank 0 starts with the half of the root holding the maximum, rank 1 the
    # other half, any further rank with nothing
    halves = bnb.split_boxes(root[None], np.array([0]))
    mine = halves[1:] if rank == 0 else (halves[:1] if rank == 1 else halves[:0])
    bb = bnb.BranchAndBound(interval_bound, root, batch=8, max_leaves=400, boxes=mine)
    before = bb.count()
    for r in range(6):
        bb.step()
        if r % 2 == 1:
            info = bnb.rebalance(bb, dist)
    U, L, total = bnb.global_bounds(bb, dist)
    q.put((rank, before, bb.count(), total, U, L, info["active"], bb.boxes.copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_rebalance_gloo_ranks(world):
    import multiprocessing as mp
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in ps]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    totals = {r[3] for r in res}
    assert len(totals) == 1 and totals.pop() == sum(r[2] for r in res)
    U, L = res[0][4], res[0][5]
    assert L <= 0.0 <= U
    # after the last rebalance every rank held work near the top of the queue,
    # including the ranks that started with nothing
    assert all(r[2] > 0 for r in res)
    # no box is duplicated across ranks
    allb = np.concatenate([r[7].reshape(len(r[7]), -1) for r in res], 0)
    assert len(np.unique(allb, axis=0)) == len(allb)
