"""Host-side multi-rank logic (box sharding, result gather, max over ranks),
on CPU with the gloo backend and world_size 2.  Boxes are independent, so the
only communication is the final gather and the timing max."""
import os
import socket

import numpy as np
import pytest

from paper_2211_14438_gb300 import sharding
from paper_2211_14438_gb300 import workloads as wl


def test_shard_ranges_cover_and_balance():
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 4, 8):
        costs = rng.uniform(0.5, 2.0, 1000)
        r = sharding.shard_ranges(costs, world)
        assert r[0][0] == 0 and r[-1][1] == 1000
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        loads = [costs[a:b].sum() for a, b in r]
        assert max(loads) - min(loads) <= 2 * costs.max() + 1e-9
    assert sharding.shard_ranges([], 3) == [(0, 0)] * 3
    assert sharding.shard_ranges([1.0], 4)[-1] == (0, 1) or sum(b - a for a, b in sharding.shard_ranges([1.0], 4)) == 1


def test_interval_cost_hand_worked():
    """A [1,1,1] net: W1 = 1, b1 = 0; W2 = 1, b2 = 0.  On [0.5, 1] the hidden
    neuron is active (cost: two layer steps, M(1,1) = 2 terms each); on
    [-1, 1] it straddles 0 and adds the pairs of a degree-1 square,
    M(M+1)/2 = 3."""
    W = [np.array([[1.0]]), np.array([[1.0]])]
    b = [np.array([0.0]), np.array([0.0])]
    boxes = np.array([[[0.5, 1.0]], [[-1.0, 1.0]], [[-2.0, -1.0]]])
    c = sharding.interval_cost([1, 1, 1], W, b, boxes, degree=2, cap=16)
    # layer steps: 1*1*M(1,1)=2 and 1*1*M(1,2)=3 after an order-2 layer
    assert c[0] == 2 + 3 and c[2] == 2 + 3
    assert c[1] == 2 + 3 + 3


def test_interval_cost_tracks_unstable_work():
    w = wl.batch_3in()
    c = sharding.interval_cost(w.net.widths, w.net.W, w.net.b, w.boxes, 2, 16)
    assert c.shape == (len(w.boxes),) and np.all(c > 0)
    # the random boxes (sides up to 0.5) are wider than the grid cells (0.125)
    assert c[4096:].mean() > c[:4096].mean()
    # a point box has no unstable neuron: the layer steps only
    pt = np.repeat(w.boxes[:1, :, :1], 2, axis=2)
    base = sum(w.net.widths[i + 1] * w.net.widths[i] * sharding._num_monomials(3, min(2 ** i, 16))
               for i in range(5))
    assert sharding.interval_cost(w.net.widths, w.net.W, w.net.b, pt, 2, 16)[0] == base


def test_box_cost_prefers_wide_boxes():
    w = wl.batch_3in()
    c = sharding.box_cost(w.boxes)
    assert c.shape == (len(w.boxes),) and np.all(c >= 1.0)
    assert c[4096:].mean() > c[:4096].mean()      # random boxes are wider than grid cells


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = wl.batch_3in(n_random=64, cells=4)
        a, b = sharding.shard_boxes(w.boxes, rank, world)
        # a stand-in per-box result that depends only on the box: its index
        # and its width sum (the real result comes from the GPU kernels)
        local = {"idx": np.arange(a, b),
                 "width": (w.boxes[a:b, :, 1] - w.boxes[a:b, :, 0]).sum(-1)}
        full = sharding.gather_results(local, rank, world, dist)
        t = sharding.max_over_ranks(float(rank + 1) * 1.5, world, dist)
        q.put((rank, full["idx"].tolist(), full["width"].tolist(), t))
    finally:
        dist.destroy_process_group()


def _fake_propagate(boxes, degree=2, cap=16):
    """A per-box result that depends only on the box (the real one comes from
    the GPU kernels): torch CPU tensors shaped like Context.propagate's."""
    import torch
    B = len(boxes)
    w = (boxes[:, :, 1] - boxes[:, :, 0]).sum(-1)
    lo = torch.from_numpy(boxes[:, :, 0].sum(-1, keepdims=True).astype(np.float32))
    hi = torch.from_numpy((boxes[:, :, 1].sum(-1, keepdims=True)).astype(np.float32))
    nt = torch.from_numpy(np.stack([np.full((B, 1), 3), np.full((B, 1), 2)], -1).astype(np.int32))
    coef = torch.from_numpy(np.repeat(w[:, None, None, None], 4, -1).repeat(2, 2)
                            .astype(np.float32))
    return {"lo": lo, "hi": hi, "n_terms": nt, "coef": coef, "keys": None}


def _sharded_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = wl.batch_3in(n_random=96, cells=6)
        res, (a, z), counts = sharding.propagate_sharded(
            _fake_propagate, w.net.widths, w.net.W, w.net.b, w.boxes, rank, world, dist)
        q.put((rank, a, z, counts, {k: (v.numpy() if v is not None else None)
                                    for k, v in res.items()}))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_propagate_sharded(world):
    """The sharded path end to end on CPU ranks: cost-balanced slices from the
    network's interval cost, each rank's result tensors gathered (padded
    all_gather per tensor) back into box order on every rank, equal to the
    unsharded result."""
    pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = wl.batch_3in(n_random=96, cells=6)
    want = {k: (v.numpy() if v is not None else None)
            for k, v in _fake_propagate(w.boxes).items()}
    costs = sharding.interval_cost(w.net.widths, w.net.W, w.net.b, w.boxes, 2, 16)
    ranges = sharding.shard_ranges(costs, world)
    loads = [costs[a:z].sum() for a, z in ranges]
    assert max(loads) - min(loads) <= 2 * costs.max()
    for rank, a, z, counts, got in res:
        assert (a, z) == ranges[rank] and sum(counts) == len(w.boxes)
        for k in ("lo", "hi", "n_terms", "coef"):
            assert np.array_equal(got[k], want[k]), k
        assert got["keys"] is None


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_gather_and_max(world):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    w = wl.batch_3in(n_random=64, cells=4)
    want_w = (w.boxes[:, :, 1] - w.boxes[:, :, 0]).sum(-1)
    for rank, idx, width, t in res:
        assert idx == list(range(len(w.boxes)))
        np.testing.assert_allclose(width, want_w)
        assert t == 1.5 * world
