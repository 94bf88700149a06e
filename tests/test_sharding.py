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
