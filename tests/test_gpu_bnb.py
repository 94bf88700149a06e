"""Branch-and-bound refinement on the GPU: the split features of the C ABI
against a numpy restatement from the same propagation result, soundness of
the search (every leaf's bounds contain the network on sampled points, the
sampled maximum never exceeds U, L <= U), and the learned split head
(labels from the plain method, GPU training, then driving the search)."""
import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import bern, bnb
from paper_2211_14438_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


def test_split_features_match_numpy(ctx):
    widths = [4, 12, 12, 2]
    net = wl.make_net(widths, 81)
    root = np.array([[-1, 1]] * 4, np.float32)
    rng = np.random.default_rng(81)
    c = rng.uniform(-0.7, 0.7, (9, 4))
    boxes = wl.box_array(c - 0.2, c + 0.25)
    W = [torch.from_numpy(x).cuda() for x in net.W]
    b = [torch.from_numpy(x).cuda() for x in net.b]
    bx = torch.from_numpy(boxes).cuda()
    out = ctx.propagate(widths, W, b, bx, degree=2, cap=16)
    x = torch.empty(9, 10, device="cuda")
    ctx.split_features(4, bx, torch.from_numpy(root).cuda(), out, 1, x)
    assert ctx.sync() == 0
    got = x.cpu().numpy()
    coef = out["coef"].cpu().numpy().astype(np.float64)
    nt = out["n_terms"].cpu().numpy()
    lo, hi = out["lo"].cpu().numpy(), out["hi"].cpu().numpy()
    ex = bern.monomials(4, 16).astype(np.float64)
    for i in range(9):
        cu = coef[i, 1, 0, :nt[i, 1, 0]]
        cl = coef[i, 1, 1, :nt[i, 1, 1]]
        m = max(len(cu), len(cl))
        cu = np.pad(cu, (0, m - len(cu)))
        cl = np.pad(cl, (0, m - len(cl)))
        s = (np.abs(cu)[:, None] * ex[:m]).sum(0)
        side = boxes[i, :, 1].astype(np.float32) - boxes[i, :, 0].astype(np.float32)
        want = np.concatenate([np.log2(side / 2.0) / 16, s / s.sum(),
                               [np.log2(hi[i, 1] - lo[i, 1]) / 8,
                                np.log2(np.abs(cu - cl).sum()) / 8]])
        assert np.allclose(got[i], want, rtol=1e-4, atol=1e-5), (i, got[i], want)


def _leaf_check(net, bb, count, rng):
    bad = 0
    for k in rng.choice(bb.count(), min(count, bb.count()), replace=False):
        box = bb.boxes[k].astype(np.float64)
        x = box[:, 0] + rng.random((2000, box.shape[0])) * (box[:, 1] - box[:, 0])
        y = oracle.network_forward(net.widths, net.W, net.b, x)[:, 0]
        e = 1e-9 * (1 + np.abs(y))
        bad += int(np.sum(y > bb.hi[k] + e) + np.sum(y < bb.lo[k] - e))
    return bad


def test_search_is_sound(ctx):
    widths = [4, 24, 24, 1]
    net = wl.make_net(widths, 71)
    root = np.array([[-1, 1]] * 4, np.float32)
    fn = bnb.gpu_bound_fn(ctx, widths, net.W, net.b, root, degree=2, cap=16)
    bb = bnb.BranchAndBound(fn, root, batch=64, max_leaves=500)
    U0 = bb.upper()
    bb.run(12)
    assert bb.count() <= 500 and bb.upper() < U0 and bb.lower() <= bb.upper()
    rng = np.random.default_rng(5)
    x = root[:, 0] + rng.random((200_000, 4)) * (root[:, 1] - root[:, 0])
    assert oracle.network_forward(widths, net.W, net.b, x)[:, 0].max() <= bb.upper()
    assert _leaf_check(net, bb, 40, rng) == 0


def test_learned_split_head(ctx):
    widths = [4, 24, 24, 1]
    net = wl.make_net(widths, 71)
    root = np.array([[-1, 1]] * 4, np.float32)
    fn = bnb.gpu_bound_fn(ctx, widths, net.W, net.b, root, degree=2, cap=16)
    boxes, feats = bnb.split_training_boxes(fn, root, rounds=10, batch=64)
    lab = bnb.split_labels(fn, boxes)
    m, loss = bnb.train_split_head(ctx, feats, lab, 4)
    z = torch.empty(len(lab), 4, device="cuda")
    ctx.mlp_forward(m, torch.from_numpy(feats).cuda(), z)
    acc = float((z.argmax(1).cpu().numpy() == lab).mean())
    chance = np.bincount(lab, minlength=4).max() / len(lab)
    assert acc > chance + 0.1, (acc, chance)
    bl = bnb.BranchAndBound(fn, root, split_fn=bnb.mlp_split_fn(ctx, m, root), batch=64,
                            max_leaves=500)
    bl.run(12)
    assert bl.lower() <= bl.upper()
    assert _leaf_check(net, bl, 40, np.random.default_rng(6)) == 0
