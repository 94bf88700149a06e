"""The seeded input recipe: shapes, seeds, draw order and box structure of
the workloads, as the design notes state them (reading R13).  Host logic
only; no method arithmetic."""
import numpy as np
import pytest

from paper_2211_14438_gb300 import workloads as wl


def test_draw_order_and_distributions():
    # per layer W (row-major) then b, from one PCG64 generator
    net = wl.make_net([3, 5, 2], seed=7)
    rng = np.random.default_rng(7)
    W1 = rng.normal(0, 1 / np.sqrt(3), (5, 3))
    b1 = rng.uniform(-0.1, 0.1, 5)
    W2 = rng.normal(0, 1 / np.sqrt(5), (2, 5))
    np.testing.assert_array_equal(net.W[0], W1.astype(np.float32))
    np.testing.assert_array_equal(net.b[0], b1.astype(np.float32))
    np.testing.assert_array_equal(net.W[1], W2.astype(np.float32))
    big = wl.make_net([64, 4096], seed=1)
    assert abs(big.W[0].std() * np.sqrt(64) - 1.0) < 0.02
    assert np.abs(big.b[0]).max() <= 0.1
    p = wl.paper_net(2, [400], seed=3)
    assert np.abs(p.W[0]).max() <= 5.0 and np.abs(p.b[0]).max() <= 5.0
    assert p.W[0].std() == pytest.approx(10 / np.sqrt(12), rel=0.05)


def test_single_boxes():
    a = wl.single_box_2in()
    assert a.net.widths == [2, 20, 20, 1] and a.net.seed == 0
    np.testing.assert_array_equal(a.boxes, [[[-1, 1], [-1, 1]]])
    b = wl.single_box_4in()
    assert b.net.widths == [4, 50, 50, 50, 2] and b.net.seed == 1
    np.testing.assert_array_equal(b.boxes, [[[-0.5, 0.5]] * 4])
    r = wl.bnb_root_6in()
    assert r.net.widths == [6, 64, 64, 64, 64, 1] and r.degree_cap == 16
    np.testing.assert_array_equal(r.boxes, [[[-1, 1]] * 6])


def test_batch_3in_structure():
    w = wl.batch_3in()
    assert w.net.widths == [3, 64, 64, 64, 64, 1] and w.boxes.shape == (5120, 3, 2)
    assert w.boxes.dtype == np.float32 and w.degree == 2 and w.degree_cap == 16
    g, r = w.boxes[:4096], w.boxes[4096:]
    side = g[..., 1] - g[..., 0]
    np.testing.assert_allclose(side, 0.125, atol=1e-6)
    # the grid cells tile [-1,1]^3 exactly: every cell's lower corner is distinct
    assert len({tuple(x) for x in g[..., 0]}) == 4096
    assert g.min() == -1.0 and g.max() == 1.0
    # random boxes: inside [-1,1]^3, sides at most 0.5, never inverted
    assert r.min() >= -1.0 and r.max() <= 1.0
    rs = r[..., 1] - r[..., 0]
    assert np.all(rs >= 0) and np.all(rs <= 0.5 + 1e-6)
    # the unclipped sides are >= 0.01
    inner = (r[..., 0] > -1.0) & (r[..., 1] < 1.0)
    assert np.all(rs[inner] >= 0.01 - 1e-6)


def test_batch_6in_structure():
    w = wl.batch_6in()
    assert w.net.widths == [6, 100, 100, 100, 2] and w.boxes.shape == (2048, 6, 2)
    assert w.prune_tau == pytest.approx(1e-7) and w.degree_cap == 16
    s = w.boxes[..., 1] - w.boxes[..., 0]
    assert np.all(s >= 0) and np.all(s <= 0.5 + 1e-6)


def test_training_boxes_are_their_own_draws():
    a = wl.batch_3in_training_boxes(800)
    assert a.shape == (800, 3, 2)
    np.testing.assert_allclose((a[:640, :, 1] - a[:640, :, 0])[
        (a[:640, :, 0] > -1) & (a[:640, :, 1] < 1)], 0.125, atol=1e-6)
    ev = wl.batch_3in().boxes
    assert not any(np.array_equal(x, y) for x in a[:50] for y in ev[4096:4146])
    assert wl.batch_6in_training_boxes(700).shape == (700, 6, 2)


def test_seeds_are_reproducible():
    a, b = wl.batch_3in(), wl.batch_3in()
    np.testing.assert_array_equal(a.boxes, b.boxes)
    for x, y in zip(a.net.W, b.net.W):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("world", [1, 2, 4])
def test_batch_3in_replicas(world):
    # weak scaling: world replicas of 5120 boxes, replica 0 the benchmark's
    # own boxes, every replica the same grid cells with its own random boxes,
    # one network
    w0 = wl.batch_3in()
    w = wl.batch_3in_replicas(world)
    assert w.boxes.shape == (5120 * world, 3, 2)
    assert np.array_equal(w.boxes[:5120], w0.boxes)
    for a, b in zip(w.net.W, w0.net.W):
        assert np.array_equal(a, b)
    reps = w.boxes.reshape(world, 5120, 3, 2)
    for r in range(1, world):
        assert np.array_equal(reps[r, :4096], w0.boxes[:4096])        # the 16^3 grid
        assert not np.array_equal(reps[r, 4096:], w0.boxes[4096:])    # fresh random boxes
        side = reps[r, 4096:, :, 1] - reps[r, 4096:, :, 0]
        assert np.all(side >= 0) and np.all(side <= 0.5 + 1e-6)
        assert np.all(reps[r, :, :, 0] >= -1) and np.all(reps[r, :, :, 1] <= 1)
    assert np.array_equal(wl.batch_3in_replicas(world).boxes, w.boxes)   # seeded
