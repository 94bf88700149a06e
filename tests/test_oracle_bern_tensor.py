"""The paper's dense Bernstein-tensor arithmetic (Sec. 4) against the
definition, and the whole BERN-NN loop on those tensors against the
power-basis oracle: the two representations give the same bounds and the
same polynomials (up to FP64 rounding), so the storage format changes cost,
not tightness."""
import numpy as np
import pytest

import oracle
from oracle import bern_tensor as bt
from paper_2211_14438_gb300 import workloads as wl


def _pts(rng, n, count=300):
    return rng.random((count, n))


@pytest.mark.parametrize("sa,sb", [((3,), (4,)), ((3, 2), (2, 4)), ((2, 3, 2), (3, 1, 2))])
def test_prod_bern_is_the_product(sa, sb):
    rng = np.random.default_rng(len(sa))
    a, b = rng.normal(size=sa), rng.normal(size=sb)
    p = bt.prod_bern(a, b)
    assert p.shape == tuple(x + y - 1 for x, y in zip(sa, sb))
    t = _pts(rng, len(sa))
    np.testing.assert_allclose(bt.evaluate(p, t), bt.evaluate(a, t) * bt.evaluate(b, t),
                               rtol=1e-11, atol=1e-11)


def test_prod_bern_hand_worked():
    # order-1 coefficients (0, 1) are t; t * t = t^2, whose order-2
    # Bernstein coefficients are (0, 0, 1)
    t = np.array([0.0, 1.0])
    np.testing.assert_allclose(bt.prod_bern(t, t), [0.0, 0.0, 1.0], atol=1e-15)
    # (1 - t) * t = t - t^2: order-2 coefficients (0, 1/2, 0)
    np.testing.assert_allclose(bt.prod_bern(np.array([1.0, 0.0]), t), [0.0, 0.5, 0.0],
                               atol=1e-15)


@pytest.mark.parametrize("sa,sb", [((2,), (5,)), ((3, 1), (1, 4)), ((2, 2, 3), (3, 2, 1))])
def test_sum_bern_and_elevation(sa, sb):
    rng = np.random.default_rng(10 + len(sa))
    a, b = rng.normal(size=sa), rng.normal(size=sb)
    s = bt.sum_bern(a, b)
    assert s.shape == tuple(max(x, y) for x, y in zip(sa, sb))
    t = _pts(rng, len(sa))
    np.testing.assert_allclose(bt.evaluate(s, t), bt.evaluate(a, t) + bt.evaluate(b, t),
                               rtol=1e-11, atol=1e-11)
    e = bt.elevate(a, [x + 2 for x in sa])
    np.testing.assert_allclose(bt.evaluate(e, t), bt.evaluate(a, t), rtol=1e-11, atol=1e-11)
    # elevation keeps the range inside the old coefficient range (Def. 2)
    assert e.min() >= a.min() - 1e-12 and e.max() <= a.max() + 1e-12


def test_pow_bern():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(2, 3))
    t = _pts(rng, 2)
    np.testing.assert_allclose(bt.evaluate(bt.pow_bern(a, 3), t), bt.evaluate(a, t) ** 3,
                               rtol=1e-10, atol=1e-10)
    assert bt.pow_bern(a, 0).shape == (1, 1)


def _compare(widths, W, b, box, d):
    n = widths[0]
    r = oracle.propagate(widths, W, b, box, d, cap=64)
    q = bt.propagate(widths, W, b, box, d)
    scale = 1 + np.abs(r["hi"]).max() + np.abs(r["lo"]).max()
    assert np.abs(q["lo"] - r["lo"]).max() <= 1e-9 * scale
    assert np.abs(q["hi"] - r["hi"]).max() <= 1e-9 * scale
    t = _pts(np.random.default_rng(d), n, 200)
    for j in range(widths[-1]):
        for name in ("upper", "lower"):
            pv = oracle.eval_poly(r[name][j], n, t)
            tv = bt.evaluate(q[name][j], t)
            assert np.abs(pv - tv).max() <= 1e-9 * (1 + np.abs(pv).max())


@pytest.mark.parametrize("d", [1, 2, 3])
def test_tensor_path_equals_power_basis_single_box_2in(d):
    w = wl.single_box_2in()
    _compare(w.net.widths, w.net.W, w.net.b, w.boxes[0], d)


def test_tensor_path_equals_power_basis_three_inputs():
    net = wl.make_net([3, 8, 8, 1], seed=9)
    _compare(net.widths, net.W, net.b, wl.box_array([-1.0] * 3, [1.0] * 3), 2)


def test_tensor_path_equals_power_basis_paper_family():
    net = wl.paper_net(2, [10, 10], seed=600)
    _compare(net.widths, net.W, net.b, wl.box_array([-1.0, -1.0], [1.0, 1.0]), 2)
