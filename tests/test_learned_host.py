"""CPU checks of the learned component's host logic: the plan family the
labels choose from, the deterministic work count behind the labels, the
choice of plans per box with the smallest width multiplier that meets the
width target, and the trace slicing helpers.  No GPU."""
import itertools

import numpy as np
import pytest
import torch

from paper_2211_14438_gb300 import learned


@pytest.mark.parametrize("n_hidden", [1, 2, 3, 4])
def test_plan_family(n_hidden):
    fam = learned.plan_family(n_hidden)
    assert len(fam) == 4 * 2 ** (n_hidden - 1) == len(set(fam))
    for p in fam:
        assert len(p) == n_hidden and p[0] in (1, 2, 3, 4)
        assert all(d in (1, 2) for d in p[1:])
    # every first order with every {1, 2} tail, the plain order-2 plan among them
    want = {(f,) + t for f in (1, 2, 3, 4) for t in itertools.product((1, 2), repeat=n_hidden - 1)}
    assert set(fam) == want and (2,) * n_hidden in fam


def test_plan_cost_counted_by_hand():
    # [2, 3, 1]: layer 1 has M(2,1) = 3 input terms: affine 3*2*3 = 18,
    # enclosure 3 * 2 * 2^2 * 3/2 = 36; then the composition and the output
    # layer at the composed degree D: affine 1*3*M(2,D), enclosure
    # 1 * 2 * (D+1)^2 (D+2)/2
    assert learned.plan_cost([2, 3, 1], (1,)) == 18 + 36 + 3 * 3 + (9 + 12)
    assert learned.plan_cost([2, 3, 1], (2,)) == 18 + 36 + 3 * 9 / 2 + (18 + 36)
    # order 3: interval Horner, 4 M sum_{k=1,2} M(2, k) = 4*3*(3+6) per neuron
    assert learned.plan_cost([2, 3, 1], (3,)) == 18 + 36 + 3 * 108 + (30 + 80)
    # the cap holds the output layer at degree 2
    assert learned.plan_cost([2, 3, 1], (3,), cap=2) == 18 + 36 + 3 * 108 + (18 + 36)


def test_plan_cost_grows_with_every_order():
    widths = [3, 64, 64, 64, 64, 1]
    for plan in learned.plan_family(4):
        c = learned.plan_cost(widths, plan)
        for i in range(4):
            if plan[i] < 4:
                up = plan[:i] + (plan[i] + 1,) + plan[i + 1:]
                assert learned.plan_cost(widths, up) > c


def _two_kinds_table():
    # plans: 0 base (cost 1.0), 1 cheap (0.5), 2 tight (2.0); boxes of kind A
    # lose nothing under plan 1, boxes of kind B widen to 1.6 there
    cost = np.array([1.0, 0.5, 2.0])
    a = np.tile([1.0, 1.0, 0.9], (50, 1))
    b = np.tile([1.0, 1.6, 0.9], (50, 1))
    return np.vstack([a, b]), cost


def test_choose_plans_smallest_multiplier_meeting_the_base_width():
    table, cost = _two_kinds_table()
    idx, lam, mean_w = learned.choose_plans(table, cost, base_idx=0)
    # B leaves plan 1 for plan 0 once 1 + lam < 0.5 + 1.6 lam, lam > 5/6;
    # then every box has width 1.0, the base mean
    assert lam == pytest.approx(5.0 / 6.0, rel=1e-6)
    assert np.all(idx[:50] == 1) and np.all(idx[50:] == 0)
    assert mean_w == pytest.approx(1.0)


def test_choose_plans_with_a_margin():
    table, cost = _two_kinds_table()
    idx, lam, mean_w = learned.choose_plans(table, cost, base_idx=0, margin=0.04)
    # target 0.96: B must take plan 2 (2 + 0.9 lam < 1 + lam, lam > 10), while
    # A keeps plan 1 up to lam = 15
    assert lam == pytest.approx(10.0, rel=1e-6)
    assert np.all(idx[:50] == 1) and np.all(idx[50:] == 2)
    assert mean_w == pytest.approx(0.95)
    # the same choice against an explicit base mean
    idx2, lam2, _ = learned.choose_plans(table, cost, base_idx=1, margin=0.04, base_mean=1.0)
    assert np.array_equal(idx, idx2) and lam2 == pytest.approx(lam)


def test_hidden_slices_and_mean_width():
    assert learned.hidden_slices([3, 64, 32, 1]) == [(1, 0, 64), (2, 64, 32)]
    assert learned.hidden_slices([2, 5, 1]) == [(1, 0, 5)]
    out = {"lo": torch.tensor([[0.0, -1.0], [1.0, 1.0]]),
           "hi": torch.tensor([[1.0, 2.0], [1.5, 3.0]])}
    assert np.allclose(learned.mean_width(out), [2.0, 1.25])
