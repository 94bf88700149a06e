"""Pins of the learned component's oracle (CPU, no GPU): the analytic
gradient against float64 finite differences, closed forms of the softmax
cross-entropy, the bfloat16 rounding rule on hand-worked values, one Adam step
in closed form, and the degree features on hand-worked items."""
import numpy as np
import pytest

from oracle import mlp as om


def rand_problem(F=8, C=4, n=37, seed=0):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.4, om.num_params(F, C))
    x = rng.normal(0, 1, (n, F)).astype(np.float32)
    y = rng.integers(0, C, n)
    w = rng.uniform(0.5, 2.0, n)
    return theta, x, y, w


@pytest.mark.parametrize("F,C", [(8, 4), (3, 2), (16, 8)])
def test_gradient_matches_finite_differences(F, C):
    theta, x, y, w = rand_problem(F, C, seed=F + C)
    _, g = om.loss_and_grad(theta, F, C, x, y, w, emulate=False)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(theta), 40, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = om.loss_and_grad(tp, F, C, x, y, w, emulate=False)
        lm, _ = om.loss_and_grad(tm, F, C, x, y, w, emulate=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1 + abs(fd)), (i, fd, g[i])


def test_zero_weights_uniform_softmax():
    F, C, n = 8, 4, 10
    theta = np.zeros(om.num_params(F, C))
    x = np.random.default_rng(2).normal(size=(n, F)).astype(np.float32)
    y = np.arange(n) % C
    loss, g = om.loss_and_grad(theta, F, C, x, y)
    assert loss == pytest.approx(np.log(C), abs=1e-15)
    # only b2 gets a gradient: mean of (1/C - onehot)
    db2 = g[-C:]
    want = np.full(C, 1.0 / C) - np.bincount(y, minlength=C) / n
    assert np.allclose(db2, want, atol=1e-15)
    assert np.all(g[:-C] == 0)


def test_softmax_shift_invariance():
    F, C = 8, 4
    theta, x, y, w = rand_problem(F, C, seed=5)
    l0, g0 = om.loss_and_grad(theta, F, C, x, y, w, emulate=False)
    t2 = theta.copy()
    t2[-C:] += 3.25
    l1, g1 = om.loss_and_grad(t2, F, C, x, y, w, emulate=False)
    assert l1 == pytest.approx(l0, rel=1e-12)
    assert np.allclose(g1, g0, atol=1e-12)


def test_bf16_rounding_hand_worked():
    # spacing of bfloat16 at 1 is 2^-7
    v = np.array([1.0, 1 + 2.0**-8, 1 + 3 * 2.0**-8, 1 + 2.0**-7, -(1 + 2.0**-8) - 2.0**-12,
                  2.0**-130, 65504.0, 0.0])
    want = np.array([1.0, 1.0, 1 + 2.0**-6, 1 + 2.0**-7, -(1 + 2.0**-7), 2.0**-130, 65536.0,
                     0.0])
    assert np.array_equal(om.bf16(v), want)


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    lr, eps = 0.01, 1e-8
    t1, m, v = om.adam(th, np.zeros(4), np.zeros(4), g, lr, 0.9, 0.999, eps, 1)
    # at t = 1 the bias-corrected moments are g and g^2
    assert np.allclose(t1, th - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_degree_features_hand_worked():
    lo = np.array([-1.0, 2.0, -3.0, -0.5], np.float32)
    hi = np.array([3.0, 4.0, -1.0, 0.5], np.float32)
    nt = np.array([1, 16, 256, 35])
    f = om.degree_features(lo, hi, nt, 2).astype(np.float64)
    assert np.allclose(f[0], [-1 / 3, 1, 2 / 8, 0.25, 0, 0, 0, 0.25])
    assert np.allclose(f[1], [0.5, 1, 1 / 8, 0.25, 4 / 16, 1, 0, 0])
    assert np.allclose(f[2], [-1, -1 / 3, 1 / 8, 0.25, 8 / 16, 0, 1, 1])
    assert np.allclose(f[3], [-1, 1, 0, 0.25, np.log2(35) / 16, 0, 0, 0.5])
