"""Pins for the oracle's Lin step (Sec. 5.3): every Lin hidden layers the
post-activation bounds are lowered to multilinear polynomials (order
[1,...,1]).  The cited algorithm is not given; the reading (R22) is the
least-squares multilinear fit on the box plus the Bernstein enclosure of the
residual, added as max (upper) or min (lower) to the constant.

Pinned against hand-worked fits, an independent numerical least squares
(weighted lstsq on Gauss-Legendre nodes), dense-grid soundness and exact
special cases.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import workloads as wl


def _d(p):
    return {k: v for k, v in oracle.to_dict(p).items()}


def _close_dicts(a, b, tol):
    for k in set(a) | set(b):
        assert abs(a.get(k, 0.0) - b.get(k, 0.0)) <= tol, (k, a.get(k), b.get(k))


def _random_poly(rng, n, deg):
    terms = {e: float(rng.normal()) for e in itertools.product(range(deg + 1), repeat=n)
             if sum(e) <= deg}
    return oracle.as_poly(terms, n)


def test_square_hand_worked():
    # t^2 on [0,1]: least-squares line t - 1/6; residual t^2 - t + 1/6 has
    # order-2 Bernstein coefficients (1/6, -1/3, 1/6)
    p = oracle.as_poly({(2,): 1.0}, 1)
    up = _d(oracle.linearize(p, 1, 2, upper=True))
    lo = _d(oracle.linearize(p, 1, 2, upper=False))
    _close_dicts(up, {(0,): 0.0, (1,): 1.0}, 1e-14)
    _close_dicts(lo, {(0,): -0.5, (1,): 1.0}, 1e-14)


def test_product_hand_worked():
    # t1^2 t2: the fit of a product of one-variable factors is the product of
    # their fits, (t1 - 1/6) t2; residual t2 (t1^2 - t1 + 1/6), whose order-3
    # Bernstein coefficients are (j/3) x (1/6, -1/6, -1/6, 1/6)
    p = oracle.as_poly({(2, 1): 1.0}, 2)
    up = _d(oracle.linearize(p, 2, 3, upper=True))
    lo = _d(oracle.linearize(p, 2, 3, upper=False))
    _close_dicts(up, {(0, 0): 1 / 6, (0, 1): -1 / 6, (1, 1): 1.0}, 1e-13)
    _close_dicts(lo, {(0, 0): -1 / 6, (0, 1): -1 / 6, (1, 1): 1.0}, 1e-13)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_multilinear_is_fixed(n):
    rng = np.random.default_rng(n)
    terms = {e: float(rng.normal()) for e in itertools.product((0, 1), repeat=n)}
    p = oracle.as_poly(terms, n)
    for upper in (True, False):
        _close_dicts(_d(oracle.linearize(p, n, n, upper=upper)), terms, 1e-12)


@pytest.mark.parametrize("n,deg", [(1, 5), (2, 4), (3, 3)])
def test_fit_matches_numerical_least_squares(n, deg):
    rng = np.random.default_rng(10 + n)
    p = _random_poly(rng, n, deg)
    # Gauss-Legendre with deg+1 nodes per axis integrates (P - A)^2 exactly
    x, w = np.polynomial.legendre.leggauss(deg + 1)
    x, w = 0.5 * (x + 1), 0.5 * w
    pts = np.array(list(itertools.product(x, repeat=n)))
    wts = np.prod(np.array(list(itertools.product(w, repeat=n))), axis=1)
    subsets = [S for S in itertools.product((0, 1), repeat=n) if sum(S) <= min(n, deg)]
    V = np.stack([np.prod(pts ** np.array(S), axis=1) for S in subsets], 1)
    y = oracle.eval_poly(p, n, pts)
    sw = np.sqrt(wts)
    a, *_ = np.linalg.lstsq(V * sw[:, None], y * sw, rcond=None)
    fit = dict(zip(subsets, a))
    up = _d(oracle.linearize(p, n, deg, upper=True))
    lo = _d(oracle.linearize(p, n, deg, upper=False))
    zero = (0,) * n
    for S in subsets:
        if S != zero:
            assert abs(up[S] - fit[S]) <= 1e-9 and abs(lo[S] - fit[S]) <= 1e-9
    # the shifts are the residual's Bernstein max and min (Def. 2)
    r = dict(oracle.to_dict(p))
    for S in subsets:
        r[S] = r.get(S, 0.0) - fit[S]
    beta = oracle.bernstein_coeffs(oracle.as_poly(r, n), n, deg)
    assert abs((up[zero] - fit[zero]) - beta.max()) <= 1e-9
    assert abs((lo[zero] - fit[zero]) - beta.min()) <= 1e-9
    # the residual has mean zero, so the shifts straddle zero
    assert up[zero] - fit[zero] >= -1e-12 and lo[zero] - fit[zero] <= 1e-12


@pytest.mark.parametrize("n,deg", [(1, 6), (2, 4), (3, 4)])
def test_sound_on_dense_grid(n, deg):
    rng = np.random.default_rng(20 + n)
    p = _random_poly(rng, n, deg)
    g = np.linspace(0, 1, {1: 2001, 2: 101, 3: 31}[n])
    pts = np.array(list(itertools.product(g, repeat=n)))
    v = oracle.eval_poly(p, n, pts)
    up = oracle.linearize(p, n, deg, upper=True)
    lo = oracle.linearize(p, n, deg, upper=False)
    assert np.all(np.asarray(up[0]) <= 1), "multilinear"
    assert np.all(oracle.eval_poly(up, n, pts) >= v - 1e-12)
    assert np.all(oracle.eval_poly(lo, n, pts) <= v + 1e-12)


def test_network_with_lin_is_sound():
    """Problem 1 with Lin = 1 on the [2,20,20,1] net over [-1,1]^2: both
    hidden layers are linearised, so the output polynomials are multilinear;
    no sampled network output leaves the bounds."""
    w = wl.single_box_2in()
    net = w.net
    r = oracle.propagate(net.widths, net.W, net.b, w.boxes[0], 2, lin=1)
    up, lo = r["upper"][0], r["lower"][0]
    assert np.asarray(up[0]).max() <= 1 and np.asarray(lo[0]).max() <= 1
    rng = np.random.default_rng(7)
    t = rng.random((200_000, 2))
    box = w.boxes[0].astype(np.float64)
    x = box[:, 0] + t * (box[:, 1] - box[:, 0])
    y = oracle.network_forward(net.widths, net.W, net.b, x)[:, 0]
    pu, pl = oracle.eval_poly(up, 2, t), oracle.eval_poly(lo, 2, t)
    assert np.all(pl <= y + 1e-9) and np.all(y <= pu + 1e-9)
    assert r["lo"][0] <= y.min() and y.max() <= r["hi"][0]
    # the Bernstein order restarts at min(n, order) after each Lin layer
    assert list(r["order"]) == [1, 2, 2]


def test_lin_beyond_depth_is_a_no_op():
    w = wl.single_box_2in()
    net = w.net
    a = oracle.propagate(net.widths, net.W, net.b, w.boxes[0], 2)
    b = oracle.propagate(net.widths, net.W, net.b, w.boxes[0], 2, lin=5)
    assert a["lo"][0] == b["lo"][0] and a["hi"][0] == b["hi"][0]


@pytest.mark.parametrize("widths,lin", [([2, 20, 20, 1], 1), ([2, 20, 20, 1], 2),
                                        ([3, 8, 8, 8, 1], 2), ([4, 6, 6, 6, 2], 3)])
def test_output_capacity_rule_covers_the_oracle(widths, lin):
    """The binding sizes output polynomials by the degree bookkeeping of the
    plan (with Lin, min(n, D) after every Lin layer); the oracle's outputs
    must fit that graded prefix."""
    from paper_2211_14438_gb300 import bern
    n = widths[0]
    net = wl.make_net(widths, seed=30 + lin)
    box = wl.box_array([-1.0] * n, [1.0] * n)
    r = oracle.propagate(net.widths, net.W, net.b, box, 2, lin=lin)
    deg = max(int(np.asarray(e).sum(axis=1).max()) for e, _ in r["upper"] + r["lower"])
    cap_terms = bern.max_output_terms(widths, 2, 16, lin)
    assert cap_terms >= bern.num_monomials(n, deg)
    assert bern.max_output_terms(widths, 2, 16, lin) <= bern.max_output_terms(widths, 2, 16)


@pytest.mark.parametrize("lin", [1, 2])
def test_exact_rational_lin_agrees_with_fp64(lin):
    """The [2,20,20,1] net over [-1,1]^2 with Lin, in exact rationals (the fit's
    normal equations solved exactly) against the FP64 oracle."""
    from oracle import exact
    w = wl.single_box_2in()
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2, lin=lin)
    q = exact.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2, lin=lin)
    assert float(q["lo"][0]) == pytest.approx(r["lo"][0], rel=1e-11, abs=1e-11)
    assert float(q["hi"][0]) == pytest.approx(r["hi"][0], rel=1e-11, abs=1e-11)
    for name in ("upper", "lower"):
        d = oracle.to_dict(r[name][0])
        qe = q[name][0]
        assert set(d) == set(qe)
        for k in d:
            assert d[k] == pytest.approx(float(qe[k]), rel=1e-9, abs=1e-10)
