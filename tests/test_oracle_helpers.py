"""Pins for the oracle's evaluation helpers, which the parity and soundness
tests lean on: polynomial evaluation, the plain network forward pass, and
Vol_relative (the mean over the box of upper minus lower bound, Sec. 6).

Each is checked against something fixed outside the oracle: hand-worked
values, and tensor Gauss-Legendre quadrature, which integrates a polynomial of
degree <= 2q-1 in every variable exactly (up to rounding).
"""
import itertools

import numpy as np
import pytest

import oracle


def _gauss_mean(fn, n, q):
    """Mean of fn over [0,1]^n by the q-point Gauss-Legendre rule per axis."""
    x, w = np.polynomial.legendre.leggauss(q)
    x = 0.5 * (x + 1.0)
    w = 0.5 * w
    pts = np.array(list(itertools.product(x, repeat=n)))
    wts = np.prod(np.array(list(itertools.product(w, repeat=n))), axis=1)
    return float(np.sum(wts * fn(pts)))


def test_eval_poly_hand_worked():
    # p(t1, t2) = 2 - 3 t1 + 0.5 t1 t2^2 + t2^3
    p = oracle.as_poly({(0, 0): 2.0, (1, 0): -3.0, (1, 2): 0.5, (0, 3): 1.0}, 2)
    t = np.array([[0.0, 0.0], [1.0, 1.0], [0.5, 0.25], [0.2, 1.0]])
    want = [2.0, 0.5, 2.0 - 1.5 + 0.5 * 0.5 * 0.0625 + 0.015625, 2.0 - 0.6 + 0.1 + 1.0]
    np.testing.assert_allclose(oracle.eval_poly(p, 2, t), want, rtol=0, atol=1e-15)


def test_network_forward_hand_worked():
    # 2 -> 2 -> 1: z = relu(W1 x + b1), y = W2 z + b2
    W = [np.array([[1.0, -2.0], [0.5, 0.5]]), np.array([[3.0, -1.0]])]
    b = [np.array([0.25, -1.0]), np.array([0.5])]
    x = np.array([[1.0, 1.0], [1.0, -1.0], [4.0, 2.0]])
    # x=(1,1):  pre (-0.75, 0)  -> z (0, 0)    -> y 0.5
    # x=(1,-1): pre (3.25, -1)  -> z (3.25, 0) -> y 10.25
    # x=(4,2):  pre (0.25, 2)   -> z (0.25, 2) -> y 0.75 - 2 + 0.5 = -0.75
    y = oracle.network_forward([2, 2, 1], W, b, x)
    np.testing.assert_allclose(y[:, 0], [0.5, 10.25, -0.75], rtol=0, atol=1e-15)


def test_vol_relative_hand_worked():
    # upper = 1 + t1 t2^2, lower = -t1: mean of (1 + t1 t2^2 + t1) = 1 + 1/6 + 1/2
    up = oracle.as_poly({(0, 0): 1.0, (1, 2): 1.0}, 2)
    lo = oracle.as_poly({(1, 0): -1.0}, 2)
    assert abs(oracle.vol_relative(up, lo, 2) - (1.0 + 1.0 / 6.0 + 0.5)) < 1e-15


@pytest.mark.parametrize("n,deg,seed", [(1, 7, 0), (2, 6, 1), (3, 4, 2)])
def test_vol_relative_matches_quadrature(n, deg, seed):
    rng = np.random.default_rng(seed)
    terms_up, terms_lo = {}, {}
    for e in itertools.product(range(deg + 1), repeat=n):
        if sum(e) <= deg:
            terms_up[e] = float(rng.normal())
            terms_lo[e] = float(rng.normal())
    up = oracle.as_poly(terms_up, n)
    lo = oracle.as_poly(terms_lo, n)
    q = deg // 2 + 1  # exact for degree <= 2q - 1 >= deg per axis
    quad = _gauss_mean(lambda t: oracle.eval_poly(up, n, t) - oracle.eval_poly(lo, n, t), n, q)
    assert abs(oracle.vol_relative(up, lo, n) - quad) <= 1e-12 * (1 + abs(quad))


def test_vol_relative_of_propagated_bounds_matches_quadrature():
    """On real output polynomials (a two-input net, order 2, degree 4)."""
    from paper_2211_14438_gb300 import workloads as wl
    w = wl.single_box_2in()
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2)
    up, lo = r["upper"][0], r["lower"][0]
    quad = _gauss_mean(lambda t: oracle.eval_poly(up, 2, t) - oracle.eval_poly(lo, 2, t), 2, 8)
    v = oracle.vol_relative(up, lo, 2)
    assert v >= 0.0
    assert abs(v - quad) <= 1e-12 * (1 + abs(quad))
