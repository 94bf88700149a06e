"""Pins for the FP64 oracle: each test checks it against something the paper or
plain mathematics fixes, never against a retyped copy of its own formulas.

A planted mistake anywhere in the oracle (dropped term, sign, index, operand
order) should fail at least one of these.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2211_14438_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def relu(y):
    return np.maximum(y, 0.0)


def random_poly(rng, n, deg, density=1.0, scale=1.0):
    terms = {}
    for e in itertools.product(range(deg + 1), repeat=n):
        if sum(e) <= deg and rng.random() < density:
            terms[e] = float(rng.normal(0, scale))
    if not terms:
        terms[(0,) * n] = 0.0
    return oracle.as_poly(terms, n)


# ------------------------------------------------------------------- Step 2

def test_table1_band_area():
    """Table 1: area between B_up and B_lo = B_up - B_up(0) on [-6,10] is
    (hi-lo) * B_up(0); the paper prints 37.5, 28.1, 16.9 for L=2,3,8."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table1_relu_band_area.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for lo, hi, d, area in rows:
        lo, hi, d, area = float(lo), float(hi), int(d), float(area)
        _, eps = oracle.relu_coeffs(lo, hi, d)
        # the band has constant height eps, so its area is eps*(hi-lo);
        # integrate numerically as well to tie the area to the two curves
        y = np.linspace(lo, hi, 20001)
        up = np.array([oracle.relu_bern_eval(lo, hi, d, v) for v in y])
        band = up - (up - oracle.relu_bern_eval(lo, hi, d, 0.0))
        num = np.trapezoid(band, y)
        assert abs(eps * (hi - lo) - area) <= 0.05 + 1e-12
        assert abs(num - area) <= 0.05 + 1e-9


@pytest.mark.parametrize("lo,hi", [(-6, 10), (-1, 1), (-0.3, 2.5), (-7.5, 0.2)])
@pytest.mark.parametrize("d", [1, 2, 3, 4, 8, 12, 16])
def test_prop1_prop2(lo, hi, d):
    """Prop. 1: B >= relu on [lo,hi]. Prop. 2: max(B - relu) = B(0), so
    B - B(0) <= relu."""
    y = np.linspace(lo, hi, 4001)
    y = np.union1d(y, [0.0])
    B = np.array([oracle.relu_bern_eval(lo, hi, d, v) for v in y])
    assert np.all(B >= relu(y) - 1e-12)
    err = B - relu(y)
    B0 = oracle.relu_bern_eval(lo, hi, d, 0.0)
    assert abs(err.max() - B0) <= 1e-12 * (1 + abs(B0))
    assert abs(y[np.argmax(err)]) <= (hi - lo) / 4000 + 1e-12
    assert np.all(B - B0 <= relu(y) + 1e-12)


def test_order1_is_chord():
    """With L=1 the Bernstein polynomial of ReLU is the chord (the linear
    convexification of Sec. 3.1)."""
    lo, hi = -2.0, 3.0
    for y in np.linspace(lo, hi, 11):
        assert oracle.relu_bern_eval(lo, hi, 1, y) == pytest.approx(hi * (y - lo) / (hi - lo), abs=1e-14)


@pytest.mark.parametrize("d", [1, 2, 3, 4, 6])
def test_power_form_matches_definition(d):
    """The power form a_j in s reproduces Def. 1: compare with numpy's
    interpolating polynomial through d+1 samples of Def. 1."""
    lo, hi = -1.7, 2.9
    a, eps = oracle.relu_coeffs(lo, hi, d)
    s = np.linspace(0, 1, d + 1)
    vals = [oracle.relu_bern_eval(lo, hi, d, lo + v * (hi - lo)) for v in s]
    fit = np.polynomial.polynomial.polyfit(s, vals, d)
    np.testing.assert_allclose(a, fit, rtol=1e-9, atol=1e-9)
    assert eps == pytest.approx(oracle.relu_bern_eval(lo, hi, d, 0.0), abs=1e-14)
    # a_0 = B(lo) = relu(lo) = 0 and sum a_j = B(hi) = hi (end-point interpolation)
    assert abs(a[0]) < 1e-14 and a.sum() == pytest.approx(hi, abs=1e-12)


@pytest.mark.parametrize("d", [8, 10, 13, 16])
def test_power_form_high_orders(d):
    """At orders up to 16 (Fig. 1's range) the power form in s still equals
    Def. 1 evaluated directly at random points (a Vandermonde fit is too
    ill-conditioned here), interpolates the end points, and its shift is
    B(0)."""
    lo, hi = -2.3, 3.1
    a, eps = oracle.relu_coeffs(lo, hi, d)
    rng = np.random.default_rng(d)
    for sv in np.r_[0.0, 1.0, rng.random(40)]:
        direct = oracle.relu_bern_eval(lo, hi, d, lo + sv * (hi - lo))
        power = sum(a[j] * sv ** j for j in range(d + 1))
        assert abs(power - direct) <= 1e-12 * (1 + np.abs(a).sum())
    assert abs(a[0]) < 1e-12 and a.sum() == pytest.approx(hi, abs=1e-10)
    assert eps == pytest.approx(oracle.relu_bern_eval(lo, hi, d, 0.0), abs=1e-14)


# ------------------------------------------------------------------- Step 1

def ber_basis(I, l, t):
    """Ber_{I,L}(t) on [0,1]^n: eq. bernpolcoeff with dlo=0, dhi=1."""
    v = 1.0
    for ik, tk in zip(I, t):
        v *= math.comb(l, ik) * tk ** ik * (1 - tk) ** (l - ik)
    return v


@pytest.mark.parametrize("n,deg,l", [(1, 4, 4), (1, 3, 6), (2, 4, 4), (2, 3, 5), (3, 2, 3)])
def test_bernstein_expansion_identity(n, deg, l):
    """The coefficients are those of the exact Bernstein expansion:
    sum_I b_I Ber_I(t) == p(t) at random points (Def. 1/2)."""
    rng = np.random.default_rng(10 * n + deg + l)
    p = random_poly(rng, n, deg)
    b = oracle.bernstein_coeffs(p, n, l)
    pts = rng.random((25, n))
    pv = oracle.eval_poly(p, n, pts)
    for t, v in zip(pts, pv):
        s = sum(b[I] * ber_basis(I, l, t) for I in itertools.product(range(l + 1), repeat=n))
        assert s == pytest.approx(v, abs=1e-11 * (1 + np.abs(p[1]).sum()))


@pytest.mark.parametrize("n,deg,l", [(2, 4, 4), (2, 4, 7), (3, 3, 3), (3, 2, 5)])
def test_bernstein_vertex_property(n, deg, l):
    """Coefficients at the corners of the grid equal p at the box corners."""
    rng = np.random.default_rng(n + 7 * deg + l)
    p = random_poly(rng, n, deg)
    b = oracle.bernstein_coeffs(p, n, l)
    for corner in itertools.product([0, 1], repeat=n):
        I = tuple(c * l for c in corner)
        v = oracle.eval_poly(p, n, np.array([corner], float))[0]
        assert b[I] == pytest.approx(v, abs=1e-12 * (1 + abs(v)))


@pytest.mark.parametrize("n,deg,l", [(1, 5, 7), (2, 4, 4), (2, 3, 6), (3, 3, 3), (3, 2, 5),
                                     (4, 2, 2), (5, 1, 2)])
def test_bernstein_factored_equals_definition(n, deg, l):
    """The factored transform (one triangular binomial transform per
    variable, used by the enclosure on large grids) gives Def. 2's
    coefficients computed term by term, and it satisfies the expansion
    identity and the vertex property itself."""
    rng = np.random.default_rng(500 + 10 * n + deg + l)
    p = random_poly(rng, n, deg)
    a = oracle.bernstein_coeffs(p, n, l)
    b = oracle.bernstein_coeffs_factored(p, n, l)
    sc = 1 + np.abs(p[1]).sum()
    assert np.max(np.abs(a - b)) <= 1e-12 * sc
    t = rng.random(n)
    s = sum(b[I] * ber_basis(I, l, t) for I in itertools.product(range(l + 1), repeat=n))
    assert s == pytest.approx(oracle.eval_poly(p, n, t[None])[0], abs=1e-11 * sc)
    for corner in itertools.product([0, 1], repeat=n):
        v = oracle.eval_poly(p, n, np.array([corner], float))[0]
        assert b[tuple(c * l for c in corner)] == pytest.approx(v, abs=1e-12 * (1 + abs(v)))


def test_enclosure_large_grid_uses_the_same_coefficients():
    """A six-variable degree-4 polynomial at order 5 (6^6 = 46,656 cells x 210
    terms, past the term-by-term threshold): the enclosure is the min/max of
    the factored coefficients, and it contains the polynomial on a grid."""
    rng = np.random.default_rng(77)
    p = random_poly(rng, 6, 4)
    mn, mx = oracle.enclosure(p, 6, 5)
    b = oracle.bernstein_coeffs_factored(p, 6, 5)
    assert mn == pytest.approx(b.min(), abs=1e-12) and mx == pytest.approx(b.max(), abs=1e-12)
    pts = rng.random((2000, 6))
    v = oracle.eval_poly(p, 6, pts)
    assert mn <= v.min() + 1e-12 and mx >= v.max() - 1e-12


@pytest.mark.parametrize("n,deg,grid", [(1, 6, 2001), (2, 4, 201), (2, 8, 201), (3, 4, 41)])
def test_enclosure_contains_dense_grid(n, deg, grid):
    """Def. 2: min b <= p(t) <= max b for every t; checked against a dense
    grid.  Also: elevating the order never loosens the enclosure."""
    rng = np.random.default_rng(100 + n + deg)
    p = random_poly(rng, n, deg)
    ax = np.linspace(0, 1, grid)
    pts = np.stack(np.meshgrid(*([ax] * n), indexing="ij"), -1).reshape(-1, n)
    v = oracle.eval_poly(p, n, pts)
    mn, mx = oracle.enclosure(p, n, deg)
    assert mn <= v.min() + 1e-12 and mx >= v.max() - 1e-12
    mn2, mx2 = oracle.enclosure(p, n, deg + 3)
    assert mn <= mn2 + 1e-12 and mx2 <= mx + 1e-12
    assert mn2 <= v.min() + 1e-12 and mx2 >= v.max() - 1e-12


def test_enclosure_linear_is_exact():
    """For an affine p = a0 + sum a_i t_i the enclosure is its exact range."""
    rng = np.random.default_rng(3)
    for n in (1, 2, 3, 5):
        a = rng.normal(size=n + 1)
        terms = {(0,) * n: a[0]}
        for i in range(n):
            e = [0] * n
            e[i] = 1
            terms[tuple(e)] = a[i + 1]
        mn, mx = oracle.enclosure(terms, n, 1)
        assert mn == pytest.approx(a[0] + np.minimum(a[1:], 0).sum(), abs=1e-14)
        assert mx == pytest.approx(a[0] + np.maximum(a[1:], 0).sum(), abs=1e-14)


def test_enclosure_budget_fallback_is_sound():
    """Budget rule R6: a smaller grid plus intervals for high-degree terms
    still encloses p (and is looser than the full grid)."""
    rng = np.random.default_rng(5)
    n, deg = 3, 6
    p = random_poly(rng, n, deg)
    ax = np.linspace(0, 1, 31)
    pts = np.stack(np.meshgrid(*([ax] * n), indexing="ij"), -1).reshape(-1, n)
    v = oracle.eval_poly(p, n, pts)
    full = oracle.enclosure(p, n, deg)
    for budget in (1, 8, 27, 64, 200):
        mn, mx = oracle.enclosure(p, n, deg, budget=budget)
        assert mn <= v.min() + 1e-12 and mx >= v.max() - 1e-12
        assert mn <= full[0] + 1e-12 and mx >= full[1] - 1e-12


# ------------------------------------------------------------------- Step 3

def test_poly_mul_brute_force():
    rng = np.random.default_rng(11)
    for n, da, db in ((1, 5, 3), (2, 4, 4), (3, 3, 2)):
        p = random_poly(rng, n, da)
        q = random_poly(rng, n, db)
        r = oracle.poly_mul(p, q, n)
        pts = rng.random((50, n))
        np.testing.assert_allclose(oracle.eval_poly(r, n, pts),
                                   oracle.eval_poly(p, n, pts) * oracle.eval_poly(q, n, pts),
                                   rtol=1e-12, atol=1e-12)
        assert len(r[1]) == len({tuple(x) for x in r[0]})


@pytest.mark.parametrize("d", [1, 2, 3, 4])
def test_compose_pointwise(d):
    """eqs. post_bounds_1/2 without truncation: the composed polynomial equals
    Def. 1's ReLU polynomial applied pointwise to P(t); the lower one is
    shifted by B(0)."""
    rng = np.random.default_rng(20 + d)
    n = 2
    P = random_poly(rng, n, 3)
    pts = rng.random((200, n))
    lo, hi = oracle.enclosure(P, n, 3)
    lo, hi = lo - 0.1, hi + 0.05
    if not (lo < 0 < hi):
        lo, hi = -abs(lo) - 0.1, abs(hi) + 0.1
    Pv = oracle.eval_poly(P, n, pts)
    want = np.array([oracle.relu_bern_eval(lo, hi, d, y) for y in Pv])
    B0 = oracle.relu_bern_eval(lo, hi, d, 0.0)
    up = oracle.compose(P, n, lo, hi, d, True, cap=64)
    lw = oracle.compose(P, n, lo, hi, d, False, cap=64)
    np.testing.assert_allclose(oracle.eval_poly(up, n, pts), want, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(oracle.eval_poly(lw, n, pts), want - B0, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("d", [6, 8, 12, 16])
def test_compose_pointwise_high_orders(d):
    """The same identity at the high orders of Fig. 1's range (the orders the
    float64 Horner composition serves): composed polynomial == Def. 1's ReLU
    polynomial applied to P(t), the lower one shifted by B(0).  The power
    form's coefficients grow like C(d, d/2) 2^(d/2), so the tolerance scales
    with the composed polynomial's coefficient mass."""
    rng = np.random.default_rng(40 + d)
    n = 2
    P = random_poly(rng, n, 2)
    pts = np.vstack([rng.random((150, n)), [[0, 0], [0, 1], [1, 0], [1, 1]]])
    lo, hi = oracle.enclosure(P, n, 2)
    lo, hi = lo - 0.05, hi + 0.05
    if not (lo < 0 < hi):
        lo, hi = -abs(lo) - 0.1, abs(hi) + 0.1
    Pv = oracle.eval_poly(P, n, pts)
    want = np.array([oracle.relu_bern_eval(lo, hi, d, y) for y in Pv])
    B0 = oracle.relu_bern_eval(lo, hi, d, 0.0)
    up = oracle.compose(P, n, lo, hi, d, True, cap=64)
    lw = oracle.compose(P, n, lo, hi, d, False, cap=64)
    assert max(sum(e) for e in up[0]) <= 2 * d          # no term was truncated
    tol = 1e-12 * (1 + np.abs(up[1]).sum())
    assert np.max(np.abs(oracle.eval_poly(up, n, pts) - want)) <= tol
    assert np.max(np.abs(oracle.eval_poly(lw, n, pts) - (want - B0))) <= tol


@pytest.mark.parametrize("cap,tau", [(3, 0.0), (4, 0.0), (6, 1e-2), (64, 5e-2)])
def test_compose_truncation_sound(cap, tau):
    """Cap truncation and pruning (R4/R5) keep upper >= B(P) >= ... >= lower."""
    rng = np.random.default_rng(cap)
    n, d = 2, 3
    P = random_poly(rng, n, 3)
    lo, hi = oracle.enclosure(P, n, 3)
    pts = rng.random((400, n))
    # at the corner t = (1,..,1) every monomial is 1, so the dropped terms'
    # remainder is attained there: a lost remainder shows up at that point
    pts[:4] = np.array(list(itertools.product([0.0, 1.0], repeat=n)))
    Pv = oracle.eval_poly(P, n, pts)
    exact_up = np.array([oracle.relu_bern_eval(lo, hi, d, y) for y in Pv])
    B0 = oracle.relu_bern_eval(lo, hi, d, 0.0)
    up = oracle.compose(P, n, lo, hi, d, True, cap=cap, tau=tau)
    lw = oracle.compose(P, n, lo, hi, d, False, cap=cap, tau=tau)
    assert max(sum(e) for e in up[0]) <= cap
    assert np.all(oracle.eval_poly(up, n, pts) >= exact_up - 1e-10)
    assert np.all(oracle.eval_poly(lw, n, pts) <= exact_up - B0 + 1e-10)


def test_compose_remainder_hand_example():
    """Hand-worked truncation (R4): P = 2t-1 on [lo,hi] = [-1,1] gives s = t;
    order 4 nodes relu(-1+k/2) = (0,0,0,1/2,1) give B(s) = 2s^3 - s^4 and
    B(1/2) = 3/16.  With cap 1 Horner drops -s^2 (upper remainder 0, lower
    -1) and then 2s^2 (upper +2); the remainders carry through the last
    product by s in [0,1].  So upper = 2 and lower = -1 - 3/16 exactly."""
    P = {(0,): -1.0, (1,): 2.0}
    a, eps = oracle.relu_coeffs(-1.0, 1.0, 4)
    np.testing.assert_allclose(a, [0, 0, 0, 2, -1], atol=1e-15)
    assert eps == pytest.approx(3 / 16, abs=1e-15)
    up = oracle.to_dict(oracle.compose(P, 1, -1.0, 1.0, 4, True, cap=1))
    lw = oracle.to_dict(oracle.compose(P, 1, -1.0, 1.0, 4, False, cap=1))
    assert up[(0,)] == pytest.approx(2.0, abs=1e-15) and abs(up.get((1,), 0.0)) < 1e-15
    assert lw[(0,)] == pytest.approx(-1.0 - 3 / 16, abs=1e-15)
    assert abs(lw.get((1,), 0.0)) < 1e-15


# ---------------------------------------------------------------- whole path

def _mc_points(rng, box, count):
    lo, hi = box[:, 0].astype(np.float64), box[:, 1].astype(np.float64)
    n = len(lo)
    t = rng.random((count, n))
    corners = np.array(list(itertools.product([0.0, 1.0], repeat=n)))
    t[: len(corners)] = corners          # the box corners are always sampled
    return t, lo + t * (hi - lo)


def test_single_box_2in_monte_carlo_soundness():
    """Problem 1 on the [2,20,20,1] net over [-1,1]^2: zero violations over 10^6 sampled inputs, and the
    enclosure lo <= NN <= hi."""
    w = wl.single_box_2in()
    box = w.boxes[0]
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, box, 2)
    rng = np.random.default_rng(0)
    t, x = _mc_points(rng, box, 1_000_000)
    nn = oracle.network_forward(w.net.widths, w.net.W, w.net.b, x)[:, 0]
    up = oracle.eval_poly(r["upper"][0], 2, t)
    lw = oracle.eval_poly(r["lower"][0], 2, t)
    e = 1e-12 * (1 + np.abs(r["upper"][0][1]).sum() + np.abs(nn))
    assert np.sum(nn > up + e) == 0
    assert np.sum(nn < lw - e) == 0
    assert np.all(nn <= r["hi"][0] + 1e-12) and np.all(nn >= r["lo"][0] - 1e-12)


def test_exact_rational_agrees_with_fp64():
    """Config 1 in exact rationals vs the FP64 oracle."""
    w = wl.single_box_2in()
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2)
    q = exact.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2)
    assert float(q["lo"][0]) == pytest.approx(r["lo"][0], rel=1e-11, abs=1e-11)
    assert float(q["hi"][0]) == pytest.approx(r["hi"][0], rel=1e-11, abs=1e-11)
    for name in ("upper", "lower"):
        d = oracle.to_dict(r[name][0])
        qe = q[name][0]
        assert set(d) == set(qe)
        for k in d:
            assert d[k] == pytest.approx(float(qe[k]), rel=1e-10, abs=1e-11)


def test_point_box_reproduces_network():
    """A degenerate box (a point): every polynomial is a constant equal to the
    network's value (stable neurons only; exact affine steps)."""
    w = wl.single_box_4in()
    rng = np.random.default_rng(4)
    for _ in range(3):
        x = rng.uniform(-0.5, 0.5, size=4).astype(np.float32)
        box = np.stack([x, x], -1)
        r = oracle.propagate(w.net.widths, w.net.W, w.net.b, box, 2)
        nn = oracle.network_forward(w.net.widths, w.net.W, w.net.b, x[None].astype(np.float64))[0]
        np.testing.assert_allclose(r["lo"], nn, rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(r["hi"], nn, rtol=1e-12, atol=1e-12)
        assert np.all(r["tr_case"] != 2)


def test_all_active_gives_exact_affine_map():
    """Large positive biases make every hidden neuron active: both output
    polynomials equal W2(W1 x + b1) + b2 exactly (as polynomials in t)."""
    rng = np.random.default_rng(8)
    W1 = rng.normal(size=(5, 2)).astype(np.float32)
    b1 = np.full(5, 50.0, np.float32)
    W2 = rng.normal(size=(1, 5)).astype(np.float32)
    b2 = np.array([0.25], np.float32)
    box = np.array([[-1.0, 1.0], [0.0, 2.0]], np.float32)
    r = oracle.propagate([2, 5, 1], [W1, W2], [b1, b2], box, 2)
    assert np.all(r["tr_case"] == 1)
    lo, wd = box[:, 0].astype(float), (box[:, 1] - box[:, 0]).astype(float)
    A = W2.astype(float) @ W1.astype(float)
    c0 = float((W2.astype(float) @ (W1.astype(float) @ lo + b1) + b2)[0])
    want = {(0, 0): c0, (1, 0): A[0, 0] * wd[0], (0, 1): A[0, 1] * wd[1]}
    for name in ("upper", "lower"):
        got = oracle.to_dict(r[name][0])
        for k, v in want.items():
            assert got[k] == pytest.approx(v, rel=1e-12, abs=1e-12)


def test_all_dead_gives_output_bias():
    rng = np.random.default_rng(9)
    W1 = rng.normal(size=(4, 3)).astype(np.float32)
    b1 = np.full(4, -50.0, np.float32)
    W2 = rng.normal(size=(2, 4)).astype(np.float32)
    b2 = np.array([0.5, -1.25], np.float32)
    box = np.array([[-1, 1]] * 3, np.float32)
    r = oracle.propagate([3, 4, 2], [W1, W2], [b1, b2], box, 3)
    assert np.all(r["tr_case"] == 0)
    np.testing.assert_allclose(r["lo"], b2, atol=0)
    np.testing.assert_allclose(r["hi"], b2, atol=0)


def test_order1_single_hidden_layer_hand_derived():
    """L=1, one hidden layer: per unstable neuron the upper is the chord
    hi(y-lo)/(hi-lo) and the lower the parallel line hi*y/(hi-lo) (Sec. 3.1,
    linear convexification); derived here by hand from interval bounds of the
    affine pre-activations."""
    rng = np.random.default_rng(12)
    n, h = 3, 7
    W1 = rng.normal(size=(h, n)).astype(np.float32)
    b1 = rng.normal(scale=0.3, size=h).astype(np.float32)
    W2 = rng.normal(size=(1, h)).astype(np.float32)
    b2 = np.array([0.1], np.float32)
    box = np.array([[-1, 0.5], [-0.25, 1.0], [0.0, 0.75]], np.float32)
    r = oracle.propagate([n, h, 1], [W1, W2], [b1, b2], box, 1)
    dl, wd = box[:, 0].astype(float), (box[:, 1] - box[:, 0]).astype(float)
    # pre-activation z_m(t) = c_m + sum_i g_mi t_i
    c = W1.astype(float) @ dl + b1
    g = W1.astype(float) * wd[None, :]
    lo = c + np.minimum(g, 0).sum(1)
    hi = c + np.maximum(g, 0).sum(1)
    up_c, up_g = np.zeros(h), np.zeros((h, n))
    lw_c, lw_g = np.zeros(h), np.zeros((h, n))
    for m in range(h):
        if hi[m] <= 0:
            continue
        if lo[m] >= 0:
            up_c[m], up_g[m], lw_c[m], lw_g[m] = c[m], g[m], c[m], g[m]
            continue
        k = hi[m] / (hi[m] - lo[m])
        up_c[m], up_g[m] = k * (c[m] - lo[m]), k * g[m]
        lw_c[m], lw_g[m] = k * c[m], k * g[m]
    w2 = W2[0].astype(float)
    wp, wn = np.maximum(w2, 0), np.minimum(w2, 0)
    U_c = wp @ up_c + wn @ lw_c + b2[0]
    U_g = wp @ up_g + wn @ lw_g
    L_c = wp @ lw_c + wn @ up_c + b2[0]
    L_g = wp @ lw_g + wn @ up_g
    np.testing.assert_allclose(r["tr_lo"], lo, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r["tr_hi"], hi, rtol=1e-12, atol=1e-12)
    for name, cc, gg in (("upper", U_c, U_g), ("lower", L_c, L_g)):
        got = oracle.to_dict(r[name][0])
        assert got.get((0, 0, 0), 0.0) == pytest.approx(cc, rel=1e-12, abs=1e-12)
        for i in range(n):
            e = [0] * n
            e[i] = 1
            assert got.get(tuple(e), 0.0) == pytest.approx(gg[i], rel=1e-12, abs=1e-12)
        assert all(sum(k) <= 1 for k in got)


def test_tightness_improves_with_order():
    """Fig. 4 trend: Vol_relative falls as the ReLU order L grows (median over
    seeded nets of the paper's [2,20,20,1] family, box [-1,1]^2)."""
    vols = {d: [] for d in (2, 3, 4)}
    for seed in range(5):
        net = wl.paper_net(2, [20, 20], seed=100 + seed)
        box = np.array([[-1, 1], [-1, 1]], np.float32)
        for d in vols:
            r = oracle.propagate(net.widths, net.W, net.b, box, d, cap=16)
            vols[d].append(oracle.vol_relative(r["upper"][0], r["lower"][0], 2))
    med = {d: float(np.median(v)) for d, v in vols.items()}
    assert med[2] > med[3] > med[4] > 0


def test_propagate_rejects_bad_input():
    w = wl.single_box_2in()
    bad = np.array([[1.0, -1.0], [0, 1]], np.float32)
    with pytest.raises(ValueError):
        oracle.propagate(w.net.widths, w.net.W, w.net.b, bad, 2)
