"""Pins of the oracle's change of variables t -> x (CPU, no GPU): a
hand-expanded example, the identity map of one coordinate, a point-box side,
and P(t(x)) evaluated directly at random points of random boxes."""
import numpy as np
import pytest

from oracle import poly_x


def nz(p):
    """The terms with a nonzero coefficient."""
    return {K: v for K, v in p.items() if v != 0.0}


def test_hand_expanded_square():
    # t = (x - 1) / 2:  t^2 = (x^2 - 2x + 1) / 4
    e = poly_x.poly_to_x({(2,): 1.0}, [1.0], [2.0])
    assert e == {(0,): 0.25, (1,): -0.5, (2,): 0.25}


def test_hand_expanded_two_variables():
    # t1 t2 + 3 with t1 = (x1 + 1) / 2, t2 = x2 / 4:
    # (x1 x2 + x2) / 8 + 3
    e = poly_x.poly_to_x({(1, 1): 1.0, (0, 0): 3.0}, [-1.0, 0.0], [2.0, 4.0])
    assert nz(e) == pytest.approx({(1, 1): 0.125, (0, 1): 0.125, (0, 0): 3.0})


def test_identity_coordinate():
    e = poly_x.poly_to_x({(0, 1, 0): 1.0}, [0.5, -2.0, 3.0], [1.0, 4.0, 0.5])
    assert nz(e) == pytest.approx({(0, 1, 0): 0.25, (0, 0, 0): 0.5})


def test_point_side_keeps_only_its_constant_terms():
    # w_2 = 0: x_2 is fixed and t_2 = 0, so every term with k_2 > 0 vanishes
    e = poly_x.poly_to_x({(1, 0): 2.0, (0, 1): 5.0, (1, 1): 7.0}, [0.0, 1.0], [1.0, 0.0])
    assert nz(e) == pytest.approx({(1, 0): 2.0})


@pytest.mark.parametrize("n,D,seed", [(1, 6, 0), (2, 5, 1), (3, 4, 2), (4, 3, 3)])
def test_matches_direct_evaluation(n, D, seed):
    rng = np.random.default_rng(seed)
    exps = [K for K in np.ndindex(*([D + 1] * n)) if sum(K) <= D]
    p = {tuple(int(k) for k in K): float(rng.normal()) for K in exps}
    dlo = rng.uniform(-2, 1, n)
    w = rng.uniform(0.1, 3, n)
    e = poly_x.poly_to_x(p, dlo, w)
    x = dlo + w * rng.random((200, n))
    t = (x - dlo) / w
    direct = np.zeros(len(x))
    for K, c in p.items():
        direct += c * np.prod(t ** np.asarray(K, np.float64), axis=1)
    mag = sum(abs(c) for c in p.values())
    assert np.max(np.abs(poly_x.eval_x(e, x) - direct)) <= 1e-11 * (1 + mag) * (1 + np.abs(dlo).max()) ** D
