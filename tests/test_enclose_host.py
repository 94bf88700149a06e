"""CPU replay of the shared-memory enclosure's pass structure (Sec. 5.1 Step
1 with Def. 2) on the library's own line table, against the oracle's
enclosure.

The replay follows the warp kernel's reading of the table: the scaled
coefficients of the graded prefix up to the item's degree are scattered into
a grid that is NOT zero-filled (here: NaN, so a read of a cell no step wrote
fails), the passes run from the last variable to the first over the lines
whose prefix digit sum is within the degree (from four variables on, only the
first C(l+k, k) (l+1)^(n-1-k) lines of pass k), a line's inputs past
degree - prefix sum are taken as zero, and terms above the grid order go to
the one-sided remainder.  Float64, no directed rounding: the check is of the
tables and the loop structure, the kernels' rounding is checked on the GPU."""
import math

import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import bern


def replay(coef, n, l):
    """(min, max) bound of the polynomial with graded coefficients coef
    (any length) on the order-l grid, the way the warp kernel computes it."""
    nt = len(coef)
    R = l + 1
    D = 0
    while bern.num_monomials(n, D) < nt:      # degree of the graded prefix
        D += 1
    Deff = min(D, l)
    m_eff = bern.num_monomials(n, Deff)
    ex = bern.monomials(n, max(D, l)).astype(int)
    grid = np.full(R ** n, np.nan)
    stride = [R ** (n - 1 - k) for k in range(n)]
    rem_lo = rem_hi = 0.0
    for r in range(max(nt, m_eff)):
        a = float(coef[r]) if r < nt else 0.0          # a ragged prefix: missing terms are 0
        if r < m_eff:
            g = sum(int(e) * stride[k] for k, e in enumerate(ex[r]))
            grid[g] = a / math.prod(math.comb(l, int(e)) for e in ex[r])
        else:                                          # above the grid order: [min(0,a), max(0,a)]
            rem_lo += min(a, 0.0)
            rem_hi += max(a, 0.0)
    lines = bern.enclose_lines(n, l)
    lo, hi = math.inf, -math.inf
    for k in range(n - 1, -1, -1):
        sk = stride[k]
        nl = math.comb(l + k, k) * R ** (n - 1 - k) if n >= 4 else R ** (n - 1)
        for base, psum in lines[k, :nl].tolist():
            if psum > Deff:
                continue
            p = Deff - psum
            x = [grid[base + j * sk] if j <= p else 0.0 for j in range(R)]
            assert not any(math.isnan(v) for v in x), "read of a cell no step wrote"
            y = [sum(math.comb(i, j) * x[j] for j in range(i + 1)) for i in range(R)]
            if k > 0:
                for i in range(R):
                    grid[base + i * sk] = y[i]
            else:
                lo, hi = min(lo, min(y)), max(hi, max(y))
    return lo + rem_lo, hi + rem_hi


CASES = [
    # (n, grid order l, polynomial degree D, ragged)
    (1, 6, 6, False), (2, 4, 4, False), (2, 5, 3, False), (3, 8, 8, False), (3, 8, 5, False),
    (3, 4, 4, True), (3, 3, 5, False), (4, 4, 4, False), (4, 6, 3, True), (5, 3, 3, False),
    (6, 2, 2, False), (6, 3, 3, False), (6, 3, 2, True), (4, 2, 4, False),
]


@pytest.mark.parametrize("n,l,D,ragged", CASES)
def test_replay_matches_the_oracle(n, l, D, ragged):
    rng = np.random.default_rng(1000 * n + 10 * l + D)
    M = bern.num_monomials(n, D)
    nt = int(rng.integers(bern.num_monomials(n, D - 1) + 1, M)) if ragged and D > 0 else M
    coef = rng.normal(size=nt)
    ex = bern.monomials(n, D)[:nt]
    if D > l:   # the oracle's budget rule lowers the order to l (R6)
        o_lo, o_hi = oracle.enclosure((ex, coef), n, D, (l + 1) ** n)
    else:
        o_lo, o_hi = oracle.enclosure((ex, coef), n, l)
    r_lo, r_hi = replay(coef, n, l)
    sc = 1.0 + float(np.abs(coef).sum())
    assert abs(r_lo - o_lo) <= 1e-12 * sc and abs(r_hi - o_hi) <= 1e-12 * sc


def test_replay_with_the_loop_over_every_line_is_the_same():
    # from four variables on, lines past the in-simplex prefix are never
    # needed: a replay over all lines of each pass gives the same bounds
    n, l = 4, 4
    rng = np.random.default_rng(5)
    coef = rng.normal(size=bern.num_monomials(n, l))
    full = bern.enclose_lines(n, l)
    part = replay(coef, n, l)
    # the full loop, written out: same steps without the prefix bound
    R = l + 1
    ex = bern.monomials(n, l).astype(int)
    stride = [R ** (n - 1 - k) for k in range(n)]
    grid = np.full(R ** n, np.nan)
    for r, e in enumerate(ex):
        grid[sum(int(v) * stride[k] for k, v in enumerate(e))] = \
            coef[r] / math.prod(math.comb(l, int(v)) for v in e)
    lo, hi = math.inf, -math.inf
    for k in range(n - 1, -1, -1):
        for base, psum in full[k].tolist():
            if psum > l:
                continue
            x = [grid[base + j * stride[k]] if j <= l - psum else 0.0 for j in range(R)]
            y = [sum(math.comb(i, j) * x[j] for j in range(i + 1)) for i in range(R)]
            if k > 0:
                for i in range(R):
                    grid[base + i * stride[k]] = y[i]
            else:
                lo, hi = min(lo, min(y)), max(hi, max(y))
    assert part == pytest.approx((lo, hi), rel=1e-14, abs=1e-14)
