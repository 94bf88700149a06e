"""FP64 oracle of the change of variables from the normalised box coordinates
t in [0,1]^n back to the input coordinates x (Sec. 5.3: the inputs enter the
network as x_i = dlo_i + w_i t_i on the box).

TEST INFRASTRUCTURE ONLY: imported by ``tests/`` alone; the library has its
own kernel and never loads this module.

For P(t) = sum_K c_K t^K and t_i = (x_i - dlo_i) / w_i the binomial theorem
gives, term by term,

    prod_i ((x_i - dlo_i) / w_i)^{k_i}
        = prod_i sum_{j_i <= k_i} C(k_i, j_i) x_i^{j_i} (-dlo_i)^{k_i - j_i} / w_i^{k_i},

so the coefficient of x^J collects c_K prod_i C(k_i, j_i) (-dlo_i)^{k_i-j_i}
w_i^{-k_i} over every K >= J.  This module expands exactly that, one term of
P at a time, in float64 (binomials from ``math.comb``).  A variable with
w_i = 0 (a point box side) is fixed at x_i = dlo_i, which is t_i = 0: only
the terms with k_i = 0 survive.  Parity: pinned by ``tests/test_oracle_poly_x.py``
(a hand-expanded example, the identity map, and P(t(x)) evaluated directly at
random points)."""
from __future__ import annotations

import itertools
import math
from typing import Dict, Sequence, Tuple

import numpy as np

Poly = Dict[Tuple[int, ...], float]


def poly_to_x(p: Poly, dlo: Sequence[float], w: Sequence[float], magnitudes: bool = False):
    """P(t) as a polynomial in x, with t_i = (x_i - dlo_i) / w_i.  With
    ``magnitudes`` also the sum of the absolute values of the terms that make
    up each coefficient (the scale of its cancellation)."""
    n = len(dlo)
    out: Poly = {}
    mag: Poly = {}
    for K, c in p.items():
        if c == 0.0:
            continue
        # per variable: the coefficients of x_i^j in ((x_i - dlo_i) / w_i)^{k_i}
        factors = []
        for i in range(n):
            k = K[i]
            if w[i] == 0.0:
                factors.append([(0, 1.0)] if k == 0 else [])
                continue
            factors.append([(j, math.comb(k, j) * (-float(dlo[i])) ** (k - j) / float(w[i]) ** k)
                            for j in range(k + 1)])
        for combo in itertools.product(*factors):
            J = tuple(j for j, _ in combo)
            v = c
            for _, f in combo:
                v *= f
            out[J] = out.get(J, 0.0) + v
            mag[J] = mag.get(J, 0.0) + abs(v)
    return (out, mag) if magnitudes else out


def eval_x(p: Poly, x: np.ndarray) -> np.ndarray:
    """sum_J e_J x^J at the rows of x ([m, n])."""
    x = np.atleast_2d(np.asarray(x, np.float64))
    v = np.zeros(x.shape[0])
    for J, e in p.items():
        v += e * np.prod(x ** np.asarray(J, np.float64), axis=1)
    return v
