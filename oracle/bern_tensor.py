"""The paper's own representation, for comparison: Bernstein polynomials as
dense n-dimensional coefficient tensors (Sec. 4.1) with the tensor arithmetic
of Sec. 4: Prod_Bern (Sec. 4.2: scale by the binomial tensors, multiply as
power series, unscale), Pow_Bern (repeated Prod_Bern), degree elevation and
Sum_Bern (Sec. 4.3), and the whole BERN-NN loop of Sec. 5 on these tensors
(FP64, plain numpy; small networks only: the tensors are dense).

TEST INFRASTRUCTURE ONLY (see the package docstring).  It shares nothing with
the power-basis oracle in bern_oracle.cpp; the tests use it to show that the
two representations give the same bounds and polynomials.

A tensor T of shape (l_1+1, ..., l_n+1) is the polynomial
sum_K T[K] prod_i C(l_i, k_i) t_i^k_i (1 - t_i)^(l_i - k_i) of t in [0,1]^n,
t_i = (x_i - dlo_i)/(dhi_i - dlo_i): the Bernstein basis on the box.
"""
from __future__ import annotations

from math import comb
from typing import List, Sequence

import numpy as np
from scipy import signal


def binom_tensor(shape) -> np.ndarray:
    """C_L: the tensor whose K-th entry is prod_i C(l_i, k_i), L = shape - 1."""
    out = np.ones(shape)
    for i, s in enumerate(shape):
        v = np.array([comb(s - 1, k) for k in range(s)], dtype=np.float64)
        out = out * v.reshape([-1 if j == i else 1 for j in range(len(shape))])
    return out


def power_prod(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Prod: the product of two power-series tensors (exponents add), i.e. the
    full n-dimensional convolution of the coefficient arrays."""
    return signal.convolve(a, b, mode="full", method="direct")


def prod_bern(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Prod_Bern (Sec. 4.2): the Bernstein tensor of the product, of order
    L1 + L2: unscale(Prod(a * C_L1, b * C_L2))."""
    p = power_prod(a * binom_tensor(a.shape), b * binom_tensor(b.shape))
    return p / binom_tensor(p.shape)


def pow_bern(a: np.ndarray, i: int) -> np.ndarray:
    """Pow_Bern: the Bernstein tensor of g^i by i - 1 applications of
    Prod_Bern (the order-0 tensor 1 for i = 0)."""
    out = np.ones([1] * a.ndim)
    for _ in range(i):
        out = prod_bern(out, a)
    return out


def elevate(a: np.ndarray, shape) -> np.ndarray:
    """Degree elevation (Sec. 4.3): Prod_Bern with the all-ones tensor of
    shape L_e - L + 1, which represents the constant 1 at order L_e - L."""
    ones = np.ones([s - t + 1 for s, t in zip(shape, a.shape)])
    return prod_bern(a, ones)


def sum_bern(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Sum_Bern (Sec. 4.3): elevate both to the element-wise larger order,
    then add element-wise."""
    shape = [max(x, y) for x, y in zip(a.shape, b.shape)]
    return elevate(a, shape) + elevate(b, shape)


def evaluate(a: np.ndarray, t: np.ndarray) -> np.ndarray:
    """The polynomial of tensor a at points t [P, n] (Def. 1's basis)."""
    t = np.asarray(t, np.float64).reshape(-1, a.ndim)
    out = np.empty(len(t))
    for p, pt in enumerate(t):
        v = a
        for i in range(a.ndim):
            l = a.shape[i] - 1
            basis = np.array([comb(l, k) * pt[i] ** k * (1 - pt[i]) ** (l - k)
                              for k in range(l + 1)])
            v = np.tensordot(basis, v, axes=(0, 0))
        out[p] = float(v)
    return out


def propagate(widths: Sequence[int], W, b, box, d: int):
    """BERN-NN on Bernstein tensors for one box with ReLU order d everywhere
    (Secs. 5.1-5.3): input init (Sec. 5.3), the layer step (Sec. 5.2) with
    Sum_Bern, Step 1 as the min / max tensor entry (Def. 2), Step 2's order-d
    Bernstein polynomial of ReLU composed in Bernstein form as
    sum_k relu(node_k) C(d,k) s^k (1-s)^(d-k) with Pow_Bern / Prod_Bern
    (Def. 1, s = (P - lo)/(hi - lo), 1 - s = (hi - P)/(hi - lo)), the lower
    bound shifted by its value at 0 (Prop. 2), stable neurons as in the
    power-basis oracle (hi <= 0: 0, lo >= 0: identity).  As in Sec. 5.4
    every neuron of a layer is elevated to the layer's order L * d, so the
    enclosure orders follow L_z = L_zhat * d.  Returns 'lo', 'hi' (o,) and
    'upper' / 'lower' (lists of output tensors)."""
    widths = [int(x) for x in widths]
    n, H = widths[0], len(widths) - 1
    box = np.asarray(box, np.float64).reshape(n, 2)
    up: List[np.ndarray] = []
    for i in range(n):
        shape = [1] * n
        shape[i] = 2
        up.append(np.array([box[i, 0], box[i, 1]]).reshape(shape))
    lo = list(up)
    for layer in range(H):
        Wl = np.asarray(W[layer], np.float64)
        bl = np.asarray(b[layer], np.float64)
        shape = [max(t.shape[i] for t in up + lo) for i in range(n)]
        eu = [elevate(t, shape) for t in up]
        el = [elevate(t, shape) for t in lo]
        pu, pl = [], []
        for m in range(Wl.shape[0]):
            su = np.full(shape, bl[m])
            sl = np.full(shape, bl[m])
            for j in range(Wl.shape[1]):
                w = Wl[m, j]
                if w > 0:
                    su = su + w * eu[j]
                    sl = sl + w * el[j]
                elif w < 0:
                    su = su + w * el[j]
                    sl = sl + w * eu[j]
            pu.append(su)
            pl.append(sl)
        if layer == H - 1:
            return {"lo": np.array([t.min() for t in pl]), "hi": np.array([t.max() for t in pu]),
                    "upper": pu, "lower": pl}
        post_shape = [(s - 1) * d + 1 for s in shape]
        up, lo = [], []
        for tu, tl in zip(pu, pl):
            l_, h_ = float(tl.min()), float(tu.max())
            if h_ <= 0.0:
                nu = np.zeros([1] * n)
                nl = np.zeros([1] * n)
            elif l_ >= 0.0:
                nu, nl = tu, tl
            else:
                nodes = [max(0.0, l_ + k * (h_ - l_) / d) for k in range(d + 1)]
                s0 = -l_ / (h_ - l_)
                eps = sum(nodes[k] * comb(d, k) * s0 ** k * (1 - s0) ** (d - k)
                          for k in range(d + 1))
                res = []
                for t in (tu, tl):
                    s = (t - l_) / (h_ - l_)
                    r = (h_ - t) / (h_ - l_)
                    acc = np.zeros([1] * n)
                    for k in range(d + 1):
                        if nodes[k] != 0.0:
                            term = prod_bern(pow_bern(s, k), pow_bern(r, d - k))
                            acc = sum_bern(acc, nodes[k] * comb(d, k) * term)
                    res.append(acc)
                nu, nl = res[0], res[1] - eps
            up.append(elevate(nu, post_shape))
            lo.append(elevate(nl, post_shape))
    raise AssertionError("unreachable")
