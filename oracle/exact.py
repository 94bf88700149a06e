"""Exact-rational BERN-NN propagation for tiny networks.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``).

Every input is a float32 value, hence a dyadic rational; every step of the
method uses only +, -, *, / and max, so with ``fractions.Fraction`` the whole
propagation is exact.  The FP64 oracle must agree with it to rounding level;
that pins the FP64 oracle's rounding (not its reading of the paper).

Steps follow the paper in order: input init (Sec. 5.3), layer step with W+/W-
(Sec. 5.2), Step 1 enclosure (eq. find_lo_hi via Def. 2), Step 2 ReLU
Bernstein polynomial (Def. 1, Prop. 1/2), Step 3 composition
(eqs. post_bounds_1/2).  Polynomials are dicts {exponent tuple: Fraction} in
t in [0,1]^n.  No truncation (the degree cap is never reached on the tiny
nets this serves) and no pruning.  With lin > 0, the Lin step of Sec. 5.3 in
the reading of the FP64 oracle (least-squares multilinear fit on the box,
Bernstein enclosure of the residual at the layer's order, outward shift) runs
after every lin-th hidden layer; the fit's normal equations are solved
exactly.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import product
from math import comb


def _mul(p, q):
    r = {}
    for ka, va in p.items():
        for kb, vb in q.items():
            k = tuple(x + y for x, y in zip(ka, kb))
            r[k] = r.get(k, Fraction(0)) + va * vb
    return r


def _bern_minmax(p, n, l):
    terms = list(p.items())
    vals = []
    for I in product(range(l + 1), repeat=n):
        b = Fraction(0)
        for J, a in terms:
            w = Fraction(1)
            for ik, jk in zip(I, J):
                if jk > ik:
                    w = Fraction(0)
                    break
                w *= Fraction(comb(ik, jk), comb(l, jk))
            b += w * a
        vals.append(b)
    return min(vals), max(vals)


def _relu_power(lo, hi, d):
    a = [Fraction(0)] * (d + 1)
    bks = []
    for k in range(d + 1):
        node = lo + (hi - lo) * k / d
        bk = node if node > 0 else Fraction(0)
        bks.append(bk)
        for m in range(d - k + 1):
            a[k + m] += bk * comb(d, k) * comb(d - k, m) * (-1) ** m
    s0 = -lo / (hi - lo)
    eps = sum(bks[k] * comb(d, k) * s0 ** k * (1 - s0) ** (d - k) for k in range(d + 1))
    return a, eps


def _linearize(P, n, order, upper):
    """Least-squares multilinear fit A of P on [0,1]^n (normal equations over
    the monomials t^S, S a set of at most min(n, deg P) variables, with the
    exact moments of t^K on the box), plus the residual's Bernstein max
    (upper) or min (lower) in the constant."""
    D = max(sum(k) for k in P)
    basis = [S for S in product((0, 1), repeat=n) if sum(S) <= min(n, D)]
    N = len(basis)

    def moment(K):
        r = Fraction(1)
        for k in K:
            r /= k + 1
        return r

    G = [[moment(tuple(x + y for x, y in zip(S, T))) for T in basis] for S in basis]
    rhs = [sum((c * moment(tuple(x + y for x, y in zip(K, S))) for K, c in P.items()),
               Fraction(0)) for S in basis]
    for col in range(N):                       # exact Gaussian elimination
        piv = next(r for r in range(col, N) if G[r][col] != 0)
        G[col], G[piv] = G[piv], G[col]
        rhs[col], rhs[piv] = rhs[piv], rhs[col]
        for r in range(col + 1, N):
            f = G[r][col] / G[col][col]
            if f:
                G[r] = [x - f * y for x, y in zip(G[r], G[col])]
                rhs[r] -= f * rhs[col]
    a = [Fraction(0)] * N
    for i in range(N - 1, -1, -1):
        a[i] = (rhs[i] - sum((G[i][j] * a[j] for j in range(i + 1, N)), Fraction(0))) / G[i][i]
    A = dict(zip(basis, a))
    R = dict(P)
    for k, v in A.items():
        R[k] = R.get(k, Fraction(0)) - v
    rmin, rmax = _bern_minmax(R, n, order)
    zero = tuple([0] * n)
    A[zero] += rmax if upper else rmin
    return A


def propagate(widths, W, b, box, degree, lin=0):
    n = widths[0]
    H = len(widths) - 1
    zero = tuple([0] * n)
    up = []
    for i in range(n):
        dl, dh = Fraction(float(box[i][0])), Fraction(float(box[i][1]))
        e = [0] * n
        e[i] = 1
        up.append({zero: dl, tuple(e): dh - dl})
    lo = [dict(p) for p in up]
    order = 1
    for layer in range(H):
        Wl = [[Fraction(float(x)) for x in row] for row in W[layer]]
        bl = [Fraction(float(x)) for x in b[layer]]
        pu, pl = [], []
        for m in range(len(bl)):
            a_up = {zero: bl[m]}
            a_lo = {zero: bl[m]}
            for j, w in enumerate(Wl[m]):
                wp = w if w > 0 else Fraction(0)
                wn = w if w < 0 else Fraction(0)
                for k, v in up[j].items():
                    a_up[k] = a_up.get(k, Fraction(0)) + wp * v
                    a_lo[k] = a_lo.get(k, Fraction(0)) + wn * v
                for k, v in lo[j].items():
                    a_up[k] = a_up.get(k, Fraction(0)) + wn * v
                    a_lo[k] = a_lo.get(k, Fraction(0)) + wp * v
            pu.append(a_up)
            pl.append(a_lo)
        if layer == H - 1:
            los = [_bern_minmax(p, n, order)[0] for p in pl]
            his = [_bern_minmax(p, n, order)[1] for p in pu]
            return {"lo": los, "hi": his, "upper": pu, "lower": pl}
        nu, nl = [], []
        for m in range(len(pu)):
            lom = _bern_minmax(pl[m], n, order)[0]
            him = _bern_minmax(pu[m], n, order)[1]
            if him <= 0:
                nu.append({zero: Fraction(0)})
                nl.append({zero: Fraction(0)})
            elif lom >= 0:
                nu.append(pu[m])
                nl.append(pl[m])
            else:
                a, eps = _relu_power(lom, him, degree)
                res = []
                for P in (pu[m], pl[m]):
                    s = {k: v / (him - lom) for k, v in P.items()}
                    s[zero] = s.get(zero, Fraction(0)) - lom / (him - lom)
                    q = {zero: a[degree]}
                    for j in range(degree - 1, -1, -1):
                        q = _mul(q, s)
                        q[zero] = q.get(zero, Fraction(0)) + a[j]
                    res.append(q)
                res[1][zero] = res[1].get(zero, Fraction(0)) - eps
                nu.append(res[0])
                nl.append(res[1])
        order = order * degree
        if lin > 0 and (layer + 1) % lin == 0:
            nu = [_linearize(P, n, order, True) for P in nu]
            nl = [_linearize(P, n, order, False) for P in nl]
            order = min(n, order)
        up, lo = nu, nl
