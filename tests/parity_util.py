"""Shared helpers for the parity tests: dense <-> sparse polynomial
conversion over the library's graded order, and float64 evaluation."""
import numpy as np

import oracle
from paper_2211_14438_gb300 import bern

_ORDER_CACHE = {}


def graded(n, D):
    key = (n, D)
    if key not in _ORDER_CACHE:
        ex = bern.monomials(n, D)
        _ORDER_CACHE[key] = (ex, {tuple(int(v) for v in row): i for i, row in enumerate(ex)})
    return _ORDER_CACHE[key]


def dense_from_dict(d, n, M, D=None):
    """Oracle polynomial (dict or (exps, coef)) -> float64 vector over the
    first M graded monomials.  Raises if a term falls outside."""
    if not isinstance(d, dict):
        d = oracle.to_dict(d)
    if D is None:
        D = 0
        while bern.num_monomials(n, D) < M:
            D += 1
    _, rank = graded(n, D)
    v = np.zeros(M)
    for k, c in d.items():
        r = rank.get(tuple(k))
        if r is None or r >= M:
            if c != 0.0:
                raise KeyError("term %s outside the first %d monomials" % (k, M))
            continue
        v[r] += c
    return v


def dict_from_dense(v, n):
    M = len(v)
    D = 0
    while bern.num_monomials(n, D) < M:
        D += 1
    ex, _ = graded(n, D)
    return {tuple(int(x) for x in ex[r]): float(v[r]) for r in range(M)}


def eval_dense(v, n, t):
    """sum_r v[r] t^{e_r} in float64 at points t [P, n]."""
    M = len(v)
    D = 0
    while bern.num_monomials(n, D) < M:
        D += 1
    ex, _ = graded(n, D)
    ex = ex[:M].astype(np.int64)
    t = np.asarray(t, np.float64)
    out = np.zeros(len(t))
    # powers table per variable
    pw = [np.ones((len(t), int(ex[:, k].max()) + 1)) for k in range(n)]
    for k in range(n):
        for e in range(1, pw[k].shape[1]):
            pw[k][:, e] = pw[k][:, e - 1] * t[:, k]
    for r in range(M):
        if v[r] == 0.0:
            continue
        term = np.full(len(t), float(v[r]))
        for k in range(n):
            if ex[r, k]:
                term *= pw[k][:, ex[r, k]]
        out += term
    return out


def random_dense(rng, n, D, scale=1.0, zero_frac=0.0):
    M = bern.num_monomials(n, D)
    v = rng.normal(0, scale, size=M)
    if zero_frac:
        v[rng.random(M) < zero_frac] = 0.0
    return v.astype(np.float32)


def l1(v):
    return float(np.abs(np.asarray(v, np.float64)).sum())


def oracle_propagate_job(args):
    """One box through the oracle, as a process-pool job (the pool is started
    with 'spawn': a process forked after the GPU is in use can hang)."""
    widths, W, b, box, degree, kw = args
    return oracle.propagate(widths, W, b, box, degree, **kw)
