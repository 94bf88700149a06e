"""FP64 CPU oracle for BERN-NN bound propagation (arxiv 2211.14438).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product library
never loads it and has no fallback to it.

The arithmetic lives in ``bern_oracle.cpp`` (plain C++, std::map polynomials,
every step written from the paper's definitions: Def. 1/2, Props. 1/2, the
Step 1-3 neuron pass of Sec. 5.1 and the layer step of Sec. 5.2).  This module
compiles it with g++ and wraps it with ctypes.

Parity status per function: all pinned by ``tests/test_oracle_pins.py``
(closed forms, Table 1, vertex/basis identities of the Bernstein expansion,
dense-grid min/max, brute-force products, exact-network special cases and
Monte-Carlo soundness), ``tests/test_oracle_helpers.py`` (evaluation helpers)
``tests/test_oracle_lin.py`` (the Lin step: hand-worked fits, numerical
least squares, soundness) and ``tests/test_oracle_bern_tensor.py`` (the
paper's dense Bernstein-tensor arithmetic in ``bern_tensor.py``, against the
definition and against the power basis), except the tightness of whole-network bounds, which
is "parity unpinned": the paper's volumes come from unseeded networks.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig
from typing import Dict, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bern_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libbern_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, -O2, no OpenMP)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    u8 = ctypes.POINTER(ctypes.c_uint8)
    lib.orc_binom.restype = ctypes.c_double
    lib.orc_binom.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.orc_relu_bern_eval.restype = ctypes.c_double
    lib.orc_relu_bern_eval.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_double]
    lib.orc_relu_coeffs.restype = None
    lib.orc_relu_coeffs.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp, dp]
    lib.orc_bernstein_coeffs.restype = ctypes.c_int
    lib.orc_bernstein_coeffs.argtypes = [ctypes.c_int, ctypes.c_int, u8, dp, ctypes.c_int, dp]
    lib.orc_bernstein_coeffs_factored.restype = ctypes.c_int
    lib.orc_bernstein_coeffs_factored.argtypes = [ctypes.c_int, ctypes.c_int, u8, dp,
                                                  ctypes.c_int, dp]
    lib.orc_enclosure.restype = ctypes.c_int
    lib.orc_enclosure.argtypes = [ctypes.c_int, ctypes.c_int, u8, dp, ctypes.c_int,
                                  ctypes.c_longlong, dp, dp]
    lib.orc_compose.restype = ctypes.c_int
    lib.orc_compose.argtypes = [ctypes.c_int, ctypes.c_int, u8, dp, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                ctypes.c_double, ctypes.c_int, ctypes.c_int, ip, u8, dp]
    lib.orc_poly_mul.restype = ctypes.c_int
    lib.orc_poly_mul.argtypes = [ctypes.c_int, ctypes.c_int, u8, dp, ctypes.c_int, u8, dp,
                                 ctypes.c_int, ip, u8, dp]
    lib.orc_affine.restype = ctypes.c_int
    lib.orc_affine.argtypes = [ctypes.c_int, ctypes.c_int, ip, u8, dp, ip, u8, dp, dp,
                               ctypes.c_double, ctypes.c_int, ip, u8, dp]
    lib.orc_eval_poly.restype = None
    lib.orc_eval_poly.argtypes = [ctypes.c_int, ctypes.c_int, u8, dp, ctypes.c_longlong, dp, dp]
    lib.orc_propagate.restype = ctypes.c_int
    lib.orc_propagate.argtypes = [ctypes.c_int, ip, dp, dp, dp, ip, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_longlong, ctypes.c_int, dp, dp,
                                  ctypes.c_int, ip, u8, dp, dp, dp, ip, ip]
    lib.orc_propagate_cb.restype = ctypes.c_int
    lib.orc_propagate_cb.argtypes = [ctypes.c_int, ip, dp, dp, dp, DEGREE_FN, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                                     ctypes.c_int, dp, dp, ctypes.c_int, ip, u8, dp, dp, dp, ip,
                                     ip, ip]
    lib.orc_linearize.restype = ctypes.c_int
    lib.orc_linearize.argtypes = [ctypes.c_int, ctypes.c_int, u8, dp, ctypes.c_int,
                                  ctypes.c_longlong, ctypes.c_int, ctypes.c_int, ip, u8, dp]
    _lib = lib
    return lib


# order chooser callback: (user, layer, neuron, lo, hi, nterms) -> order
DEGREE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                             ctypes.c_double, ctypes.c_double, ctypes.c_longlong)


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _u8(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))


# A polynomial is a pair (exps uint8 [T, n], coef float64 [T]) in t in [0,1]^n.
Poly = Tuple[np.ndarray, np.ndarray]


def as_poly(p, n: int) -> Poly:
    if isinstance(p, dict):
        keys = list(p.keys())
        e = np.array(keys, dtype=np.uint8).reshape(len(keys), n)
        c = np.array([p[k] for k in keys], dtype=np.float64)
        return e, c
    e, c = p
    return (np.ascontiguousarray(e, dtype=np.uint8).reshape(-1, n),
            np.ascontiguousarray(c, dtype=np.float64).reshape(-1))


def to_dict(p: Poly) -> Dict[tuple, float]:
    e, c = p
    out: Dict[tuple, float] = {}
    for row, v in zip(e, c):
        k = tuple(int(x) for x in row)
        out[k] = out.get(k, 0.0) + float(v)
    return out


def binom(n: int, k: int) -> float:
    return _load().orc_binom(n, k)


def relu_bern_eval(lo: float, hi: float, d: int, y: float) -> float:
    """Def. 1 applied to ReLU on [lo,hi]: the order-d Bernstein polynomial at y."""
    return _load().orc_relu_bern_eval(lo, hi, d, y)


def relu_coeffs(lo: float, hi: float, d: int):
    """Power form a_0..a_d in s=(y-lo)/(hi-lo) and the shift eps = B(0) (Prop. 2)."""
    a = np.zeros(d + 1)
    eps = ctypes.c_double()
    _load().orc_relu_coeffs(lo, hi, d, _dp(a), ctypes.byref(eps))
    return a, eps.value


def bernstein_coeffs(p, n: int, l: int) -> np.ndarray:
    """Bernstein coefficients on [0,1]^n, order l per variable, shape (l+1,)*n
    (Def. 2 term by term)."""
    e, c = as_poly(p, n)
    out = np.zeros((l + 1) ** n)
    rc = _load().orc_bernstein_coeffs(n, len(c), _u8(e), _dp(c), l, _dp(out))
    if rc:
        raise ValueError("polynomial exponent exceeds Bernstein order")
    return out.reshape((l + 1,) * n)


def bernstein_coeffs_factored(p, n: int, l: int) -> np.ndarray:
    """The same coefficients by the weight's factorisation over the variables
    (one triangular transform per variable), which the enclosure uses on large
    grids."""
    e, c = as_poly(p, n)
    out = np.zeros((l + 1) ** n)
    rc = _load().orc_bernstein_coeffs_factored(n, len(c), _u8(e), _dp(c), l, _dp(out))
    if rc:
        raise ValueError("polynomial exponent exceeds Bernstein order")
    return out.reshape((l + 1,) * n)


def enclosure(p, n: int, l: int, budget: int = 0):
    """(min, max) of the Bernstein coefficients (Def. 2); budget rule R6."""
    e, c = as_poly(p, n)
    mn, mx = ctypes.c_double(), ctypes.c_double()
    rc = _load().orc_enclosure(n, len(c), _u8(e), _dp(c), l, budget,
                               ctypes.byref(mn), ctypes.byref(mx))
    if rc:
        raise ValueError("polynomial exponent exceeds Bernstein order")
    return mn.value, mx.value


def _out_poly(n, cap_terms):
    return (np.zeros(1, np.int32), np.zeros(cap_terms * n, np.uint8),
            np.zeros(cap_terms, np.float64))


def compose(p, n: int, lo: float, hi: float, d: int, upper: bool, cap: int = 64,
            tau: float = 0.0, cap_terms: int = 1 << 16) -> Poly:
    """Step 3 for one bound of one neuron (eqs. post_bounds_1/2)."""
    e, c = as_poly(p, n)
    on, oe, oc = _out_poly(n, cap_terms)
    rc = _load().orc_compose(n, len(c), _u8(e), _dp(c), lo, hi, d, cap, tau,
                             1 if upper else 0, cap_terms, _ip(on), _u8(oe), _dp(oc))
    if rc:
        raise ValueError("compose failed (%d)" % rc)
    k = int(on[0])
    return oe[: k * n].reshape(k, n).copy(), oc[:k].copy()


def poly_mul(p, q, n: int, cap_terms: int = 1 << 18) -> Poly:
    ea, ca = as_poly(p, n)
    eb, cb = as_poly(q, n)
    on, oe, oc = _out_poly(n, cap_terms)
    rc = _load().orc_poly_mul(n, len(ca), _u8(ea), _dp(ca), len(cb), _u8(eb), _dp(cb),
                              cap_terms, _ip(on), _u8(oe), _dp(oc))
    if rc:
        raise ValueError("poly_mul capacity")
    k = int(on[0])
    return oe[: k * n].reshape(k, n).copy(), oc[:k].copy()


def affine(up, lo, n: int, w_row, bias: float, cap_terms: int = 1 << 16):
    """Sec. 5.2 layer step for ONE output neuron: up/lo are lists of input
    polynomials; returns (pre_up, pre_lo)."""
    ups = [as_poly(p, n) for p in up]
    los = [as_poly(p, n) for p in lo]
    nt_u = np.array([len(c) for _, c in ups], np.int32)
    nt_l = np.array([len(c) for _, c in los], np.int32)
    e_u = np.ascontiguousarray(np.concatenate([e for e, _ in ups]).reshape(-1), np.uint8)
    c_u = np.ascontiguousarray(np.concatenate([c for _, c in ups]), np.float64)
    e_l = np.ascontiguousarray(np.concatenate([e for e, _ in los]).reshape(-1), np.uint8)
    c_l = np.ascontiguousarray(np.concatenate([c for _, c in los]), np.float64)
    w = np.ascontiguousarray(np.asarray(w_row, np.float64).reshape(-1))
    on = np.zeros(2, np.int32)
    oe = np.zeros(2 * cap_terms * n, np.uint8)
    oc = np.zeros(2 * cap_terms)
    rc = _load().orc_affine(n, len(ups), _ip(nt_u), _u8(e_u), _dp(c_u), _ip(nt_l), _u8(e_l),
                            _dp(c_l), _dp(w), float(bias), cap_terms, _ip(on), _u8(oe), _dp(oc))
    if rc:
        raise ValueError("affine failed (%d)" % rc)
    oe = oe.reshape(2, cap_terms, n)
    oc = oc.reshape(2, cap_terms)
    return ((oe[0, : on[0]].copy(), oc[0, : on[0]].copy()),
            (oe[1, : on[1]].copy(), oc[1, : on[1]].copy()))


def eval_poly(p, n: int, t: np.ndarray) -> np.ndarray:
    """Evaluate sum_K c_K t^K at points t (shape [P, n]) in FP64."""
    e, c = as_poly(p, n)
    t = np.ascontiguousarray(t, dtype=np.float64).reshape(-1, n)
    out = np.zeros(len(t))
    _load().orc_eval_poly(n, len(c), _u8(e), _dp(c), len(t), _dp(t), _dp(out))
    return out


def linearize(p, n: int, order: int, upper: bool, budget: int = 0,
              cap_terms: int = 1 << 12) -> Poly:
    """Lin step (Sec. 5.3, reading R22) on one polynomial: its least-squares
    multilinear fit on the box plus the Bernstein enclosure (order `order`)
    of the residual, max for the upper bound, min for the lower."""
    e, c = as_poly(p, n)
    ne = np.zeros(1, np.int32)
    oe = np.zeros(cap_terms * n, np.uint8)
    oc = np.zeros(cap_terms)
    rc = _load().orc_linearize(n, len(c), _u8(e), _dp(c), order, budget, int(bool(upper)),
                               cap_terms, _ip(ne), _u8(oe), _dp(oc))
    if rc:
        raise ValueError("oracle linearize failed (%d)" % rc)
    k = int(ne[0])
    return oe.reshape(cap_terms, n)[:k].copy(), oc[:k].copy()


def propagate(widths: Sequence[int], W, b, box, degrees, cap: int = 16,
              tau: float = 0.0, budget: int = 0, cap_terms: int = 1 << 16, lin: int = 0):
    """Whole-network bounds for ONE box.

    widths: [n, h_1, ..., o]; W, b: per-layer float arrays (float32 values are
    taken exactly); box: array (n, 2); degrees: an int (every hidden neuron),
    an array with one ReLU order per hidden neuron, or a callable
    choose(layer, neuron, lo, hi, nterms) -> order called for every hidden
    neuron once its pre-activation enclosure is known (layer is 1-based;
    nterms is the dense term count M(n, D) of its pre-activation polynomials).
    Returns a dict with 'lo', 'hi' (o,), 'upper'/'lower' (lists of polys),
    and the per-hidden-neuron trace 'tr_lo', 'tr_hi', 'tr_case', 'degree' and
    the per-layer Bernstein order 'order'.  lin > 0 linearises the
    post-activation bounds after every lin-th hidden layer (Sec. 5.3, R22).
    """
    widths = [int(w) for w in widths]
    H = len(widths) - 1
    n, o = widths[0], widths[-1]
    Wa = np.concatenate([np.asarray(w, dtype=np.float64).reshape(-1) for w in W])
    ba = np.concatenate([np.asarray(x, dtype=np.float64).reshape(-1) for x in b])
    bx = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(n, 2))
    n_hidden = sum(widths[1:-1])
    wid = np.array(widths, np.int32)
    out_lo = np.zeros(o)
    out_hi = np.zeros(o)
    nterms = np.zeros(o * 2, np.int32)
    exps = np.zeros(o * 2 * cap_terms * n, np.uint8)
    coef = np.zeros(o * 2 * cap_terms)
    nh = max(n_hidden, 1)
    tr_lo, tr_hi = np.zeros(nh), np.zeros(nh)
    tr_case = np.zeros(nh, np.int32)
    tr_deg = np.zeros(nh, np.int32)
    tr_order = np.zeros(H, np.int32)
    if callable(degrees):
        err = []

        def _cb(user, layer, m, lo, hi, nt):
            try:
                return int(degrees(int(layer), int(m), float(lo), float(hi), int(nt)))
            except Exception as ex:   # report, never raise through C
                err.append(ex)
                return 0

        fn = DEGREE_FN(_cb)
        rc = _load().orc_propagate_cb(H, _ip(wid), _dp(Wa), _dp(ba), _dp(bx), fn, None, cap, tau,
                                      budget, int(lin), _dp(out_lo), _dp(out_hi), cap_terms, _ip(nterms),
                                      _u8(exps), _dp(coef), _dp(tr_lo), _dp(tr_hi),
                                      _ip(tr_case), _ip(tr_order), _ip(tr_deg))
        if err:
            raise err[0]
    else:
        if np.isscalar(degrees):
            deg = np.full(nh, int(degrees), np.int32)
        else:
            deg = np.ascontiguousarray(np.asarray(degrees, dtype=np.int32).reshape(-1))
            if len(deg) < n_hidden:
                raise ValueError("need one degree per hidden neuron")
            if len(deg) == 0:
                deg = np.ones(1, np.int32)
        tr_deg[:n_hidden] = deg[:n_hidden]
        rc = _load().orc_propagate(H, _ip(wid), _dp(Wa), _dp(ba), _dp(bx), _ip(deg), cap, tau,
                                   budget, int(lin), _dp(out_lo), _dp(out_hi), cap_terms, _ip(nterms),
                                   _u8(exps), _dp(coef), _dp(tr_lo), _dp(tr_hi), _ip(tr_case),
                                   _ip(tr_order))
    if rc:
        raise ValueError("oracle propagate failed (%d)" % rc)
    exps = exps.reshape(o, 2, cap_terms, n)
    coef = coef.reshape(o, 2, cap_terms)
    nterms = nterms.reshape(o, 2)
    upper = [(exps[j, 0, : nterms[j, 0]].copy(), coef[j, 0, : nterms[j, 0]].copy()) for j in range(o)]
    lower = [(exps[j, 1, : nterms[j, 1]].copy(), coef[j, 1, : nterms[j, 1]].copy()) for j in range(o)]
    return {"lo": out_lo, "hi": out_hi, "upper": upper, "lower": lower,
            "tr_lo": tr_lo[:n_hidden], "tr_hi": tr_hi[:n_hidden],
            "tr_case": tr_case[:n_hidden], "degree": tr_deg[:n_hidden], "order": tr_order}


def network_forward(widths: Sequence[int], W, b, x: np.ndarray) -> np.ndarray:
    """Plain FP64 forward pass of the ReLU network (Sec. 2) at points x [P, n]."""
    z = np.asarray(x, dtype=np.float64)
    H = len(widths) - 1
    for i in range(H):
        z = z @ np.asarray(W[i], dtype=np.float64).T + np.asarray(b[i], dtype=np.float64)
        if i < H - 1:
            z = np.maximum(z, 0.0)
    return z


def vol_relative(upper: Poly, lower: Poly, n: int) -> float:
    """Mean over the box of (p_up - p_lo): the paper's Vol_relative (Sec. 6),
    in closed form for monomials: the mean of t^K over [0,1]^n is
    prod_i 1/(k_i+1)."""
    tot = 0.0
    for (e, c), sgn in ((upper, 1.0), (lower, -1.0)):
        e = np.asarray(e, dtype=np.float64).reshape(-1, n)
        tot += sgn * float(np.sum(np.asarray(c) / np.prod(e + 1.0, axis=1)))
    return tot
