"""Python binding of libbern.so (the C ABI in include/bern.h).

Argument marshalling only: every step of the bound propagation runs in the
library's CUDA kernels.  PyTorch supplies device memory and the stream.  If
the shared library is missing or cannot be loaded this module raises; there
is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

BERN_OK = 0
BERN_E_INVALID = 1
BERN_E_CAPACITY = 2
BERN_E_NONFINITE = 3
BERN_E_TIMEOUT = 4
BERN_E_CUDA = 5
BERN_E_UNSUPPORTED = 6
BERN_E_NOMEM = 7
BERN_MEM_DEVICE = 0
BERN_MEM_HOST = 1
BERN_DEG_GLOBAL = 0
BERN_DEG_PER_LAYER = 1
BERN_DEG_PER_NEURON = 2
BERN_DEG_LEARNED = 3
BERN_MLP_HIDDEN = 64
BERN_DEGREE_FEATURES = 8
BERN_DEGREE_CLASSES = 4
BERN_MAX_ORDER = 16
BERN_MAX_GRID = 24576
BERN_MAX_BIG_GRID = 4194304
BERN_MAX_ENCLOSE_ORDER = 24
COEF_STRIDE = BERN_MAX_ORDER + 1


def effective_budget(budget: int = 0, noalloc: bool = False) -> int:
    """The Bernstein-grid budget the library applies: 0 means 2^20; clamped
    to BERN_MAX_BIG_GRID (grids above BERN_MAX_GRID run in the context's
    global-memory workspace, at orders up to 16), or to BERN_MAX_GRID for
    bern_propagate_noalloc, which has no workspace."""
    b = budget if budget > 0 else 1 << 20
    return min(b, BERN_MAX_GRID if noalloc else BERN_MAX_BIG_GRID)

EXPORTS = [
    "bern_create", "bern_destroy", "bern_set_pointer_mode", "bern_set_graphs",
    "bern_strerror", "bern_sync", "bern_kernel_launches", "bern_num_monomials",
    "bern_monomials", "bern_propagate", "bern_init_inputs", "bern_affine",
    "bern_enclose", "bern_relu_coeffs", "bern_compose", "bern_propagate_noalloc",
    "bern_mlp_num_params", "bern_degree_features", "bern_mlp_forward", "bern_mlp_backward",
    "bern_mlp_adam", "bern_propagate_traced", "bern_split_features",
    "bern_set_horner_smem_limit", "bern_set_autotune", "bern_force_variant",
    "bern_poly_to_x", "bern_linearize", "bern_fma_throughput", "bern_layer", "bern_set_fused",
    "bern_bernstein_square",
    "bern_bernstein_elevate",
    "bern_bernstein_affine",
    "bern_enclose_lines",
    "bern_enclose_scales",
    "bern_compose_rows",
    "bern_pair_lists",
]


class BernError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__("%s: %s (%d)" % (where, strerror(code), code))
        self.code = code


class bern_net(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int), ("widths", ctypes.POINTER(ctypes.c_int)),
                ("W", ctypes.POINTER(ctypes.c_void_p)), ("b", ctypes.POINTER(ctypes.c_void_p))]


class bern_mlp(ctypes.Structure):
    _fields_ = [("n_features", ctypes.c_int), ("n_classes", ctypes.c_int),
                ("W1", ctypes.c_void_p), ("b1", ctypes.c_void_p),
                ("W2", ctypes.c_void_p), ("b2", ctypes.c_void_p)]


class bern_degree_plan(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("global_d", ctypes.c_int),
                ("per_layer", ctypes.POINTER(ctypes.c_int)),
                ("per_neuron", ctypes.POINTER(ctypes.c_uint8)),
                ("degree_cap", ctypes.c_int), ("prune_tau", ctypes.c_float),
                ("bern_budget", ctypes.c_int64),
                ("mlp", ctypes.POINTER(bern_mlp)), ("min_conf", ctypes.c_float),
                ("lin_every", ctypes.c_int)]


class bern_trace(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("nterms", ctypes.c_void_p),
                ("degree", ctypes.c_void_p)]


class bern_result(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_void_p), ("hi", ctypes.c_void_p), ("n_terms", ctypes.c_void_p),
                ("keys", ctypes.c_void_p), ("coef", ctypes.c_void_p), ("cap_terms", ctypes.c_int64)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libbern.so (building it first if it is absent and allowed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError("libbern.so is not built (%s)" % path)
        _build.build()
    lib = ctypes.CDLL(path)
    V, I, I64, F = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_float
    sig = {
        "bern_create": (I, [ctypes.POINTER(V), I, V]),
        "bern_destroy": (I, [V]),
        "bern_set_pointer_mode": (I, [V, I]),
        "bern_set_graphs": (I, [V, I]),
        "bern_set_horner_smem_limit": (I, [V, I64]),
        "bern_set_autotune": (I, [V, I]),
        "bern_force_variant": (I, [V, ctypes.c_char_p, I]),
        "bern_poly_to_x": (I, [V, I, I64, I, V, V, V, I64, V]),
        "bern_strerror": (ctypes.c_char_p, [I]),
        "bern_sync": (I, [V]),
        "bern_kernel_launches": (I64, [V]),
        "bern_fma_throughput": (I, [I, V, I, I, ctypes.POINTER(ctypes.c_double)]),
        "bern_num_monomials": (I64, [I, I]),
        "bern_monomials": (I, [I, I, V]),
        "bern_enclose_lines": (I, [I, I, V, I64]),
        "bern_enclose_scales": (I, [I, I, V, I64]),
        "bern_compose_rows": (I, [I, I, V, I64, V]),
        "bern_pair_lists": (I, [I, I, I, I, V, I64, V, I64, V]),
        "bern_propagate": (I, [V, ctypes.POINTER(bern_net), V, I64,
                               ctypes.POINTER(bern_degree_plan), ctypes.POINTER(bern_result)]),
        "bern_init_inputs": (I, [V, I, I64, V, V, V, I64, V]),
        "bern_affine": (I, [V, I64, I, I, V, V, V, V, I64, V, V, V, I64, V]),
        "bern_enclose": (I, [V, I, I64, I, I, I64, V, V, I64, V, V, V]),
        "bern_linearize": (I, [V, I, I64, I, I, I64, V, V, I64, V, V, V, I64, V, V, V]),
        "bern_relu_coeffs": (I, [V, I64, V, V, V, I, V, V, V]),
        "bern_compose": (I, [V, I, I64, I, I, F, V, V, V, V, I, V, V, V, V, I64, V, V, V, I64,
                             V]),
        "bern_layer": (I, [V, I, I64, I, I, I64, I, I, V, V, I64, V, I, V, V, V, V, I64, V]),
        "bern_set_fused": (I, [V, I]),
        "bern_bernstein_square": (I, [V, I, I, I64, V, V, V]),
        "bern_bernstein_elevate": (I, [V, I, I, I, I64, V, V, V, V]),
        "bern_bernstein_affine": (I, [V, I64, I, I, V, V, I64, V, V, V, V]),
        "bern_propagate_noalloc": (I, [ctypes.POINTER(bern_net), V, I64,
                                       ctypes.POINTER(bern_degree_plan),
                                       ctypes.POINTER(bern_result), V]),
        "bern_propagate_traced": (I, [V, ctypes.POINTER(bern_net), V, I64,
                                      ctypes.POINTER(bern_degree_plan),
                                      ctypes.POINTER(bern_result), ctypes.POINTER(bern_trace)]),
        "bern_split_features": (I, [V, I, I64, V, V, ctypes.POINTER(bern_result), I, I, V]),
        "bern_mlp_num_params": (I64, [I, I]),
        "bern_degree_features": (I, [V, I64, V, V, V, I, V]),
        "bern_mlp_forward": (I, [V, ctypes.POINTER(bern_mlp), I64, V, V]),
        "bern_mlp_backward": (I, [V, ctypes.POINTER(bern_mlp), I64, V, V, V, V, V]),
        "bern_mlp_adam": (I, [V, I, I, V, V, V, V, F, F, F, F, I, V, V]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def strerror(code: int) -> str:
    return load().bern_strerror(code).decode()


def _check(code: int, where: str):
    if code != BERN_OK:
        raise BernError(code, where)


def fma_throughput(device: int = 0, stream=None, directed: bool = True, reps: int = 5) -> float:
    """Measured FP32 FMA throughput of the device in TFLOP/s (bern_fma_throughput)."""
    out = ctypes.c_double(0.0)
    h = 0 if stream is None else int(stream.cuda_stream)
    _check(load().bern_fma_throughput(int(device), ctypes.c_void_p(h), 1 if directed else 0,
                                     int(reps), ctypes.byref(out)), "bern_fma_throughput")
    return float(out.value)


def num_monomials(n: int, D: int) -> int:
    return int(load().bern_num_monomials(n, D))


def monomials(n: int, D: int) -> np.ndarray:
    """The library's graded monomial order: array [M(n,D), n] of exponents."""
    m = num_monomials(n, D)
    out = np.zeros((m, n), np.uint8)
    _check(load().bern_monomials(n, D, out.ctypes.data), "bern_monomials")
    return out


def enclose_lines(n: int, l: int) -> np.ndarray:
    """The enclosure's line table for order l (bern_enclose_lines): array
    [n, (l+1)^(n-1), 2] of (grid index of the line's first cell, digit sum of
    the variables before the line's variable)."""
    nl = (l + 1) ** (n - 1)
    out = np.zeros((n, nl, 2), np.int32)
    _check(load().bern_enclose_lines(n, l, out.ctypes.data, out.size), "bern_enclose_lines")
    return out


def enclose_scales(n: int, l: int) -> np.ndarray:
    """The enclosure's reciprocal brackets for order l (bern_enclose_scales):
    array [M(n,l), 2] of float32 (lo, hi) around 1 / prod_k C(l, j_k), in the
    graded order."""
    out = np.zeros((num_monomials(n, l), 2), np.float32)
    _check(load().bern_enclose_scales(n, l, out.ctypes.data, out.size), "bern_enclose_scales")
    return out


def compose_rows(n: int, D: int) -> dict:
    """The composition's row tables for input degree D (bern_compose_rows):
    pos_in [M], hdr [rows, 4], in_off [rows], pairs [n_pairs, 4], out_ranks,
    and row_split."""
    sizes = np.zeros(5, np.int64)
    lib = load()
    _check(lib.bern_compose_rows(n, D, None, 0, sizes.ctypes.data), "bern_compose_rows")
    m_in, rows, split, npairs, nout = (int(v) for v in sizes)
    out = np.zeros(m_in + 5 * rows + 4 * npairs + nout, np.int32)
    _check(lib.bern_compose_rows(n, D, out.ctypes.data, out.size, sizes.ctypes.data),
           "bern_compose_rows")
    o = np.cumsum([0, m_in, 4 * rows, rows, 4 * npairs, nout])
    return {"pos_in": out[o[0]:o[1]], "hdr": out[o[1]:o[2]].reshape(rows, 4),
            "in_off": out[o[2]:o[3]], "pairs": out[o[3]:o[4]].reshape(npairs, 4),
            "out_ranks": out[o[4]:o[5]], "row_split": split}


def pair_lists(n: int, Dq: int, Ds: int, square: bool):
    """The composition's output-stationary pair lists (bern_pair_lists):
    (ptr [M(n, Dq+Ds)+1], pairs [n_pairs, 2] of graded ranks (I, J))."""
    sizes = np.zeros(2, np.int64)
    lib = load()
    _check(lib.bern_pair_lists(n, Dq, Ds, int(square), None, 0, None, 0, sizes.ctypes.data),
           "bern_pair_lists")
    ptr = np.zeros(int(sizes[0]), np.int32)
    pairs = np.zeros((int(sizes[1]), 2), np.int32)
    _check(lib.bern_pair_lists(n, Dq, Ds, int(square), ptr.ctypes.data, ptr.size,
                               pairs.ctypes.data, pairs.size, sizes.ctypes.data),
           "bern_pair_lists")
    return ptr, pairs


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class Context:
    """Owns a bern_ctx on one CUDA device, bound to a torch stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        h = ctypes.c_void_p()
        _check(lib.bern_create(ctypes.byref(h), device, ctypes.c_void_p(stream.cuda_stream)),
               "bern_create")
        self.h = h
        self.device = device
        self.lib = lib

    def close(self):
        if getattr(self, "h", None):
            self.lib.bern_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- control
    def sync(self) -> int:
        return int(self.lib.bern_sync(self.h))

    def check(self, where="bern_sync"):
        _check(self.sync(), where)

    def kernel_launches(self) -> int:
        return int(self.lib.bern_kernel_launches(self.h))

    def set_graphs(self, on: bool):
        _check(self.lib.bern_set_graphs(self.h, 1 if on else 0), "bern_set_graphs")

    def set_autotune(self, on: bool):
        _check(self.lib.bern_set_autotune(self.h, 1 if on else 0), "bern_set_autotune")

    def force_variant(self, kind: str, variant: int):
        """Force variant `variant` (-1: none) of kernel family `kind`
        ("affine" or "enclose") for later launches (tests and tuning)."""
        _check(self.lib.bern_force_variant(self.h, kind.encode(), int(variant)),
               "bern_force_variant")

    def bernstein_square(self, n, l, a, c_hi, c_lo):
        """bern_bernstein_square: Prod_Bern squares of dense Bernstein tensors
        a [P, (l+1)^n] into coefficient intervals [c_lo, c_hi] [P, (2l+1)^n]."""
        _check(self.lib.bern_bernstein_square(self.h, n, l, int(a.shape[0]), _ptr(a), _ptr(c_hi),
                                              _ptr(c_lo)), "bern_bernstein_square")

    def bernstein_elevate(self, n, l, r, a_hi, a_lo, c_hi, c_lo):
        """bern_bernstein_elevate: interval tensors [a_lo, a_hi] [P, (l+1)^n]
        elevated to order l + r: [c_lo, c_hi] [P, (l+r+1)^n]."""
        _check(self.lib.bern_bernstein_elevate(self.h, n, l, r, int(a_hi.shape[0]), _ptr(a_hi),
                                               _ptr(a_lo), _ptr(c_hi), _ptr(c_lo)),
               "bern_bernstein_elevate")

    def bernstein_affine(self, n_boxes, h_out, h_in, W, b, n_coef, in_hi, in_lo, out_hi, out_lo):
        """bern_bernstein_affine: the layer sum on dense Bernstein tensors in
        the layer-block layout [B, n_coef, h] (bias on every coefficient)."""
        _check(self.lib.bern_bernstein_affine(self.h, int(n_boxes), h_out, h_in, _ptr(W), _ptr(b),
                                              int(n_coef), _ptr(in_hi), _ptr(in_lo), _ptr(out_hi),
                                              _ptr(out_lo)), "bern_bernstein_affine")

    def set_fused(self, on: bool):
        _check(self.lib.bern_set_fused(self.h, 1 if on else 0), "bern_set_fused")

    def layer(self, n, n_boxes, h, order, budget, global_d, cap, pre_up, pre_lo, pre_ld,
              pre_nterms, h_next, W_next, b_next, next_up, next_lo, next_ld, next_nterms):
        """bern_layer: one fused hidden layer (a2-a4) plus the next layer's a1."""
        _check(self.lib.bern_layer(self.h, n, n_boxes, h, order, budget, global_d, cap,
                                   _ptr(pre_up), _ptr(pre_lo), pre_ld, _ptr(pre_nterms), h_next,
                                   _ptr(W_next), _ptr(b_next), _ptr(next_up), _ptr(next_lo),
                                   next_ld, _ptr(next_nterms)), "bern_layer")

    def set_horner_smem_limit(self, nbytes: int):
        _check(self.lib.bern_set_horner_smem_limit(self.h, int(nbytes)),
               "bern_set_horner_smem_limit")

    def set_pointer_mode(self, mode: int):
        _check(self.lib.bern_set_pointer_mode(self.h, mode), "bern_set_pointer_mode")

    # ------------------------------------------------------------- steps
    # Layer blocks: coefficient r of neuron m of box b at ((b*ld + r)*h + m).
    def init_inputs(self, n, boxes, z_up, z_lo, ld, nterms):
        _check(self.lib.bern_init_inputs(self.h, n, boxes.shape[0], _ptr(boxes), _ptr(z_up),
                                         _ptr(z_lo), ld, _ptr(nterms)), "bern_init_inputs")

    def affine(self, n_boxes, h_out, h_in, W, b, in_up, in_lo, in_ld, in_nterms,
               out_up, out_lo, out_ld, out_nterms):
        _check(self.lib.bern_affine(self.h, n_boxes, h_out, h_in, _ptr(W), _ptr(b), _ptr(in_up),
                                    _ptr(in_lo), in_ld, _ptr(in_nterms), _ptr(out_up),
                                    _ptr(out_lo), out_ld, _ptr(out_nterms)), "bern_affine")

    def poly_to_x(self, boxes, n_terms, coef, out=None):
        """Output polynomials of ``propagate`` (``n_terms`` [B, o, 2], ``coef``
        [B, o, 2, cap]) rewritten in the input coordinates x of their boxes
        (``boxes`` [B, n, 2]); the constant terms carry the rounding remainder
        outward.  Returns ``out`` (a tensor shaped like ``coef``)."""
        B, n = int(boxes.shape[0]), int(boxes.shape[1])
        o, cap = int(coef.shape[1]), int(coef.shape[3])
        if out is None:
            out = coef.new_zeros(coef.shape)
        _check(self.lib.bern_poly_to_x(self.h, n, B, o, _ptr(boxes), _ptr(n_terms), _ptr(coef),
                                       cap, _ptr(out)), "bern_poly_to_x")
        return out

    def enclose(self, n, n_boxes, h, order, budget, pre_up, pre_lo, ld, nterms, lo, hi):
        _check(self.lib.bern_enclose(self.h, n, n_boxes, h, order, budget, _ptr(pre_up),
                                     _ptr(pre_lo), ld, _ptr(nterms), _ptr(lo), _ptr(hi)),
               "bern_enclose")

    def linearize(self, n, n_boxes, h, order, budget, post_up, post_lo, ld, nterms, lin_up,
                  lin_lo, lin_ld, lin_nterms, res_lo, res_hi):
        _check(self.lib.bern_linearize(self.h, n, n_boxes, h, order, budget, _ptr(post_up),
                                       _ptr(post_lo), ld, _ptr(nterms), _ptr(lin_up),
                                       _ptr(lin_lo), lin_ld, _ptr(lin_nterms), _ptr(res_lo),
                                       _ptr(res_hi)), "bern_linearize")

    def relu_coeffs(self, n_items, lo, hi, degrees, global_d, kind, coef, eps):
        _check(self.lib.bern_relu_coeffs(self.h, n_items, _ptr(lo), _ptr(hi), _ptr(degrees),
                                         global_d, _ptr(kind), _ptr(coef), _ptr(eps)),
               "bern_relu_coeffs")

    def compose(self, n, n_boxes, h, cap, tau, kind, coef, eps, degrees, global_d, lo, hi,
                pre_up, pre_lo, pre_ld, pre_nterms, post_up, post_lo, post_ld, post_nterms):
        _check(self.lib.bern_compose(self.h, n, n_boxes, h, cap, tau, _ptr(kind), _ptr(coef),
                                     _ptr(eps), _ptr(degrees), global_d, _ptr(lo), _ptr(hi),
                                     _ptr(pre_up), _ptr(pre_lo), pre_ld, _ptr(pre_nterms),
                                     _ptr(post_up), _ptr(post_lo), post_ld,
                                     _ptr(post_nterms)), "bern_compose")

    # ------------------------------------------------------------- learned component
    def degree_features(self, n_items, lo, hi, nterms, layer, x):
        _check(self.lib.bern_degree_features(self.h, n_items, _ptr(lo), _ptr(hi), _ptr(nterms),
                                             int(layer), _ptr(x)), "bern_degree_features")

    def split_features(self, n, boxes, root, out, output, x):
        """Split-dimension features (bern_split_features) of the boxes of a
        propagate() result `out` (device tensors; out must hold coef)."""
        B = int(boxes.shape[0])
        o = int(out["lo"].shape[1])
        res = bern_result(_ptr(out["lo"]), _ptr(out["hi"]), _ptr(out["n_terms"]), None,
                          _ptr(out["coef"]), int(out["coef"].shape[-1]))
        _check(self.lib.bern_split_features(self.h, n, B, _ptr(boxes), _ptr(root),
                                            ctypes.byref(res), o, int(output), _ptr(x)),
               "bern_split_features")

    def mlp_forward(self, mlp: "Mlp", x, logits):
        _check(self.lib.bern_mlp_forward(self.h, ctypes.byref(mlp.struct()), int(x.shape[0]),
                                         _ptr(x), _ptr(logits)), "bern_mlp_forward")

    def mlp_backward(self, mlp: "Mlp", x, labels, w, grad, loss):
        _check(self.lib.bern_mlp_backward(self.h, ctypes.byref(mlp.struct()), int(x.shape[0]),
                                          _ptr(x), _ptr(labels), _ptr(w), _ptr(grad),
                                          _ptr(loss)), "bern_mlp_backward")

    def mlp_adam(self, mlp: "Mlp", grad, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        mlp.t += 1
        _check(self.lib.bern_mlp_adam(self.h, mlp.F, mlp.C, _ptr(mlp.param), _ptr(mlp.m),
                                      _ptr(mlp.v), _ptr(grad), lr, beta1, beta2, eps, mlp.t,
                                      _ptr(mlp.W1), _ptr(mlp.W2)), "bern_mlp_adam")

    # ------------------------------------------------------------- whole path
    def propagate(self, widths: Sequence[int], W, b, boxes, degree=2, cap: int = 16,
                  tau: float = 0.0, budget: int = 0, cap_terms: Optional[int] = None,
                  out=None, keys: bool = False, sync: bool = True, trace: bool = False,
                  lin: int = 0):
        """bern_propagate on device tensors (W, b: lists of float32 CUDA tensors;
        boxes: float32 CUDA tensor [B, n, 2]).  degree: int (global), list of
        per-hidden-layer ints, or a uint8 array with one order per hidden
        neuron.  lin > 0 linearises every lin-th hidden layer (Sec. 5.3).
        Returns a dict of CUDA tensors."""
        torch = self.torch
        widths = [int(x) for x in widths]
        H = len(widths) - 1
        o = widths[-1]
        B = int(boxes.shape[0])
        plan, keep = make_plan(degree, widths, cap, tau, budget, lin)
        if cap_terms is None:
            cap_terms = max_output_terms(widths, degree, cap, lin)
        dev = boxes.device
        if out is None:
            out = {
                "lo": torch.empty(B, o, device=dev, dtype=torch.float32),
                "hi": torch.empty(B, o, device=dev, dtype=torch.float32),
                "n_terms": torch.empty(B, o, 2, device=dev, dtype=torch.int32),
                "coef": torch.empty(B, o, 2, cap_terms, device=dev, dtype=torch.float32),
                "keys": (torch.empty(B, o, 2, cap_terms, device=dev, dtype=torch.int64)
                         if keys else None),
            }
        net, keep2 = make_net(widths, [_ptr(w) for w in W], [_ptr(x) for x in b])
        res = bern_result(_ptr(out["lo"]), _ptr(out["hi"]), _ptr(out["n_terms"]),
                          _ptr(out.get("keys")), _ptr(out.get("coef")), cap_terms)
        if trace:
            nh = sum(widths[1:-1])
            out["tr_lo"] = torch.empty(B, nh, device=dev, dtype=torch.float32)
            out["tr_hi"] = torch.empty(B, nh, device=dev, dtype=torch.float32)
            out["tr_nterms"] = torch.empty(B, nh, device=dev, dtype=torch.int32)
            out["tr_degree"] = torch.empty(B, nh, device=dev, dtype=torch.uint8)
            tr = bern_trace(_ptr(out["tr_lo"]), _ptr(out["tr_hi"]), _ptr(out["tr_nterms"]),
                            _ptr(out["tr_degree"]))
            rc = self.lib.bern_propagate_traced(self.h, ctypes.byref(net),
                                                ctypes.c_void_p(_ptr(boxes)), B,
                                                ctypes.byref(plan), ctypes.byref(res),
                                                ctypes.byref(tr))
        else:
            rc = self.lib.bern_propagate(self.h, ctypes.byref(net), ctypes.c_void_p(_ptr(boxes)),
                                         B, ctypes.byref(plan), ctypes.byref(res))
        _check(rc, "bern_propagate")
        if sync:
            self.check("bern_propagate")
        return out

    def propagate_host(self, widths, W, b, boxes, degree=2, cap: int = 16, tau: float = 0.0,
                       budget: int = 0, cap_terms: Optional[int] = None, out=None, lin: int = 0):
        """bern_propagate with host buffers (numpy arrays, ideally pinned):
        copies in, runs, copies out and synchronises inside the call."""
        widths = [int(x) for x in widths]
        o = widths[-1]
        B = int(boxes.shape[0])
        plan, keep = make_plan(degree, widths, cap, tau, budget, lin)
        if cap_terms is None:
            cap_terms = max_output_terms(widths, degree, cap, lin)
        if out is None:
            out = {"lo": np.empty((B, o), np.float32), "hi": np.empty((B, o), np.float32),
                   "n_terms": np.empty((B, o, 2), np.int32),
                   "coef": np.empty((B, o, 2, cap_terms), np.float32)}
        Wp = [np.ascontiguousarray(w, np.float32) for w in W]
        bp = [np.ascontiguousarray(x, np.float32) for x in b]
        net, keep2 = make_net(widths, [w.ctypes.data for w in Wp], [x.ctypes.data for x in bp])
        bx = np.ascontiguousarray(boxes, np.float32)
        res = bern_result(out["lo"].ctypes.data, out["hi"].ctypes.data,
                          out["n_terms"].ctypes.data, 0,
                          out["coef"].ctypes.data if out.get("coef") is not None else 0,
                          cap_terms)
        self.set_pointer_mode(BERN_MEM_HOST)
        try:
            rc = self.lib.bern_propagate(self.h, ctypes.byref(net), bx.ctypes.data, B,
                                         ctypes.byref(plan), ctypes.byref(res))
        finally:
            self.set_pointer_mode(BERN_MEM_DEVICE)
        _check(rc, "bern_propagate(host)")
        return out


def propagate_noalloc(widths, W, b, boxes, out, degree=2, cap: int = 16, tau: float = 0.0,
                      budget: int = 0, stream=None) -> int:
    """bern_propagate_noalloc on caller-allocated CUDA tensors (W, b lists,
    boxes [B, n, 2], out dict with 'lo', 'hi', 'n_terms', 'coef' and optional
    'keys').  The library allocates nothing for this call; it returns the
    status code (0 on success) after synchronising the stream."""
    widths = [int(x) for x in widths]
    plan, keep = make_plan(degree, widths, cap, tau, budget)
    net, keep2 = make_net(widths, [_ptr(w) for w in W], [_ptr(x) for x in b])
    cap_terms = int(out["coef"].shape[-1]) if out.get("coef") is not None else 0
    res = bern_result(_ptr(out["lo"]), _ptr(out["hi"]), _ptr(out["n_terms"]),
                      _ptr(out.get("keys")), _ptr(out.get("coef")), cap_terms)
    h = 0 if stream is None else int(stream.cuda_stream)
    return int(load().bern_propagate_noalloc(ctypes.byref(net), ctypes.c_void_p(_ptr(boxes)),
                                             int(boxes.shape[0]), ctypes.byref(plan),
                                             ctypes.byref(res), ctypes.c_void_p(h)))


class Mlp:
    """Device state of one MLP of the learned component: the FP32 master
    parameter vector (W1, b1, W2, b2), its Adam moments and the BF16 copies
    of W1 and W2 that the kernels read.  Tensors are torch CUDA tensors."""

    def __init__(self, torch, n_features: int, n_classes: int, theta=None, device="cuda"):
        self.F, self.C = int(n_features), int(n_classes)
        P = int(load().bern_mlp_num_params(self.F, self.C))
        if P < 0:
            raise ValueError("unsupported MLP shape")
        H = BERN_MLP_HIDDEN
        if theta is None:
            theta = np.zeros(P, np.float32)
        theta = np.asarray(theta, np.float32)
        self.param = torch.from_numpy(theta.copy()).to(device)
        self.m = torch.zeros_like(self.param)
        self.v = torch.zeros_like(self.param)
        self.t = 0
        oW1, ob1, oW2 = H * self.F, H * self.F + H, H * self.F + H + self.C * H
        self.b1 = self.param[oW1:ob1]
        self.b2 = self.param[oW2:]
        # bf16 copies (round to nearest even), as raw 16-bit words
        self.W1 = self.param[:oW1].to(torch.bfloat16).view(torch.int16).contiguous()
        self.W2 = self.param[ob1:oW2].to(torch.bfloat16).view(torch.int16).contiguous()
        self.n_params = P
        self._s = None

    def struct(self):
        if self._s is None:
            self._s = bern_mlp(self.F, self.C, _ptr(self.W1), _ptr(self.b1), _ptr(self.W2),
                               _ptr(self.b2))
        return self._s

    def theta(self) -> np.ndarray:
        return self.param.detach().cpu().numpy().astype(np.float64)


def make_net(widths, W_ptrs, b_ptrs):
    H = len(widths) - 1
    wid = (ctypes.c_int * (H + 1))(*widths)
    Wa = (ctypes.c_void_p * H)(*W_ptrs)
    ba = (ctypes.c_void_p * H)(*b_ptrs)
    net = bern_net(H, wid, Wa, ba)
    return net, (wid, Wa, ba)


class Learned:
    """A learned degree plan: the degree MLP (an Mlp with BERN_DEGREE_FEATURES
    features and BERN_DEGREE_CLASSES classes), the confidence below which a
    neuron falls back to the plain order, and that order."""

    def __init__(self, mlp: "Mlp", min_conf: float = 0.0, fallback: int = 2, max_per_layer=None):
        self.mlp, self.min_conf, self.fallback = mlp, float(min_conf), int(fallback)
        self.max_per_layer = None if max_per_layer is None else [int(x) for x in max_per_layer]


def make_plan(degree, widths, cap, tau, budget, lin: int = 0):
    H = len(widths) - 1
    keep = []
    if isinstance(degree, Learned):
        ms = degree.mlp.struct()
        keep.append(ms)
        caps = None
        if degree.max_per_layer is not None:
            caps = (ctypes.c_int * len(degree.max_per_layer))(*degree.max_per_layer)
            keep.append(caps)
        plan = bern_degree_plan(BERN_DEG_LEARNED, degree.fallback, caps, None, cap, tau, budget,
                                ctypes.pointer(ms), degree.min_conf)
    elif isinstance(degree, (int, np.integer)):
        plan = bern_degree_plan(BERN_DEG_GLOBAL, int(degree), None, None, cap, tau, budget)
    else:
        arr = np.asarray(degree)
        if arr.dtype == np.uint8 or len(arr) == sum(widths[1:-1]) and len(arr) != H - 1:
            a = np.ascontiguousarray(arr, np.uint8)
            keep.append(a)
            plan = bern_degree_plan(BERN_DEG_PER_NEURON, 0, None,
                                    a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), cap, tau,
                                    budget)
        else:
            a = (ctypes.c_int * len(arr))(*[int(x) for x in arr])
            keep.append(a)
            plan = bern_degree_plan(BERN_DEG_PER_LAYER, 0, a, None, cap, tau, budget)
    plan.lin_every = int(lin)
    return plan, keep


def layer_degrees(widths, degree):
    H = len(widths) - 1
    if isinstance(degree, Learned):
        if degree.max_per_layer is not None:
            return list(degree.max_per_layer)
        return [max(BERN_DEGREE_CLASSES, degree.fallback)] * (H - 1)
    if isinstance(degree, (int, np.integer)):
        return [int(degree)] * (H - 1)
    arr = np.asarray(degree)
    if arr.dtype == np.uint8 or len(arr) == sum(widths[1:-1]) and len(arr) != H - 1:
        out, base = [], 0
        for h in widths[1:-1]:
            out.append(int(arr[base:base + h].max()))
            base += h
        return out
    return [int(x) for x in arr]


def max_output_terms(widths, degree, cap, lin: int = 0) -> int:
    """Worst-case term count of an output polynomial (the graded prefix of
    total degree min(prod d_i, cap); with Lin every lin-th hidden layer
    lowers the degree to min(n, D))."""
    n = int(widths[0])
    D = 1
    for i, d in enumerate(layer_degrees(widths, degree)):
        D = min(D * d, cap)
        if lin > 0 and (i + 1) % lin == 0:
            D = min(n, D)
    return num_monomials(n, D)
