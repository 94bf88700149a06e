"""The allocation-free entry point (bern_propagate_noalloc) against the
regular one (bern_propagate).

bern_propagate_noalloc exists for callers that may not allocate device
memory (a framework that owns all GPU memory, a loop where cudaMalloc is not
allowed): it keeps its workspace in a fixed device array inside the library.
This file is collected last; it must pass alone in a fresh process (the first
call does the per-device set-up) and after every other test.

The comparison is within the parity tolerance, not bit for bit: the
allocation-free path always runs the per-step kernels, while bern_propagate
may run other kernels for the same plan, whose sums can be ordered
differently (every sum is rounded outward, so both results are sound)."""
import time

import numpy as np
import pytest

from paper_2211_14438_gb300 import bern
from paper_2211_14438_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-4      # the whole-path tolerance of the parity tests


def _dev(net):
    return ([torch.from_numpy(w).cuda() for w in net.W],
            [torch.from_numpy(x).cuda() for x in net.b])


def _out(B, o, cap_terms, keys=False):
    return {"lo": torch.empty(B, o, device="cuda"), "hi": torch.empty(B, o, device="cuda"),
            "n_terms": torch.empty(B, o, 2, dtype=torch.int32, device="cuda"),
            "coef": torch.zeros(B, o, 2, cap_terms, device="cuda"),
            "keys": (torch.zeros(B, o, 2, cap_terms, dtype=torch.int64, device="cuda")
                     if keys else None)}


def _close(a, b):
    if a.get("keys") is not None:
        ka, kb, nt = a["keys"].cpu().numpy(), b["keys"].cpu().numpy(), b["n_terms"].cpu().numpy()
        for i, j, s in np.ndindex(*nt.shape):
            assert np.array_equal(ka[i, j, s, :nt[i, j, s]], kb[i, j, s, :nt[i, j, s]])
    a = {k: v.cpu().numpy().astype(np.float64) for k, v in a.items() if k != "keys" and v is not None}
    b = {k: v.cpu().numpy().astype(np.float64) for k, v in b.items() if k != "keys" and v is not None}
    assert np.array_equal(a["n_terms"], b["n_terms"])
    for k in ("lo", "hi"):
        assert np.all(np.abs(a[k] - b[k]) <= TOL * (1 + np.abs(b[k])))
    B, o = a["lo"].shape
    for i in range(B):
        for j in range(o):
            for s in range(2):
                nt = int(b["n_terms"][i, j, s])
                d = np.abs(a["coef"][i, j, s, :nt] - b["coef"][i, j, s, :nt]).sum()
                assert d <= TOL * (1 + np.abs(b["coef"][i, j, s, :nt]).sum())


@pytest.mark.parametrize("which", ["single_box_2in", "batch_3in_subset",
                                   "batch_3in_per_layer_keys"])
def test_noalloc_matches_propagate_twice(which):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    keys = which == "batch_3in_per_layer_keys"
    if which == "single_box_2in":
        w = wl.single_box_2in()
        boxes = w.boxes
        degree = w.degree
    else:
        w = wl.batch_3in()
        boxes = np.ascontiguousarray(w.boxes[::40])   # 128 boxes: several workspace chunks
        degree = [2, 1, 2, 2] if keys else w.degree
    W, b = _dev(w.net)
    bx = torch.from_numpy(boxes).cuda()
    B, o = len(boxes), w.net.n_out
    cap_terms = bern.max_output_terms(w.net.widths, degree, w.degree_cap)
    ctx = bern.Context(0)
    want = ctx.propagate(w.net.widths, W, b, bx, degree=degree, cap=w.degree_cap,
                         cap_terms=cap_terms, keys=keys)
    want = {k: v for k, v in want.items() if v is not None}
    for call in range(2):                   # two calls in a row share the static workspace
        got = _out(B, o, cap_terms, keys)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = bern.propagate_noalloc(w.net.widths, W, b, bx, got, degree=degree,
                                    cap=w.degree_cap)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert rc == bern.BERN_OK, bern.strerror(rc)
        # once the library's device image is loaded (lazily, on the first call
        # in a process: it holds the fixed arrays), a call allocates nothing
        if call > 0:
            assert free1 == free0, (call, free0, free1)
        _close(got, want)
    ctx.close()


def test_noalloc_rejects_oversized_tables_fast():
    """A narrow six-input net whose last hidden layer squares degree-15
    polynomials (54,264 terms, ~1.5e9 square pairs) has a small per-box
    workspace but tables far beyond the static table area: rejected from the
    plan alone, before any table is built."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    widths = [6, 2, 2, 2, 2, 2, 1]
    W = [torch.full((widths[i + 1], widths[i]), 0.1, device="cuda") for i in range(6)]
    b = [torch.zeros(widths[i + 1], device="cuda") for i in range(6)]
    bx = torch.from_numpy(wl.box_array([-1] * 6, [1] * 6)[None]).cuda()
    out = _out(1, 1, 16)
    t0 = time.perf_counter()
    rc = bern.propagate_noalloc(widths, W, b, bx, out, degree=2, cap=15)
    assert rc == bern.BERN_E_UNSUPPORTED
    assert time.perf_counter() - t0 < 1.0


def test_noalloc_rejects_oversized_network():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    widths = [6, 2000, 2000, 2000, 1]     # layer-3 polynomials need ~48 MB per box
    W = [torch.zeros(widths[i + 1], widths[i], device="cuda") for i in range(4)]
    b = [torch.zeros(widths[i + 1], device="cuda") for i in range(4)]
    bx = torch.from_numpy(wl.box_array([-1] * 6, [1] * 6)[None]).cuda()
    out = _out(1, 1, 16)
    rc = bern.propagate_noalloc(widths, W, b, bx, out, degree=2, cap=16)
    assert rc == bern.BERN_E_UNSUPPORTED


def test_noalloc_rejects_horner_plans():
    """Orders >= 3 and pruning need the Horner product tables, which the
    static table area does not hold: rejected before any GPU work."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    w = wl.single_box_2in()
    W = [torch.from_numpy(x).cuda() for x in w.net.W]
    b = [torch.from_numpy(x).cuda() for x in w.net.b]
    bx = torch.from_numpy(w.boxes).cuda()
    out = _out(1, 1, 256)
    assert bern.propagate_noalloc(w.net.widths, W, b, bx, out, degree=3, cap=16) == \
        bern.BERN_E_UNSUPPORTED
    assert bern.propagate_noalloc(w.net.widths, W, b, bx, out, degree=2, cap=16, tau=1e-3) == \
        bern.BERN_E_UNSUPPORTED
