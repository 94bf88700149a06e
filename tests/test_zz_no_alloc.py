"""The allocation-free entry point (bern_propagate_noalloc) against the
regular one (bern_propagate).

bern_propagate_noalloc exists for callers that may not allocate device
memory (a framework that owns all GPU memory, a loop where cudaMalloc is not
allowed): it keeps its workspace in a fixed device array inside the library.
This file is collected last; it must pass alone in a fresh process (the first
call does the per-device set-up) and after every other test."""
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


def _out(B, o, cap_terms):
    return {"lo": torch.empty(B, o, device="cuda"), "hi": torch.empty(B, o, device="cuda"),
            "n_terms": torch.empty(B, o, 2, dtype=torch.int32, device="cuda"),
            "coef": torch.zeros(B, o, 2, cap_terms, device="cuda")}


def _close(a, b):
    a = {k: v.cpu().numpy().astype(np.float64) for k, v in a.items()}
    b = {k: v.cpu().numpy().astype(np.float64) for k, v in b.items()}
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


@pytest.mark.parametrize("which", ["single_box_2in", "batch_3in_subset"])
def test_noalloc_matches_propagate_twice(which):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    if which == "single_box_2in":
        w = wl.single_box_2in()
        boxes = w.boxes
    else:
        w = wl.batch_3in()
        boxes = np.ascontiguousarray(w.boxes[::40])   # 128 boxes: several workspace chunks
    W, b = _dev(w.net)
    bx = torch.from_numpy(boxes).cuda()
    B, o = len(boxes), w.net.n_out
    cap_terms = bern.max_output_terms(w.net.widths, w.degree, w.degree_cap)
    ctx = bern.Context(0)
    want = ctx.propagate(w.net.widths, W, b, bx, degree=w.degree, cap=w.degree_cap,
                         cap_terms=cap_terms)
    want = {k: v for k, v in want.items() if v is not None}
    for _ in range(2):                      # two calls in a row share the static workspace
        got = _out(B, o, cap_terms)
        rc = bern.propagate_noalloc(w.net.widths, W, b, bx, got, degree=w.degree,
                                    cap=w.degree_cap)
        assert rc == bern.BERN_OK, bern.strerror(rc)
        _close(got, want)
    ctx.close()


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
