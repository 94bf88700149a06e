"""bern_poly_to_x (output polynomials in the input coordinates x) against the
oracle's float64 binomial expansion of the same t-polynomials, its outward
constant terms, Monte-Carlo soundness of the converted bounds in x, a box
with a zero-width side, and the term-count check.

Tolerances follow the kernel's own bound.  With E_J the sum of the
magnitudes of the terms behind coefficient J (from the oracle) and
g = 2 (n (4D + 3) + nt + 4) 2^-53, each coefficient but the constant lies
within 2^-24 |e_J| + 2 g E_J of the oracle's; the constant is outward (>= the
oracle's for an upper polynomial, <= for a lower one) by at most twice
R = sum_{J != 0} (2^-24 |e_J| + g E_J) X^J + g E_0, X_i = max |x_i| on the
box, plus one float ulp of its own directed rounding.  In x the monomial basis is badly conditioned on small boxes far from
the origin (E_J can exceed |e_J| by many orders), which R reflects."""
import numpy as np
import pytest

import oracle
from oracle import poly_x
from paper_2211_14438_gb300 import bern
from paper_2211_14438_gb300 import workloads as wl
from parity_util import dict_from_dense, graded
from test_gpu_propagate import run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


def lib_w(box):
    """The library's side lengths: dhi - dlo in float32, rounded up."""
    lo = box[:, 0].astype(np.float32)
    w = box[:, 1].astype(np.float64) - lo.astype(np.float64)
    wf = w.astype(np.float32)
    return np.where(wf.astype(np.float64) < w, np.nextafter(wf, np.float32(np.inf)), wf)


def exps_of(n, nt):
    """Exponents of the first nt monomials of the graded order."""
    D = 0
    while bern.num_monomials(n, D) < nt:
        D += 1
    ex, _ = graded(n, D)
    return ex[:nt]


def convert(ctx, boxes, g):
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = ctx.poly_to_x(dev(boxes), dev(g["n_terms"]), dev(g["coef"]))
    assert ctx.sync() == 0
    return out.cpu().numpy().astype(np.float64)


def check_box(net, box, g, cx, bi, rng, n_mc=4000):
    n, o = net.n_in, net.n_out
    dlo = box[:, 0].astype(np.float32).astype(np.float64)
    w = lib_w(box).astype(np.float64)
    X = np.maximum(np.abs(box[:, 0]), np.abs(box[:, 1])).astype(np.float64)
    x = box[:, 0] + rng.random((n_mc, n)) * (box[:, 1] - box[:, 0])
    x = np.vstack([x, box[:, 0], box[:, 1]]).astype(np.float64)
    nn = oracle.network_forward(net.widths, net.W, net.b, x)
    for j in range(o):
        for k in (0, 1):
            nt = int(g["n_terms"][bi, j, k])
            pt = dict_from_dense(g["coef"][bi, j, k, :nt].astype(np.float64), n)
            e, E = poly_x.poly_to_x(pt, dlo, w, magnitudes=True)
            exps = exps_of(n, nt)
            D = int(max(sum(int(v) for v in ex) for ex in exps))
            gam = 2.0 * (n * (4 * D + 3) + nt + 4) * 2.0 ** -53
            R = gam * E.get((0,) * n, 0.0)
            for r in range(1, nt):
                J = tuple(int(v) for v in exps[r])
                want, EJ = e.get(J, 0.0), E.get(J, 0.0)
                assert abs(cx[bi, j, k, r] - want) <= 2.0 ** -24 * abs(want) + 2 * gam * EJ
                R += (2.0 ** -24 * abs(want) + gam * EJ) * np.prod(X ** np.asarray(J, np.float64))
            e0 = e.get((0,) * n, 0.0)
            c0 = cx[bi, j, k, 0]
            ulp = 2.0 ** -23 * abs(c0) + 1e-44            # the constant's directed rounding
            if k == 0:
                assert c0 >= e0 and c0 - e0 <= 2 * R + ulp
            else:
                assert c0 <= e0 and e0 - c0 <= 2 * R + ulp
            mag = sum(abs(v) * np.prod(X ** np.asarray(J, np.float64)) for J, v in e.items())
            px = {tuple(int(v) for v in exps[r]): cx[bi, j, k, r] for r in range(nt)}
            vals = poly_x.eval_x(px, x)
            tol = 1e-9 * (1 + mag + np.abs(nn[:, j]))
            if k == 0:
                assert np.all(nn[:, j] <= vals + tol)
            else:
                assert np.all(nn[:, j] >= vals - tol)


def test_batch_3in_boxes(ctx):
    w = wl.batch_3in(n_random=8, cells=2)
    g = run_gpu(ctx, w.net, w.boxes)
    cx = convert(ctx, w.boxes, g)
    rng = np.random.default_rng(3)
    for bi in range(0, len(w.boxes), 2):
        check_box(w.net, w.boxes[bi], g, cx, bi, rng)


def test_single_box_2in_and_orders(ctx):
    w = wl.single_box_2in()
    for d in (1, 2, 3):
        g = run_gpu(ctx, w.net, w.boxes, degree=d)
        cx = convert(ctx, w.boxes, g)
        check_box(w.net, w.boxes[0], g, cx, 0, np.random.default_rng(d))


def test_zero_width_side(ctx):
    net = wl.make_net([3, 12, 12, 2], 61)
    boxes = wl.box_array(np.array([[-0.4, 0.3, 0.1], [0.2, -0.5, 0.7]]),
                         np.array([[0.1, 0.3, 0.6], [0.2, 0.1, 0.9]]))
    g = run_gpu(ctx, net, boxes)
    cx = convert(ctx, boxes, g)
    rng = np.random.default_rng(61)
    for bi in range(len(boxes)):
        check_box(net, boxes[bi], g, cx, bi, rng)


def test_term_count_above_capacity_is_reported(ctx):
    w = wl.single_box_2in()
    g = run_gpu(ctx, w.net, w.boxes)
    nt = g["n_terms"].copy()
    nt[0, 0, 0] = g["coef"].shape[3] + 1
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx.poly_to_x(dev(w.boxes), dev(nt), dev(g["coef"]))
    assert ctx.sync() == bern.BERN_E_INVALID
    assert ctx.sync() == 0
