"""Lin linearisation (Sec. 5.3) through the C ABI against the FP64 oracle.

Reading R22: every Lin hidden layers each neuron's bounds become their
least-squares multilinear fit on the box plus the Bernstein enclosure of the
residual (max for the upper bound, min for the lower).  The oracle solves the
normal equations of the fit; the kernel uses the closed form in shifted
Legendre products, so agreement checks the two derivations against each
other.  Tolerances as in the whole-path parity tests: bounds within
1e-4 * (1 + |bound|), polynomials within 1e-4 * (1 + ||p||_1) in the sum of
absolute coefficient differences; plus Monte-Carlo soundness."""
import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import bern
from paper_2211_14438_gb300 import workloads as wl
from parity_util import dense_from_dict, eval_dense, graded, l1
from test_gpu_propagate import compare_box, mc_check, near_tie, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


def _multilinear_only(g, bi, j, n):
    for k in (0, 1):
        nt = int(g["n_terms"][bi, j, k])
        ex, _ = graded(n, n)
        assert nt <= len(ex)
        c = g["coef"][bi, j, k, :nt]
        assert np.all(c[ex[:nt].max(axis=1) > 1] == 0.0)


@pytest.mark.parametrize("lin", [1, 2])
def test_lin_single_box_2in(ctx, lin):
    w = wl.single_box_2in()
    g = run_gpu(ctx, w.net, w.boxes, lin=lin)
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2, lin=lin)
    assert not near_tie(r)
    compare_box(g, 0, r, 2, 1)
    assert mc_check(g, 0, w.net, w.boxes[0], 200_000, np.random.default_rng(3)) == 0
    if lin == 1:
        # the last hidden layer was linearised: the output bounds are multilinear
        _multilinear_only(g, 0, 0, 2)


@pytest.mark.parametrize("lin", [1, 2])
def test_lin_single_box_4in(ctx, lin):
    w = wl.single_box_4in()
    g = run_gpu(ctx, w.net, w.boxes, lin=lin)
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2, lin=lin)
    assert not near_tie(r)
    compare_box(g, 0, r, 4, 2)
    assert mc_check(g, 0, w.net, w.boxes[0], 100_000, np.random.default_rng(4)) == 0


@pytest.mark.parametrize("lin,count", [(1, 16), (2, 4), (3, 16)])
def test_lin_batch_3in_subset(ctx, lin, count):
    """Grid-cell and random boxes of the [3,64x4,1] net, all in one call."""
    w = wl.batch_3in(n_random=8, cells=2)
    boxes = w.boxes[:count] if count == 16 else w.boxes[::4][:count]
    g = run_gpu(ctx, w.net, boxes, lin=lin)
    rng = np.random.default_rng(5)
    for bi in range(len(boxes)):
        r = oracle.propagate(w.net.widths, w.net.W, w.net.b, boxes[bi], 2, lin=lin)
        if not near_tie(r):
            compare_box(g, bi, r, 3, 1)
        assert mc_check(g, bi, w.net, boxes[bi], 20_000, rng) == 0


@pytest.mark.parametrize("lin", [1, 2])
def test_lin_paper_deep_net(ctx, lin):
    """The paper's deepest ablation shape (Fig. 7: [2,20x5,1], W and b
    U(-5,5)) on [-1,1]^2 at cap 64: without Lin its output degree is 32, with
    it at most 4."""
    net = wl.paper_net(2, [20] * 5, seed=522)
    box = wl.box_array([-1.0, -1.0], [1.0, 1.0])
    g = run_gpu(ctx, net, box[None], cap=64, lin=lin)
    r = oracle.propagate(net.widths, net.W, net.b, box, 2, cap=64, lin=lin)
    assert not near_tie(r)
    compare_box(g, 0, r, 2, 1)
    assert mc_check(g, 0, net, box, 100_000, np.random.default_rng(6)) == 0


@pytest.mark.parametrize("widths", [[6, 10, 10, 1], [8, 6, 6, 1]])
def test_lin_many_inputs(ctx, widths):
    """Six and eight inputs: 64 and 256 variable sets in the fit (more sets
    than lanes), and with eight inputs Bernstein grids above the library's
    limit, lowered by the budget rule on both sides."""
    n = widths[0]
    net = wl.make_net(widths, seed=40 + n)
    box = wl.box_array([-0.5] * n, [0.5] * n)
    budget = 1 << 20              # the plans' default budget
    g = run_gpu(ctx, net, box[None], lin=1)
    r = oracle.propagate(net.widths, net.W, net.b, box, 2, lin=1, budget=budget)
    if not near_tie(r):
        compare_box(g, 0, r, n, 1)
    assert mc_check(g, 0, net, box, 50_000, np.random.default_rng(n)) == 0


def test_lin_beyond_depth_is_the_plain_method(ctx):
    w = wl.batch_3in(n_random=8, cells=2)
    a = run_gpu(ctx, w.net, w.boxes)
    b = run_gpu(ctx, w.net, w.boxes, lin=9)
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])


def test_lin_graph_replay_is_stable(ctx):
    w = wl.batch_3in(n_random=8, cells=2)
    a = run_gpu(ctx, w.net, w.boxes, lin=2)
    b = run_gpu(ctx, w.net, w.boxes, lin=2)
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])
    assert np.array_equal(a["coef"], b["coef"])


def test_lin_rejects_negative(ctx):
    w = wl.single_box_2in()
    with pytest.raises(bern.BernError):
        run_gpu(ctx, w.net, w.boxes, lin=-1)


def test_linearize_step_matches_oracle(ctx):
    """bern_linearize on a layer block of random polynomials (full and short
    graded prefixes, and an empty one) against the oracle's Lin step."""
    n, D, order, h, B = 3, 4, 4, 8, 3
    ld = bern.num_monomials(n, D)                 # 35
    lin_ld = bern.num_monomials(n, min(n, order))  # 20
    rng = np.random.default_rng(11)
    up = rng.normal(0, 1, (B, ld, h)).astype(np.float32)
    lo = (up - np.abs(rng.normal(0, 0.1, (B, ld, h)))).astype(np.float32)
    nt = np.full((B, h), ld, np.int32)
    nt[0, 1] = bern.num_monomials(n, 2)
    nt[1, 2] = bern.num_monomials(n, 1)
    nt[2, 3] = 0
    dev = torch.device("cuda", 0)
    t_up, t_lo = torch.from_numpy(up).to(dev), torch.from_numpy(lo).to(dev)
    t_nt = torch.from_numpy(nt).to(dev)
    l_up = torch.zeros(B, lin_ld, h, device=dev)
    l_lo = torch.zeros(B, lin_ld, h, device=dev)
    l_nt = torch.zeros(B, h, dtype=torch.int32, device=dev)
    r_lo = torch.zeros(B, h, device=dev)
    r_hi = torch.zeros(B, h, device=dev)
    ctx.linearize(n, B, h, order, 0, t_up, t_lo, ld, t_nt, l_up, l_lo, lin_ld, l_nt, r_lo, r_hi)
    ctx.check("bern_linearize")
    L_up, L_lo = l_up.cpu().numpy(), l_lo.cpu().numpy()
    R_up, R_lo = t_up.cpu().numpy(), t_lo.cpu().numpy()
    L_nt = l_nt.cpu().numpy()
    ex, _ = graded(n, D)
    pts = rng.random((4000, n))
    for b in range(B):
        for m in range(h):
            k = int(nt[b, m])
            assert L_nt[b, m] == min(k, lin_ld)
            if k == 0:
                continue
            kl = int(L_nt[b, m])
            for src, res, lin, upper in ((up, R_up, L_up, True), (lo, R_lo, L_lo, False)):
                p = {tuple(int(x) for x in ex[r]): float(src[b, r, m]) for r in range(k)}
                want = dense_from_dict(oracle.linearize(oracle.as_poly(p, n), n, order, upper),
                                       n, kl)
                got = lin[b, :kl, m].astype(np.float64)
                assert np.abs(got - want).sum() <= TOL * (1 + l1(want)), (b, m, upper)
                # residual + fit reproduces the input (the fit without its shift)
                fit = got.copy()
                fit[0] = 0.0
                back = res[b, :k, m].astype(np.float64)
                back[:kl] += fit
                orig = src[b, :k, m].astype(np.float64)
                scale = 1 + max(np.abs(orig).max(), np.abs(fit).max())
                assert np.abs(back[1:] - orig[1:]).max() <= 1e-5 * scale
                # soundness against the float32 input, evaluated in float64
                pv = eval_dense(orig, n, pts)
                lv = eval_dense(got, n, pts)
                e = 1e-9 * (1 + l1(orig) + l1(got))
                if upper:
                    assert np.all(lv >= pv - e)
                else:
                    assert np.all(lv <= pv + e)
