"""Learned degree plans (BERN_DEG_LEARNED) through bern_propagate: the GPU's
run-time order proposals and the bounds they lead to against the oracle's
propagation driven by the oracle MLP (same seeded weights, bf16-emulated), the
degenerate proposal rules against the plain plans they reduce to (bit for
bit), and Monte-Carlo soundness whatever the MLP proposes.

A box whose oracle decisions include a near-tie (two class probabilities, or
the largest one and min_conf, within 1e-3) may legitimately take another
order in float32; it is checked for soundness only."""
import numpy as np
import pytest

import oracle
from oracle import mlp as om
from paper_2211_14438_gb300 import bern
from paper_2211_14438_gb300 import workloads as wl
from test_gpu_propagate import compare_box, mc_check, near_tie, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

F, C = bern.BERN_DEGREE_FEATURES, bern.BERN_DEGREE_CLASSES


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


def random_theta(seed, scale=1.0):
    return (np.random.default_rng(seed).normal(0, scale, om.num_params(F, C))).astype(np.float32)


def const_theta(cls):
    """Zero weights and a bias that makes class `cls` the sure winner."""
    th = np.zeros(om.num_params(F, C), np.float32)
    th[-C + cls] = 10.0
    return th


@pytest.mark.parametrize("widths,seed,tseed", [([2, 20, 20, 1], 0, 1), ([3, 10, 10, 2], 22, 2),
                                               ([2, 8, 8, 8, 1], 23, 3)])
def test_learned_plan_matches_oracle(ctx, widths, seed, tseed):
    net = wl.make_net(widths, seed)
    rng = np.random.default_rng(seed)
    n = widths[0]
    c = rng.uniform(-1, 1, (4, n))
    s = rng.uniform(0.2, 1.5, (4, n))
    boxes = wl.box_array(c - s / 2, c + s / 2)
    theta = random_theta(tseed, 0.8)
    m = bern.Mlp(torch, F, C, theta)
    plan = bern.Learned(m, min_conf=0.0, fallback=2)
    g = run_gpu(ctx, net, boxes, degree=plan)
    checked = 0
    for bi in range(len(boxes)):
        ch = om.DegreeChooser(theta, 0.0, 2)
        r = oracle.propagate(widths, net.W, net.b, boxes[bi], ch,
                             budget=1 << 20)
        if ch.margin > 1e-3 and not near_tie(r):
            compare_box(g, bi, r, n, widths[-1])
            checked += 1
        assert mc_check(g, bi, net, boxes[bi], 20_000, rng) == 0
    assert checked >= 2


def run_per_step(ctx, *a, **kw):
    """The plain plan through the per-step kernels (the default; learned plans
    always run them, while the fused layer kernels order the output layer's
    sums differently)."""
    ctx.set_fused(False)
    return run_gpu(ctx, *a, **kw)


@pytest.mark.parametrize("cls", [0, 1, 2, 3])
def test_sure_proposal_equals_global_plan(ctx, cls):
    """An MLP that always proposes order cls+1 gives exactly the global plan
    (both through the per-step kernels, which learned plans always use: the
    fused layer kernels order the output layer's sums differently)."""
    w = wl.batch_3in(n_random=8, cells=2)
    m = bern.Mlp(torch, F, C, const_theta(cls))
    a = run_gpu(ctx, w.net, w.boxes, degree=bern.Learned(m), cap=16)
    b = run_per_step(ctx, w.net, w.boxes, degree=cls + 1, cap=16)
    for k in ("lo", "hi", "n_terms"):
        assert np.array_equal(a[k], b[k]), k
    for bi in range(len(w.boxes)):
        nt = b["n_terms"][bi, 0, 0]
        assert np.array_equal(a["coef"][bi, 0, :, :nt], b["coef"][bi, 0, :, :nt])


def test_low_confidence_falls_back_to_plain(ctx):
    w = wl.batch_3in(n_random=8, cells=2)
    m = bern.Mlp(torch, F, C, random_theta(5))
    a = run_gpu(ctx, w.net, w.boxes, degree=bern.Learned(m, min_conf=1.01, fallback=2))
    b = run_per_step(ctx, w.net, w.boxes, degree=2)
    for k in ("lo", "hi", "n_terms"):
        assert np.array_equal(a[k], b[k]), k


def test_any_proposal_is_sound(ctx):
    """Random MLPs propose arbitrary mixed orders: the bounds stay sound."""
    w = wl.batch_3in(n_random=24, cells=2)
    rng = np.random.default_rng(7)
    for seed in (11, 12):
        m = bern.Mlp(torch, F, C, random_theta(seed, 2.0))
        g = run_gpu(ctx, w.net, w.boxes, degree=bern.Learned(m))
        assert np.all(g["lo"] <= g["hi"])
        for bi in range(0, len(w.boxes), 4):
            assert mc_check(g, bi, w.net, w.boxes[bi], 5_000, rng) == 0


def test_trained_mlp_gains_over_plain(ctx):
    """The learned component trained on the GPU (labels from plain-method
    widths on the training boxes) against the plain method on held-out boxes
    of the benchmark's distribution: no looser on average (1% slack for the
    held-out generalisation) and much less polynomial work (the term counts
    every hidden layer and the output carry)."""
    from paper_2211_14438_gb300 import learned as lm
    w = wl.batch_3in()
    net = w.net
    held = w.boxes[np.r_[0:4096:8, 4096:5120:2]]         # 512 grid cells + 512 random
    info = lm.fit(ctx, net.widths, net.W, net.b, wl.batch_3in_training_boxes(800), cap=16)
    assert info["n_samples"] >= 200_000
    plan = info["plan"]
    gp = run_gpu(ctx, net, held, degree=2, trace=True)
    gl = run_gpu(ctx, net, held, degree=plan, trace=True)
    wp = float(np.mean(gp["hi"] - gp["lo"]))
    wlr = float(np.mean(gl["hi"] - gl["lo"]))
    assert wlr <= 1.01 * wp, (wlr, wp)
    work = lambda g: float(g["tr_nterms"].astype(np.int64).sum() + g["n_terms"].sum())
    assert work(gl) < 0.8 * work(gp), (work(gl), work(gp))
    # the proposals actually vary, and every bound is sound on a sample of boxes
    assert len(np.unique(gl["tr_degree"])) >= 2
    rng = np.random.default_rng(17)
    for bi in range(0, len(held), 64):
        assert mc_check(gl, bi, net, held[bi], 5_000, rng) == 0


def test_per_layer_caps_clamp_proposals(ctx):
    """With per-layer caps the proposals are clamped: an MLP sure of order 4
    under caps of 2 everywhere gives exactly the order-2 plan, and caps
    (4, 1, 1, 1) give the per-layer plan (4, 1, 1, 1)."""
    w = wl.batch_3in(n_random=8, cells=2)
    m = bern.Mlp(torch, F, C, const_theta(3))
    a = run_gpu(ctx, w.net, w.boxes, degree=bern.Learned(m, max_per_layer=[2, 2, 2, 2]))
    b = run_per_step(ctx, w.net, w.boxes, degree=2)
    for k in ("lo", "hi", "n_terms"):
        assert np.array_equal(a[k], b[k]), k
    a = run_gpu(ctx, w.net, w.boxes, degree=bern.Learned(m, max_per_layer=[4, 1, 1, 1]))
    b = run_per_step(ctx, w.net, w.boxes, degree=[4, 1, 1, 1])
    for k in ("lo", "hi", "n_terms"):
        assert np.array_equal(a[k], b[k]), k
