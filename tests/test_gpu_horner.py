"""Composition by Horner's rule on the GPU (ReLU orders 3 to 16 in float32
below order 6 and float64 from there, mixed per-layer and per-neuron orders,
degree-cap truncation and pruning) against the FP64 oracle, plus Monte-Carlo
soundness.  Same tolerances as the other
whole-path tests: bounds within 1e-4 * (1 + |bound|), polynomials within
1e-4 * (1 + ||p||_1) in summed absolute coefficient difference."""
import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import bern
from paper_2211_14438_gb300 import workloads as wl
from parity_util import dense_from_dict, l1
from test_gpu_propagate import compare_box, mc_check, near_tie, run_gpu

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


def random_boxes(n, k, seed, lo=0.05, hi=1.0):
    rng = np.random.default_rng(seed)
    c = rng.uniform(-1, 1, (k, n))
    s = rng.uniform(lo, hi, (k, n))
    return wl.box_array(c - s / 2, c + s / 2)


def check_all(ctx, net, boxes, degree, cap=16, tau=0.0, mc=20_000, seed=0):
    g = run_gpu(ctx, net, boxes, degree=degree, cap=cap, tau=tau)
    widths = net.widths
    if isinstance(degree, (int, np.integer)):
        degs = int(degree)
    else:
        arr = np.asarray(degree)
        if len(arr) == len(widths) - 2 and arr.dtype != np.uint8:
            degs = np.concatenate([np.full(h, d) for h, d in zip(widths[1:-1], arr)])
        else:
            degs = arr.astype(np.int64)
    rng = np.random.default_rng(seed)
    checked = 0
    for bi in range(len(boxes)):
        r = oracle.propagate(widths, net.W, net.b, boxes[bi], degs, cap=cap, tau=tau,
                             budget=1 << 20)
        if not near_tie(r):
            compare_box(g, bi, r, widths[0], widths[-1])
            checked += 1
        assert mc_check(g, bi, net, boxes[bi], mc, rng) == 0
    assert checked >= max(1, len(boxes) - 1)
    return g


@pytest.mark.parametrize("d", [3, 4, 5])
def test_single_box_2in_orders_above_two(ctx, d):
    w = wl.single_box_2in()
    check_all(ctx, w.net, w.boxes, d, mc=200_000, seed=d)


def test_order8_single_composition_parity(ctx):
    """Order 8 with one hidden layer (the degree cap truncates nothing):
    parity with the oracle and Monte-Carlo soundness."""
    net = wl.make_net([2, 12, 1], 51)
    check_all(ctx, net, random_boxes(2, 4, 51, 0.2, 1.0), 8, cap=16, seed=51)


@pytest.mark.parametrize("widths,d,cap,seed", [([2, 12, 1], 12, 16, 52), ([2, 12, 1], 9, 16, 62),
                                               ([3, 8, 2], 12, 16, 60), ([3, 6, 2], 10, 16, 63),
                                               ([2, 8, 8, 1], 6, 16, 56), ([3, 6, 6, 1], 6, 16, 58)])
def test_orders_above_5_parity(ctx, widths, d, cap, seed):
    """Orders 6 to 12 compose in float64 (the power-form coefficients of the
    order-d ReLU polynomial grow like C(d, d/2) 2^(d/2) (hi - lo) / d, far
    beyond what float32 rounding of the intermediate polynomials tolerates):
    parity with the oracle at the whole-path tolerance, on one composition up
    to order 12 and on two compositions at order 6, and Monte-Carlo
    soundness."""
    net = wl.make_net(widths, seed)
    check_all(ctx, net, random_boxes(widths[0], 4, seed, 0.2, 1.0), d, cap=cap, mc=50_000,
              seed=seed)


@pytest.mark.parametrize("widths,seed", [([2, 12, 1], 53), ([3, 8, 2], 55)])
def test_order16_parity(ctx, widths, seed):
    """Order 16 (the top of Fig. 1's range) on one composition.  The composed
    polynomials have l1 norms of 3e2 to 9e3 in the power basis of t for
    bounds of about 0.2, so their float32 storage alone (u = 2^-24 per
    coefficient) moves a bound by up to u ||p||_1 -- more than 1e-4.  The
    tolerance adds 16 u ||p||_1 (p the oracle's output polynomial of that
    side) to the whole-path one: one rounding of every stored coefficient,
    the affine step's product and sum, and the enclosure's per-variable
    transforms, each at most a few u of the coefficient magnitudes."""
    net = wl.make_net(widths, seed)
    boxes = random_boxes(widths[0], 4, seed, 0.2, 1.0)
    g = run_gpu(ctx, net, boxes, degree=16, cap=16)
    rng = np.random.default_rng(seed)
    M = bern.num_monomials(widths[0], 16)
    for bi in range(len(boxes)):
        r = oracle.propagate(widths, net.W, net.b, boxes[bi], 16, cap=16, budget=1 << 20)
        for j in range(widths[-1]):
            for key, name in (("hi", "upper"), ("lo", "lower")):
                nrm = l1(dense_from_dict(r[name][j], widths[0], M))
                dv = abs(float(g[key][bi, j]) - r[key][j])
                assert dv <= 1e-4 * (1 + abs(r[key][j])) + 16 * 2.0 ** -24 * nrm, (bi, j, key)
        assert mc_check(g, bi, net, boxes[bi], 50_000, rng) == 0


@pytest.mark.parametrize("widths,d,cap,seed", [([1, 6, 6, 1], 8, 64, 54), ([2, 8, 8, 1], 7, 16, 57),
                                               ([3, 6, 6, 1], 10, 16, 58),
                                               ([2, 6, 6, 1], 12, 24, 61)])
def test_two_compositions_high_orders_sound(ctx, widths, d, cap, seed):
    """Two compositions above order 6: the first layer's composed polynomials
    (l1 norms up to 1e12 in the power basis of t) are stored in float32 and
    composed again, which multiplies their rounding by the coefficient size
    of B'(s(t)); the bounds (|bound| of 1e5 to 1e14 in the oracle too, from
    the truncated remainders) stay sound and finite but do not reach the
    oracle's within 1e-4."""
    net = wl.make_net(widths, seed)
    boxes = random_boxes(widths[0], 4, seed, 0.2, 1.0)
    g = run_gpu(ctx, net, boxes, degree=d, cap=cap)
    rng = np.random.default_rng(seed)
    assert np.all(np.isfinite(g["lo"])) and np.all(g["lo"] <= g["hi"])
    for bi in range(len(boxes)):
        assert mc_check(g, bi, net, boxes[bi], 50_000, rng) == 0


def test_single_box_2in_order8_two_layers_parity(ctx):
    """Two hidden layers of 20 at order 8 with cap 16 (the truncated
    remainders make the bounds loose in both the oracle and the GPU path):
    parity and soundness; at order 16 the same net stays sound."""
    w = wl.single_box_2in()
    g = run_gpu(ctx, w.net, w.boxes, degree=8, cap=16)
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 8, cap=16, budget=1 << 20)
    assert not near_tie(r)
    compare_box(g, 0, r, 2, 1)
    assert mc_check(g, 0, w.net, w.boxes[0], 200_000, np.random.default_rng(8)) == 0
    g = run_gpu(ctx, w.net, w.boxes, degree=16, cap=16)
    assert np.all(np.isfinite(g["lo"])) and np.all(g["lo"] <= g["hi"])
    assert mc_check(g, 0, w.net, w.boxes[0], 200_000, np.random.default_rng(16)) == 0


def test_per_neuron_orders_both_precisions(ctx):
    """Per-neuron orders 3..10 in one layer: items below order 6 run the
    float32 Horner kernel and the rest the float64 one in the same call;
    parity with the oracle and soundness."""
    widths = [2, 10, 10, 1]
    net = wl.make_net(widths, 59)
    degs = np.random.default_rng(59).integers(3, 11, sum(widths[1:-1])).astype(np.uint8)
    assert degs.min() < 6 <= degs.max()
    check_all(ctx, net, random_boxes(2, 4, 59, 0.3, 1.2), degs, mc=50_000, seed=59)


@pytest.mark.parametrize("d", [6, 12])
def test_global_workspace_path_matches_shared_f64(ctx, d):
    """The float64 Horner kernel computes the same bits with its buffers in
    the global workspace as in shared memory."""
    widths = [3, 8, 8, 1]
    net = wl.make_net(widths, 92)
    boxes = random_boxes(3, 3, 92, 0.3, 1.2)
    a = run_gpu(ctx, net, boxes, degree=d)
    ctx.set_horner_smem_limit(0)
    try:
        b = run_gpu(ctx, net, boxes, degree=d)
    finally:
        ctx.set_horner_smem_limit(200 * 1024)
    for k in ("lo", "hi", "n_terms", "coef"):
        assert np.array_equal(a[k], b[k]), k


@pytest.mark.parametrize("widths,degree,seed", [
    ([2, 6, 5, 3], [3, 2], 21), ([3, 10, 10, 2], [1, 4], 22), ([1, 8, 8, 1], 4, 23),
    ([4, 8, 8, 1], [2, 3], 24), ([3, 7, 6, 5, 1], [3, 3, 2], 25)])
def test_per_layer_orders(ctx, widths, degree, seed):
    net = wl.make_net(widths, seed)
    check_all(ctx, net, random_boxes(widths[0], 4, seed), degree, seed=seed)


def test_per_neuron_orders(ctx):
    widths = [2, 8, 8, 1]
    net = wl.make_net(widths, 31)
    degs = np.random.default_rng(31).integers(1, 5, sum(widths[1:-1])).astype(np.uint8)
    check_all(ctx, net, random_boxes(2, 4, 31, 0.3, 1.5), degs, seed=31)


@pytest.mark.parametrize("cap", [3, 5, 7])
def test_degree_cap_truncation_with_horner(ctx, cap):
    """Low caps force truncation (and remainder carrying) inside Horner."""
    widths = [2, 6, 6, 1]
    net = wl.make_net(widths, 41)
    check_all(ctx, net, random_boxes(2, 4, 41, 0.5, 2.0), 3, cap=cap, seed=cap)


@pytest.mark.parametrize("tau,degree", [(1e-3, 2), (1e-2, 2), (1e-3, 3), (3e-3, 1)])
def test_pruning(ctx, tau, degree):
    widths = [3, 10, 10, 2]
    net = wl.make_net(widths, 51)
    boxes = random_boxes(3, 4, 51, 0.3, 1.5)
    g = check_all(ctx, net, boxes, degree, tau=tau, seed=52)
    # pruning only ever removes terms: term counts never exceed the unpruned ones
    g0 = run_gpu(ctx, net, boxes, degree=degree)
    assert np.all(g["n_terms"] <= g0["n_terms"])


def test_pruning_shrinks_terms_on_small_boxes(ctx):
    """On small boxes the high-degree terms are tiny and pruning drops whole
    degrees: the term count falls below the unpruned graded prefix."""
    w = wl.batch_3in()
    idx = np.arange(0, 4096, 512)
    g0 = run_gpu(ctx, w.net, w.boxes[idx])
    g = run_gpu(ctx, w.net, w.boxes[idx], tau=1e-4)
    assert np.all(g["n_terms"] <= g0["n_terms"])
    assert np.any(g["n_terms"] < g0["n_terms"])
    for k, bi in enumerate(idx):
        r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[bi], 2, tau=1e-4)
        if not near_tie(r):
            compare_box(g, k, r, 3, 1)


@pytest.mark.parametrize("d", [3, 12])
def test_step_compose_matches_oracle(ctx, d):
    """bern_compose (step ABI) on order-3 (float32 Horner) and order-12
    (float64 Horner) items against the oracle's compose of each item's
    polynomial."""
    n, h, B = 2, 3, 2
    D = 3
    Mpre = bern.num_monomials(n, D)
    cap = 8
    Mpost = bern.num_monomials(n, min(d * D, cap))
    rng = np.random.default_rng(61)
    pre = rng.normal(0, 0.3, (B, Mpre, h)).astype(np.float32)
    # bracket each item's range loosely so that s lies in [0,1]
    mag = np.abs(pre).sum(1)
    lo = (pre[:, 0, :] - mag - 0.1).astype(np.float32)
    hi = (pre[:, 0, :] + mag + 0.2).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    kind = torch.full((B * h,), 2, dtype=torch.int8, device="cuda")
    coef = torch.zeros((B * h, bern.COEF_STRIDE), dtype=torch.float32, device="cuda")
    eps = torch.zeros(B * h, dtype=torch.float32, device="cuda")
    lo_d, hi_d = dev(lo.reshape(-1)), dev(hi.reshape(-1))
    ctx.relu_coeffs(B * h, lo_d, hi_d, None, d, kind, coef, eps)
    nt = torch.full((B * h,), Mpre, dtype=torch.int32, device="cuda")
    pu, pl = dev(pre), dev(pre)
    qu = torch.zeros((B, Mpost, h), dtype=torch.float32, device="cuda")
    ql = torch.zeros_like(qu)
    qn = torch.zeros(B * h, dtype=torch.int32, device="cuda")
    ctx.compose(n, B, h, cap, 0.0, kind, coef, eps, None, d, lo_d, hi_d, pu, pl, Mpre, nt,
                qu, ql, Mpost, qn)
    assert ctx.sync() == 0
    qu, ql, qn = qu.cpu().numpy(), ql.cpu().numpy(), qn.cpu().numpy()
    ex = bern.monomials(n, D)
    for b in range(B):
        for m in range(h):
            assert qn[b * h + m] == Mpost
            for name, arr, upper in (("u", qu, True), ("l", ql, False)):
                ref = oracle.compose((ex, pre[b, :, m].astype(np.float64)), n, float(lo[b, m]),
                                     float(hi[b, m]), d, upper, cap=cap)
                ov = dense_from_dict(oracle.to_dict(ref), n, Mpost)
                gv = arr[b, :, m].astype(np.float64)
                assert np.abs(gv - ov).sum() <= 1e-4 * (1 + l1(ov)), (b, m, name)


@pytest.mark.parametrize("degree,tau", [(3, 0.0), (2, 1e-3), (4, 0.0)])
def test_global_workspace_path_matches_shared(ctx, degree, tau):
    """The Horner kernel with its buffers in the global workspace computes
    the same bits as with them in shared memory."""
    widths = [3, 10, 10, 2]
    net = wl.make_net(widths, 91)
    boxes = random_boxes(3, 5, 91, 0.3, 1.5)
    a = run_gpu(ctx, net, boxes, degree=degree, tau=tau)
    ctx.set_horner_smem_limit(0)
    try:
        b = run_gpu(ctx, net, boxes, degree=degree, tau=tau)
    finally:
        ctx.set_horner_smem_limit(200 * 1024)
    for k in ("lo", "hi", "n_terms", "coef"):
        assert np.array_equal(a[k], b[k]), k


def test_six_inputs_cap16_pruned(ctx):
    """The branch-and-bound network shape ([6, 64 x 4, 1], cap 16) with
    pruning: the order-2 items of the last hidden layer (3003-term inputs,
    74613-term outputs) run in the global-workspace Horner path.  Bounds are
    sound, term counts never exceed the unpruned ones, and the pruned bounds
    stay close to the unpruned ones on small boxes."""
    w = wl.bnb_root_6in()
    rng = np.random.default_rng(101)
    c = rng.uniform(-0.8, 0.8, (3, 6))
    boxes = wl.box_array(c - 0.06, c + 0.06)
    g0 = run_gpu(ctx, w.net, boxes, degree=2, cap=16)
    g1 = run_gpu(ctx, w.net, boxes, degree=2, cap=16, tau=1e-7)
    assert np.all(g1["n_terms"] <= g0["n_terms"])
    assert np.all(g1["lo"] <= g1["hi"])
    scale = 1 + np.abs(g0["hi"]) + np.abs(g0["lo"])
    assert np.all(np.abs(g1["hi"] - g0["hi"]) <= 1e-3 * scale)
    assert np.all(np.abs(g1["lo"] - g0["lo"]) <= 1e-3 * scale)
    for bi in range(len(boxes)):
        assert mc_check(g1, bi, w.net, boxes[bi], 5_000, rng) == 0
