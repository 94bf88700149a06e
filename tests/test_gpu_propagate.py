"""Whole-path parity (bern_propagate through the C ABI) against the FP64
oracle, Monte-Carlo soundness, and the edge cases of the boundary.

Tolerance (float32 path vs float64 oracle): every output bound within
1e-4 * (1 + |bound|), and every output polynomial within 1e-4 * (1 + ||p||_1)
in the sum of absolute coefficient differences (a sup-norm bound of the
difference on the box, since each monomial lies in [0,1]).  A box where the
oracle sees a hidden neuron with |lo| or |hi| within 1e-5 relative of 0 is a
genuine tie (float32 and float64 may take different ReLU cases there); such a
box is checked for soundness only."""
import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import bern
from paper_2211_14438_gb300 import workloads as wl
from parity_util import dense_from_dict, eval_dense, l1

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


def run_gpu(ctx, net, boxes, degree=2, cap=16, **kw):
    W = [torch.from_numpy(w).cuda() for w in net.W]
    b = [torch.from_numpy(x).cuda() for x in net.b]
    out = ctx.propagate(net.widths, W, b, torch.from_numpy(np.ascontiguousarray(boxes)).cuda(),
                        degree=degree, cap=cap, **kw)
    return {k: (v.cpu().numpy() if v is not None else None) for k, v in out.items()}


def near_tie(r, rel=1e-5):
    lo, hi = r["tr_lo"], r["tr_hi"]
    sc = 1 + np.maximum(np.abs(lo), np.abs(hi))
    return bool(np.any(np.minimum(np.abs(lo), np.abs(hi)) <= rel * sc))


def gpu_t(box, x):
    """The library's normalised coordinates: t = (x - dlo) / w, w = fl_up(dhi - dlo)."""
    lo = box[:, 0].astype(np.float32)
    w = (box[:, 1].astype(np.float64) - lo.astype(np.float64))
    wf = w.astype(np.float32)
    wf = np.where(wf.astype(np.float64) < w, np.nextafter(wf, np.float32(np.inf)), wf)
    return (x - lo.astype(np.float64)) / np.where(wf > 0, wf, 1.0).astype(np.float64)


def compare_box(g, bi, r, n, o, check_polys=True):
    for j in range(o):
        lo_g, hi_g = float(g["lo"][bi, j]), float(g["hi"][bi, j])
        assert abs(lo_g - r["lo"][j]) <= TOL * (1 + abs(r["lo"][j])), (bi, j, lo_g, r["lo"][j])
        assert abs(hi_g - r["hi"][j]) <= TOL * (1 + abs(r["hi"][j])), (bi, j, hi_g, r["hi"][j])
        if not check_polys:
            continue
        for k, name in ((0, "upper"), (1, "lower")):
            nt = int(g["n_terms"][bi, j, k])
            gv = g["coef"][bi, j, k, :nt].astype(np.float64)
            ov = dense_from_dict(r[name][j], n, nt)
            assert np.abs(gv - ov).sum() <= TOL * (1 + l1(ov)), (bi, j, name)


def mc_check(g, bi, net, box, count, rng):
    n, o = net.n_in, net.n_out
    t = rng.random((count, n))
    corners = np.array(np.meshgrid(*([[0.0, 1.0]] * n), indexing="ij")).reshape(n, -1).T
    t[: min(len(corners), count)] = corners[: min(len(corners), count)]
    lo = box[:, 0].astype(np.float64)
    hi = box[:, 1].astype(np.float64)
    x = lo + t * (hi - lo)
    nn = oracle.network_forward(net.widths, net.W, net.b, x)
    tg = gpu_t(box, x)
    viol = 0
    for j in range(o):
        nt_u, nt_l = int(g["n_terms"][bi, j, 0]), int(g["n_terms"][bi, j, 1])
        up = eval_dense(g["coef"][bi, j, 0, :nt_u].astype(np.float64), n, tg)
        lw = eval_dense(g["coef"][bi, j, 1, :nt_l].astype(np.float64), n, tg)
        e = 1e-12 * (1 + np.abs(nn[:, j]) + l1(g["coef"][bi, j, 0, :nt_u]))
        viol += int(np.sum(nn[:, j] > up + e)) + int(np.sum(nn[:, j] < lw - e))
        viol += int(np.sum(nn[:, j] > g["hi"][bi, j] + e)) + int(np.sum(nn[:, j] < g["lo"][bi, j] - e))
    return viol


def test_single_box_2in_parity_and_soundness(ctx):
    w = wl.single_box_2in()
    g = run_gpu(ctx, w.net, w.boxes)
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2)
    assert not near_tie(r)
    compare_box(g, 0, r, 2, 1)
    assert mc_check(g, 0, w.net, w.boxes[0], 1_000_000, np.random.default_rng(1)) == 0


def test_single_box_4in_parity_and_soundness(ctx):
    w = wl.single_box_4in()
    g = run_gpu(ctx, w.net, w.boxes)
    r = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], 2)
    assert not near_tie(r)
    compare_box(g, 0, r, 4, 2)
    assert mc_check(g, 0, w.net, w.boxes[0], 200_000, np.random.default_rng(2)) == 0


def test_batch_3in_full_batch_sampled(ctx):
    """The benchmark's launch configuration: all 5120 boxes in one call;
    64 sampled boxes (the grid's corners and both ends of the random part,
    the rest drawn) are checked against the oracle one by one (a spawned
    process pool runs the oracle), and every box against properties that hold
    at any size."""
    import multiprocessing as mp
    import os
    from parity_util import oracle_propagate_job
    w = wl.batch_3in()
    g = run_gpu(ctx, w.net, w.boxes)
    B = len(w.boxes)
    assert np.all(np.isfinite(g["lo"])) and np.all(g["lo"] <= g["hi"])
    nt = g["n_terms"][:, 0, 0]
    assert np.all(nt >= 1) and np.all(nt <= bern.num_monomials(3, 16))
    rng = np.random.default_rng(3)
    fixed = [0, 1, 15, 255, 2047, 4095, 4096, 5119]
    rest = rng.choice(np.setdiff1d(np.arange(B), fixed), 64 - len(fixed), replace=False)
    sample = fixed + [int(x) for x in rest]
    jobs = [(w.net.widths, w.net.W, w.net.b, w.boxes[bi], 2, {}) for bi in sample]
    with mp.get_context("spawn").Pool(max(1, min(16, os.cpu_count() or 1))) as pool:
        refs = pool.map(oracle_propagate_job, jobs, chunksize=1)
    checked = 0
    for k, (bi, r) in enumerate(zip(sample, refs)):
        if not near_tie(r):
            compare_box(g, bi, r, 3, 1)
            checked += 1
        assert mc_check(g, bi, w.net, w.boxes[bi], 100_000 if k < 8 else 10_000, rng) == 0
    assert checked >= len(sample) - 4
    # every box: the bound contains the network at the box centre and corners
    for bi in range(0, B, 97):
        box = w.boxes[bi]
        assert mc_check(g, bi, w.net, box, 9, rng) == 0


def test_batch_3in_small_batch_matches_full(ctx):
    """A ragged batch (37 boxes, several tiles and a tail) gives the same
    numbers as the same boxes inside the full batch (no cross-box state)."""
    w = wl.batch_3in()
    idx = np.r_[0:20, 4096:4113]
    g_small = run_gpu(ctx, w.net, w.boxes[idx])
    g_full = run_gpu(ctx, w.net, w.boxes)
    assert np.array_equal(g_small["lo"], g_full["lo"][idx])
    assert np.array_equal(g_small["hi"], g_full["hi"][idx])
    assert np.array_equal(g_small["n_terms"], g_full["n_terms"][idx])


@pytest.mark.parametrize("widths,degree,seed", [
    ([1, 8, 8, 1], 2, 11), ([2, 6, 5, 3], [2, 1], 12), ([3, 10, 10, 2], 1, 13),
    ([5, 12, 7, 1], 2, 14), ([8, 6, 4, 2], 2, 15), ([2, 20, 20, 1], 2, 16)])
def test_small_nets_parity(ctx, widths, degree, seed):
    net = wl.make_net(widths, seed)
    rng = np.random.default_rng(seed)
    n = widths[0]
    c = rng.uniform(-1, 1, (5, n))
    s = rng.uniform(0.05, 1.0, (5, n))
    boxes = wl.box_array(c - s / 2, c + s / 2)
    g = run_gpu(ctx, net, boxes, degree=degree)
    dl = degree if isinstance(degree, int) else None
    for bi in range(len(boxes)):
        if dl is None:
            degs = np.concatenate([np.full(h, d) for h, d in zip(widths[1:-1], degree)])
        else:
            degs = dl
        r = oracle.propagate(widths, net.W, net.b, boxes[bi], degs,
                             budget=1 << 20)
        if near_tie(r):
            continue
        compare_box(g, bi, r, n, widths[-1])
        assert mc_check(g, bi, net, boxes[bi], 20_000, rng) == 0


def test_paper_family_nets(ctx):
    """The paper's own ablation family (weights U(-5,5)), [2,20,20,1] on
    [-1,1]^2 with L = 2, 3, 4: parity and soundness."""
    net = wl.paper_net(2, [20, 20], seed=101)
    box = wl.box_array([-1, -1], [1, 1])[None]
    for d in (2, 3, 4):
        g = run_gpu(ctx, net, box, degree=d)
        r = oracle.propagate(net.widths, net.W, net.b, box[0], d)
        if not near_tie(r):
            compare_box(g, 0, r, 2, 1)
        assert mc_check(g, 0, net, box[0], 200_000, np.random.default_rng(d)) == 0


# ------------------------------------------------------------ edge cases
def test_empty_batch(ctx):
    w = wl.single_box_2in()
    g = run_gpu(ctx, w.net, w.boxes[:0])
    assert g["lo"].shape == (0, 1)


def test_point_box_gives_network_value(ctx):
    w = wl.single_box_4in()
    x = np.array([0.1, -0.2, 0.3, 0.05], np.float32)
    box = np.stack([x, x], -1)[None]
    g = run_gpu(ctx, w.net, box)
    nn = oracle.network_forward(w.net.widths, w.net.W, w.net.b, x[None].astype(np.float64))[0]
    assert np.all(g["lo"][0] <= nn + 1e-5 * (1 + abs(nn)))
    assert np.all(g["hi"][0] >= nn - 1e-5 * (1 + abs(nn)))
    assert np.all(g["hi"][0] - g["lo"][0] <= 1e-4 * (1 + abs(nn)))


def test_invalid_box_reported(ctx):
    w = wl.single_box_2in()
    bad = np.array([[[0.5, -0.5], [0.0, 1.0]]], np.float32)
    with pytest.raises(bern.BernError) as ei:
        run_gpu(ctx, w.net, bad)
    assert ei.value.code == bern.BERN_E_INVALID
    bad = np.array([[[np.nan, 0.5], [0.0, 1.0]]], np.float32)
    with pytest.raises(bern.BernError):
        run_gpu(ctx, w.net, bad)
    assert ctx.sync() == 0


def test_capacity_too_small_reports_need(ctx):
    w = wl.single_box_2in()
    with pytest.raises(bern.BernError) as ei:
        run_gpu(ctx, w.net, w.boxes, cap_terms=4)
    assert ei.value.code == bern.BERN_E_CAPACITY


def test_all_dead_and_all_active(ctx):
    rng = np.random.default_rng(9)
    W1 = rng.normal(size=(4, 3)).astype(np.float32)
    W2 = rng.normal(size=(2, 4)).astype(np.float32)
    b2 = np.array([0.5, -1.25], np.float32)
    box = np.array([[[-1, 1]] * 3], np.float32)
    dead = wl.Net([3, 4, 2], [W1, W2], [np.full(4, -50, np.float32), b2])
    g = run_gpu(ctx, dead, box)
    assert np.array_equal(g["lo"][0], b2) and np.array_equal(g["hi"][0], b2)
    act = wl.Net([3, 4, 2], [W1, W2], [np.full(4, 50, np.float32), b2])
    g = run_gpu(ctx, act, box)
    r = oracle.propagate([3, 4, 2], act.W, act.b, box[0], 2)
    compare_box(g, 0, r, 3, 2)


def test_host_mode_matches_device_mode(ctx):
    w = wl.batch_3in(n_random=8, cells=2)
    g = run_gpu(ctx, w.net, w.boxes)
    h = ctx.propagate_host(w.net.widths, w.net.W, w.net.b, w.boxes, degree=2)
    assert np.array_equal(h["lo"], g["lo"]) and np.array_equal(h["hi"], g["hi"])
    assert np.array_equal(h["n_terms"], g["n_terms"])
    for bi in range(len(w.boxes)):
        nt = g["n_terms"][bi, 0, 0]
        assert np.array_equal(h["coef"][bi, 0, :, :nt], g["coef"][bi, 0, :, :nt])


def test_graphs_on_off_identical_and_counted(ctx):
    w = wl.batch_3in(n_random=16, cells=4)
    before = ctx.kernel_launches()
    ctx.set_graphs(False)
    a = run_gpu(ctx, w.net, w.boxes)
    mid = ctx.kernel_launches()
    ctx.set_graphs(True)
    b = run_gpu(ctx, w.net, w.boxes)
    c = run_gpu(ctx, w.net, w.boxes)
    after = ctx.kernel_launches()
    assert mid > before and after > mid
    for k in ("lo", "hi", "n_terms", "coef"):
        assert np.array_equal(a[k], b[k]) and np.array_equal(b[k], c[k])


def test_output_keys_are_graded_monomials(ctx):
    w = wl.single_box_2in()
    g = run_gpu(ctx, w.net, w.boxes, keys=True)
    nt = int(g["n_terms"][0, 0, 0])
    ex = bern.monomials(2, 4)[:nt].astype(np.int64)
    want = ex[:, 0] | (ex[:, 1] << 8)
    assert np.array_equal(g["keys"][0, 0, 0, :nt], want)
    assert np.array_equal(g["keys"][0, 0, 1, :nt], want)


@pytest.mark.parametrize("widths,seed", [([3, 64, 64, 64, 64, 1], 2), ([6, 100, 100, 2], 3),
                                        ([3, 40, 72, 48, 4], 5)])
def test_forced_variants_identical(ctx, widths, seed):
    """Every variant of the wide-layer affine kernel (persistent
    register-blocked 8x4, 8x2 and 8x1 thread tiles, 64x32 block tiles) and of the
    enclosure (8, 4, 2 items per block with a warp per polynomial, a block per
    polynomial for the larger grids) gives the same bits, on layers 64 and 100
    wide and on widths that are not multiples of 64 (the six-input net's
    enclosures reach 5^6 = 15625 cells)."""
    net = wl.make_net(widths, seed)
    rng = np.random.default_rng(seed)
    n = widths[0]
    c = rng.uniform(-1, 1, (24, n))
    s = rng.uniform(0.05, 0.6, (24, n))
    boxes = wl.box_array(c - s / 2, c + s / 2)
    ref = None
    try:
        for kind, nv in (("affine", 5), ("enclose", 5)):
            for v in range(nv):
                ctx.force_variant(kind, v)
                g = run_gpu(ctx, net, boxes)
                ctx.force_variant(kind, -1)
                if ref is None:
                    ref = g
                for k in ("lo", "hi", "n_terms", "coef"):
                    assert np.array_equal(g[k], ref[k]), (kind, v, k)
    finally:
        ctx.force_variant("affine", -1)
        ctx.force_variant("enclose", -1)
    r = oracle.propagate(widths, net.W, net.b, boxes[0], 2)
    if not near_tie(r):
        compare_box(ref, 0, r, n, widths[-1])


def test_autotune_on_off_identical(ctx):
    """Every tunable variant computes the same values: results with the
    autotuner's choices equal those with the built-in defaults, bit for bit."""
    w = wl.batch_3in(n_random=40, cells=4)
    ctx.set_autotune(False)
    try:
        a = run_gpu(ctx, w.net, w.boxes)
    finally:
        ctx.set_autotune(True)
    b = run_gpu(ctx, w.net, w.boxes)
    c = run_gpu(ctx, w.net, w.boxes)
    for k in ("lo", "hi", "n_terms", "coef"):
        assert np.array_equal(a[k], b[k]) and np.array_equal(b[k], c[k]), k


def test_stability_screen_matches_full_enclosure(ctx):
    """Untraced plain runs decide the hidden items whose coefficient signs
    show them stable without enclosing them; traced runs enclose every item.
    The outputs agree: bit for bit on (nearly) every box, and within the
    parity tolerance where a Bernstein bound within rounding of 0 takes the
    other ReLU case."""
    w = wl.batch_3in(n_random=64, cells=4)
    ctx.set_fused(False)          # the per-step kernels (the default), as traced runs use
    a = run_gpu(ctx, w.net, w.boxes)
    b = run_gpu(ctx, w.net, w.boxes, trace=True)
    # the fused layer kernels screen the same way; their output layer's sums
    # run in another order
    ctx.set_fused(True)
    try:
        f = run_gpu(ctx, w.net, w.boxes)
    finally:
        ctx.set_fused(False)
    assert np.array_equal(f["n_terms"], a["n_terms"])
    assert np.all(np.abs(f["lo"] - a["lo"]) <= 1e-5 * (1 + np.abs(a["lo"])))
    assert np.all(np.abs(f["hi"] - a["hi"]) <= 1e-5 * (1 + np.abs(a["hi"])))
    same = np.all(a["lo"] == b["lo"], axis=1) & np.all(a["hi"] == b["hi"], axis=1)
    assert same.mean() >= 0.95
    assert np.all(np.abs(a["lo"] - b["lo"]) <= TOL * (1 + np.abs(b["lo"])))
    assert np.all(np.abs(a["hi"] - b["hi"]) <= TOL * (1 + np.abs(b["hi"])))
    # the traced run's Bernstein bounds confirm every hidden case the screen decided
    assert np.array_equal(a["n_terms"][same], b["n_terms"][same])
