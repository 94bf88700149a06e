"""The fused layer kernel (bern_layer: a2 + a3 + a4 of one hidden layer and a1
of the next, Sec. 5.1 Steps 1-3 and the layer step of Sec. 5.2) through the
C ABI:

* against the FP64 oracle step by step (enclosure, ReLU coefficients,
  composition and the next layer's affine map, each by the oracle), at the
  step tolerances of the per-step tests;
* bit for bit against the per-step kernels (bern_enclose, bern_relu_coeffs,
  bern_compose, bern_affine) where the kernel promises the same arithmetic:
  wide next layers, no cap truncation;
* whole-path bern_propagate with the fused kernels against the per-step path;
* edge cases: all-dead and all-identity boxes, ragged term counts, narrow
  and odd next-layer widths, cap truncation, one input variable, no boxes,
  and the shapes the kernel declines."""
import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import bern
from paper_2211_14438_gb300 import workloads as wl
from parity_util import dense_from_dict, dict_from_dense, l1, random_dense

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_block(rng, n, D, B, h, mode="mixed", ragged=False):
    """Random pre-activation bounds [B, h, M]: a mix of neurons that are
    clearly dead, clearly active and straddling 0."""
    M = bern.num_monomials(n, D)
    deg = np.array([sum(r) for r in bern.monomials(n, D)], np.float64)
    up = np.zeros((B, h, M), np.float32)
    lo = np.zeros((B, h, M), np.float32)
    nt = np.full((B, h), M, np.int32)
    for b in range(B):
        for m in range(h):
            k = M
            if ragged and (b + m) % 5 == 0:
                k = bern.num_monomials(n, max(0, D - 1))
            nt[b, m] = k
            base = random_dense(rng, n, D, scale=0.4) * (0.6 ** deg).astype(np.float32)
            gap = np.abs(random_dense(rng, n, D, scale=0.02)) * (0.6 ** deg).astype(np.float32)
            kind = mode if mode != "mixed" else ["dead", "active", "cross", "cross"][(b * 7 + m) % 4]
            c0 = {"dead": -3.0, "active": 3.0, "cross": 0.0}[kind]
            base[0] = c0 + rng.normal(0, 0.05)
            up[b, m, :k] = (base + gap)[:k]
            lo[b, m, :k] = (base - gap)[:k]
    return up, lo, nt


def to_layer_block(a):
    """[B, h, M] -> the layer-block layout [B, M, h] (flat)."""
    return np.ascontiguousarray(a.transpose(0, 2, 1)).reshape(-1)


def from_layer_block(t, B, M, h):
    return t.cpu().numpy().reshape(B, M, h).transpose(0, 2, 1).astype(np.float64)


def run_layer(ctx, n, up, lo, nt, order, d, cap, W, bias, budget=0):
    B, h, M = up.shape
    hn = W.shape[0]
    D = 0
    while bern.num_monomials(n, D) < M:
        D += 1
    Dn = min(d * D, cap)
    Mn = bern.num_monomials(n, Dn)
    nu = torch.full((B * Mn * hn,), np.nan, device="cuda")
    nl = torch.full_like(nu, np.nan)
    nnt = torch.zeros(B * hn, dtype=torch.int32, device="cuda")
    ctx.layer(n, B, h, order, budget, d, cap, dev(to_layer_block(up)), dev(to_layer_block(lo)),
              M, dev(nt), hn, dev(W), dev(bias), nu, nl, Mn, nnt)
    assert ctx.sync() == 0
    return nu, nl, nnt.cpu().numpy().reshape(B, hn), Mn


def run_steps(ctx, n, up, lo, nt, order, d, cap, W, bias, budget=0):
    """The same layer through the per-step kernels."""
    B, h, M = up.shape
    hn = W.shape[0]
    D = 0
    while bern.num_monomials(n, D) < M:
        D += 1
    Mp = bern.num_monomials(n, min(d * D, cap))
    items = B * h
    glo = torch.zeros(items, device="cuda")
    ghi = torch.zeros(items, device="cuda")
    pu, pl, pnt = dev(to_layer_block(up)), dev(to_layer_block(lo)), dev(nt)
    ctx.enclose(n, B, h, order, budget, pu, pl, M, pnt, glo, ghi)
    kind = torch.zeros(items, dtype=torch.int8, device="cuda")
    coef = torch.zeros(items * bern.COEF_STRIDE, device="cuda")
    eps = torch.zeros(items, device="cuda")
    ctx.relu_coeffs(items, glo, ghi, None, d, kind, coef, eps)
    qu = torch.zeros(B * Mp * h, device="cuda")
    ql = torch.zeros_like(qu)
    qnt = torch.zeros(items, dtype=torch.int32, device="cuda")
    ctx.compose(n, B, h, cap, 0.0, kind, coef, eps, None, d, glo, ghi, pu, pl, M, pnt, qu, ql, Mp,
                qnt)
    nu = torch.full((B * Mp * hn,), np.nan, device="cuda")
    nl = torch.full_like(nu, np.nan)
    nnt = torch.zeros(B * hn, dtype=torch.int32, device="cuda")
    ctx.affine(B, hn, h, dev(W), dev(bias), qu, ql, Mp, qnt, nu, nl, Mp, nnt)
    assert ctx.sync() == 0
    return nu, nl, nnt.cpu().numpy().reshape(B, hn), Mp


def oracle_layer(n, up, lo, nt, order, d, cap, W, bias, budget):
    """The oracle's Steps 1-3 for every neuron, then its layer step."""
    B, h, M = up.shape
    outs = []
    for b in range(B):
        post_u, post_l = [], []
        for m in range(h):
            k = int(nt[b, m])
            Pu = dict_from_dense(up[b, m, :k].astype(np.float64), n) if k else {(0,) * n: 0.0}
            Pl = dict_from_dense(lo[b, m, :k].astype(np.float64), n) if k else {(0,) * n: 0.0}
            L = oracle.enclosure(Pl, n, order, budget)[0]
            H = oracle.enclosure(Pu, n, order, budget)[1]
            if H <= 0:
                post_u.append({(0,) * n: 0.0})
                post_l.append({(0,) * n: 0.0})
            elif L >= 0:
                post_u.append(Pu)
                post_l.append(Pl)
            else:
                post_u.append(oracle.to_dict(oracle.compose(Pu, n, L, H, d, True, cap=cap)))
                post_l.append(oracle.to_dict(oracle.compose(Pl, n, L, H, d, False, cap=cap)))
        rows = []
        for mp in range(W.shape[0]):
            ou, ol = oracle.affine(post_u, post_l, n, W[mp].astype(np.float64), float(bias[mp]))
            rows.append((oracle.to_dict(ou), oracle.to_dict(ol)))
        outs.append((rows, post_u, post_l))
    return outs


@pytest.mark.parametrize("n,D,h,hn,d,cap,B,ragged", [
    (3, 4, 64, 64, 2, 16, 3, False),     # the benchmark net's third hidden layer
    (3, 8, 64, 1, 2, 16, 2, False),      # its fourth, into the output neuron
    (2, 2, 20, 20, 2, 16, 4, True),      # ragged term counts
    (3, 4, 37, 7, 2, 16, 3, False),      # odd widths: a scalar next-layer tile
    (3, 4, 24, 16, 2, 6, 3, False),      # cap 6 < 2D: truncation remainders
    (4, 2, 50, 50, 2, 16, 2, False),
    (3, 4, 64, 8, 1, 16, 3, True),       # order 1
    (1, 8, 9, 3, 2, 16, 3, False),       # one input variable
])
def test_layer_against_oracle(ctx, n, D, h, hn, d, cap, B, ragged):
    rng = np.random.default_rng(31 * n + 7 * D + h + hn + d + cap)
    up, lo, nt = make_block(rng, n, D, B, h, ragged=ragged)
    W = (rng.normal(size=(hn, h)) / np.sqrt(h)).astype(np.float32)
    bias = rng.uniform(-0.1, 0.1, hn).astype(np.float32)
    order = D
    nu, nl, nnt, Mn = run_layer(ctx, n, up, lo, nt, order, d, cap, W, bias)
    gu = from_layer_block(nu, B, Mn, hn)
    gl = from_layer_block(nl, B, Mn, hn)
    want = oracle_layer(n, up, lo, nt, order, d, cap, W, bias, 1 << 20)
    for b in range(B):
        rows, post_u, post_l = want[b]
        k = int(nnt[b, 0])
        assert np.all(nnt[b] == k) and 1 <= k <= Mn
        sc = [l1(list(pu.values())) + l1(list(pl.values())) for pu, pl in zip(post_u, post_l)]
        for mp in range(hn):
            ou = dense_from_dict(rows[mp][0], n, Mn)
            ol = dense_from_dict(rows[mp][1], n, Mn)
            scale = 1 + np.abs(W[mp]).astype(np.float64) @ np.array(sc) + abs(float(bias[mp]))
            g_u = np.where(np.arange(Mn) < k, gu[b, mp], 0.0)
            g_l = np.where(np.arange(Mn) < k, gl[b, mp], 0.0)
            assert np.all(np.isfinite(g_u)) and np.all(np.isfinite(g_l))
            assert np.abs(g_u - ou).sum() <= 1e-4 * scale, (b, mp, np.abs(g_u - ou).sum(), scale)
            assert np.abs(g_l - ol).sum() <= 1e-4 * scale, (b, mp, np.abs(g_l - ol).sum(), scale)


@pytest.mark.parametrize("n,D,h,hn,d,B", [
    (3, 4, 64, 64, 2, 5), (3, 8, 64, 32, 2, 3), (2, 4, 40, 12, 2, 4), (3, 2, 64, 64, 1, 4),
    (5, 2, 30, 12, 2, 3)])
def test_layer_bitwise_against_step_kernels(ctx, n, D, h, hn, d, B):
    """Next layers wider than 8 neurons (the per-step affine kernels for them
    sum every input neuron in index order, as the fused kernel does over the
    live ones; dead neurons add exact zeros) and no truncation: the fused
    kernel reproduces the per-step kernels' values exactly."""
    rng = np.random.default_rng(100 + n + D + h + hn + d)
    up, lo, nt = make_block(rng, n, D, B, h)
    W = (rng.normal(size=(hn, h)) / np.sqrt(h)).astype(np.float32)
    bias = rng.uniform(-0.1, 0.1, hn).astype(np.float32)
    a = run_layer(ctx, n, up, lo, nt, D, d, 16, W, bias)
    s = run_steps(ctx, n, up, lo, nt, D, d, 16, W, bias)
    assert a[3] == s[3]
    assert np.array_equal(a[2], s[2])
    for b in range(B):
        k = int(a[2][b, 0])
        fu = from_layer_block(a[0], B, a[3], hn)[b][:, :k]
        su = from_layer_block(s[0], B, s[3], hn)[b][:, :k]
        fl = from_layer_block(a[1], B, a[3], hn)[b][:, :k]
        sl = from_layer_block(s[1], B, s[3], hn)[b][:, :k]
        assert np.array_equal(fu, su), (b, np.abs(fu - su).max())
        assert np.array_equal(fl, sl), (b, np.abs(fl - sl).max())


@pytest.mark.parametrize("mode", ["dead", "active", "cross"])
def test_layer_uniform_boxes(ctx, mode):
    """Every neuron dead (the next layer is its bias), every neuron active
    (the next layer is the plain affine map of the block), every neuron
    unstable."""
    n, D, h, hn, B = 3, 4, 32, 16, 3
    rng = np.random.default_rng({"dead": 1, "active": 2, "cross": 3}[mode])
    up, lo, nt = make_block(rng, n, D, B, h, mode=mode)
    W = (rng.normal(size=(hn, h)) / np.sqrt(h)).astype(np.float32)
    bias = rng.uniform(-0.1, 0.1, hn).astype(np.float32)
    a = run_layer(ctx, n, up, lo, nt, D, 2, 16, W, bias)
    s = run_steps(ctx, n, up, lo, nt, D, 2, 16, W, bias)
    k = a[2][:, 0]
    assert np.array_equal(a[2], s[2])
    if mode == "dead":
        assert np.all(k == 1)
        gu = from_layer_block(a[0], B, a[3], hn)[:, :, 0]
        gl = from_layer_block(a[1], B, a[3], hn)[:, :, 0]
        assert np.array_equal(gu, np.broadcast_to(bias, gu.shape))
        assert np.array_equal(gl, np.broadcast_to(bias, gl.shape))
    if mode == "active":
        assert np.all(k == bern.num_monomials(n, D))
    for b in range(B):
        fu = from_layer_block(a[0], B, a[3], hn)[b][:, :k[b]]
        su = from_layer_block(s[0], B, s[3], hn)[b][:, :k[b]]
        assert np.array_equal(fu, su)


def test_layer_zero_boxes_and_declined_shapes(ctx):
    n, D, h, hn = 3, 4, 16, 8
    M = bern.num_monomials(n, D)
    z = torch.zeros(16, device="cuda")
    zi = torch.zeros(16, dtype=torch.int32, device="cuda")
    W = torch.zeros(hn * h, device="cuda")
    ctx.layer(n, 0, h, D, 0, 2, 16, z, z, M, zi, hn, W, z, z, z, M, zi)    # no boxes: no-op
    assert ctx.sync() == 0
    # order 3, more than 256 neurons, and an input degree beyond the row tables
    for args in ((n, 1, h, D, 0, 3, 16, M), (n, 1, 300, D, 0, 2, 16, M),
                 (6, 1, h, 8, 0, 2, 16, bern.num_monomials(6, 8))):
        with pytest.raises(bern.BernError) as ei:
            nn, B, hh, order, budget, d, cap, ld = args
            ctx.layer(nn, B, hh, order, budget, d, cap, z, z, ld, zi, hn, W, z, z, z, ld, zi)
        assert ei.value.code == bern.BERN_E_UNSUPPORTED


def test_propagate_fused_matches_step_path(ctx):
    """bern_propagate on 256 boxes of the benchmark workload with the fused
    layer kernels and with the per-step kernels: the same term counts, and
    bounds and polynomials equal up to the order of the output layer's sums
    (the per-step narrow affine kernel reduces across lanes)."""
    w = wl.batch_3in()
    boxes = np.ascontiguousarray(w.boxes[::20])
    W = [dev(x) for x in w.net.W]
    b = [dev(x) for x in w.net.b]
    bx = dev(boxes)
    ct = bern.max_output_terms(w.net.widths, 2, 16)
    def run_twice():
        # the second call replays the captured graph (no autotuning probes)
        ctx.propagate(w.net.widths, W, b, bx, degree=2, cap=16, cap_terms=ct)
        n0 = ctx.kernel_launches()
        r = ctx.propagate(w.net.widths, W, b, bx, degree=2, cap=16, cap_terms=ct)
        return r, ctx.kernel_launches() - n0

    ctx.set_fused(True)
    try:
        fa, launches_fused = run_twice()
    finally:
        ctx.set_fused(False)
    st, launches_step = run_twice()
    # one launch per hidden layer instead of the per-step sequence
    assert 0 < launches_fused < launches_step
    assert np.array_equal(fa["n_terms"].cpu().numpy(), st["n_terms"].cpu().numpy())
    for k in ("lo", "hi"):
        x, y = fa[k].cpu().numpy().astype(np.float64), st[k].cpu().numpy().astype(np.float64)
        assert np.all(np.abs(x - y) <= 1e-5 * (1 + np.abs(y)))
    cf, cs = fa["coef"].cpu().numpy().astype(np.float64), st["coef"].cpu().numpy().astype(np.float64)
    nt = st["n_terms"].cpu().numpy()
    for i in range(len(boxes)):
        for s in range(2):
            k = int(nt[i, 0, s])
            assert np.abs(cf[i, 0, s, :k] - cs[i, 0, s, :k]).sum() <= \
                1e-5 * (1 + np.abs(cs[i, 0, s, :k]).sum())


def test_propagate_fused_then_in_place_layer(ctx):
    """A six-input net whose last hidden layer is too large for the fused
    kernel (input degree 8 beyond the row path): the fused kernels of the
    first layers write that layer's pre-activation block at its in-place row
    stride (the stride of its post-activation block), and the per-step
    kernels compose it in place.  The same results as the per-step path."""
    net = wl.make_net([6, 12, 12, 12, 12, 1], 71)
    rng = np.random.default_rng(71)
    c = rng.uniform(-0.8, 0.8, (16, 6))
    s = rng.uniform(0.05, 0.3, (16, 6))
    boxes = dev(wl.box_array(c - s / 2, c + s / 2))
    W = [dev(x) for x in net.W]
    b = [dev(x) for x in net.b]
    ct = bern.max_output_terms(net.widths, 2, 16)
    ctx.set_fused(True)
    try:
        fa = ctx.propagate(net.widths, W, b, boxes, degree=2, cap=16, cap_terms=ct)
    finally:
        ctx.set_fused(False)
    st = ctx.propagate(net.widths, W, b, boxes, degree=2, cap=16, cap_terms=ct)
    assert np.array_equal(fa["n_terms"].cpu().numpy(), st["n_terms"].cpu().numpy())
    for k in ("lo", "hi"):
        x, y = fa[k].cpu().numpy().astype(np.float64), st[k].cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(x))
        assert np.all(np.abs(x - y) <= 1e-5 * (1 + np.abs(y)))
