"""GPU parity of each step of the path (init, affine, enclosure, ReLU
coefficients, composition) against the FP64 oracle, through the C ABI.

Bar: every GPU coefficient/bound lies on the sound side of the oracle's value
(outward rounding) and within the float32 tolerance written in each test."""
import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import bern
from parity_util import dense_from_dict, eval_dense, l1, random_dense

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


# ---------------------------------------------------------------- a0
# Layer blocks: coefficient r of neuron m of box b at ((b*ld + r)*h + m).

def test_init_inputs(ctx):
    rng = np.random.default_rng(0)
    n, B = 3, 37
    lo = rng.uniform(-2, 1, (B, n)).astype(np.float32)
    hi = (lo + rng.uniform(0, 1.5, (B, n))).astype(np.float32)
    hi[5] = lo[5]                                   # a point box
    boxes = np.stack([lo, hi], -1)
    ld = n + 2
    zu = torch.zeros(B * ld * n, device="cuda")
    zl = torch.zeros_like(zu)
    nt = torch.zeros(B * n, dtype=torch.int32, device="cuda")
    ctx.init_inputs(n, dev(boxes), zu, zl, ld, nt)
    assert ctx.sync() == 0
    zu = zu.cpu().numpy().reshape(B, ld, n)
    assert np.array_equal(zu, zl.cpu().numpy().reshape(B, ld, n))
    assert np.all(nt.cpu().numpy() == n + 1)
    w = hi.astype(np.float64) - lo.astype(np.float64)
    for b in range(B):
        for i in range(n):
            assert zu[b, 0, i] == lo[b, i]
            assert zu[b, 1 + i, i] >= w[b, i] and zu[b, 1 + i, i] - w[b, i] <= 2 ** -23 * (w[b, i] + 1e-30) * 2
            others = [zu[b, 1 + k, i] for k in range(n) if k != i]
            assert all(x == 0 for x in others)


def test_init_rejects_inverted_box(ctx):
    boxes = np.array([[[0.5, 0.25], [0, 1]]], np.float32)
    zu = torch.zeros(3 * 2, device="cuda")
    zl = torch.zeros_like(zu)
    nt = torch.zeros(2, dtype=torch.int32, device="cuda")
    ctx.init_inputs(2, dev(boxes), zu, zl, 3, nt)
    assert ctx.sync() == bern.BERN_E_INVALID
    assert ctx.sync() == 0                           # the status word was cleared


# ---------------------------------------------------------------- a1
@pytest.mark.parametrize("n,D,h_in,h_out,B", [
    (2, 2, 5, 7, 3), (3, 4, 20, 9, 5), (4, 3, 33, 17, 2), (3, 8, 64, 1, 3), (2, 3, 6, 3, 4),
    (3, 2, 7, 5, 2), (3, 8, 64, 64, 2), (2, 4, 40, 33, 3), (6, 2, 100, 100, 2), (1, 6, 3, 2, 5),
    # a warp per box at exactly 16 rows; the register-blocked kernel with
    # h_in > 128 and a ragged neuron slice; the quad kernel at G = 4 and 32
    (1, 15, 20, 40, 3), (3, 4, 150, 70, 2), (2, 4, 4, 1, 3), (2, 3, 128, 2, 3)])
def test_affine_step(ctx, n, D, h_in, h_out, B):
    rng = np.random.default_rng(n * 100 + D)
    M = bern.num_monomials(n, D)
    up = np.zeros((B, h_in, M), np.float32)
    lo = np.zeros((B, h_in, M), np.float32)
    nt = np.zeros((B, h_in), np.int32)
    choices = [0, 1] + [bern.num_monomials(n, g) for g in range(1, D + 1)]
    for b in range(B):
        for j in range(h_in):
            k = int(rng.choice(choices))
            nt[b, j] = k
            base = random_dense(rng, n, D)[:k]
            gap = np.abs(random_dense(rng, n, D))[:k]
            up[b, j, :k] = base + gap
            lo[b, j, :k] = base - gap
    nt[0, :] = np.minimum(nt[0, :], 1)              # a box whose inputs are all constants/empty
    W = rng.normal(size=(h_out, h_in)).astype(np.float32)
    W[rng.random(W.shape) < 0.1] = 0.0
    bias = rng.normal(size=h_out).astype(np.float32)
    out_u = torch.full((B * M * h_out,), np.nan, device="cuda")
    out_l = torch.full_like(out_u, np.nan)
    out_nt = torch.zeros(B * h_out, dtype=torch.int32, device="cuda")
    # entries beyond a neuron's term count hold garbage that must not be read
    up_blk = np.where(np.arange(M)[None, None, :] < nt[:, :, None], up, np.float32(1e30))
    lo_blk = np.where(np.arange(M)[None, None, :] < nt[:, :, None], lo, np.float32(-1e30))
    up_blk = np.ascontiguousarray(up_blk.transpose(0, 2, 1))
    lo_blk = np.ascontiguousarray(lo_blk.transpose(0, 2, 1))
    ctx.affine(B, h_out, h_in, dev(W), dev(bias), dev(up_blk), dev(lo_blk), M, dev(nt), out_u,
               out_l, M, out_nt)
    assert ctx.sync() == 0
    out_u = out_u.cpu().numpy().reshape(B, M, h_out).transpose(0, 2, 1).astype(np.float64)
    out_l = out_l.cpu().numpy().reshape(B, M, h_out).transpose(0, 2, 1).astype(np.float64)
    out_nt = out_nt.cpu().numpy().reshape(B, h_out)
    from parity_util import dict_from_dense
    for b in range(B):
        Mb = max(1, int(nt[b].max()))
        assert np.all(out_nt[b] == Mb)
        ups = [dict_from_dense(up[b, j, : nt[b, j]].astype(np.float64), n) if nt[b, j] else {(0,) * n: 0.0}
               for j in range(h_in)]
        los = [dict_from_dense(lo[b, j, : nt[b, j]].astype(np.float64), n) if nt[b, j] else {(0,) * n: 0.0}
               for j in range(h_in)]
        scale = np.abs(W).astype(np.float64) @ np.array(
            [l1(up[b, j]) + l1(lo[b, j]) for j in range(h_in)]) + np.abs(bias)
        for m in range(h_out):
            pu, pl = oracle.affine(ups, los, n, W[m].astype(np.float64), float(bias[m]))
            ou = dense_from_dict(pu, n, Mb)
            ol = dense_from_dict(pl, n, Mb)
            tol = 1e-6 * (1 + scale[m])
            gu, gl = out_u[b, m, :Mb], out_l[b, m, :Mb]
            assert np.all(gu >= ou - 1e-12 * (1 + scale[m]))       # rounded up
            assert np.all(gl <= ol + 1e-12 * (1 + scale[m]))       # rounded down
            assert np.max(np.abs(gu - ou)) <= tol and np.max(np.abs(gl - ol)) <= tol


# ---------------------------------------------------------------- a2
@pytest.mark.parametrize("n,D,order,budget", [
    (1, 6, 6, 0), (2, 4, 4, 0), (2, 4, 7, 0), (3, 8, 8, 0), (3, 8, 16, 0), (3, 6, 4, 0),
    (4, 4, 4, 0), (4, 8, 8, 0), (3, 8, 8, 100), (5, 2, 2, 0), (2, 1, 1, 0),
    # six inputs at order 8 (the branch-and-bound network's fourth hidden layer)
    (6, 8, 8, 0)])
def test_enclose_step(ctx, n, D, order, budget):
    rng = np.random.default_rng(7 * n + D + order)
    M = bern.num_monomials(n, D)
    h, B = 3, 8
    items = B * h
    up = np.zeros((items, M), np.float32)
    lo = np.zeros((items, M), np.float32)
    nt = np.zeros(items, np.int32)
    for i in range(items):
        k = M if i % 3 else bern.num_monomials(n, int(rng.integers(0, D + 1)))
        nt[i] = k
        base = random_dense(rng, n, D)[:k]
        up[i, :k] = base + 0.1
        lo[i, :k] = base - 0.1
    # layer block [B][M][h]; unused entries are poison
    blk_u = np.where(np.arange(M)[None, :] < nt[:, None], up, np.float32(np.nan))
    blk_l = np.where(np.arange(M)[None, :] < nt[:, None], lo, np.float32(np.nan))
    blk_u = np.ascontiguousarray(blk_u.reshape(B, h, M).transpose(0, 2, 1))
    blk_l = np.ascontiguousarray(blk_l.reshape(B, h, M).transpose(0, 2, 1))
    glo = torch.zeros(items, device="cuda")
    ghi = torch.zeros(items, device="cuda")
    ctx.enclose(n, B, h, order, budget, dev(blk_u), dev(blk_l), M, dev(nt), glo, ghi)
    assert ctx.sync() == 0
    glo, ghi = glo.cpu().numpy().astype(np.float64), ghi.cpu().numpy().astype(np.float64)
    eff_budget = budget if budget > 0 else 1 << 20    # the default budget, honoured
    from parity_util import dict_from_dense
    for i in range(items):
        pu = dict_from_dense(up[i, : nt[i]].astype(np.float64), n)
        pl = dict_from_dense(lo[i, : nt[i]].astype(np.float64), n)
        o_lo = oracle.enclosure(pl, n, min(order, 24), eff_budget)[0]
        o_hi = oracle.enclosure(pu, n, min(order, 24), eff_budget)[1]
        sc = 1 + l1(up[i]) + l1(lo[i])
        assert glo[i] <= o_lo + 1e-12 * sc and ghi[i] >= o_hi - 1e-12 * sc
        assert o_lo - glo[i] <= 1e-5 * sc and ghi[i] - o_hi <= 1e-5 * sc


# ---------------------------------------------------------------- a3
@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 8, 12, 16])
def test_relu_coeffs_step(ctx, d):
    rng = np.random.default_rng(d)
    N = 64
    lo = rng.uniform(-3, 1, N).astype(np.float32)
    hi = (lo + rng.uniform(0.01, 4, N)).astype(np.float32)
    lo[:4] = [0.0, -1.0, -2.0, 1e-30]
    hi[:4] = [1.0, 0.0, -1.0, 2.0]
    lo[4], hi[4] = -6.0, 10.0                       # the interval of Table 1
    kind = torch.zeros(N, dtype=torch.int8, device="cuda")
    coef = torch.zeros(N * bern.COEF_STRIDE, device="cuda")
    eps = torch.zeros(N, device="cuda")
    ctx.relu_coeffs(N, dev(lo), dev(hi), None, d, kind, coef, eps)
    assert ctx.sync() == 0
    kind = kind.cpu().numpy()
    coef = coef.cpu().numpy().reshape(N, -1).astype(np.float64)
    eps = eps.cpu().numpy().astype(np.float64)
    for i in range(N):
        l, h = float(lo[i]), float(hi[i])
        want = 0 if h <= 0 else (1 if l >= 0 else 2)
        assert kind[i] == want
        if want != 2:
            continue
        a, e = oracle.relu_coeffs(l, h, d)
        mag = (h - l) * 2 ** d
        assert np.all(coef[i, : d + 1] >= a - 1e-14 * mag)
        assert np.all(coef[i, : d + 1] - a <= 2.5e-7 * np.abs(a) + 1e-9 * mag)
        assert eps[i] >= e and eps[i] - e <= 1e-6 * (1 + abs(e)) + 2.5e-7 * np.abs(a).sum()
    # Table 1: the shift on [-6,10] times the width is the printed band area
    if d in (2, 3, 8):
        area = {2: 37.5, 3: 28.1, 8: 16.9}[d]
        assert abs(eps[4] * 16 - area) <= 0.05 + 1e-5


# ---------------------------------------------------------------- a4
@pytest.mark.parametrize("n,D,d,cap", [(2, 2, 2, 16), (3, 4, 2, 16), (3, 8, 2, 16), (2, 4, 2, 6),
                                       (4, 4, 2, 8), (3, 4, 1, 16), (1, 8, 2, 16), (6, 2, 2, 16)])
def test_compose_step(ctx, n, D, d, cap):
    rng = np.random.default_rng(1000 + 10 * n + D + cap)
    M = bern.num_monomials(n, D)
    Mout = bern.num_monomials(n, min(d * D, cap))
    h, B = 4, 3
    items = h * B
    pu = np.zeros((items, M), np.float32)
    pl = np.zeros((items, M), np.float32)
    nt = np.full(items, M, np.int32)
    nt[3] = bern.num_monomials(n, max(0, D - 1))      # ragged: lower degree
    lo = np.zeros(items, np.float32)
    hi = np.zeros(items, np.float32)
    from parity_util import dict_from_dense
    for i in range(items):
        base = random_dense(rng, n, D, scale=0.5)
        base[nt[i]:] = 0
        gap = np.abs(random_dense(rng, n, D, scale=0.05))
        gap[nt[i]:] = 0
        pu[i] = base + gap
        pl[i] = base - gap
        l_, _ = oracle.enclosure(dict_from_dense(pl[i, : nt[i]].astype(np.float64), n), n, D)
        _, h_ = oracle.enclosure(dict_from_dense(pu[i, : nt[i]].astype(np.float64), n), n, D)
        lo[i] = np.nextafter(np.float32(l_), np.float32(-np.inf))
        hi[i] = np.nextafter(np.float32(h_), np.float32(np.inf))
        if not (lo[i] < 0 < hi[i]):
            shift = np.float32((float(lo[i]) + float(hi[i])) / 2)
            pu[i, 0] -= shift
            pl[i, 0] -= shift
            lo[i] = np.float32(lo[i] - shift) - np.float32(1e-3)
            hi[i] = np.float32(hi[i] - shift) + np.float32(1e-3)
    kind = torch.zeros(items, dtype=torch.int8, device="cuda")
    coef = torch.zeros(items * bern.COEF_STRIDE, device="cuda")
    eps = torch.zeros(items, device="cuda")
    glo, ghi = dev(lo), dev(hi)
    ctx.relu_coeffs(items, glo, ghi, None, d, kind, coef, eps)
    blk_u = np.ascontiguousarray(pu.reshape(B, h, M).transpose(0, 2, 1))
    blk_l = np.ascontiguousarray(pl.reshape(B, h, M).transpose(0, 2, 1))
    qu = torch.full((B * Mout * h,), np.nan, device="cuda")
    ql = torch.full_like(qu, np.nan)
    qnt = torch.zeros(items, dtype=torch.int32, device="cuda")
    ctx.compose(n, B, h, cap, 0.0, kind, coef, eps, None, d, glo, ghi, dev(blk_u), dev(blk_l), M,
                dev(nt), qu, ql, Mout, qnt)
    assert ctx.sync() == 0
    assert np.all(kind.cpu().numpy() == 2)
    qu = qu.cpu().numpy().reshape(B, Mout, h).transpose(0, 2, 1).reshape(items, Mout).astype(np.float64)
    ql = ql.cpu().numpy().reshape(B, Mout, h).transpose(0, 2, 1).reshape(items, Mout).astype(np.float64)
    qnt = qnt.cpu().numpy()
    pts = rng.random((300, n))
    pts[0] = 1.0
    pts[1] = 0.0
    for i in range(items):
        Di = 0
        while bern.num_monomials(n, Di) < nt[i]:
            Di += 1
        Mi = bern.num_monomials(n, min(d * Di, cap))
        assert qnt[i] == Mi
        P_u = dict_from_dense(pu[i, : nt[i]].astype(np.float64), n)
        P_l = dict_from_dense(pl[i, : nt[i]].astype(np.float64), n)
        ou = dense_from_dict(oracle.compose(P_u, n, float(lo[i]), float(hi[i]), d, True, cap=cap), n, Mi)
        ol = dense_from_dict(oracle.compose(P_l, n, float(lo[i]), float(hi[i]), d, False, cap=cap), n, Mi)
        gu, gl = qu[i, :Mi], ql[i, :Mi]
        tol = 1e-4 * (1 + l1(ou))
        assert np.abs(gu - ou).sum() <= tol and np.abs(gl - ol).sum() <= tol
        # sound side, value-wise on the box
        sc = 1e-9 * (1 + l1(ou))
        assert np.all(eval_dense(gu, n, pts) >= eval_dense(ou, n, pts) - sc)
        assert np.all(eval_dense(gl, n, pts) <= eval_dense(ol, n, pts) + sc)


def test_compose_stable_cases(ctx):
    """Identity items copy their input, zero items produce no terms (one box,
    three neurons)."""
    n, D = 2, 2
    M = bern.num_monomials(n, D)
    rng = np.random.default_rng(3)
    pu = random_dense(rng, n, D).reshape(1, M).repeat(3, 0)
    pl = (pu - 0.25).astype(np.float32)
    lo = np.array([-2, 0.5, -1], np.float32)
    hi = np.array([-0.5, 2, 1], np.float32)
    nt = np.full(3, M, np.int32)
    kind = torch.zeros(3, dtype=torch.int8, device="cuda")
    coef = torch.zeros(3 * bern.COEF_STRIDE, device="cuda")
    eps = torch.zeros(3, device="cuda")
    ctx.relu_coeffs(3, dev(lo), dev(hi), None, 2, kind, coef, eps)
    Mout = bern.num_monomials(n, 2 * D)
    qu = torch.zeros(Mout * 3, device="cuda")
    ql = torch.zeros_like(qu)
    qnt = torch.zeros(3, dtype=torch.int32, device="cuda")
    ctx.compose(n, 1, 3, 16, 0.0, kind, coef, eps, None, 2, dev(lo), dev(hi),
                dev(np.ascontiguousarray(pu.T)), dev(np.ascontiguousarray(pl.T)), M, dev(nt), qu,
                ql, Mout, qnt)
    assert ctx.sync() == 0
    assert list(kind.cpu().numpy()) == [0, 1, 2]
    qnt = qnt.cpu().numpy()
    assert qnt[0] == 0 and qnt[1] == M and qnt[2] == Mout
    qu = qu.cpu().numpy().reshape(Mout, 3).T
    ql = ql.cpu().numpy().reshape(Mout, 3).T
    assert np.array_equal(qu[1, :M], pu[1]) and np.array_equal(ql[1, :M], pl[1])


@pytest.mark.parametrize("n,D,d,cap,tau", [(3, 4, 2, 16, 0.0), (3, 8, 2, 16, 0.0),
                                           (2, 4, 3, 16, 0.0), (3, 4, 2, 16, 1e-3),
                                           (4, 4, 2, 8, 0.0), (2, 4, 1, 16, 0.0)])
def test_compose_in_place_matches_separate_blocks(ctx, n, D, d, cap, tau):
    """bern_compose in place (post block = pre block, the post stride) gives
    the bits of the separate-block call, including identity items (whose
    coefficients stay where they are) and zero items, on the row, Horner and
    linear paths.  (In place the step entry point sizes its kernels by the
    stride, so shapes whose pair-list inputs would not fit shared memory at
    that stride are declined; bern_propagate passes the true capacity.)"""
    rng = np.random.default_rng(2000 + 100 * n + 10 * D + d)
    M = bern.num_monomials(n, D)
    Mout = bern.num_monomials(n, min(max(d, 1) * D, cap))
    h, B = 8, 3
    items = h * B
    base = rng.normal(0, 0.3, (items, M)).astype(np.float32)
    gap = np.abs(rng.normal(0, 0.01, (items, M))).astype(np.float32)
    pu, pl = base + gap, base - gap
    mag = np.abs(pu).sum(1) + np.abs(pl).sum(1)
    lo = (-mag - 0.1).astype(np.float32)
    hi = (mag + 0.2).astype(np.float32)
    # a dead and an identity item in every box
    for b in range(B):
        hi[b * h + 1] = -0.5
        lo[b * h + 1] = -1.0
        lo[b * h + 2] = 0.5
        hi[b * h + 2] = 1.5
    glo, ghi = dev(lo), dev(hi)
    kind = torch.zeros(items, dtype=torch.int8, device="cuda")
    coef = torch.zeros(items * bern.COEF_STRIDE, device="cuda")
    eps = torch.zeros(items, device="cuda")
    ctx.relu_coeffs(items, glo, ghi, None, d, kind, coef, eps)
    nt = dev(np.full(items, M, np.int32))

    def block(a, ld):
        out = np.zeros((B, ld, h), np.float32)
        out[:, :M, :] = a.reshape(B, h, M).transpose(0, 2, 1)
        return dev(out.reshape(-1))

    su, sl = block(pu, M), block(pl, M)
    qu = torch.full((B * Mout * h,), np.nan, device="cuda")
    ql = torch.full_like(qu, np.nan)
    qn = torch.zeros(items, dtype=torch.int32, device="cuda")
    ctx.compose(n, B, h, cap, tau, kind, coef, eps, None, d, glo, ghi, su, sl, M, nt, qu, ql, Mout,
                qn)
    iu, il = block(pu, Mout), block(pl, Mout)
    qn2 = torch.zeros(items, dtype=torch.int32, device="cuda")
    ctx.compose(n, B, h, cap, tau, kind, coef, eps, None, d, glo, ghi, iu, il, Mout, nt, iu, il,
                Mout, qn2)
    assert ctx.sync() == 0
    qn, qn2 = qn.cpu().numpy(), qn2.cpu().numpy()
    assert np.array_equal(qn, qn2)
    a_u = qu.cpu().numpy().reshape(B, Mout, h)
    a_l = ql.cpu().numpy().reshape(B, Mout, h)
    b_u = iu.cpu().numpy().reshape(B, Mout, h)
    b_l = il.cpu().numpy().reshape(B, Mout, h)
    for b in range(B):
        for m in range(h):
            k = int(qn[b * h + m])
            assert np.array_equal(a_u[b, :k, m], b_u[b, :k, m]), (b, m)
            assert np.array_equal(a_l[b, :k, m], b_l[b, :k, m]), (b, m)


def test_compose_partial_alias_rejected(ctx):
    """Aliasing only one bound, or in place at two strides, is BERN_E_INVALID."""
    n, D = 2, 2
    M = bern.num_monomials(n, D)
    Mo = bern.num_monomials(n, 4)
    z = torch.zeros(4 * Mo, device="cuda")
    z2 = torch.zeros(4 * Mo, device="cuda")
    kind = torch.zeros(4, dtype=torch.int8, device="cuda")
    coef = torch.zeros(4 * bern.COEF_STRIDE, device="cuda")
    f = torch.zeros(4, device="cuda")
    nt = torch.full((4,), M, dtype=torch.int32, device="cuda")
    qn = torch.zeros(4, dtype=torch.int32, device="cuda")
    for pu, pl, qu, ql, pld, qld in ((z, z2, z, torch.zeros_like(z), Mo, Mo),
                                     (z, z2, z, z2, M, Mo)):
        with pytest.raises(bern.BernError) as ei:
            ctx.compose(n, 1, 4, 16, 0.0, kind, coef, f, None, 2, f, f, pu, pl, pld, nt, qu, ql,
                        qld, qn)
        assert ei.value.code == bern.BERN_E_INVALID

