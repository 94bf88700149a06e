"""The paper's dense Bernstein-tensor product on the GPU (bern_bernstein_square,
Prod_Bern of Sec. 4.2) against the FP64 tensor arithmetic of
oracle/bern_tensor.py: every exact coefficient of the square lies in the GPU
interval [c_lo, c_hi].  The interval is the round-to-nearest sum widened by
its a-posteriori bound, gamma_m times the sum of the terms' magnitudes (the
coefficient of the square of |a|), with gamma_m = m u / (1 - m u), u = 2^-24
and m = (l+1)^n + 2n + 6 (every product a cell can sum, plus the scaling,
binomial and division roundings); the bound enters twice on each side (the
numerator and the binomial bracket), so the width is at most 4.5 gamma_m
(1 + magnitude)."""
import numpy as np
import pytest

from oracle import bern_tensor as bt
from paper_2211_14438_gb300 import bern

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,l,P", [(1, 6, 9), (2, 4, 7), (3, 4, 5), (3, 8, 4), (4, 4, 3), (2, 8, 3),
                                   (3, 0, 2)])
def test_bernstein_square_contains_exact(ctx, n, l, P):
    rng = np.random.default_rng(100 * n + l)
    a = rng.normal(0, 1, (P,) + (l + 1,) * n).astype(np.float32)
    a[0] = np.abs(a[0])                       # one all-positive tensor (no cancellation)
    ga = torch.from_numpy(a.reshape(P, -1)).cuda()
    Go = (2 * l + 1) ** n
    hi = torch.full((P, Go), np.nan, device="cuda")
    lo = torch.full((P, Go), np.nan, device="cuda")
    ctx.bernstein_square(n, l, ga, hi, lo)
    assert ctx.sync() == 0
    hi = hi.cpu().numpy().astype(np.float64)
    lo = lo.cpu().numpy().astype(np.float64)
    for p in range(P):
        a64 = a[p].astype(np.float64)
        exact = bt.prod_bern(a64, a64).reshape(-1)
        mag = bt.prod_bern(np.abs(a64), np.abs(a64)).reshape(-1)
        tol64 = 1e-12 * (1 + mag)                # the float64 reference's own rounding
        assert np.all(lo[p] <= exact + tol64), p
        assert np.all(hi[p] >= exact - tol64), p
        m = (l + 1) ** n + 2 * n + 6
        gamma = m * 2.0 ** -24 / (1 - m * 2.0 ** -24)
        assert np.all(hi[p] - lo[p] <= 4.5 * gamma * (1 + mag)), p


def test_bernstein_square_declines_large_weights(ctx):
    """(max_k C(l,k))^n must stay below 2^24 (exact float weights): n = 4 at
    order 8 (70^4) is declined."""
    a = torch.zeros(1, 9 ** 4, device="cuda")
    out = torch.zeros(1, 17 ** 4, device="cuda")
    with pytest.raises(bern.BernError) as ei:
        ctx.bernstein_square(4, 8, a, out, out)
    assert ei.value.code == bern.BERN_E_UNSUPPORTED


@pytest.mark.parametrize("n,l,r,P", [(1, 6, 5, 7), (2, 4, 4, 5), (3, 8, 8, 3), (3, 4, 12, 3),
                                     (4, 3, 3, 3), (2, 0, 5, 4), (3, 2, 0, 4)])
def test_bernstein_elevate_contains_exact(ctx, n, l, r, P):
    """Degree elevation (Sec. 4.3) of interval tensors against the float64
    elevation of oracle/bern_tensor.py: the exact elevation of the upper
    (lower) tensor lies below c_hi (above c_lo), and the directed passes
    widen it by at most n passes of l + 3 roundings relative to the elevated
    magnitudes."""
    rng = np.random.default_rng(1000 * n + 10 * l + r)
    a = rng.normal(0, 1, (P,) + (l + 1,) * n)
    e = np.abs(rng.normal(0, 1e-3, a.shape))
    a_hi = (a + e).astype(np.float32)
    a_lo = (a - e).astype(np.float32)
    gi, go = (l + 1) ** n, (l + r + 1) ** n
    t_hi, t_lo = (torch.from_numpy(x.reshape(P, gi)).cuda() for x in (a_hi, a_lo))
    c_hi = torch.full((P, go), np.nan, device="cuda")
    c_lo = torch.full((P, go), np.nan, device="cuda")
    ctx.bernstein_elevate(n, l, r, t_hi, t_lo, c_hi, c_lo)
    assert ctx.sync() == 0
    c_hi = c_hi.cpu().numpy().astype(np.float64)
    c_lo = c_lo.cpu().numpy().astype(np.float64)
    shape = (l + r + 1,) * n
    for p in range(P):
        eh = bt.elevate(a_hi[p].astype(np.float64), shape).reshape(-1)
        el = bt.elevate(a_lo[p].astype(np.float64), shape).reshape(-1)
        mag = bt.elevate(np.maximum(np.abs(a_hi[p]), np.abs(a_lo[p])).astype(np.float64),
                         shape).reshape(-1)
        tol64 = 1e-12 * (1 + mag)
        assert np.all(c_hi[p] >= eh - tol64) and np.all(c_lo[p] <= el + tol64), p
        slack = 2 * n * (l + 3) * 2.0 ** -24 * (1 + mag)
        assert np.all(c_hi[p] - eh <= slack) and np.all(el - c_lo[p] <= slack), p


def test_bernstein_elevate_declines_out_of_range(ctx):
    a = torch.zeros(1, 16, device="cuda")
    out = torch.zeros(1, 16, device="cuda")
    for n, l, r in ((1, 12, 13), (4, 6, 6)):      # binomials past 2^24; 13^4 cells past 200 KB
        with pytest.raises(bern.BernError) as ei:
            ctx.bernstein_elevate(n, l, r, a, a, out, out)
        assert ei.value.code == bern.BERN_E_UNSUPPORTED


@pytest.mark.parametrize("B,h_out,h_in,G", [(3, 64, 64, 729), (4, 1, 64, 4913), (2, 20, 12, 27),
                                            (3, 64, 64, 10)])
def test_bernstein_affine_bounds_exact(ctx, B, h_out, h_in, G):
    """The layer sum on Bernstein tensors (Sum_Bern with weights, the bias on
    every coefficient) against the sign-split sums in float64: every exact
    output coefficient lies in [out_lo, out_hi], within a few float32
    roundings of the summed magnitudes."""
    rng = np.random.default_rng(B * 1000 + h_out + G)
    x = rng.normal(0, 1, (B, G, h_in))
    e = np.abs(rng.normal(0, 1e-2, x.shape))
    hi = (x + e).astype(np.float32)
    lo = (x - e).astype(np.float32)
    W = (rng.normal(size=(h_out, h_in)) / np.sqrt(h_in)).astype(np.float32)
    b = rng.uniform(-0.5, 0.5, h_out).astype(np.float32)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    oh = torch.full((B, G, h_out), np.nan, device="cuda")
    ol = torch.full((B, G, h_out), np.nan, device="cuda")
    ctx.bernstein_affine(B, h_out, h_in, dev(W), dev(b), G, dev(hi), dev(lo), oh, ol)
    assert ctx.sync() == 0
    oh = oh.cpu().numpy().astype(np.float64)
    ol = ol.cpu().numpy().astype(np.float64)
    Wp, Wm = np.maximum(W, 0).astype(np.float64), np.minimum(W, 0).astype(np.float64)
    h64, l64 = hi.astype(np.float64), lo.astype(np.float64)
    up = b + h64 @ Wp.T + l64 @ Wm.T
    dn = b + l64 @ Wp.T + h64 @ Wm.T
    scale = 1 + np.abs(b) + np.maximum(np.abs(h64), np.abs(l64)) @ np.abs(W.astype(np.float64)).T
    assert np.all(oh >= up - 1e-12 * scale) and np.all(ol <= dn + 1e-12 * scale)
    slack = 4 * (h_in + 2) * 2.0 ** -24 * scale
    assert np.all(oh - up <= slack) and np.all(dn - ol <= slack)
