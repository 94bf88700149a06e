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
