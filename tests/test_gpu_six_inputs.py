"""GPU parity of the six-input composition paths against the FP64 oracle.

The branch-and-bound network ([6,64x4,1], cap 16) squares degree-8
polynomials in six variables at its fourth hidden layer: 3003 input terms,
74,613 output terms.  Six inputs are beyond the row-convolution kernel, so
order 2 runs on the per-item pair lists, and with pruning (tau > 0) on the
Horner kernel whose buffers (about 1.2 MB per item) live in a global
workspace.  Both are compared here element by element with the oracle's
Step 3 (Sec. 5.1, eqs. post_bounds_1/2), at the whole-path tolerance
1e-4 (1 + ||p||_1) in summed absolute coefficient difference, plus the sound
side at sampled points of the box."""
import numpy as np
import pytest

import oracle
from paper_2211_14438_gb300 import bern
from parity_util import dense_from_dict, dict_from_dense, eval_dense, l1, random_dense

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

N, D, CAP = 6, 8, 16
M = bern.num_monomials(N, D)               # 3003
MOUT = bern.num_monomials(N, 2 * D)        # 74613 (2D = cap)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _items(seed, B, h):
    """Random degree-8 pre-activation bounds with an interval [lo, hi] that
    contains them on the box and straddles 0 (unstable items)."""
    rng = np.random.default_rng(seed)
    items = B * h
    pu = np.zeros((items, M), np.float32)
    pl = np.zeros((items, M), np.float32)
    lo = np.zeros(items, np.float32)
    hi = np.zeros(items, np.float32)
    for i in range(items):
        # coefficients shrink with the degree, as in a network's layer blocks
        deg = np.array([sum(r) for r in bern.monomials(N, D)], np.float64)
        base = random_dense(rng, N, D, scale=0.3) * (0.5 ** deg).astype(np.float32)
        gap = np.abs(random_dense(rng, N, D, scale=0.01)) * (0.5 ** deg).astype(np.float32)
        pu[i] = base + gap
        pl[i] = base - gap
        pu[i, 0] = pl[i, 0] = 0.0
        # every monomial lies in [0,1] on the box: the coefficient-sign interval
        # contains each polynomial; centre it on 0 so the item is unstable
        l_ = float(np.minimum(pl[i, 1:], 0).sum())
        h_ = float(np.maximum(pu[i, 1:], 0).sum())
        shift = np.float32(-(l_ + h_) / 2)
        pu[i, 0] = shift + np.float32(0.001)
        pl[i, 0] = shift - np.float32(0.001)
        lo[i] = np.float32(l_ + float(pl[i, 0]) - 1e-3)
        hi[i] = np.float32(h_ + float(pu[i, 0]) + 1e-3)
        assert lo[i] < 0 < hi[i]
    return pu, pl, lo, hi


def _run(ctx, pu, pl, lo, hi, B, h, tau):
    items = B * h
    kind = torch.zeros(items, dtype=torch.int8, device="cuda")
    coef = torch.zeros(items * bern.COEF_STRIDE, device="cuda")
    eps = torch.zeros(items, device="cuda")
    glo, ghi = dev(lo), dev(hi)
    ctx.relu_coeffs(items, glo, ghi, None, 2, kind, coef, eps)
    blk_u = pu.reshape(B, h, M).transpose(0, 2, 1)
    blk_l = pl.reshape(B, h, M).transpose(0, 2, 1)
    qu = torch.full((B * MOUT * h,), np.nan, device="cuda")
    ql = torch.full_like(qu, np.nan)
    qnt = torch.zeros(items, dtype=torch.int32, device="cuda")
    nt = np.full(items, M, np.int32)
    ctx.compose(N, B, h, CAP, tau, kind, coef, eps, None, 2, glo, ghi, dev(blk_u), dev(blk_l),
                M, dev(nt), qu, ql, MOUT, qnt)
    assert ctx.sync() == 0
    assert np.all(kind.cpu().numpy() == 2)
    qu = qu.cpu().numpy().reshape(B, MOUT, h).transpose(0, 2, 1).reshape(items, MOUT)
    ql = ql.cpu().numpy().reshape(B, MOUT, h).transpose(0, 2, 1).reshape(items, MOUT)
    return qu.astype(np.float64), ql.astype(np.float64), qnt.cpu().numpy()


def _check(qu, ql, qnt, pu, pl, lo, hi, tau, rng):
    pts = rng.random((64, N))
    pts[0] = 1.0
    pts[1] = 0.0
    for i in range(len(lo)):
        Pu = dict_from_dense(pu[i].astype(np.float64), N)
        Pl = dict_from_dense(pl[i].astype(np.float64), N)
        ou = dense_from_dict(oracle.compose(Pu, N, float(lo[i]), float(hi[i]), 2, True, cap=CAP,
                                            tau=tau, cap_terms=1 << 17), N, MOUT)
        ol = dense_from_dict(oracle.compose(Pl, N, float(lo[i]), float(hi[i]), 2, False, cap=CAP,
                                            tau=tau, cap_terms=1 << 17), N, MOUT)
        k = int(qnt[i])
        assert 0 < k <= MOUT
        gu = np.zeros(MOUT)
        gl = np.zeros(MOUT)
        gu[:k], gl[:k] = qu[i, :k], ql[i, :k]
        assert np.all(np.isfinite(gu)) and np.all(np.isfinite(gl))
        tol_u, tol_l = 1e-4 * (1 + l1(ou)), 1e-4 * (1 + l1(ol))
        assert np.abs(gu - ou).sum() <= tol_u, (i, np.abs(gu - ou).sum(), tol_u)
        assert np.abs(gl - ol).sum() <= tol_l, (i, np.abs(gl - ol).sum(), tol_l)
        sc_u, sc_l = 1e-9 * (1 + l1(ou)), 1e-9 * (1 + l1(ol))
        if tau == 0.0:
            assert np.all(eval_dense(gu, N, pts) >= eval_dense(ou, N, pts) - sc_u)
            assert np.all(eval_dense(gl, N, pts) <= eval_dense(ol, N, pts) + sc_l)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    yield c
    c.close()


def test_compose_pairs_six_inputs_degree8(ctx):
    """Order 2 at input degree 8, tau = 0: the pair-list kernel."""
    B, h = 2, 2
    pu, pl, lo, hi = _items(601, B, h)
    qu, ql, qnt = _run(ctx, pu, pl, lo, hi, B, h, 0.0)
    assert np.all(qnt == MOUT)
    _check(qu, ql, qnt, pu, pl, lo, hi, 0.0, np.random.default_rng(6010))


def test_compose_horner_global_workspace_six_inputs_degree8():
    """Order 2 with pruning (tau = 1e-7, the branch-and-bound setting): the
    Horner kernel with its buffers in the global workspace (a shared-memory
    limit of 0 forces that path).  The oracle prunes the same terms up to
    rounding at the threshold (either choice is sound; the difference is
    within 2 tau ||q||_1 per product)."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    c = bern.Context(0)
    try:
        c.set_horner_smem_limit(0)
        B, h = 2, 2
        pu, pl, lo, hi = _items(602, B, h)
        qu, ql, qnt = _run(c, pu, pl, lo, hi, B, h, 1e-7)
        _check(qu, ql, qnt, pu, pl, lo, hi, 1e-7, np.random.default_rng(6020))
    finally:
        c.close()
