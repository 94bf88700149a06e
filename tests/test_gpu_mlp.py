"""The learned component's BF16 kernels (features, inference, gradient, Adam)
through the C ABI against the CPU oracle (oracle/mlp.py), and GPU training on
a separable toy problem.

Tolerances: the GPU and the oracle round the same inputs and weights to
bfloat16; the GPU accumulates in float32, the oracle in float64, so a hidden
activation near a bfloat16 rounding boundary may land one bfloat16 ulp
(2^-8 relative) apart.  Logits: every sample within 1e-2 * (1 + |z|) and 99%
of them within 1e-4 * (1 + |z|).  Gradients: within 1e-3 of the largest
gradient entry.  Loss: 1e-5 relative."""
import numpy as np
import pytest

from oracle import mlp as om
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


def problem(F, C, n, seed):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.5, om.num_params(F, C)).astype(np.float32)
    x = rng.normal(0, 1, (n, F)).astype(np.float32)
    y = rng.integers(0, C, n).astype(np.int32)
    w = rng.uniform(0.5, 2.0, n).astype(np.float32)
    return theta, x, y, w


@pytest.mark.parametrize("F,C,n", [(8, 4, 1000), (3, 2, 37), (16, 8, 5000), (8, 4, 1)])
def test_forward_matches_oracle(ctx, F, C, n):
    theta, x, _, _ = problem(F, C, n, F * C + n)
    m = bern.Mlp(torch, F, C, theta)
    xd = torch.from_numpy(x).cuda()
    z = torch.empty(n, C, device="cuda")
    ctx.mlp_forward(m, xd, z)
    assert ctx.sync() == 0
    zg = z.cpu().numpy().astype(np.float64)
    zo, _ = om.forward(theta.astype(np.float64), F, C, x, emulate=True)
    err = np.abs(zg - zo) / (1 + np.abs(zo))
    assert np.all(err <= 1e-2)
    assert np.mean(err.max(axis=1) <= 1e-4) >= 0.99


@pytest.mark.parametrize("F,C,n,weighted", [(8, 4, 3000, False), (8, 4, 1500, True),
                                            (5, 3, 7, True), (16, 8, 2049, False)])
def test_backward_matches_oracle(ctx, F, C, n, weighted):
    theta, x, y, w = problem(F, C, n, 100 + n)
    m = bern.Mlp(torch, F, C, theta)
    P = om.num_params(F, C)
    g = torch.empty(P, device="cuda")
    loss = torch.empty(1, device="cuda")
    wd = torch.from_numpy(w).cuda() if weighted else None
    ctx.mlp_backward(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), wd, g, loss)
    assert ctx.sync() == 0
    lo, go = om.loss_and_grad(theta.astype(np.float64), F, C, x, y, w if weighted else None,
                              emulate=True)
    assert float(loss.item()) == pytest.approx(lo, rel=1e-5)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(gg - go)) <= 1e-3 * np.max(np.abs(go))
    # deterministic: a second call gives the same bits
    g2 = torch.empty_like(g)
    ctx.mlp_backward(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), wd, g2, loss)
    assert torch.equal(g, g2)


def test_adam_step_matches_oracle(ctx):
    F, C = 8, 4
    theta, x, y, _ = problem(F, C, 500, 7)
    m = bern.Mlp(torch, F, C, theta)
    P = om.num_params(F, C)
    g = torch.empty(P, device="cuda")
    loss = torch.empty(1, device="cuda")
    th = theta.astype(np.float64)
    mo, vo = np.zeros(P), np.zeros(P)
    for t in range(1, 4):
        ctx.mlp_backward(m, torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), None, g, loss)
        gh = g.cpu().numpy().astype(np.float64)
        ctx.mlp_adam(m, g, 1e-2)
        th, mo, vo = om.adam(th, mo, vo, gh, 1e-2, 0.9, 0.999, 1e-8, t)
        assert ctx.sync() == 0
        got = m.theta()
        assert np.max(np.abs(got - th)) <= 1e-6 * (1 + np.max(np.abs(th)))
        th = got          # continue from the GPU's float32 state
        mo = m.m.cpu().numpy().astype(np.float64)
        vo = m.v.cpu().numpy().astype(np.float64)
    # the bf16 copies are the round-to-nearest-even images of the masters
    H = bern.BERN_MLP_HIDDEN
    p = m.param.cpu().numpy()
    w1 = m.W1.cpu().view(torch.bfloat16).float().numpy()
    w2 = m.W2.cpu().view(torch.bfloat16).float().numpy()
    assert np.array_equal(w1, om.bf16(p[:H * F]).astype(np.float32))
    assert np.array_equal(w2, om.bf16(p[H * F + H:H * F + H + C * H]).astype(np.float32))


def test_degree_features_match_oracle(ctx):
    rng = np.random.default_rng(3)
    n = 4000
    lo = rng.normal(0, 2, n).astype(np.float32)
    hi = (lo + rng.exponential(1.0, n)).astype(np.float32)
    lo[:10] = np.float32(0.0)
    hi[10:20] = np.float32(0.0)
    nt = rng.integers(1, 5000, n).astype(np.int32)
    x = torch.empty(n, bern.BERN_DEGREE_FEATURES, device="cuda")
    ctx.degree_features(n, torch.from_numpy(lo).cuda(), torch.from_numpy(hi).cuda(),
                        torch.from_numpy(nt).cuda(), 3, x)
    assert ctx.sync() == 0
    got = x.cpu().numpy()
    want = om.degree_features(lo, hi, nt, 3)
    assert np.array_equal(got[:, [3, 5, 6]], want[:, [3, 5, 6]])
    assert np.max(np.abs(got - want)) <= 1e-6


def test_training_on_gpu_learns_a_separable_rule(ctx):
    """Labels from a fixed linear teacher on the features: GPU training with
    the library's own backward and Adam kernels reaches high accuracy."""
    F, C, n = 8, 4, 20000
    rng = np.random.default_rng(11)
    x = rng.normal(0, 1, (n, F)).astype(np.float32)
    T = rng.normal(0, 1, (C, F))
    y = np.argmax(x @ T.T, axis=1).astype(np.int32)
    theta = rng.normal(0, 0.1, om.num_params(F, C)).astype(np.float32)
    m = bern.Mlp(torch, F, C, theta)
    xd, yd = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    g = torch.empty(m.n_params, device="cuda")
    loss = torch.empty(1, device="cuda")
    first = None
    for it in range(400):
        ctx.mlp_backward(m, xd, yd, None, g, loss)
        if first is None:
            first = float(loss.item())
        ctx.mlp_adam(m, g, 3e-3)
    assert ctx.sync() == 0
    z = torch.empty(n, C, device="cuda")
    ctx.mlp_forward(m, xd, z)
    acc = float((z.argmax(1).cpu().numpy() == y).mean())
    assert float(loss.item()) < 0.5 * first
    assert acc >= 0.9
