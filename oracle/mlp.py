"""Oracle of the learned component: the two-layer MLP (plain numpy, float64).

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline leg, never by the library.

The model (not from the paper; the paper has no learned part): features x,
hidden width H = 64,

    a = relu(W1 x + b1),   z = W2 a + b2,   p = softmax(z),
    L = (1/n) sum_s w_s * (-log p_s[y_s]).

`emulate=True` applies the BF16 roundings the GPU kernels use (x, W1, W2 and
the activations a rounded to bfloat16, round to nearest even) and keeps
everything else in float64; `emulate=False` is the plain float64 model that
the finite-difference pins check.  The flat parameter vector holds W1 [H x F]
(row-major), b1 [H], W2 [C x H], b2 [C] in that order.

The degree features follow the library's definition of the (box, neuron)
features; they are computed here in float64 and returned as float32.
"""
import numpy as np

H = 64


def num_params(F: int, C: int) -> int:
    return H * F + H + C * H + C


def unpack(theta, F: int, C: int):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + H * F].reshape(H, F); o += H * F
    b1 = theta[o:o + H]; o += H
    W2 = theta[o:o + C * H].reshape(C, H); o += C * H
    b2 = theta[o:o + C]
    return W1, b1, W2, b2


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) from the float32 value of x;
    returns float64 holding the bfloat16 values."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    # add half an ulp of the 16 dropped bits, plus one if the kept lsb is odd
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


def forward(theta, F: int, C: int, x, emulate: bool = True):
    """Logits z [n x C], plus the intermediates (xb, z1, a)."""
    W1, b1, W2, b2 = unpack(theta, F, C)
    x = np.asarray(x, dtype=np.float64).reshape(-1, F)
    if emulate:
        W1, W2, xb = bf16(W1), bf16(W2), bf16(x)
    else:
        xb = x
    z1 = xb @ W1.T + b1
    a = np.maximum(z1, 0.0)
    if emulate:
        a = bf16(a)
    z = a @ W2.T + b2
    return z, (xb, z1, a)


def loss_and_grad(theta, F: int, C: int, x, labels, w=None, emulate: bool = True):
    """Mean weighted softmax cross-entropy and its gradient with respect to
    the flat parameter vector (the roundings count as the identity in the
    derivative)."""
    W1, b1, W2, b2 = unpack(theta, F, C)
    if emulate:
        W2 = bf16(W2)
    z, (xb, z1, a) = forward(theta, F, C, x, emulate)
    n = z.shape[0]
    y = np.asarray(labels, dtype=np.int64)
    w = np.ones(n) if w is None else np.asarray(w, dtype=np.float64)
    zs = z - z.max(axis=1, keepdims=True)
    e = np.exp(zs)
    s = e.sum(axis=1, keepdims=True)
    p = e / s
    ce = np.log(s[:, 0]) - zs[np.arange(n), y]
    loss = float(np.sum(w * ce) / n)
    onehot = np.zeros_like(p)
    onehot[np.arange(n), y] = 1.0
    dz = w[:, None] * (p - onehot) / n
    dW2 = dz.T @ a
    db2 = dz.sum(axis=0)
    dz1 = (dz @ W2) * (z1 > 0)
    dW1 = dz1.T @ xb
    db1 = dz1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2])
    return loss, g


def adam(theta, m, v, g, lr, beta1, beta2, eps, t):
    """One Adam step (Kingma & Ba 2015, Algorithm 1) with bias correction."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def degree_features(lo, hi, nterms, layer: int) -> np.ndarray:
    """The 8 features of (box, neuron) items for degree proposals."""
    lo = np.asarray(lo, dtype=np.float32).astype(np.float64)
    hi = np.asarray(hi, dtype=np.float32).astype(np.float64)
    nt = np.maximum(np.asarray(nterms, dtype=np.float64), 1.0)
    s = np.maximum(np.maximum(np.abs(lo), np.abs(hi)), 1e-30)
    width = np.asarray(hi.astype(np.float32) - lo.astype(np.float32), dtype=np.float64)
    kink = np.where(lo >= 0, 0.0, np.where(hi <= 0, 1.0,
                                           np.clip(-lo / np.where(width > 0, width, 1.0), 0, 1)))
    f = np.stack([lo / s, hi / s, np.log2(np.maximum(width, 1e-30)) / 8,
                  np.full_like(lo, layer / 8.0), np.log2(nt) / 16,
                  (lo >= 0).astype(np.float64), (hi <= 0).astype(np.float64), kink], axis=-1)
    return f.astype(np.float32)


class DegreeChooser:
    """Order proposals of a degree MLP for the oracle's propagation (a
    callable for oracle.propagate): features -> bf16-emulated forward ->
    the first maximum of the softmax; below min_conf the fallback order.
    Records the smallest decision margin seen (the gap between the two
    largest probabilities, and the distance of the largest from min_conf),
    so that a caller can tell a genuine near-tie from a disagreement."""

    def __init__(self, theta, min_conf: float = 0.0, fallback: int = 2, classes: int = 4):
        self.theta = np.asarray(theta, dtype=np.float64)
        self.min_conf, self.fallback, self.C = float(min_conf), int(fallback), int(classes)
        self.margin = np.inf
        self.chosen = []

    def __call__(self, layer, m, lo, hi, nterms):
        x = degree_features([lo], [hi], [nterms], layer)
        z, _ = forward(self.theta, x.shape[1], self.C, x, emulate=True)
        z = z[0]
        p = np.exp(z - z.max())
        p /= p.sum()
        order = np.argsort(-p, kind="stable")
        best, second = p[order[0]], p[order[1]]
        self.margin = min(self.margin, best - second)
        if self.min_conf > 0:
            self.margin = min(self.margin, abs(best - self.min_conf))
        d = int(order[0]) + 1 if best >= self.min_conf else self.fallback
        self.chosen.append(d)
        return d
