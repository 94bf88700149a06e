"""The learned component: per-neuron ReLU-order proposals from a small BF16
MLP, trained on the GPU with the library's own forward/backward/Adam kernels
on labels that the plain method itself produces.

Labels (the method has no learned part; this is the project's reading of
"labelled by plain-method bound widths"):

* For every training box b, hidden layer i and candidate order d in {1..4},
  the plain method runs with order d at layer i and the base order (2)
  everywhere else; W[b, i, d] is the box's mean output-bound width and
  cost[i, d] the plan's measured GPU time per box.
* Each (box, layer) gets the order minimising  cost[i, d] + lam * W[b, i, d];
  lam is the smallest value for which the predicted mean width (the base
  width plus the per-layer width changes) does not exceed the base plan's
  mean width, so the labels trade time for width only where it is cheap and
  never loosen the batch on average.
* Every hidden neuron of (b, i) is a training sample with that label and the
  features of bern_degree_features taken from the base plan's trace.

The plain method computes sound bounds for whatever order the MLP proposes
(BERN_DEG_LEARNED); a neuron whose largest class probability is below
min_conf uses the base order (the fallback).
"""
from __future__ import annotations

import time
from typing import Dict, List, Sequence, Tuple

import numpy as np

from . import bern

CLASSES = bern.BERN_DEGREE_CLASSES        # class c proposes order c + 1
FEATURES = bern.BERN_DEGREE_FEATURES


def _torch():
    import torch
    return torch


def _dev_net(widths, W, b):
    torch = _torch()
    return ([torch.as_tensor(np.asarray(w, np.float32)).cuda() for w in W],
            [torch.as_tensor(np.asarray(x, np.float32)).cuda() for x in b])


def hidden_slices(widths) -> List[Tuple[int, int, int]]:
    """(layer (1-based), offset, width) of every hidden layer in the trace."""
    out, off = [], 0
    for i, h in enumerate(widths[1:-1]):
        out.append((i + 1, off, int(h)))
        off += int(h)
    return out


def mean_width(out) -> np.ndarray:
    """Per box: the mean over outputs of hi - lo."""
    return (out["hi"] - out["lo"]).float().mean(dim=1).cpu().numpy().astype(np.float64)


def timed_propagate(ctx, widths, Wd, bd, boxes_d, degree, cap, reps=3, **kw):
    """One warm-up plus `reps` timed runs (CUDA events); returns (out, ms)."""
    torch = _torch()
    out = ctx.propagate(widths, Wd, bd, boxes_d, degree=degree, cap=cap, **kw)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        ctx.propagate(widths, Wd, bd, boxes_d, degree=degree, cap=cap, out=out, sync=False,
                      **kw)
    ev1.record()
    torch.cuda.synchronize()
    ctx.check("propagate")
    return out, ev0.elapsed_time(ev1) / reps


def width_table(ctx, widths, W, b, boxes, cap=16, base=2):
    """W[b, i, d-1] and cost[i, d-1] (ms per box) for every hidden layer i
    and order d in 1..CLASSES, with the base order elsewhere."""
    torch = _torch()
    Wd, bd = _dev_net(widths, W, b)
    boxes_d = torch.as_tensor(np.ascontiguousarray(boxes, np.float32)).cuda()
    B = boxes.shape[0]
    H1 = len(widths) - 2
    table = np.zeros((B, H1, CLASSES))
    cost = np.zeros((H1, CLASSES))
    for i in range(H1):
        for d in range(1, CLASSES + 1):
            plan = [base] * H1
            plan[i] = d
            out, ms = timed_propagate(ctx, widths, Wd, bd, boxes_d, plan, cap)
            table[:, i, d - 1] = mean_width(out)
            cost[i, d - 1] = ms / B
    return table, cost


def choose_labels(table, cost, base=2, iters=60):
    """Per (box, layer) class labels and the multiplier lam (see the module
    docstring)."""
    B, H1, _ = table.shape
    w_base = table[:, 0, base - 1]
    target = w_base.mean()

    def labels_for(lam):
        score = cost[None, :, :] + lam * table
        lab = np.argmin(score, axis=2)
        chosen = np.take_along_axis(table, lab[:, :, None], axis=2)[:, :, 0]
        pred = w_base + (chosen - w_base[:, None]).sum(axis=1)
        return lab, pred.mean()

    lo, hi = 0.0, 1.0
    while labels_for(hi)[1] > target and hi < 1e12:
        hi *= 4.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if labels_for(mid)[1] > target:
            lo = mid
        else:
            hi = mid
    lab, pred = labels_for(hi)
    return lab, hi, pred


def trace_features(ctx, widths, W, b, boxes, cap=16, base=2):
    """Features [B, N_hidden, FEATURES] of the base plan's trace (GPU)."""
    torch = _torch()
    Wd, bd = _dev_net(widths, W, b)
    boxes_d = torch.as_tensor(np.ascontiguousarray(boxes, np.float32)).cuda()
    out = ctx.propagate(widths, Wd, bd, boxes_d, degree=base, cap=cap, trace=True)
    B = boxes.shape[0]
    nh = sum(widths[1:-1])
    X = torch.empty(B, nh, FEATURES, device="cuda")
    for layer, off, h in hidden_slices(widths):
        lo = out["tr_lo"][:, off:off + h].contiguous()
        hi = out["tr_hi"][:, off:off + h].contiguous()
        nt = out["tr_nterms"][:, off:off + h].contiguous()
        x = torch.empty(B * h, FEATURES, device="cuda")
        ctx.degree_features(B * h, lo, hi, nt, layer, x)
        X[:, off:off + h] = x.view(B, h, FEATURES)
    ctx.check("degree_features")
    return X


def train(ctx, X, y, steps=400, lr=3e-3, seed=0, w=None):
    """Full-batch Adam on the GPU with the library's kernels; X [n, F] and
    y [n] CUDA tensors.  Returns (Mlp, loss history)."""
    torch = _torch()
    rng = np.random.default_rng(seed)
    F = X.shape[1]
    P = int(bern.load().bern_mlp_num_params(F, CLASSES))
    H = bern.BERN_MLP_HIDDEN
    theta = np.zeros(P, np.float32)
    theta[:H * F] = rng.normal(0, np.sqrt(2.0 / F), H * F)
    o = H * F + H
    theta[o:o + CLASSES * H] = rng.normal(0, np.sqrt(1.0 / H), CLASSES * H)
    m = bern.Mlp(torch, F, CLASSES, theta)
    g = torch.empty(P, device="cuda")
    loss = torch.empty(1, device="cuda")
    hist = []
    for it in range(steps):
        ctx.mlp_backward(m, X, y, w, g, loss)
        ctx.mlp_adam(m, g, lr)
        if it % 50 == 0 or it == steps - 1:
            hist.append(float(loss.item()))
    ctx.check("train")
    return m, hist


def fit(ctx, widths, W, b, boxes, cap=16, base=2, steps=400, lr=3e-3, seed=0) -> Dict:
    """Labels from the plain method on `boxes`, then GPU training.  Returns a
    dict with the trained Mlp and what was learned from."""
    torch = _torch()
    t0 = time.time()
    table, cost = width_table(ctx, widths, W, b, boxes, cap, base)
    lab, lam, pred = choose_labels(table, cost, base)
    X = trace_features(ctx, widths, W, b, boxes, cap, base)
    B = boxes.shape[0]
    ys = []
    for (layer, off, h) in hidden_slices(widths):
        ys.append(np.repeat(lab[:, layer - 1][:, None], h, axis=1))
    y = np.concatenate(ys, axis=1).astype(np.int32).reshape(-1)
    Xf = X.reshape(-1, FEATURES).contiguous()
    yd = torch.as_tensor(y).cuda()
    m, hist = train(ctx, Xf, yd, steps, lr, seed)
    z = torch.empty(Xf.shape[0], CLASSES, device="cuda")
    ctx.mlp_forward(m, Xf, z)
    acc = float((z.argmax(1).cpu().numpy() == y).mean())
    return {"mlp": m, "labels": lab, "lam": lam, "pred_width": pred,
            "base_width": float(table[:, 0, base - 1].mean()), "table": table, "cost": cost,
            "n_samples": int(y.size), "loss": hist, "train_acc": acc,
            "label_hist": np.bincount(y, minlength=CLASSES).tolist(),
            "seconds": time.time() - t0}
