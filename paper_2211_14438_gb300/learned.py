"""The learned component: per-neuron ReLU-order proposals from a small BF16
MLP, trained on the GPU with the library's own forward/backward/Adam kernels
on labels that the plain method itself produces.

Labels (the method has no learned part; this is the project's reading of
"labelled by plain-method bound widths"):

* A family of per-layer order plans (every layer in {1, 2}, plus order 3 or
  4 at the first hidden layer with {1, 2} after it; plans with more than four
  times the base plan's counted work, or beyond the library's limits, are
  left out) runs with the plain method over all training boxes: W[b, p] is
  box b's mean output-bound width under plan p and cost[p] the plan's
  arithmetic work per box (plan_cost: a deterministic count, so the labels do
  not depend on timing noise).
* The learned plan caps each layer's proposals; the caps must form a plan the
  library runs, and among such cap vectors the one whose plans reach the
  width target at the least work is kept.
* Each box takes the plan minimising  cost[p] + lam * W[b, p];  lam is the
  smallest value for which the mean of the chosen widths does not exceed
  (1 - margin) times the base plan's mean width, so boxes buy speed with
  width where it is cheap and tightness where it is cheap, and the batch is
  never looser on average.
* Every hidden neuron of box b at layer i is a training sample labelled
  with the order its box's plan uses at layer i, with the features of
  bern_degree_features taken from the trace of that same plan (so the
  features at layer i reflect the orders chosen before it, as they will
  when the MLP drives the propagation).

The plain method computes sound bounds for whatever order the MLP proposes
(BERN_DEG_LEARNED); a neuron whose largest class probability is below
min_conf uses the base order (the fallback).
"""
from __future__ import annotations

import itertools
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


def plan_family(n_hidden: int) -> List[Tuple[int, ...]]:
    """The per-layer order plans the labels choose from."""
    fam = []
    for first in (1, 2, 3, 4):
        for k in range(2 ** (n_hidden - 1)):
            rest = tuple(1 + ((k >> j) & 1) for j in range(n_hidden - 1))
            fam.append((first,) + rest)
    return fam


def _monomials(n: int, D: int) -> int:
    r = 1
    for i in range(1, n + 1):
        r = r * (D + i) // i
    return r


def plan_cost(widths, plan, cap=16) -> float:
    """Fused multiply-adds per box of a per-layer order plan when every hidden
    neuron is unstable: the affine steps (h_i h_{i-1} M_pre), the Bernstein
    enclosures (h_i n (l+1)^n (l+2)/2 at order l = the pre-activation degree)
    and the compositions (order 1: M_pre; order 2: M_pre^2 / 2; order d >= 3:
    4 M_pre sum_k M(n, min(k D, cap)) for the interval Horner products)."""
    n = int(widths[0])
    D = 1
    total = 0.0
    for i in range(1, len(widths)):
        h_in, h = int(widths[i - 1]), int(widths[i])
        M = _monomials(n, D)
        total += h * h_in * M + h * n * (D + 1) ** n * (D + 2) / 2.0
        if i < len(widths) - 1:
            d = int(plan[i - 1])
            if d == 1:
                total += h * M
            elif d == 2:
                total += h * M * M / 2.0
            else:
                total += h * 4.0 * M * sum(_monomials(n, min(k * D, cap)) for k in range(1, d))
            D = min(D * d, cap)
    return total


def width_table(ctx, widths, W, b, boxes, plans, cap=16, skip=None):
    """W[b, p] (mean output width of box b under plan p) and the plan's
    measured GPU time per box (ms, for reporting); plans in `skip`, and plans
    the library rejects, get infinite width and time."""
    torch = _torch()
    Wd, bd = _dev_net(widths, W, b)
    boxes_d = torch.as_tensor(np.ascontiguousarray(boxes, np.float32)).cuda()
    B = boxes.shape[0]
    table = np.zeros((B, len(plans)))
    cost = np.zeros(len(plans))
    for k, plan in enumerate(plans):
        if skip is not None and skip[k]:
            table[:, k] = np.inf
            cost[k] = np.inf
            continue
        try:
            out, ms = timed_propagate(ctx, widths, Wd, bd, boxes_d, list(plan), cap)
        except bern.BernError:
            ctx.sync()                       # clear any device-side status of the attempt
            table[:, k] = np.inf             # beyond the library's limits: never chosen
            cost[k] = np.inf
            continue
        table[:, k] = mean_width(out)
        cost[k] = ms / B
    return table, cost


def choose_plans(table, cost, base_idx, margin=0.0, iters=60, base_mean=None):
    """Per box the plan index minimising cost + lam * width, with the
    smallest lam that keeps the mean chosen width <= (1 - margin) * base
    (base: the mean width of plan base_idx, or base_mean when given)."""
    bm = table[:, base_idx].mean() if base_mean is None else base_mean
    target = (1.0 - margin) * bm

    def pick(lam):
        idx = np.argmin(cost[None, :] + lam * table, axis=1)
        return idx, table[np.arange(len(idx)), idx].mean()

    lo, hi = 0.0, 1e-6
    while pick(hi)[1] > target and hi < 1e12:
        hi *= 4.0
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if pick(mid)[1] > target:
            lo = mid
        else:
            hi = mid
    idx, mean_w = pick(hi)
    return idx, hi, mean_w


def trace_features(ctx, widths, W, b, boxes, cap=16, base=2):
    """Features [B, N_hidden, FEATURES] of the trace of plan `base` (an
    order or a per-layer list) over `boxes` (GPU)."""
    torch = _torch()
    Wd, bd = _dev_net(widths, W, b)
    boxes_d = torch.as_tensor(np.ascontiguousarray(boxes, np.float32)).cuda()
    deg = list(base) if isinstance(base, (tuple, list)) else base
    out = ctx.propagate(widths, Wd, bd, boxes_d, degree=deg, cap=cap, trace=True)
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


def _labels_and_features(ctx, widths, W, b, boxes, plans, idx, cap):
    torch = _torch()
    lab = np.array([plans[k] for k in idx], np.int32) - 1          # [B, H1] classes
    nh = sum(widths[1:-1])
    X = torch.empty(boxes.shape[0], nh, FEATURES, device="cuda")
    for k in np.unique(idx):
        sel = np.nonzero(idx == k)[0]
        X[torch.as_tensor(sel).cuda()] = trace_features(ctx, widths, W, b, boxes[sel], cap,
                                                        plans[k])
    ys = [np.repeat(lab[:, layer - 1][:, None], h, axis=1)
          for (layer, off, h) in hidden_slices(widths)]
    y = np.concatenate(ys, axis=1).astype(np.int32).reshape(-1)
    return X.reshape(-1, FEATURES).contiguous(), y


def _runnable(ctx, widths, W, b, boxes, plan, cap):
    torch = _torch()
    Wd, bd = _dev_net(widths, W, b)
    try:
        ctx.propagate(widths, Wd, bd, torch.as_tensor(np.ascontiguousarray(boxes)).cuda(),
                      degree=list(plan), cap=cap)
        return True
    except bern.BernError:
        ctx.sync()
        return False


def evaluate(ctx, widths, W, b, boxes, degree, cap=16, reps=3):
    """(mean output width, ms per box) of a plan over `boxes`."""
    torch = _torch()
    Wd, bd = _dev_net(widths, W, b)
    boxes_d = torch.as_tensor(np.ascontiguousarray(boxes, np.float32)).cuda()
    out, ms = timed_propagate(ctx, widths, Wd, bd, boxes_d, degree, cap, reps=reps)
    return float(mean_width(out).mean()), ms / boxes.shape[0]


def fit(ctx, widths, W, b, boxes, cap=16, base=2, steps=600, lr=3e-3, seed=0,
        margins=(0.02, 0.03, 0.04, 0.05, 0.065, 0.08, 0.1, 0.12, 0.16, 0.24),
        slack=0.005, max_work=4.0) -> Dict:
    """Labels from the plain method on `boxes`, GPU training, and a check of
    the trained MLP driving the propagation on the same boxes.  The label
    margin grows until the learned plan's measured mean width is at most
    (1 - slack) times the base plan's (the smallest such margin buys the
    least tightness, so it keeps the most speed).
    Returns a dict with the trained Mlp and what was learned from."""
    torch = _torch()
    t0 = time.time()
    H1 = len(widths) - 2
    plans = plan_family(H1)
    base_plan = tuple([base] * H1)
    if base_plan not in plans:
        plans.append(base_plan)
    base_idx = plans.index(base_plan)
    # plans with more than max_work times the base plan's counted work are not
    # run at all (they would never be chosen, and the largest need tables of
    # hundreds of millions of entries on six inputs)
    work = np.array([plan_cost(widths, p, cap) for p in plans])
    skip = work > max_work * work[base_idx]
    table, ms_per_box = width_table(ctx, widths, W, b, boxes, plans, cap, skip)
    cost = np.where(np.isfinite(ms_per_box), work, np.inf)
    base_mean = float(table[:, base_idx].mean())
    # the per-layer caps size the learned plan and must form a runnable plan;
    # among the runnable cap vectors keep the one whose plans reach the width
    # target at the least work (or, if none does, the tightest)
    feasible = [p for k, p in enumerate(plans) if np.isfinite(cost[k])]
    top = [max(p[i] for p in feasible) for i in range(H1)]
    best_key, caps = None, None
    for c in itertools.product(*[range(1, t + 1) for t in top]):
        sel = np.array([np.isfinite(cost[k]) and all(p[i] <= c[i] for i in range(H1))
                        for k, p in enumerate(plans)])
        if not sel.any() or not _runnable(ctx, widths, W, b, boxes[:1], c, cap):
            continue
        t2 = np.where(sel[None, :], table, np.inf)
        c2 = np.where(sel, cost, np.inf)
        idx, _, mw = choose_plans(t2, c2, base_idx, margins[0], base_mean=base_mean)
        ok = mw <= (1.0 - margins[0]) * base_mean
        key = (0, float(c2[idx].mean())) if ok else (1, float(mw))
        if best_key is None or key < best_key:
            best_key, caps = key, list(c)
    if caps is None:
        raise RuntimeError("no runnable order plan")
    for k, p in enumerate(plans):
        if any(p[i] > caps[i] for i in range(H1)):
            cost[k] = np.inf
            table[:, k] = np.inf
    base_w = base_mean
    tried, best = [], None
    for margin in margins:
        idx, lam, mean_w = choose_plans(table, cost, base_idx, margin, base_mean=base_mean)
        Xf, y = _labels_and_features(ctx, widths, W, b, boxes, plans, idx, cap)
        m, hist = train(ctx, Xf, torch.as_tensor(y).cuda(), steps, lr, seed)
        z = torch.empty(Xf.shape[0], CLASSES, device="cuda")
        ctx.mlp_forward(m, Xf, z)
        acc = float((z.argmax(1).cpu().numpy() == y).mean())
        w_l, c_l = evaluate(ctx, widths, W, b, boxes, bern.Learned(m, 0.0, base, caps), cap)
        rec = {"margin": margin, "lam": lam, "label_width": float(mean_w),
               "label_work": float(cost[idx].mean() / work[base_idx]), "learned_width": w_l,
               "learned_ms_per_box": c_l, "train_acc": acc, "loss": hist,
               "label_hist": np.bincount(y, minlength=CLASSES).tolist(),
               "plan_of_box": idx}
        tried.append(rec)
        if w_l <= (1.0 - slack) * base_w:   # the smallest margin that meets the target
            best = (rec, m)
            break
    if best is None:    # no margin met the width target: keep the tightest one
        k = int(np.argmin([r["learned_width"] for r in tried]))
        idx, lam, _ = choose_plans(table, cost, base_idx, tried[k]["margin"],
                                   base_mean=base_mean)
        Xf, y = _labels_and_features(ctx, widths, W, b, boxes, plans, idx, cap)
        m, _ = train(ctx, Xf, torch.as_tensor(y).cuda(), steps, lr, seed)
        best = (tried[k], m)
    rec, m = best
    return {"mlp": m, "plan": bern.Learned(m, 0.0, base, caps), "max_per_layer": caps,
            "plans": plans, "base_width": base_w, "base_work": float(work[base_idx]),
            "table": table, "cost": cost, "ms_per_box": ms_per_box, "tried": tried,
            "chosen": rec,
            "n_samples": int(Xf.shape[0]), "seconds": time.time() - t0}
