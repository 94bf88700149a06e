"""Seeded synthetic inputs: ReLU networks and input boxes.

This module only draws random numbers. It holds none of the bound-propagation
arithmetic, so both the CUDA path and the FP64 oracle can take their inputs
from it.

Networks follow the paper's model (Sec. 2, "Notation pertaining to neural
networks"): H affine layers, ReLU after every layer but the last. Weights are
stored row-major, W[i] has shape (h_i, h_{i-1}), in float32, because the CUDA
path computes in float32 and the oracle reads the same float32 values exactly
as float64.

Draw order for a network with seed s (numpy PCG64, ``default_rng(s)``):
for each layer i = 1..H, W[i] row-major then b[i]; boxes are drawn afterwards
from the same generator.  W ~ N(0, 1/fan_in), b ~ U(-0.1, 0.1).  The paper's
own ablation nets use W, b ~ U(-5, 5) (Sec. 6.1, Figs. 4-7); ``paper_net``
draws those.

Boxes are float32 arrays of shape (n_boxes, n, 2): [..., 0] is the lower and
[..., 1] the upper corner coordinate.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass
class Net:
    widths: List[int]
    W: List[np.ndarray]
    b: List[np.ndarray]
    seed: int = 0

    @property
    def n_in(self) -> int:
        return self.widths[0]

    @property
    def n_out(self) -> int:
        return self.widths[-1]

    @property
    def n_layers(self) -> int:
        return len(self.widths) - 1


@dataclass
class Workload:
    name: str
    net: Net
    boxes: np.ndarray           # (n_boxes, n, 2) float32
    degree: int = 2             # Bernstein ReLU order L (the paper's L)
    degree_cap: int = 16
    prune_tau: float = 0.0
    notes: dict = field(default_factory=dict)


def _draw_net(rng: np.random.Generator, widths, dist: str) -> tuple:
    W, b = [], []
    for i in range(1, len(widths)):
        fan_in, fan_out = widths[i - 1], widths[i]
        if dist == "gauss":
            w = rng.normal(0.0, 1.0 / np.sqrt(fan_in), size=(fan_out, fan_in))
            bb = rng.uniform(-0.1, 0.1, size=fan_out)
        elif dist == "paper":
            w = rng.uniform(-5.0, 5.0, size=(fan_out, fan_in))
            bb = rng.uniform(-5.0, 5.0, size=fan_out)
        else:
            raise ValueError(dist)
        W.append(np.ascontiguousarray(w, dtype=np.float32))
        b.append(np.ascontiguousarray(bb, dtype=np.float32))
    return W, b


def make_net(widths, seed: int, dist: str = "gauss", rng=None) -> Net:
    rng = np.random.default_rng(seed) if rng is None else rng
    W, b = _draw_net(rng, list(widths), dist)
    return Net(list(widths), W, b, seed)


def box_array(lo, hi) -> np.ndarray:
    lo = np.asarray(lo, dtype=np.float32)
    hi = np.asarray(hi, dtype=np.float32)
    return np.stack([lo, hi], axis=-1).astype(np.float32)


def grid_boxes(n: int, cells: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Uniform split of [lo,hi]^n into cells^n boxes (last dimension fastest)."""
    edges = np.linspace(lo, hi, cells + 1, dtype=np.float64)
    idx = np.stack(np.meshgrid(*([np.arange(cells)] * n), indexing="ij"), -1).reshape(-1, n)
    blo = edges[idx]
    bhi = edges[idx + 1]
    return box_array(blo, bhi)


def random_boxes(rng: np.random.Generator, count: int, n: int, side_lo: float,
                 side_hi: float, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Boxes with centres U(lo,hi)^n and per-dimension side lengths
    U(side_lo, side_hi), clipped to [lo,hi]^n."""
    c = rng.uniform(lo, hi, size=(count, n))
    s = rng.uniform(side_lo, side_hi, size=(count, n))
    blo = np.clip(c - s / 2, lo, hi)
    bhi = np.clip(c + s / 2, lo, hi)
    out = box_array(blo, bhi)
    # float32 rounding can never invert a box, but keep the invariant explicit
    bad = out[..., 0] > out[..., 1]
    out[..., 1][bad] = out[..., 0][bad]
    return out


# --------------------------------------------------------------------------
# The five workload shapes.  Sizes and draw recipes are those of the paper's
# experiments (Sec. 6) widened to batches of sub-boxes.
# --------------------------------------------------------------------------

def single_box_2in() -> Workload:
    """[2,20,20,1], seed 0, one box [-1,1]^2, degree 2 (shape of Fig. 4)."""
    net = make_net([2, 20, 20, 1], seed=0)
    return Workload("mlp2-20-20-1_box1_d2", net, box_array([-1, -1], [1, 1])[None], degree=2)


def single_box_4in() -> Workload:
    """[4,50,50,50,2], seed 1, one box [-0.5,0.5]^4, degree 2."""
    net = make_net([4, 50, 50, 50, 2], seed=1)
    return Workload("mlp4-50x3-2_box1_d2", net,
                    box_array([-0.5] * 4, [0.5] * 4)[None], degree=2)


def batch_3in(n_random: int = 1024, cells: int = 16) -> Workload:
    """[3,64,64,64,64,1], seed 2: the cells^3 grid over [-1,1]^3 plus n_random
    boxes with centres U(-1,1)^3 and sides U(0.01,0.5), clipped."""
    rng = np.random.default_rng(2)
    net = make_net([3, 64, 64, 64, 64, 1], seed=2, rng=rng)
    g = grid_boxes(3, cells)
    r = random_boxes(rng, n_random, 3, 0.01, 0.5)
    return Workload("mlp3-64x4-1_boxes%d_d2" % (len(g) + len(r)), net,
                    np.concatenate([g, r], 0), degree=2)


def batch_3in_replicas(world: int) -> Workload:
    """The batched workload for `world` ranks at fixed work per rank (weak
    scaling): replica 0 is batch_3in's 5120 boxes; replica r >= 1 is the same
    16^3 grid plus 1024 random boxes drawn like batch_3in's from the generator
    seeded 2000 + r.  The network is batch_3in's."""
    w = batch_3in()
    parts = [w.boxes]
    for r in range(1, int(world)):
        rng = np.random.default_rng(2000 + r)
        parts.append(np.concatenate([grid_boxes(3, 16), random_boxes(rng, 1024, 3, 0.01, 0.5)],
                                    0))
    return Workload("mlp3-64x4-1_boxes%d_d2" % sum(len(x) for x in parts), w.net,
                    np.ascontiguousarray(np.concatenate(parts, 0)), degree=2)


def batch_3in_training_boxes(count: int = 800, seed: int = 1002) -> np.ndarray:
    """Training boxes for the learned component on the [3,64x4,1] network, drawn
    like the benchmark's boxes (4/5 grid-cell sized, 1/5 random sized) but from
    their own seed: cells of the 16^3 grid's size (side 0.125) at random
    centres, and boxes with sides U(0.01, 0.5); all clipped to [-1,1]^3."""
    rng = np.random.default_rng(seed)
    k = (count * 4) // 5
    c = rng.uniform(-1 + 0.0625, 1 - 0.0625, (k, 3))
    cells = box_array(c - 0.0625, c + 0.0625)
    return np.concatenate([cells, random_boxes(rng, count - k, 3, 0.01, 0.5)], 0)


def batch_6in(n_boxes: int = 2048) -> Workload:
    """[6,100,100,100,2], seed 3, random sub-boxes of [-1,1]^6 with sides
    U(0.05,0.5); degrees in {1..4} with total-degree cap 16."""
    rng = np.random.default_rng(3)
    net = make_net([6, 100, 100, 100, 2], seed=3, rng=rng)
    return Workload("mlp6-100x3-2_boxes%d" % n_boxes, net,
                    random_boxes(rng, n_boxes, 6, 0.05, 0.5), degree=2,
                    degree_cap=16, prune_tau=1e-7)


def batch_6in_training_boxes(count: int = 700, seed: int = 1003) -> np.ndarray:
    """Training boxes for the learned component on the [6,100x3,2] network:
    random sub-boxes of [-1,1]^6 with sides U(0.05, 0.5), like the workload's,
    from their own seed (700 boxes x 300 hidden neurons = 210,000 samples)."""
    return random_boxes(np.random.default_rng(seed), count, 6, 0.05, 0.5)


def bnb_root_6in() -> Workload:
    """[6,64,64,64,64,1], seed 4, root box [-1,1]^6 (branch-and-bound root)."""
    net = make_net([6, 64, 64, 64, 64, 1], seed=4)
    return Workload("mlp6-64x4-1_root", net, box_array([-1] * 6, [1] * 6)[None],
                    degree=2, degree_cap=16, prune_tau=1e-7)


def paper_net(n: int, hidden: List[int], seed: int) -> Net:
    """A net of the paper's ablation family (weights and biases U(-5,5))."""
    return make_net([n] + list(hidden) + [1], seed=seed, dist="paper")


WORKLOADS = {"single_box_2in": single_box_2in, "single_box_4in": single_box_4in, "batch_3in": batch_3in,
             "batch_6in": batch_6in, "bnb_root_6in": bnb_root_6in}
