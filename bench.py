"""Benchmark: input boxes propagated per second (BERN-NN bounds) on GB300.

Workload: the batched plain method, ReLU MLP [3, 64, 64, 64, 64, 1] (seed 2),
5120 boxes (the 16^3 grid of [-1,1]^3 plus 1024 random boxes with sides
U(0.01,0.5)), Bernstein ReLU order 2, total-degree cap 16.  A step is one
bern_propagate over all 5120 boxes (init, then per hidden layer the affine step
with the stability screen, the enclosure of the undecided pre-activations with
their ReLU coefficients, and the in-place composition of the unstable neurons;
the output layer's affine step, its enclosure and copy-out), replayed as one
CUDA graph.  The fused
per-layer kernel (one launch per hidden layer) is timed beside it as an
alternate path (--fused makes it the headline).  L2 is flushed (256 MB
write) before every timed step, outside the timed interval; each step is
timed with CUDA events on the launching stream.

Multi-GPU (torchrun, weak scaling): N replicas of the 5120-box batch (the
same grid cells, fresh random boxes per replica) are split into N contiguous
slices of equal estimated cost (interval arithmetic counts each box's
straddling neurons, weighted by the term pairs of their squares); every rank
bounds its slice, and the per-box bounds and term counts come back to every
rank by one NCCL all_gather per tensor inside the timed step.  Barrier and
max over ranks of the timed region.

Also reported: per-kernel durations (a second K-step pass through the
step-level C ABI, events around every launch), the roofline of the dominant
kernel, the end-to-end rate through bern_propagate with host buffers, the
FP64 oracle on the host cores, and SM clocks sampled during the timed region.

--impl reference times the FP64 oracle (the reference arm: there is no
installable reference implementation of the method) on the host cores with the
same metric and workload.
"""
from __future__ import annotations

import argparse
import datetime
import hashlib
import json
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "input boxes propagated/sec at fixed mean output-bound width; % of HBM roofline"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
FP32_LANES_PER_SM = 128


# ---------------------------------------------------------------- helpers
def load_peaks():
    if os.path.exists(PEAKS_FILE):
        with open(PEAKS_FILE) as f:
            p = json.load(f)
        return p, "measured"
    return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": 2070.0}, "fallback"


def oracle_box(args):
    """One box through the FP64 oracle (runs in a spawned worker)."""
    import oracle as orc
    widths, W, b, box, degree = args
    t0 = time.perf_counter()
    orc.propagate(widths, W, b, box, degree)
    return time.perf_counter() - t0


def oracle_rate(pool, cores, w, sample_idx):
    """Boxes/s of the pool on the sample, its wall time, and the per-box
    single-thread times measured inside the workers."""
    jobs = [(w.net.widths, w.net.W, w.net.b, w.boxes[i], w.degree) for i in sample_idx]
    t0 = time.perf_counter()
    per_box = pool.map(oracle_box, jobs, chunksize=1)
    wall = time.perf_counter() - t0
    return len(sample_idx) / wall, wall, per_box


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms; the samples
    whose timestamps fall inside the timed region (marked by begin()/end())
    give the reported median clock and the reasons."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)                     # first sample before the timed region

    def begin(self):
        self.t0 = datetime.datetime.now()

    def end(self):
        self.t1 = datetime.datetime.now()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        time.sleep(2.5 * self.PERIOD_MS / 1000.0)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                parts[0] = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
            except ValueError:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        t0, t1 = self.t0 or rows[0][0], self.t1 or rows[-1][0]
        inside = [r for r in rows if t0 <= r[0] <= t1]
        # a timed region shorter than the sampling period: the samples nearest to it
        half = datetime.timedelta(milliseconds=self.PERIOD_MS)
        window = inside or [r for r in rows if t0 - half <= r[0] <= t1 + half]
        sm = [num(r[2]) for r in window if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in window:
            for name, v in zip(names, r[6:10]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": num(rows[0][3]), "reasons": sorted(reasons),
                "samples": len(rows), "samples_in_timed_region": len(inside),
                "samples_used": len(window),
                "timed_region_ms": round((t1 - t0).total_seconds() * 1000.0, 1),
                "power_w_max": max((num(r[4]) or 0.0) for r in window) if window else None}


# ----------------------------------------------------- per-kernel timing pass
class KernelPass:
    """Drives the kernels bern_propagate runs for this workload through the
    step-level C ABI on torch-allocated buffers, with CUDA events around every
    launch on the launching stream.  With fused=False (the default path): init,
    the first layer's affine step, per hidden layer the per-step kernels
    (bern_enclose, bern_relu_coeffs, bern_compose, bern_affine) and the output
    enclosure; that pass also supplies the ReLU cases and term counts for the
    algorithmic-work counts.  With fused=True the hidden layers run as one
    bern_layer launch each (enclosure, ReLU coefficients, composition and the
    next layer's affine step), timed after the per-step pass that supplies the
    counts."""

    def __init__(self, ctx, torch, w, Wd, bd, boxes_d, fused=True):
        from paper_2211_14438_gb300 import bern
        self.bern, self.torch, self.ctx = bern, torch, ctx
        self.w, self.Wd, self.bd, self.boxes = w, Wd, bd, boxes_d
        self.fused = fused
        widths = w.net.widths
        self.n, self.B, self.H = widths[0], len(w.boxes), len(widths) - 1
        dev = boxes_d.device
        n, B = self.n, self.B
        f32, i32 = torch.float32, torch.int32
        self.z = [torch.empty(B * n * (n + 1), device=dev, dtype=f32) for _ in range(2)]
        self.znt = torch.empty(B * n, device=dev, dtype=i32)
        self.layers = []
        D = 1
        order = 1
        for i in range(self.H):
            h = widths[i + 1]
            hidden = i < self.H - 1
            Mpre = bern.num_monomials(n, D)
            # hidden layers compose in place, as bern_propagate does: the
            # pre-activation block has the post-activation block's row stride
            ld = bern.num_monomials(n, min(D * w.degree, w.degree_cap)) if hidden else Mpre
            L = {"h_in": widths[i], "h": h, "hidden": hidden, "D": D, "order": order,
                 "Mpre": Mpre, "ld": ld,
                 "pre": [torch.empty(B * h * ld, device=dev, dtype=f32) for _ in range(2)],
                 "pre_nt": torch.empty(B * h, device=dev, dtype=i32),
                 "lo": torch.empty(B * h, device=dev, dtype=f32),
                 "hi": torch.empty(B * h, device=dev, dtype=f32)}
            if hidden:
                Dp = min(D * w.degree, w.degree_cap)
                Mpost = bern.num_monomials(n, Dp)
                L.update({"Mpost": Mpost,
                          "kind": torch.empty(B * h, device=dev, dtype=torch.int8),
                          "coef": torch.empty(B * h * bern.COEF_STRIDE, device=dev, dtype=f32),
                          "eps": torch.empty(B * h, device=dev, dtype=f32),
                          "post": L["pre"],
                          "post_nt": torch.empty(B * h, device=dev, dtype=i32)})
                D, order = Dp, min(order * w.degree, w.degree_cap)
            self.layers.append(L)
        self.times = {}

    def _timed(self, name, fn):
        t = self.torch
        s, e = t.cuda.Event(enable_timing=True), t.cuda.Event(enable_timing=True)
        st = self.ctx.stream
        s.record(st)
        fn()
        e.record(st)
        self.pending.append((name, s, e))

    def step(self):
        if self.fused:
            self.step_fused()
        else:
            self.step_per_kernel()

    def step_fused(self):
        # the fused layer kernels keep separate blocks: pre-activation rows at
        # the layer's own stride (the buffers are large enough)
        ctx, w = self.ctx, self.w
        n, B = self.n, self.B
        self.pending = []
        self._timed("init", lambda: ctx.init_inputs(n, self.boxes, self.z[0], self.z[1], n + 1,
                                                    self.znt))
        L0 = self.layers[0]
        self._timed("affine_L1", lambda: ctx.affine(
            B, L0["h"], L0["h_in"], self.Wd[0], self.bd[0], self.z[0], self.z[1], n + 1,
            self.znt, L0["pre"][0], L0["pre"][1], L0["Mpre"], L0["pre_nt"]))
        for i, L in enumerate(self.layers):
            if not L["hidden"]:
                self._timed("enclose_L%d" % (i + 1), lambda: ctx.enclose(
                    n, B, L["h"], L["order"], 0, L["pre"][0], L["pre"][1], L["Mpre"],
                    L["pre_nt"], L["lo"], L["hi"]))
                break
            N = self.layers[i + 1]
            self._timed("layer_L%d" % (i + 1), lambda: ctx.layer(
                n, B, L["h"], L["order"], 0, w.degree, w.degree_cap, L["pre"][0], L["pre"][1],
                L["Mpre"], L["pre_nt"], N["h"], self.Wd[i + 1], self.bd[i + 1], N["pre"][0],
                N["pre"][1], N["Mpre"], N["pre_nt"]))

    def step_per_kernel(self):
        ctx, w = self.ctx, self.w
        n, B = self.n, self.B
        self.pending = []
        self._timed("init", lambda: ctx.init_inputs(n, self.boxes, self.z[0], self.z[1], n + 1,
                                                    self.znt))
        in_u, in_l, in_nt, in_stride = self.z[0], self.z[1], self.znt, n + 1
        for i, L in enumerate(self.layers):
            self._timed("affine_L%d" % (i + 1), lambda: ctx.affine(
                B, L["h"], L["h_in"], self.Wd[i], self.bd[i], in_u, in_l, in_stride, in_nt,
                L["pre"][0], L["pre"][1], L["ld"], L["pre_nt"]))
            self._timed("enclose_L%d" % (i + 1), lambda: ctx.enclose(
                n, B, L["h"], L["order"], 0, L["pre"][0], L["pre"][1], L["ld"], L["pre_nt"],
                L["lo"], L["hi"]))
            if not L["hidden"]:
                break
            self._timed("relu_L%d" % (i + 1), lambda: ctx.relu_coeffs(
                B * L["h"], L["lo"], L["hi"], None, w.degree, L["kind"], L["coef"], L["eps"]))
            self._timed("compose_L%d" % (i + 1), lambda: ctx.compose(
                n, B, L["h"], w.degree_cap, 0.0, L["kind"], L["coef"], L["eps"], None, w.degree,
                L["lo"], L["hi"], L["pre"][0], L["pre"][1], L["ld"], L["pre_nt"],
                L["post"][0], L["post"][1], L["ld"], L["post_nt"]))
            in_u, in_l, in_nt, in_stride = L["post"][0], L["post"][1], L["post_nt"], L["ld"]

    def collect(self):
        self.torch.cuda.synchronize()
        for name, s, e in self.pending:
            self.times.setdefault(name, []).append(s.elapsed_time(e))

    def work(self):
        """Algorithmic bytes and flops per launch of every kernel, from the
        intermediates of a per-step pass (actual term counts and ReLU cases).
        Bytes: every polynomial coefficient a launch must read or write once
        (both bounds, float32).  Flops: two per fused multiply-add of the
        method's arithmetic (the sign-split layer step: one FMA per product
        and bound; the enclosure's line transforms; the square's pair
        products and the ReLU polynomial's terms)."""
        bern = self.bern
        n, B = self.n, self.B
        saved = self.pending if hasattr(self, "pending") else []
        self.step_per_kernel()                       # fills the intermediates
        self.torch.cuda.synchronize()
        self.pending = saved
        out = {}
        in_nt = self.znt.cpu().numpy().reshape(B, n).astype(np.int64)
        for i, L in enumerate(self.layers):
            h = L["h"]
            pre_nt = L["pre_nt"].cpu().numpy().reshape(B, h).astype(np.int64)
            Mb = pre_nt[:, 0]
            rd = 2 * 4 * in_nt.sum()
            wr = 2 * 4 * h * Mb.sum()
            affine = {"bytes": float(rd + wr), "flops": float(4 * h * in_nt.sum())}
            out["affine_L%d" % (i + 1)] = affine
            lb = L["order"]
            g_lines = n * (lb + 1) ** (n - 1) * lb * (lb + 1) // 2
            enc = {"bytes": float(2 * 4 * pre_nt.sum() + 8 * B * h),
                   "flops": float(2 * B * h * g_lines)}
            out["enclose_L%d" % (i + 1)] = enc
            if not L["hidden"]:
                break
            kind = L["kind"].cpu().numpy().reshape(B, h)
            post_nt = L["post_nt"].cpu().numpy().reshape(B, h).astype(np.int64)
            act = kind == 1
            unst = kind == 2
            rd = 2 * 4 * (pre_nt[act].sum() + pre_nt[unst].sum())
            wr = 2 * 4 * (post_nt[act].sum() + post_nt[unst].sum())
            Mp = pre_nt[unst]
            pairs = (Mp * (Mp + 1) // 2).sum()
            comp_flops = float(2 * 2 * pairs + 2 * 2 * post_nt[unst].sum())
            out["compose_L%d" % (i + 1)] = {"bytes": float(rd + wr), "flops": comp_flops,
                                            "unstable": int(unst.sum()), "active": int(act.sum()),
                                            "items": int(B * h)}
            out["relu_L%d" % (i + 1)] = {"bytes": float(8 * B * h + 41 * unst.sum()), "flops": 0.0}
            # the fused launch: reads this layer's block, writes the next one; its
            # flops are the enclosures of the unstable items, their compositions
            # and the next layer's step over the live (active or unstable) items
            hn = self.layers[i + 1]["h"]
            Mn = post_nt.max(axis=1).clip(min=1)
            live_nt = (post_nt * (act | unst)).sum()
            out["layer_L%d" % (i + 1)] = {
                "bytes": float(2 * 4 * pre_nt.sum() + 2 * 4 * hn * Mn.sum()),
                "flops": float(2 * 2 * unst.sum() * g_lines) + comp_flops + float(4 * hn * live_nt),
                "unstable": int(unst.sum()), "active": int(act.sum()), "items": int(B * h)}
            in_nt = post_nt
        out["init"] = {"bytes": float(B * n * 8 + 2 * B * n * (n + 1) * 4), "flops": 0.0}
        return out


def source_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


KERNEL_SOURCES = {"affine": "k_affine.cu", "enclose": "k_enclose.cu", "compose": "k_compose.cu",
                  "relu": "k_enclose.cu", "init": "k_io.cu", "layer": "k_layer.cu"}


def ncu_traffic(kernel_key):
    """DRAM bytes per launch from a committed ncu summary, if its kernel
    source is unchanged since the counters were taken."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    rec = d.get(kernel_key)
    if not rec:
        return None
    src = os.path.join(ROOT, "paper_2211_14438_gb300", "csrc",
                       KERNEL_SOURCES[kernel_key.split("_")[0]])
    if rec.get("source_sha") != source_sha(src):
        return None
    return rec.get("dram_bytes_per_launch")


# ------------------------------------------------------ Lin linearisation
def lin_entries(ctx, torch, dev, flush, args, w, Wd, bd, boxes_d, plain_ms, plain_width, world,
                dist):
    """Throughput and mean output-bound width with the bounds linearised after
    every lin-th hidden layer (Sec. 5.3), on the benchmark workload and on the
    paper's deepest ablation shape (Fig. 7: [2,20x5,1], W and b U(-5,5), the
    net of the paper-shaped sweeps), each next to the plain method.  Timed
    like the headline step: CUDA events on the stream, L2 flushed before
    every timed call."""
    from paper_2211_14438_gb300 import bern
    from paper_2211_14438_gb300 import workloads as wl
    from paper_2211_14438_gb300.sharding import max_over_ranks
    stream = ctx.stream

    def timed(net, Wd_, bd_, bx_, degree, cap, lin):
        nb, o_ = int(bx_.shape[0]), net.n_out
        ct = bern.max_output_terms(net.widths, degree, cap, lin)
        outx = {"lo": torch.empty(nb, o_, device=dev), "hi": torch.empty(nb, o_, device=dev),
                "n_terms": torch.empty(nb, o_, 2, device=dev, dtype=torch.int32),
                "coef": torch.empty(nb, o_, 2, ct, device=dev), "keys": None}

        def st():
            ctx.propagate(net.widths, Wd_, bd_, bx_, degree=degree, cap=cap, lin=lin,
                          cap_terms=ct, out=outx, sync=False)
        for _ in range(args.warmup):
            st()
        if ctx.sync() != 0:
            raise RuntimeError("propagate failed (lin %d)" % lin)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for s_, e_ in ev:
            flush.zero_()
            s_.record(stream)
            st()
            e_.record(stream)
        torch.cuda.synchronize()
        if ctx.sync() != 0:
            raise RuntimeError("propagate failed (lin %d)" % lin)
        ms = max_over_ranks(float(np.mean([s_.elapsed_time(e_) for s_, e_ in ev])), world, dist,
                            dev)
        return {"value": round(world * nb / (ms / 1e3), 1), "unit": "boxes/s",
                "ms_per_step": round(ms, 4),
                "mean_output_width": round(float((outx["hi"] - outx["lo"]).mean().item()), 6)}

    nb = int(boxes_d.shape[0])
    res = {"workload": "the benchmark workload above",
           "plain": {"value": round(world * nb / (plain_ms / 1e3), 1), "unit": "boxes/s",
                     "ms_per_step": round(plain_ms, 4),
                     "mean_output_width": round(plain_width, 6)}}
    for lin in (1, 2):
        res["lin%d" % lin] = timed(w.net, Wd, bd, boxes_d, w.degree, w.degree_cap, lin)
    net = wl.paper_net(2, [20] * 5, seed=522)
    rng = np.random.default_rng(1022)
    c = rng.uniform(-1, 1, (4096, 2))
    sd = rng.uniform(0.05, 0.5, (4096, 2))
    bx = torch.from_numpy(wl.box_array(np.clip(c - sd / 2, -1, 1),
                                       np.clip(c + sd / 2, -1, 1))).to(dev)
    Wp = [torch.from_numpy(x).to(dev) for x in net.W]
    bp = [torch.from_numpy(x).to(dev) for x in net.b]
    deep = {"workload": "paper deep shape [2,20,20,20,20,20,1], W and b U(-5,5) seed 522, 4096 "
                        "random sub-boxes of [-1,1]^2 (sides U(0.05,0.5)), ReLU order 2, cap 64"}
    for lin in (0, 1, 2):
        deep["plain" if lin == 0 else "lin%d" % lin] = timed(net, Wp, bp, bx, 2, 64, lin)
    res["deep_2in"] = deep
    return res


# ------------------------------------------- Bernstein-tensor arithmetic (Sec. 4)
def bernstein_basis_entry(ctx, torch, dev, flush, args):
    """One layer step in the paper's representation against the power basis,
    on the layer-4 size of the benchmark net (three variables, degree 8):
    P = 4096 items of the power-basis composition at order 2 (both bounds:
    two squares of 165-term polynomials per item, the library's row kernels,
    plus the queue, the linear term and the epilogue), against 2P Prod_Bern
    squares of order-8 Bernstein tensors (9^3 = 729 coefficients, 729^2 term
    products each, bern_bernstein_square); the degree elevation of 2P order-8
    tensors to order 16 (bern_bernstein_elevate); and the layer sums
    (bern_affine on 165- and 969-coefficient blocks against
    bern_bernstein_affine on 729- and 4913-coefficient tensors).  Random
    seeded coefficients; CUDA events, L2 flushed before every timed call."""
    from paper_2211_14438_gb300 import bern
    n, D, P, h = 3, 8, 4096, 64
    B = P // h
    M, Mo = bern.num_monomials(n, D), bern.num_monomials(n, 2 * D)
    rng = np.random.default_rng(4242)
    deg = np.array([sum(r) for r in bern.monomials(n, D)], np.float64)
    base = (rng.normal(0, 0.3, (P, M)) * 0.6 ** deg).astype(np.float32)
    gap = np.abs(rng.normal(0, 0.01, (P, M)) * 0.6 ** deg).astype(np.float32)
    up, lo_p = base + gap, base - gap
    mag = np.abs(up).sum(1) + np.abs(lo_p).sum(1)
    lo = (-mag - 1.0).astype(np.float32)                 # every item unstable
    hi = (mag + 1.0).astype(np.float32)
    blk = lambda a: torch.from_numpy(np.ascontiguousarray(a.reshape(B, h, M).transpose(0, 2, 1))).to(dev)
    pu, pl = blk(up), blk(lo_p)
    nt = torch.full((P,), M, dtype=torch.int32, device=dev)
    glo, ghi = torch.from_numpy(lo).to(dev), torch.from_numpy(hi).to(dev)
    kind = torch.zeros(P, dtype=torch.int8, device=dev)
    coef = torch.zeros(P * bern.COEF_STRIDE, device=dev)
    eps = torch.zeros(P, device=dev)
    ctx.relu_coeffs(P, glo, ghi, None, 2, kind, coef, eps)
    qu = torch.empty(B * Mo * h, device=dev)
    ql = torch.empty_like(qu)
    qnt = torch.empty(P, dtype=torch.int32, device=dev)
    tens = torch.from_numpy(rng.normal(0, 1, (2 * P, (D + 1) ** n)).astype(np.float32)).to(dev)
    chi = torch.empty(2 * P, (2 * D + 1) ** n, device=dev)
    clo = torch.empty_like(chi)
    stream = ctx.stream

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        if ctx.sync() != 0:
            raise RuntimeError("bernstein-basis comparison failed")
        return float(np.median(ms))

    ms_pow = timed(lambda: ctx.compose(n, B, h, 16, 0.0, kind, coef, eps, None, 2, glo, ghi, pu,
                                       pl, M, nt, qu, ql, Mo, qnt))
    ms_bern = timed(lambda: ctx.bernstein_square(n, D, tens, chi, clo))
    # Sum_Bern: degree elevation (order 8 -> 16, what an identity neuron's
    # tensor needs before the next sum) and the layer sums: 64 -> 64 neurons on
    # the layer-4 pre-activation size and 64 -> 1 on the output layer's input,
    # against the affine step on the power-basis blocks of the same items
    ms_elev = timed(lambda: ctx.bernstein_elevate(n, D, D, tens, tens, chi, clo))
    W4 = torch.from_numpy((rng.normal(size=(h, h)) / np.sqrt(h)).astype(np.float32)).to(dev)
    b4 = torch.from_numpy(rng.uniform(-0.1, 0.1, h).astype(np.float32)).to(dev)
    W5 = torch.from_numpy((rng.normal(size=(1, h)) / np.sqrt(h)).astype(np.float32)).to(dev)
    b5 = torch.from_numpy(rng.uniform(-0.1, 0.1, 1).astype(np.float32)).to(dev)
    G8, G16 = (D + 1) ** n, (2 * D + 1) ** n
    a4u, a4l = torch.empty(B * M * h, device=dev), torch.empty(B * M * h, device=dev)
    a4nt = torch.empty(P, dtype=torch.int32, device=dev)
    a5u, a5l = torch.empty(B * Mo, device=dev), torch.empty(B * Mo, device=dev)
    a5nt = torch.empty(B, dtype=torch.int32, device=dev)
    ms_pow_a4 = timed(lambda: ctx.affine(B, h, h, W4, b4, pu, pl, M, nt, a4u, a4l, M, a4nt))
    ms_pow_a5 = timed(lambda: ctx.affine(B, 1, h, W5, b5, qu, ql, Mo, qnt, a5u, a5l, Mo, a5nt))
    del a4u, a4l, a5u, a5l
    t8 = torch.from_numpy(rng.normal(0, 1, (B, G8, h)).astype(np.float32)).to(dev)
    o8u, o8l = torch.empty(B * G8 * h, device=dev), torch.empty(B * G8 * h, device=dev)
    ms_bern_a4 = timed(lambda: ctx.bernstein_affine(B, h, h, W4, b4, G8, t8, t8, o8u, o8l))
    del t8, o8u, o8l
    t16 = torch.from_numpy(rng.normal(0, 1, (B, G16, h)).astype(np.float32)).to(dev)
    o16u, o16l = torch.empty(B * G16, device=dev), torch.empty(B * G16, device=dev)
    ms_bern_a5 = timed(lambda: ctx.bernstein_affine(B, 1, h, W5, b5, G16, t16, t16, o16u, o16l))
    del t16
    layer_pow = ms_pow_a4 + ms_pow + ms_pow_a5
    layer_bern = ms_bern_a4 + ms_bern + ms_elev + ms_bern_a5
    return {"workload": "4096 items of three variables at degree 8 (the benchmark net's layer-4 "
                        "size, 64 boxes of 64 neurons), both bounds: 8192 squares in each "
                        "representation, 8192 elevations of order-8 tensors to order 16, and "
                        "the layer sums 64 -> 64 (pre-activation size) and 64 -> 1 (the output "
                        "layer's input)",
            "power_basis_composition_ms": round(ms_pow, 4),
            "bernstein_prod_bern_squares_ms": round(ms_bern, 4),
            "bernstein_over_power_time": round(ms_bern / ms_pow, 2),
            "bernstein_elevate_ms": round(ms_elev, 4),
            "affine_64_64_ms": {"power_basis": round(ms_pow_a4, 4),
                                "bernstein": round(ms_bern_a4, 4)},
            "affine_64_1_ms": {"power_basis": round(ms_pow_a5, 4),
                               "bernstein": round(ms_bern_a5, 4)},
            "layer_step_ms": {"power_basis": round(layer_pow, 4),
                              "bernstein": round(layer_bern, 4),
                              "bernstein_over_power": round(layer_bern / layer_pow, 2),
                              "note": "sum + square + output sum; the Bernstein step adds the "
                                      "elevation its identity neurons need (timed for all items)"},
            "term_products_per_square": {"power_basis": M * (M + 1) // 2,
                                         "bernstein_tensor": ((D + 1) ** n) ** 2},
            "coefficients": {"power_basis_in_out": [M, Mo],
                             "bernstein_in_out": [G8, G16]}}


# ---------------------------------------------------------------- our arm
def run_ours(args, rank, world, local_rank, dist):
    import torch
    from paper_2211_14438_gb300 import bern, build
    from paper_2211_14438_gb300 import workloads as wl

    pool = None
    cores = 0
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        pool = mp.get_context("spawn").Pool(cores)   # before the first GPU call
    build.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    w = wl.batch_3in()
    if args.n_boxes:
        # an evenly strided subset keeps the mix of grid cells and random boxes
        pick = np.linspace(0, len(w.boxes) - 1, args.n_boxes).astype(int)
        w.boxes = np.ascontiguousarray(w.boxes[pick])
    B_total = len(w.boxes)
    counts = [B_total]
    if world > 1:
        # weak scaling: world replicas of the batch (5120 boxes each), split
        # into cost-balanced contiguous slices, one per rank; the per-box
        # results come back to every rank by one all_gather per tensor
        from paper_2211_14438_gb300 import sharding
        wg = wl.batch_3in_replicas(world)
        if args.n_boxes:
            pick = np.linspace(0, len(wg.boxes) - 1, args.n_boxes * world).astype(int)
            wg.boxes = np.ascontiguousarray(wg.boxes[pick])
        costs = sharding.interval_cost(wg.net.widths, wg.net.W, wg.net.b, wg.boxes, wg.degree,
                                       wg.degree_cap)
        ranges = sharding.shard_ranges(costs, world)
        a0, z0 = ranges[rank]
        counts = [r1 - r0 for r0, r1 in ranges]
        w.boxes = np.ascontiguousarray(wg.boxes[a0:z0])
        B_total = len(wg.boxes)
    B = len(w.boxes)
    ctx = bern.Context(local_rank, stream=torch.cuda.current_stream(dev))
    stream = ctx.stream
    Wd = [torch.from_numpy(x).to(dev) for x in w.net.W]
    bd = [torch.from_numpy(x).to(dev) for x in w.net.b]
    boxes_d = torch.from_numpy(w.boxes).to(dev)
    cap_terms = bern.max_output_terms(w.net.widths, w.degree, w.degree_cap)
    o = w.net.n_out
    out = {"lo": torch.empty(B, o, device=dev), "hi": torch.empty(B, o, device=dev),
           "n_terms": torch.empty(B, o, 2, device=dev, dtype=torch.int32),
           "coef": torch.empty(B, o, 2, cap_terms, device=dev), "keys": None}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        ctx.propagate(w.net.widths, Wd, bd, boxes_d, degree=w.degree, cap=w.degree_cap,
                      cap_terms=cap_terms, out=out, sync=False)
        if world > 1:
            sharding.gather_tensors({"lo": out["lo"], "hi": out["hi"],
                                     "n_terms": out["n_terms"]}, B, counts, dist)

    ctx.set_fused(bool(args.fused))
    from paper_2211_14438_gb300.sharding import max_over_ranks
    sampler = ClockSampler(local_rank)
    sampler.start()
    for _ in range(args.warmup):
        step()
    rc = ctx.sync()
    if rc != 0:
        raise RuntimeError("propagate failed: %s" % bern.strerror(rc))
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.kernel_launches()
    sampler.begin()
    for k in range(args.steps):
        flush.zero_()
        starts[k].record(stream)
        step()
        ends[k].record(stream)
    torch.cuda.synchronize()
    sampler.end()
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop()
    launches = ctx.kernel_launches() - launches0
    rc = ctx.sync()
    if rc != 0:
        raise RuntimeError("propagate failed: %s" % bern.strerror(rc))
    ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ms_local = float(np.sum(ms)) / args.steps
    ms_step = max_over_ranks(ms_local, world, dist, dev)
    value = B_total / (ms_step / 1e3)

    lo = out["lo"].cpu().numpy()[:, 0].astype(np.float64)
    hi = out["hi"].cpu().numpy()[:, 0].astype(np.float64)

    # ---- the same step through the other path (fused layer launches when the
    # headline runs the per-step kernels, and the reverse), timed the same way
    alt = None
    if not args.no_alt_path:
        ctx.set_fused(not args.fused)
        try:
            for _ in range(args.warmup):
                step()
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                step()
                ends[k].record(stream)
            torch.cuda.synchronize()
            if ctx.sync() != 0:
                raise RuntimeError("alternate path failed")
            ms_alt = max_over_ranks(float(np.mean([s_.elapsed_time(e_) for s_, e_ in
                                                   zip(starts, ends)])), world, dist, dev)
            w_alt = float((out["hi"] - out["lo"]).float().mean().item())
            alt = {"fused_layers": not args.fused, "ms_per_step": round(ms_alt, 4),
                   "value": round(B_total / (ms_alt / 1e3), 1), "unit": "boxes/s",
                   "mean_output_width": round(w_alt, 6),
                   "note": "bern_propagate with bern_set_fused(%d)" % (0 if args.fused else 1)}
        finally:
            ctx.set_fused(bool(args.fused))
    nt = out["n_terms"].cpu().numpy()[:, 0, 0]
    coef = out["coef"].cpu().numpy()[:, 0].astype(np.float64)
    ex = bern.monomials(w.net.n_in, w.degree_cap).astype(np.float64)
    inv = 1.0 / np.prod(ex + 1.0, axis=1)
    vol = np.array([((coef[i, 0, :nt[i]] - coef[i, 1, :nt[i]]) * inv[:nt[i]]).sum()
                    for i in range(B)])

    # ---- per-kernel pass (same kernels through the step ABI)
    kp = KernelPass(ctx, torch, w, Wd, bd, boxes_d, fused=bool(args.fused))
    for _ in range(max(1, args.warmup)):
        kp.step()
    kp.collect()
    kp.times = {}
    for _ in range(args.steps):
        flush.zero_()
        kp.step()
        kp.collect()
    rc = ctx.sync()
    if rc != 0:
        raise RuntimeError("kernel pass failed: %s" % bern.strerror(rc))
    work = kp.work()
    avg = {k: float(np.mean(v)) for k, v in kp.times.items()}
    fused_kernels = None
    if not args.fused and not args.no_alt_path:
        kf = KernelPass(ctx, torch, w, Wd, bd, boxes_d, fused=True)
        for _ in range(max(1, args.warmup)):
            kf.step()
        kf.collect()
        kf.times = {}
        for _ in range(args.steps):
            flush.zero_()
            kf.step()
            kf.collect()
        if ctx.sync() != 0:
            raise RuntimeError("fused kernel pass failed")
        fwork = kf.work()
        fused_kernels = {}
        for k_, v_ in sorted(kf.times.items(), key=lambda kv: -float(np.mean(kv[1]))):
            ms_ = float(np.mean(v_))
            wk_ = fwork.get(k_, {"bytes": 0.0, "flops": 0.0})
            fused_kernels[k_] = {"ms": round(ms_, 4),
                                 "GBps": round(wk_["bytes"] / (ms_ / 1e3) / 1e9, 1),
                                 "TFLOPs": round(wk_["flops"] / (ms_ / 1e3) / 1e12, 3)}
    total_kernel_ms = sum(avg.values())
    dom = max(avg, key=lambda k: avg[k])
    peaks, peak_kind = load_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_nominal = (sm_count * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0))
                    * 1e6 / 1e12)
    # the FP32 roof is measured: round-up FMAs (what the bound kernels issue)
    # on every resident thread, fastest of five launches
    fp32_peak = bern.fma_throughput(local_rank, stream, directed=True, reps=5)
    fp32_rn = bern.fma_throughput(local_rank, stream, directed=False, reps=5)
    wk = work.get(dom, {"bytes": 0.0, "flops": 0.0})
    sec = avg[dom] / 1e3
    gbs = wk["bytes"] / sec / 1e9
    tfs = wk["flops"] / sec / 1e12
    # the bound is whichever roof the kernel's arithmetic intensity hits first
    ridge = fp32_peak * 1e12 / (hbm * 1e9)
    inten = wk["flops"] / max(wk["bytes"], 1.0)
    if inten < ridge:
        roof = {"bound": "hbm", "achieved": round(gbs, 2), "peak": hbm, "unit": "GB/s",
                "frac": round(gbs / hbm, 4)}
    else:
        roof = {"bound": "alu", "achieved": round(tfs, 3), "peak": round(fp32_peak, 2),
                "unit": "TFLOP/s", "frac": round(tfs / fp32_peak, 4)}
    roof["kernel"] = dom
    roof["peak_source"] = ("%s (%s)" % (PEAKS_FILE.split("/")[-1], peak_kind)
                           if roof["bound"] == "hbm" else
                           "measured: bern_fma_throughput, round-up FMAs, 8 chains per thread "
                           "on every resident thread (nominal %d SMs x 128 lanes x 2 x %.0f MHz "
                           "= %.1f TFLOP/s)" % (sm_count, float(peaks.get("sm_max_mhz", 2070.0)),
                                                fp32_nominal))
    roof["fp32_measured_tflops"] = {"round_up": round(fp32_peak, 2),
                                    "round_to_nearest": round(fp32_rn, 2),
                                    "nominal": round(fp32_nominal, 2)}
    roof["traffic"] = ncu_traffic(dom)
    roof["algorithmic_bytes"] = wk["bytes"]
    roof["algorithmic_flops"] = wk["flops"]
    roof["avg_launch_ms"] = round(avg[dom], 4)
    def kernel_entry(k, v):
        wk_ = work.get(k, {"bytes": 0.0, "flops": 0.0})
        gbs_ = wk_["bytes"] / (v / 1e3) / 1e9
        tfs_ = wk_["flops"] / (v / 1e3) / 1e12
        alu = wk_["flops"] / max(wk_["bytes"], 1.0) >= ridge
        return {"ms": round(v, 4), "share": round(v / total_kernel_ms, 4),
                "GBps": round(gbs_, 1), "TFLOPs": round(tfs_, 3),
                "bound": "alu" if alu else "hbm",
                "frac": round(tfs_ / fp32_peak if alu else gbs_ / hbm, 4)}
    kernels = {k: kernel_entry(k, v) for k, v in sorted(avg.items(), key=lambda kv: -kv[1])}

    # ---- end to end through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        boxes_h = pin(w.boxes)
        W_h = [pin(x) for x in w.net.W]
        b_h = [pin(x) for x in w.net.b]
        out_h = {"lo": pin(np.empty((B, o), np.float32)), "hi": pin(np.empty((B, o), np.float32)),
                 "n_terms": pin(np.empty((B, o, 2), np.int32)),
                 "coef": pin(np.empty((B, o, 2, cap_terms), np.float32))}
        for _ in range(max(1, args.warmup)):
            ctx.propagate_host(w.net.widths, W_h, b_h, boxes_h, degree=w.degree,
                               cap=w.degree_cap, cap_terms=cap_terms, out=out_h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.propagate_host(w.net.widths, W_h, b_h, boxes_h, degree=w.degree,
                               cap=w.degree_cap, cap_terms=cap_terms, out=out_h)
        wall = (time.perf_counter() - t0) / args.steps
        wall = max_over_ranks(wall, world, dist, dev)
        h2d = boxes_h.nbytes + sum(x.nbytes for x in W_h) + sum(x.nbytes for x in b_h)
        d2h = sum(v.nbytes for v in out_h.values())
        e2e = {"value": round(B_total / wall, 1), "unit": "boxes/s",
               "note": ("each rank its own slice through host buffers, no gather"
                        if world > 1 else "host buffers in, host buffers out"),
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": round(wall * 1e3, 3)}

    # ---- the learned form: degree MLP trained on the GPU, then timed like the plain form
    learned = None
    learned4 = None
    if not args.no_learned and world == 1:
        from paper_2211_14438_gb300 import learned as lm

        def timed(net, Wd_, bd_, bx_, degree, ct, o_, tau=0.0):
            outx = {"lo": torch.empty(bx_.shape[0], o_, device=dev),
                    "hi": torch.empty(bx_.shape[0], o_, device=dev),
                    "n_terms": torch.empty(bx_.shape[0], o_, 2, device=dev, dtype=torch.int32),
                    "coef": torch.empty(bx_.shape[0], o_, 2, ct, device=dev), "keys": None}

            def st():
                ctx.propagate(net.widths, Wd_, bd_, bx_, degree=degree, cap=16, tau=tau,
                              cap_terms=ct, out=outx, sync=False)
            for _ in range(args.warmup):
                st()
            if ctx.sync() != 0:
                raise RuntimeError("propagate failed")
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            for k in range(args.steps):
                flush.zero_()
                starts[k].record(stream)
                st()
                ends[k].record(stream)
            torch.cuda.synchronize()
            if ctx.sync() != 0:
                raise RuntimeError("propagate failed")
            msx = max_over_ranks(float(np.mean([s_.elapsed_time(e_) for s_, e_ in
                                                zip(starts, ends)])), world, dist, dev)
            return msx, float((outx["hi"] - outx["lo"]).float().mean().item())

        def learned_entry(net, train_boxes, plain_ms, plain_width, bx_, Wd_, bd_, ct, o_):
            info = lm.fit(ctx, net.widths, net.W, net.b, train_boxes, cap=16)
            plan = info["plan"]
            ms_l, width_l = timed(net, Wd_, bd_, bx_, plan, ct, o_)
            tr = ctx.propagate(net.widths, Wd_, bd_, bx_, degree=plan, cap=16, cap_terms=ct,
                               trace=True)
            hist = np.bincount(tr["tr_degree"].cpu().numpy().reshape(-1), minlength=5)[1:]
            ch = info["chosen"]
            nb = int(bx_.shape[0])
            return {
                "value": round(world * nb / (ms_l / 1e3), 1), "unit": "boxes/s",
                "ms_per_step": round(ms_l, 4),
                "plain_value": round(world * nb / (plain_ms / 1e3), 1),
                "mean_output_width": round(width_l, 6),
                "plain_mean_output_width": round(plain_width, 6),
                "speedup_vs_plain": round(plain_ms / ms_l, 4),
                "order_histogram_1_to_4": hist.tolist(),
                "train": {"boxes": int(len(train_boxes)), "neurons": info["n_samples"],
                          "seconds": round(info["seconds"], 2), "label_margin": ch["margin"],
                          "train_acc": round(ch["train_acc"], 4),
                          "learned_width_on_training_boxes": round(ch["learned_width"], 6),
                          "plain_width_on_training_boxes": round(info["base_width"], 6)},
                "plan": "BERN_DEG_LEARNED, fallback order 2, min_conf 0, per-layer caps %s"
                        % info["max_per_layer"],
            }

        learned = learned_entry(w.net, wl.batch_3in_training_boxes(800), ms_step,
                                float(np.mean(hi - lo)), boxes_d, Wd, bd, cap_terms, o)
        learned["workload"] = "the benchmark workload above"
        if not args.n_boxes:
            w4 = wl.batch_6in()
            Wd4 = [torch.from_numpy(x).to(dev) for x in w4.net.W]
            bd4 = [torch.from_numpy(x).to(dev) for x in w4.net.b]
            bx4 = torch.from_numpy(w4.boxes).to(dev)
            ct4 = bern.max_output_terms(w4.net.widths, 4, 16)
            ms4, width4 = timed(w4.net, Wd4, bd4, bx4, 2, ct4, w4.net.n_out)
            learned4 = learned_entry(w4.net, wl.batch_6in_training_boxes(700), ms4, width4, bx4,
                                     Wd4, bd4, ct4, w4.net.n_out)
            learned4["workload"] = ("learned-degree shape: MLP [6,100,100,100,2] seed 3, "
                                    "2048 boxes with sides U(0.05,0.5) in [-1,1]^6, cap 16; "
                                    "plain = order 2 everywhere")

    # ---- branch-and-bound refinement of the [6,64x4,1] root box [-1,1]^6 (wall clock,
    # host work included), plain orders against the learned form
    bnb5 = None
    if not args.no_learned and not args.no_bnb and not args.n_boxes and world == 1:
        from paper_2211_14438_gb300 import bnb
        from paper_2211_14438_gb300 import learned as lm
        w5 = wl.bnb_root_6in()
        root5 = w5.boxes[0]
        rng5 = np.random.default_rng(1005)
        c5 = rng5.uniform(-1, 1, (400, 6))
        s5 = rng5.uniform(0.1, 0.7, (400, 6))
        tr5 = wl.box_array(np.clip(c5 - s5 / 2, -1, 1), np.clip(c5 + s5 / 2, -1, 1))
        t0 = time.time()
        info5 = lm.fit(ctx, w5.net.widths, w5.net.W, w5.net.b, tr5, cap=16)
        train5 = time.time() - t0
        bnb5 = {"workload": "branch-and-bound network [6,64x4,1] seed 4, root [-1,1]^6, best-first "
                            "refinement of output 0 in rounds of 1024 splits until %d "
                            "leaves: plain order 2 and the learned degrees with the widest "
                            "side split, and the learned degrees with the learned split head; "
                            "boxes/s counts every bounded child, wall clock with host work"
                            % args.bnb_leaves,
                "learned_caps": info5["max_per_layer"], "train_seconds": round(train5, 2)}
        # the split head: trained on the leaves of a widest-side and a random-side
        # search, labelled by the plain method (the dimension whose halving
        # gives the smallest larger child upper bound)
        t0 = time.time()
        fn_plain = bnb.gpu_bound_fn(ctx, w5.net.widths, w5.net.W, w5.net.b, root5, 2, 16, 0.0)
        sb, sf = bnb.split_training_boxes(fn_plain, root5, rounds=10, batch=64)
        slab = bnb.split_labels(fn_plain, sb)
        head, head_loss = bnb.train_split_head(ctx, sf, slab, 6)
        split_fn = bnb.mlp_split_fn(ctx, head, root5)
        bnb5["split_head"] = {"train_boxes": int(len(sb)), "train_seconds": round(time.time() - t0, 2),
                              "loss": round(head_loss, 4),
                              "label_histogram": np.bincount(slab, minlength=6).tolist()}
        arms = (("plain", 2, None), ("learned", info5["plan"], None),
                ("learned_split", info5["plan"], split_fn))
        for name, deg, sfn in arms:
            fn = bnb.gpu_bound_fn(ctx, w5.net.widths, w5.net.W, w5.net.b, root5, deg, 16, 0.0)
            fn(root5[None])                                   # warm-up (tuning, graphs)
            bb = bnb.BranchAndBound(fn, root5, split_fn=sfn, batch=1024,
                                    max_leaves=args.bnb_leaves)
            torch.cuda.synchronize()
            t0 = time.time()
            bb.run(64)
            torch.cuda.synchronize()
            dt = time.time() - t0
            bnb5[name] = {"boxes_per_s": round((bb.propagated - 1) / dt, 1),
                          "leaves": bb.count(), "rounds": len(bb.history),
                          "U": round(bb.upper(), 5), "L": round(bb.lower(), 5),
                          "seconds": round(dt, 3)}

    # ---- the paper's Bernstein-tensor squares against the power basis (context)
    bern_basis = None
    if world == 1 and not args.no_bernstein_basis:
        try:
            bern_basis = bernstein_basis_entry(ctx, torch, dev, flush, args)
        except Exception as ex:
            bern_basis = {"error": "%s: %s" % (type(ex).__name__, ex)}

    # ---- Lin linearisation (Sec. 5.3); reported beside the headline, which
    # it can never cost: an error here is recorded, not raised
    lin_res = None
    if not args.no_lin and world == 1:
        try:
            lin_res = lin_entries(ctx, torch, dev, flush, args, w, Wd, bd, boxes_d, ms_step,
                                  float(np.mean(hi - lo)), world, dist)
        except Exception as ex:
            lin_res = {"error": "%s: %s" % (type(ex).__name__, ex)}

    cpu = None
    if pool is not None:
        idx = np.linspace(0, B - 1, 2 * cores).astype(int)
        rate, wall, per_box = oracle_rate(pool, cores, w, idx)
        pool.close()
        cpu = {"value": round(rate, 4), "unit": "boxes/s", "cores": cores, "kind": "oracle",
               "nproc": os.cpu_count(),
               "single_thread_boxes_per_s": round(len(per_box) / float(np.sum(per_box)), 4),
               "sample": "%d of the 5120 boxes (evenly strided), one per worker process, "
                         "FP64 oracle, %.1f s wall, %.1f s of CPU time; the single-thread "
                         "figure is the mean per-box time inside the workers"
                         % (len(idx), wall, float(np.sum(per_box)))}

    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "boxes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded networks and boxes)",
        "config": {"workload": "batched plain method: MLP [3,64,64,64,64,1] seed 2, "
                               "5120 boxes (16^3 grid of [-1,1]^3 + 1024 random, sides "
                               "U(0.01,0.5)), ReLU order 2, cap 16" +
                               (" (%d strided boxes only)" % B if args.n_boxes else ""),
                   "n_boxes_per_gpu": B, "degree": w.degree, "degree_cap": w.degree_cap,
                   "mean_output_width": round(float(np.mean(hi - lo)), 6),
                   "mean_vol_relative": round(float(np.mean(vol)), 6),
                   "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": ("box-sharded dp%d: %d replicas of the batch split into "
                                   "cost-balanced slices (interval-arithmetic term-pair cost), "
                                   "results all_gathered (lo, hi, n_terms) every step"
                                   % (world, world)) if world > 1 else "single GPU",
                   "boxes_total": B_total,
                   "graphs": True, "fused_layers": bool(args.fused)},
        "roofline": roof, "kernels": kernels, "alternate_path": alt,
        "fused_layer_kernels": fused_kernels,
        "kernel_pass_ms_per_step": round(total_kernel_ms, 4),
        "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
        "learned": learned, "learned_6in": learned4, "bnb_6in": bnb5, "lin": lin_res,
        "bernstein_basis": bern_basis,
        "clocks": clocks,
    }
    return line


# ---------------------------------------------------------------- reference
def run_reference(args, rank, world):
    from paper_2211_14438_gb300 import workloads as wl
    if rank != 0:
        return None
    cores = os.cpu_count() or 1
    pool = mp.get_context("spawn").Pool(cores)
    w = wl.batch_3in()
    B = len(w.boxes)
    rng = np.random.default_rng(0)
    for _ in range(args.warmup):
        oracle_rate(pool, cores, w, rng.choice(B, cores, replace=False))
    total_boxes, total_wall = 0, 0.0
    for _ in range(args.steps):
        idx = rng.choice(B, cores, replace=False)
        r, wall, _ = oracle_rate(pool, cores, w, idx)
        total_boxes += len(idx)
        total_wall += wall
    pool.close()
    value = total_boxes / total_wall
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "boxes/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * total_wall / args.steps, 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded networks and boxes)",
        "config": {"workload": "batched plain method: MLP [3,64,64,64,64,1] seed 2, "
                               "5120 boxes, ReLU order 2, cap 16",
                   "sample_per_step": "%d random boxes of the 5120, one per process" % cores},
        "cpu_baseline": {"value": round(value, 4), "unit": "boxes/s", "cores": cores,
                         "kind": "oracle",
                         "sample": "%d steps x %d boxes, FP64 oracle" % (args.steps, cores)},
        "e2e": {"value": round(value, 4), "unit": "boxes/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


# ------------------------------------------------- paper-shaped sweeps (context)
def run_paper_sweeps(args):
    """Context runs on the shapes of the paper's ablations (Figs. 4-7): weights
    and biases U(-5,5) (seeded here, unseeded in the paper), box [-1,1]^n,
    degree cap 64.  Per setting: the latency of one box per call (the paper's
    unit: graph replay, CUDA events, median of 20 calls after warm-up), the
    throughput of 4096 random sub-boxes per call (sides U(0.05,0.5)), and the
    mean over the box of upper minus lower polynomial (Vol_relative).  Not the
    headline metric; one JSON line."""
    import torch
    from paper_2211_14438_gb300 import bern
    from paper_2211_14438_gb300 import workloads as wl
    dev = torch.device("cuda:0")
    ctx = bern.Context(0, stream=torch.cuda.current_stream(dev))
    settings = [("fig4", 2, [20, 20], L) for L in (2, 3, 4, 5, 6)]
    settings += [("fig5", n, [20, 20], 2) for n in range(2, 9)]
    settings += [("fig6", 2, [ne, ne], 2) for ne in (10, 20, 40, 60, 80, 100)]
    settings += [("fig7", 2, [20] * k, 2) for k in range(1, 6)]
    cap = 64
    rows = []
    for si, (fig, n, hidden, L) in enumerate(settings):
        net = wl.paper_net(n, hidden, seed=500 + si)
        Wd = [torch.from_numpy(x).to(dev) for x in net.W]
        bd = [torch.from_numpy(x).to(dev) for x in net.b]
        ct = bern.max_output_terms(net.widths, L, cap)

        def timed(boxes_d, reps):
            B = int(boxes_d.shape[0])
            out = {"lo": torch.empty(B, 1, device=dev), "hi": torch.empty(B, 1, device=dev),
                   "n_terms": torch.empty(B, 1, 2, device=dev, dtype=torch.int32),
                   "coef": torch.empty(B, 1, 2, ct, device=dev), "keys": None}
            for _ in range(3):
                ctx.propagate(net.widths, Wd, bd, boxes_d, degree=L, cap=cap, cap_terms=ct,
                              out=out, sync=False)
            if ctx.sync() != 0:
                raise RuntimeError("propagate failed on %s %s" % (fig, net.widths))
            ms = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(ctx.stream)
                ctx.propagate(net.widths, Wd, bd, boxes_d, degree=L, cap=cap, cap_terms=ct,
                              out=out, sync=False)
                e1.record(ctx.stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            if ctx.sync() != 0:
                raise RuntimeError("propagate failed on %s %s" % (fig, net.widths))
            return float(np.median(ms)), out

        one = torch.from_numpy(wl.box_array([-1.0] * n, [1.0] * n)[None]).to(dev)
        t1, out = timed(one, 20)
        nt = int(out["n_terms"][0, 0, 0])
        D = 0
        while bern.num_monomials(n, D) < nt:
            D += 1
        ex = bern.monomials(n, D)[:nt].astype(np.float64)
        cf = out["coef"][0, 0].cpu().numpy().astype(np.float64)
        vol = float(((cf[0, :nt] - cf[1, :nt]) / np.prod(ex + 1.0, axis=1)).sum())
        rng = np.random.default_rng(900 + si)
        c = rng.uniform(-1, 1, (4096, n))
        sd = rng.uniform(0.05, 0.5, (4096, n))
        many = torch.from_numpy(wl.box_array(np.clip(c - sd / 2, -1, 1),
                                             np.clip(c + sd / 2, -1, 1))).to(dev)
        tb, _ = timed(many, 5)
        rows.append({"setting": fig, "widths": net.widths, "relu_order": L,
                     "one_box_ms": round(t1, 4), "boxes_per_s_4096": round(4096 / (tb / 1e3), 1),
                     "vol_relative": round(vol, 3),
                     "lo": round(float(out["lo"][0, 0]), 4), "hi": round(float(out["hi"][0, 0]), 4)})
    return {"metric": "paper-shaped sweeps (context, not the headline metric)",
            "data": "synthetic: paper ablation shapes, weights and biases U(-5,5) seeded 500+i, "
                    "box [-1,1]^n; throughput on 4096 random sub-boxes",
            "degree_cap": cap, "rows": rows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--bnb-leaves", type=int, default=65536,
                    help="leaf budget of the branch-and-bound refinement (65536: the stated size)")
    ap.add_argument("--no-bnb", action="store_true",
                    help="skip the branch-and-bound refinement of the [6,64x4,1] root box [-1,1]^6")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip training and timing the learned-degree form")
    ap.add_argument("--no-lin", action="store_true",
                    help="skip timing the Lin-linearised forms")
    ap.add_argument("--no-bernstein-basis", action="store_true",
                    help="skip the Bernstein-tensor (Prod_Bern) comparison")
    ap.add_argument("--fused", action="store_true",
                    help="headline through the fused layer kernels (bern_set_fused(1))")
    ap.add_argument("--no-alt-path", action="store_true",
                    help="skip timing the other path (fused / per-step) beside the headline")
    ap.add_argument("--n-boxes", type=int, default=0,
                    help="use N evenly strided boxes of the workload (small cases for ncu)")
    ap.add_argument("--paper-sweeps", action="store_true",
                    help="instead of the benchmark, time the paper's ablation shapes (context)")
    args = ap.parse_args()
    if args.paper_sweeps:
        print(json.dumps(run_paper_sweeps(args)))
        return
    args.warmup = max(args.warmup, 3)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
        dist = tdist
    if args.impl == "reference":
        line = run_reference(args, rank, world)
    else:
        line = run_ours(args, rank, world, local_rank, dist)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if line is not None and rank == 0:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
