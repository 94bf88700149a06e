"""CPU checks of the oracle's run-time order choice (the learned plan's
reference): a chooser that returns fixed orders reproduces the fixed-order
propagation exactly, the term counts handed to the chooser are the dense
graded counts M(n, D) of the pre-activation polynomials, the per-box order
follows min(cap, order * max d), and the oracle MLP chooser's decision rule."""
import numpy as np

import oracle
from oracle import mlp as om
from paper_2211_14438_gb300 import workloads as wl


def test_callback_with_fixed_orders_reproduces_fixed_plan():
    w = wl.single_box_2in()
    degs = np.random.default_rng(0).integers(1, 5, 40)
    a = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], degs)
    seen = []

    def choose(layer, m, lo, hi, nt):
        k = (layer - 1) * 20 + m
        seen.append((layer, m, nt))
        return int(degs[k])

    b = oracle.propagate(w.net.widths, w.net.W, w.net.b, w.boxes[0], choose)
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])
    assert np.array_equal(a["tr_lo"], b["tr_lo"]) and np.array_equal(b["degree"], degs)
    for k in range(2):
        assert np.array_equal(a["upper"][0][k], b["upper"][0][k])
    # layer 1 sees degree-1 polynomials: M(2,1) = 3 terms; layer 2 sees the
    # degree max over layer-1 orders of its unstable neurons (graded count)
    assert all(nt == 3 for (layer, m, nt) in seen if layer == 1)
    D2 = max([degs[m] for m in range(20) if b["tr_case"][m] == 2] + [1])
    assert all(nt == (D2 + 1) * (D2 + 2) // 2 for (layer, m, nt) in seen if layer == 2)
    # per-box order bookkeeping: order_2 = min(16, max over layer-1 orders)
    assert b["order"][0] == 1 and b["order"][1] == min(16, int(degs[:20].max()))


def test_oracle_chooser_rule():
    th = np.zeros(om.num_params(8, 4))
    th[-4 + 2] = 10.0
    ch = om.DegreeChooser(th, 0.0, 2)
    assert ch(1, 0, -1.0, 2.0, 3) == 3
    # below min_conf: the fallback order
    th0 = np.zeros(om.num_params(8, 4))
    ch = om.DegreeChooser(th0, 0.5, 2)
    assert ch(1, 0, -1.0, 2.0, 3) == 2      # uniform softmax: 0.25 < 0.5
    assert ch.margin == 0.0                 # an exact tie is recorded as margin 0
