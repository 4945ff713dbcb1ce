"""The oracle against the stored golden values (CPU only)."""
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows():
    for line in open(os.path.join(GOLDEN, "hand_worked.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        name, a, b, W, V, qty, val = [s.strip() for s in line.split("|")]
        yield (name, np.array([float(x) for x in a.split(",")]),
               np.array([float(x) for x in b.split(",")]), int(W), int(V), qty,
               [float(x) for x in val.split(",")])


def test_hand_worked_examples(orc):
    n = 0
    for name, a, b, W, V, qty, val in _rows():
        U, Lo = orc.envelope(b, W)
        if qty == "dtw":
            got = [orc.dtw(a, b, W)]
        elif qty == "env_u":
            got = list(U)
        elif qty == "env_l":
            got = list(Lo)
        elif qty == "lb_keogh":
            got = [orc.lb_keogh(a, U, Lo)]
        elif qty == "lb_enhanced":
            got = [orc.lb_enhanced(a, b, U, Lo, W, V)]
        elif qty == "lb_enh_improved":
            got = [orc.lb_enhanced_improved(a, b, U, Lo, W, V)]
        elif qty == "lb_improved":
            got = [orc.lb_improved(a, b, U, Lo, W)]
        elif qty == "lb_new":
            got = [orc.lb_new(a, b, W)]
        else:
            raise AssertionError(qty)
        assert got == val, (name, qty, got, val)
        n += 1
    assert n == 30


def test_tiny_golden_regression(orc):
    from paper_1808_09617_gb300 import synth
    ds = synth.make_tiny()
    rows = [l.split() for l in open(os.path.join(GOLDEN, "tiny_nn.txt")) if not l.startswith("#")]
    idx, lab, dist = orc.nn_brute(ds.train, ds.train_labels, ds.test, ds.W)
    assert len(rows) == ds.Q
    for q, r in enumerate(rows):
        assert int(r[0]) == q
        assert idx[q] == int(r[1]) and lab[q] == int(r[2])
        assert dist[q] == float.fromhex(r[3])
