"""Write the stored expected values for the 'tiny' workload.

Calls only ``oracle/`` (and the seeded input generator for its inputs).  Run
from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1808_09617_gb300 import synth  # noqa: E402


def main():
    ds = synth.make_tiny()
    orc = oracle.get()
    idx, lab, dist = orc.nn_brute(ds.train, ds.train_labels, ds.test, ds.W)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_nn.txt")
    with open(out, "w") as f:
        f.write("# 1-NN of the 'tiny' workload (train 64, test 32, L=128, W=13), FP64 oracle\n")
        f.write("# brute force, ties to the lowest index.  Written by tests/golden/make_golden.py\n")
        f.write("# query nn_index nn_label nn_dist(hex float)\n")
        for q in range(ds.Q):
            f.write(f"{q} {idx[q]} {lab[q]} {float(dist[q]).hex()}\n")


if __name__ == "__main__":
    main()
