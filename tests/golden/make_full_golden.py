"""Write the stored 1-NN results of the full-size workloads, for the parity
tests that compare every query of the GPU search with the oracle.

Calls only ``oracle/`` (the paper's pruned search, Sec. 4, in FP64; equal to
the exhaustive 1-NN, which the oracle tests pin) and the seeded input
generator for its inputs.  Run from the repository root:

    python tests/golden/make_full_golden.py precision   # 3 windows x 2,000 queries
    python tests/golden/make_full_golden.py batched     # 64 datasets, 35,843 queries
    python tests/golden/make_full_golden.py serving     # 16 resident sets, 24 queries each
    python tests/golden/make_full_golden.py large       # Q x N above 2^31, 24 sampled queries
    python tests/golden/make_full_golden.py varlen      # unequal lengths, 2,000 queries

Each file is gzip-compressed text, one query per line:
``[dataset] query nn_index nn_label nn_dist(hex float)``.
"""
import gzip
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1808_09617_gb300 import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
PRECISION_RATIOS = (0.1, 0.5, 1.0)
SERVING_QUERIES_PER_SET = 24


def precision_path(ratio):
    return os.path.join(HERE, f"precision_r{int(round(ratio * 100)):03d}_nn.txt.gz")


BATCHED_PATH = os.path.join(HERE, "batched_nn.txt.gz")
LARGE_PATH = os.path.join(HERE, "large_nn.txt.gz")
# a search whose Q x N (50,000 x 43,000 = 2.15e9) is above 2^31, on short series
LARGE_N, LARGE_Q, LARGE_L, LARGE_W, LARGE_V = 50_000, 43_000, 16, 2, 2
LARGE_SAMPLE = 24


def large_inputs():
    """The large search's inputs: seeded z-normalised random walks, labels
    uniform over 5 classes, and the sampled query indices."""
    import numpy as np
    train = synth.random_series(7101, LARGE_N, LARGE_L)
    test = synth.random_series(7102, LARGE_Q, LARGE_L)
    rng = np.random.default_rng(7103)
    labels = rng.integers(0, 5, LARGE_N).astype(np.int32)
    sample = np.sort(rng.choice(LARGE_Q, LARGE_SAMPLE, replace=False))
    return train, labels, test, sample


SERVING_PATH = os.path.join(HERE, "serving_nn.txt.gz")
VARLEN_PATH = os.path.join(HERE, "varlen_nn.txt.gz")


def _write(path, header, rows):
    tmp = path + ".tmp"
    with gzip.open(tmp, "wt") as f:
        for h in header:
            f.write(f"# {h}\n")
        for r in rows:
            f.write(" ".join(r) + "\n")
    os.replace(tmp, path)


def _rows(prefix, idx, lab, dist, queries=None):
    qs = range(len(idx)) if queries is None else queries
    return [[*prefix, str(q), str(int(i)), str(int(l)), float(d).hex()]
            for q, i, l, d in zip(qs, idx, lab, dist)]


def make_precision(threads=None):
    orc = oracle.get()
    for r in PRECISION_RATIOS:
        ds = synth.make_precision(r)
        t0 = time.time()
        idx, lab, dist, _ = orc.nn_pruned(ds.train, ds.train_labels, ds.test, ds.W, ds.V,
                                          threads=threads)
        _write(precision_path(r),
               [f"1-NN of every query of the precision workload ({ds.N} x {ds.Q}, L={ds.L}, "
                f"W={ds.W}, V={ds.V}), FP64 oracle (pruned search, ties to the lowest index)",
                "written by tests/golden/make_full_golden.py",
                "query nn_index nn_label nn_dist(hex float)"],
               _rows([], idx, lab, dist))
        print(f"precision W={ds.W}: {ds.Q} queries in {time.time() - t0:.0f} s", flush=True)


def make_batched(threads=None):
    orc = oracle.get()
    rows = []
    t0 = time.time()
    for d, spec in enumerate(synth.batched_specs(64)):
        ds = synth.make_batched_dataset(d, spec)
        idx, lab, dist, _ = orc.nn_pruned(ds.train, ds.train_labels, ds.test, ds.W, ds.V,
                                          threads=threads)
        rows += _rows([str(d)], idx, lab, dist)
    _write(BATCHED_PATH,
           ["1-NN of every query of the 64 datasets of the batched workload, FP64 oracle "
            "(pruned search, ties to the lowest index)",
            "written by tests/golden/make_full_golden.py",
            "dataset query nn_index nn_label nn_dist(hex float)"], rows)
    print(f"batched: {len(rows)} queries in {time.time() - t0:.0f} s", flush=True)


def make_serving(threads=None):
    orc = oracle.get()
    rows = []
    t0 = time.time()
    k = SERVING_QUERIES_PER_SET
    for d, spec in enumerate(synth.serving_specs(16)):
        ds = synth.make_serving_set(d, spec)
        qs, _ = synth.serving_queries(d, spec, k, offset=0)
        idx, lab, dist, _ = orc.nn_pruned(ds.train, ds.train_labels, qs, ds.W, ds.V,
                                          threads=threads)
        rows += _rows([str(d)], idx, lab, dist)
    _write(SERVING_PATH,
           [f"1-NN of serving queries 0..{k - 1} of each of the 16 resident sets of the serving "
            "workload, FP64 oracle (pruned search, ties to the lowest index)",
            "written by tests/golden/make_full_golden.py",
            "set query nn_index nn_label nn_dist(hex float)"], rows)
    print(f"serving: {len(rows)} queries in {time.time() - t0:.0f} s", flush=True)


def make_large(threads=None):
    orc = oracle.get()
    train, labels, test, sample = large_inputs()
    t0 = time.time()
    idx, lab, dist, _ = orc.nn_pruned(train, labels, test[sample], LARGE_W, LARGE_V,
                                      threads=threads)
    _write(LARGE_PATH,
           [f"1-NN of {LARGE_SAMPLE} sampled queries of a search with Q x N above 2^31 "
            f"(train {LARGE_N}, test {LARGE_Q}, L={LARGE_L}, W={LARGE_W}, V={LARGE_V}), FP64 "
            "oracle (pruned search, ties to the lowest index)",
            "written by tests/golden/make_full_golden.py",
            "query nn_index nn_label nn_dist(hex float)"],
           _rows([], idx, lab, dist, queries=sample))
    print(f"large: {LARGE_SAMPLE} queries in {time.time() - t0:.0f} s", flush=True)


def make_varlen(threads=None):
    orc = oracle.get()
    ds = synth.make_varlen()
    tv, to = ds.pack(ds.train)
    qv, qo = ds.pack(ds.test)
    t0 = time.time()
    idx, lab, dist, _ = orc.nn_pruned_var(tv, to, ds.train_labels, qv, qo, ds.W, ds.V,
                                          threads=threads)
    _write(VARLEN_PATH,
           [f"1-NN of every query of the unequal-length workload ({ds.N} x {ds.Q}, lengths "
            f"{ds.extra['L0'] - ds.extra['dL']}..{ds.extra['L0'] + ds.extra['dL']}, W={ds.W}, "
            f"V={ds.V}), FP64 oracle (pruned search, ties to the lowest index; -1 without a "
            "warping path)",
            "written by tests/golden/make_full_golden.py",
            "query nn_index nn_label nn_dist(hex float)"],
           _rows([], idx, lab, dist))
    print(f"varlen: {ds.Q} queries in {time.time() - t0:.0f} s", flush=True)


def read(path):
    """Rows of a stored file as lists of ints, the distance as a float."""
    out = []
    with gzip.open(path, "rt") as f:
        for line in f:
            if line.startswith("#"):
                continue
            parts = line.split()
            out.append([int(x) for x in parts[:-1]] + [float.fromhex(parts[-1])])
    return out


if __name__ == "__main__":
    what = sys.argv[1:] or ["precision", "batched", "serving"]
    th = int(os.environ.get("ORACLE_THREADS", "0")) or None
    for w in what:
        {"precision": make_precision, "batched": make_batched, "serving": make_serving,
         "large": make_large, "varlen": make_varlen}[w](th)
