"""Seeded synthetic time-series datasets (stand-ins for the UCR archive).

This module only draws data.  It holds none of the method's arithmetic
(no distance, envelope, bound or search), so both the CUDA path's tests and
the CPU oracle may take their inputs from it.

Recipes (one per workload; every draw comes from numpy's PCG64 seeded with
``SeedSequence([1808096170, workload, dataset, split])``):

* base series: a Gaussian random walk with unit steps, z-normalised per series
  (mean 0, standard deviation 1), then a class shape is added (no
  re-normalisation) and, where stated, N(0, sigma^2) noise;
* labels: uniform over the classes;
* integer windows from a fraction r of the length: W = floor(r * L + 0.5).

=========  ==================================================================
tiny       train 64, test 32, L=128, W=13, V=5, float64; 4 classes, class c is a
           sinusoid of period L/(2+c), amplitude 1.5, random phase.
pairs      train 500, test 500, L=256, W=26, V in {1,2,5}, float32; 8 classes:
           even c a sinusoid of period L/(2+c/2), odd c a Gaussian bump
           (sigma L/16, height 1.5) centred at (c+0.5)L/8; plus N(0, 0.3^2).
precision  train 10,000, test 2,000, L=1024, W in {102, 512, 1023}, V=5,
           float32; 16 classes: sinusoid of period L/(2 + c mod 8) (amplitude
           1.5, random phase) plus a continuous two-piece linear trend whose
           breakpoint (c+1)L/17 and slopes (uniform in [-2, 2]/L) are drawn
           once per class.
batched    64 datasets; L log-uniform in [24, 2048], train size log-uniform in
           [16, 8000], test size train//2, W = round(r L) with r drawn from
           {0, .05, .1, .2, .5, 1}, V uniform in 1..8, 2..32 classes; class c
           a sinusoid of period L/(2 + c mod 8) with a class phase.
serving    16 resident training sets; L cycles through {128, 512, 1500}; size
           log-uniform in [1000, 20000]; W = round(0.1 L), V=5, 8 classes as in
           ``tiny``; queries are drawn one at a time (split "serve").
varlen     series of unequal lengths (ragged sets): train 8,000, test 2,000,
           each series' length uniform in [L0 - dL, L0 + dL] (L0 = 512,
           dL = 64), W = round(0.2 L0) = 102, V=5, float32; 8 classes, class c
           a sinusoid of period (own length)/(2 + c) (the class pattern
           stretched to the series' length), amplitude 1.5, random phase,
           added to the series' own z-normalised walk.
=========  ==================================================================
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_ROOT = 1808096170
WORKLOADS = {"tiny": 0, "pairs": 1, "precision": 2, "batched": 3, "serving": 4, "varlen": 5}
SPLITS = {"train": 0, "test": 1, "meta": 2, "serve": 3, "class": 4}


def rng_for(workload: str, dataset: int, split: str) -> np.random.Generator:
    ss = np.random.SeedSequence([SEED_ROOT, WORKLOADS[workload], int(dataset), SPLITS[split]])
    return np.random.Generator(np.random.PCG64(ss))


def window_from_ratio(r: float, L: int) -> int:
    """Integer window for a fractional one: floor(r * L + 0.5)."""
    return int(math.floor(r * L + 0.5))


def znormed_walks(rng: np.random.Generator, n: int, L: int) -> np.ndarray:
    w = np.cumsum(rng.standard_normal((n, L)), axis=1)
    mu = w.mean(axis=1, keepdims=True)
    sd = w.std(axis=1, keepdims=True)
    sd[sd == 0] = 1.0
    return (w - mu) / sd


@dataclass
class Dataset:
    name: str
    train: np.ndarray
    train_labels: np.ndarray
    test: np.ndarray
    test_labels: np.ndarray
    W: int
    V: int
    n_classes: int
    extra: dict = field(default_factory=dict)

    @property
    def L(self) -> int:
        return int(self.train.shape[1])

    @property
    def N(self) -> int:
        return int(self.train.shape[0])

    @property
    def Q(self) -> int:
        return int(self.test.shape[0])


def _sinusoid(L: int, period: float, phase: np.ndarray, amp: float = 1.5) -> np.ndarray:
    i = np.arange(L)[None, :]
    return amp * np.sin(2.0 * np.pi * i / period + phase[:, None])


def _shapes_tiny(rng, labels, L):
    phase = rng.uniform(0, 2 * np.pi, size=labels.shape[0])
    out = np.zeros((labels.shape[0], L))
    for c in np.unique(labels):
        m = labels == c
        out[m] = _sinusoid(L, L / (2.0 + c), phase[m])
    return out


def _draw_tiny_like(workload, dataset, n_train, n_test, L, n_classes, shapes):
    parts = []
    for split, n in (("train", n_train), ("test", n_test)):
        rng = rng_for(workload, dataset, split)
        labels = rng.integers(0, n_classes, size=n).astype(np.int32)
        x = znormed_walks(rng, n, L) + shapes(rng, labels, L)
        parts.append((x, labels))
    return parts


def make_tiny() -> Dataset:
    L = 128
    (tr, trl), (te, tel) = _draw_tiny_like("tiny", 0, 64, 32, L, 4, _shapes_tiny)
    return Dataset("tiny", tr.astype(np.float64), trl, te.astype(np.float64), tel,
                   W=window_from_ratio(0.1, L), V=5, n_classes=4)


def _shapes_pairs(rng, labels, L):
    n = labels.shape[0]
    phase = rng.uniform(0, 2 * np.pi, size=n)
    i = np.arange(L)[None, :]
    out = np.zeros((n, L))
    for c in np.unique(labels):
        m = labels == c
        if c % 2 == 0:
            out[m] = _sinusoid(L, L / (2.0 + c // 2), phase[m])
        else:
            mu = (c + 0.5) * L / 8.0
            sig = L / 16.0
            out[m] = np.broadcast_to(1.5 * np.exp(-0.5 * ((i - mu) / sig) ** 2), (int(m.sum()), L))
    return out + rng.normal(0.0, 0.3, size=(n, L))


def make_pairs(V: int = 5) -> Dataset:
    L = 256
    (tr, trl), (te, tel) = _draw_tiny_like("pairs", 0, 500, 500, L, 8, _shapes_pairs)
    return Dataset("pairs", tr.astype(np.float32), trl, te.astype(np.float32), tel,
                   W=window_from_ratio(0.1, L), V=V, n_classes=8)


def _class_trends(L: int, n_classes: int):
    rng = rng_for("precision", 0, "class")
    bps = [(c + 1) * L / 17.0 for c in range(n_classes)]
    slopes = rng.uniform(-2.0 / L, 2.0 / L, size=(n_classes, 2))
    i = np.arange(L, dtype=np.float64)
    trends = np.empty((n_classes, L))
    for c in range(n_classes):
        bp = bps[c]
        s1, s2 = slopes[c]
        trends[c] = np.where(i <= bp, s1 * i, s1 * bp + s2 * (i - bp))
    return trends


def make_precision(W_ratio: float = 0.1, n_train: int = 10_000, n_test: int = 2_000,
                   L: int = 1024) -> Dataset:
    n_classes = 16
    trends = _class_trends(L, n_classes)
    parts = []
    for split, n in (("train", n_train), ("test", n_test)):
        rng = rng_for("precision", 0, split)
        labels = rng.integers(0, n_classes, size=n).astype(np.int32)
        x = znormed_walks(rng, n, L)
        phase = rng.uniform(0, 2 * np.pi, size=n)
        for c in np.unique(labels):
            m = labels == c
            x[m] += _sinusoid(L, L / (2.0 + c % 8), phase[m]) + trends[c][None, :]
        parts.append((x.astype(np.float32), labels))
    W = min(window_from_ratio(W_ratio, L), L - 1)
    (tr, trl), (te, tel) = parts
    return Dataset(f"precision_w{W}", tr, trl, te, tel, W=W, V=5, n_classes=n_classes)


def batched_specs(n_datasets: int = 64):
    """Shape parameters of the heterogeneous batch (drawn, not data)."""
    rng = rng_for("batched", 0, "meta")
    ratios = [0.0, 0.05, 0.1, 0.2, 0.5, 1.0]
    specs = []
    for d in range(n_datasets):
        L = int(round(math.exp(rng.uniform(math.log(24), math.log(2048)))))
        N = int(round(math.exp(rng.uniform(math.log(16), math.log(8000)))))
        r = ratios[int(rng.integers(0, len(ratios)))]
        V = int(rng.integers(1, 9))
        k = int(rng.integers(2, 33))
        specs.append(dict(L=L, N=N, Q=max(1, N // 2), W=min(window_from_ratio(r, L), L - 1),
                          V=V, n_classes=k, ratio=r))
    return specs


def make_batched_dataset(d: int, spec: dict) -> Dataset:
    L, N, Q, k = spec["L"], spec["N"], spec["Q"], spec["n_classes"]
    class_phase = rng_for("batched", d, "class").uniform(0, 2 * np.pi, size=k)
    parts = []
    for split, n in (("train", N), ("test", Q)):
        rng = rng_for("batched", d, split)
        labels = rng.integers(0, k, size=n).astype(np.int32)
        x = znormed_walks(rng, n, L)
        for c in np.unique(labels):
            m = labels == c
            x[m] += _sinusoid(L, L / (2.0 + c % 8), np.full(int(m.sum()), class_phase[c]))
        parts.append((x.astype(np.float32), labels))
    (tr, trl), (te, tel) = parts
    return Dataset(f"batched_{d}", tr, trl, te, tel, W=spec["W"], V=spec["V"], n_classes=k,
                   extra=dict(spec))


def make_batched(n_datasets: int = 64, max_n: int | None = None):
    """The heterogeneous batch; ``max_n`` caps train sizes for quick tests."""
    out = []
    for d, spec in enumerate(batched_specs(n_datasets)):
        spec = dict(spec)
        if max_n is not None and spec["N"] > max_n:
            spec["N"] = max_n
            spec["Q"] = max(1, max_n // 2)
        out.append(make_batched_dataset(d, spec))
    return out


SERVING_LENGTHS = (128, 512, 1500)


def serving_specs(n_sets: int = 16):
    rng = rng_for("serving", 0, "meta")
    specs = []
    for d in range(n_sets):
        L = SERVING_LENGTHS[d % len(SERVING_LENGTHS)]
        N = int(round(math.exp(rng.uniform(math.log(1000), math.log(20000)))))
        specs.append(dict(L=L, N=N, W=window_from_ratio(0.1, L), V=5, n_classes=8))
    return specs


def make_serving_set(d: int, spec: dict, max_n: int | None = None) -> Dataset:
    L, k = spec["L"], spec["n_classes"]
    N = spec["N"] if max_n is None else min(spec["N"], max_n)
    rng = rng_for("serving", d, "train")
    labels = rng.integers(0, k, size=N).astype(np.int32)
    x = znormed_walks(rng, N, L) + _shapes_tiny(rng, labels, L)
    return Dataset(f"serving_{d}", x.astype(np.float32), labels,
                   np.zeros((0, L), np.float32), np.zeros(0, np.int32),
                   W=spec["W"], V=spec["V"], n_classes=k, extra=dict(spec))


def serving_queries(d: int, spec: dict, n: int, offset: int = 0):
    """``n`` queries for serving set ``d``; query ``offset + k`` is always the
    same series whatever ``n`` is, so a query can be regenerated alone."""
    L, k = spec["L"], spec["n_classes"]
    xs = np.empty((n, L), np.float32)
    ys = np.empty(n, np.int32)
    for r in range(n):
        ss = np.random.SeedSequence([SEED_ROOT, WORKLOADS["serving"], d, SPLITS["serve"],
                                     offset + r])
        rng = np.random.Generator(np.random.PCG64(ss))
        lab = rng.integers(0, k, size=1).astype(np.int32)
        xs[r] = (znormed_walks(rng, 1, L) + _shapes_tiny(rng, lab, L))[0]
        ys[r] = lab[0]
    return xs, ys


def arrival_times(rate_qps: float, duration_s: float, seed_index: int = 0) -> np.ndarray:
    """Poisson arrival instants (seconds) at the given rate."""
    ss = np.random.SeedSequence([SEED_ROOT, WORKLOADS["serving"], 10_000 + seed_index,
                                 SPLITS["meta"]])
    rng = np.random.Generator(np.random.PCG64(ss))
    n = int(rate_qps * duration_s * 1.5) + 16
    t = np.cumsum(rng.exponential(1.0 / rate_qps, size=n))
    return t[t < duration_s]


def random_series(seed: int, n: int, L: int, dtype=np.float32) -> np.ndarray:
    """Plain z-normalised walks for property tests."""
    ss = np.random.SeedSequence([SEED_ROOT, 99, seed, 0])
    rng = np.random.Generator(np.random.PCG64(ss))
    return znormed_walks(rng, n, L).astype(dtype)


@dataclass
class RaggedDataset:
    """A dataset whose series have unequal lengths: lists of 1-D arrays."""
    name: str
    train: list
    train_labels: np.ndarray
    test: list
    test_labels: np.ndarray
    W: int
    V: int
    n_classes: int
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return len(self.train)

    @property
    def Q(self) -> int:
        return len(self.test)

    @property
    def max_len(self) -> int:
        return max(max(len(x) for x in self.train), max(len(x) for x in self.test))

    @staticmethod
    def pack(series):
        """(values, offsets): series k is values[offsets[k]:offsets[k+1]]."""
        off = np.zeros(len(series) + 1, np.int64)
        off[1:] = np.cumsum([len(x) for x in series])
        return np.concatenate(series).astype(np.float32), off


def make_varlen(n_train: int = 8000, n_test: int = 2000, L0: int = 512, dL: int = 64,
                W_ratio: float = 0.2, V: int = 5, n_classes: int = 8,
                dataset: int = 0) -> RaggedDataset:
    parts = []
    for split, n in (("train", n_train), ("test", n_test)):
        rng = rng_for("varlen", dataset, split)
        labels = rng.integers(0, n_classes, size=n).astype(np.int32)
        lengths = rng.integers(L0 - dL, L0 + dL + 1, size=n)
        phase = rng.uniform(0, 2 * np.pi, size=n)
        xs = []
        for k in range(n):
            m = int(lengths[k])
            x = znormed_walks(rng, 1, m)[0]
            x += _sinusoid(m, m / (2.0 + labels[k]), phase[k:k + 1])[0]
            xs.append(x.astype(np.float32))
        parts.append((xs, labels))
    (tr, trl), (te, tel) = parts
    W = window_from_ratio(W_ratio, L0)
    return RaggedDataset(f"varlen_{dataset}", tr, trl, te, tel, W=W, V=V, n_classes=n_classes,
                         extra=dict(L0=L0, dL=dL))

