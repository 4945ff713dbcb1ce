"""Parity of the unequal-length path (ragged sets, through the C ABI) with the
FP64 oracle's unequal-length routines (Sec. 2: the equal-length exposition
generalises).

Tolerances as for equal lengths: FP32 bounds and DTW values within 1e-4
relative; +inf (no warping path inside the window) exactly where the oracle
has it; envelopes bit-exact; NN indices and labels bit-identical, -1 where
no training series fits the window.
"""
import math
import os

import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL32 = 1e-4
HERE = os.path.dirname(os.path.abspath(__file__))


def _series_set(seed, n, lo, hi):
    rng = np.random.default_rng(seed)
    out = []
    for m in rng.integers(lo, hi + 1, n):
        x = rng.standard_normal(int(m)).cumsum()
        x = (x - x.mean()) / (x.std() or 1.0)
        out.append(x.astype(np.float32))
    return out


def _pack(xs):
    return synth.RaggedDataset.pack(xs)


def _close_or_inf(got, want, rtol=RTOL32):
    got = np.asarray(got, np.float64)
    want = np.asarray(want, np.float64)
    inf_w = np.isinf(want)
    np.testing.assert_array_equal(np.isinf(got), inf_w)
    np.testing.assert_allclose(got[~inf_w], want[~inf_w], rtol=rtol, atol=1e-6)


# --------------------------------------------------------------- envelopes

ENV_CASES = [(2, 9, 0), (2, 9, 1), (5, 40, 3), (20, 130, 13), (100, 300, 33), (100, 300, 150),
             (448, 576, 102), (1000, 1100, 40), (2, 64, 500), (3000, 4500, 1200),
             (30, 31, 31), (7000, 8192, 700)]


@pytest.mark.parametrize("lo,hi,W", ENV_CASES)
def test_envelopes_varlen_bit_exact(lib, orc, lo, hi, W):
    xs = _series_set(lo * 31 + hi + W, 23, lo, hi)
    ml = max(len(x) for x in xs)
    Weff = min(W, ml - 1)
    env = lib.nn_dtw_build_envelopes_varlen(lib.ragged(xs), W).cpu().numpy()
    assert env.shape == (len(xs), ml, 2)
    for t, x in enumerate(xs):
        rows = min(len(x) + Weff, ml)
        U, Lo = orc.envelope_var(x, Weff, E=rows)
        np.testing.assert_array_equal(env[t, :rows, 0], U.astype(np.float32), err_msg=str(t))
        np.testing.assert_array_equal(env[t, :rows, 1], Lo.astype(np.float32), err_msg=str(t))


# ------------------------------------------------------------------ bounds

LB_CASES = [(20, 60, 5, 3), (20, 60, 40, 5), (2, 10, 1, 2), (2, 10, 8, 5), (100, 200, 13, 5),
            (448, 576, 102, 5), (30, 34, 0, 1), (60, 64, 63, 8), (1500, 2100, 300, 5)]


@pytest.mark.parametrize("lo,hi,W,V", LB_CASES)
def test_lb_enhanced_varlen_parity(lib, orc, lo, hi, W, V):
    tr = _series_set(lo + 7 * W + V, 70, lo, hi)
    te = _series_set(lo + 7 * W + V + 1, 40, lo, hi)
    ml = max(max(map(len, tr)), max(map(len, te)))
    Weff = min(W, ml - 1)
    rtr, rte = lib.ragged(tr), lib.ragged(te)
    env = lib.nn_dtw_build_envelopes_varlen(rtr, W, max_len=ml)
    tv, to = _pack(tr)
    qv, qo = _pack(te)
    for keogh in (False, True):
        kind = "keogh" if keogh else "enhanced"
        want = orc.lb_matrix_var(qv, qo, tv, to, Weff, V, kind=kind)
        got = lib.lb_enhanced_varlen(rte, rtr, env, W, V, keogh=keogh).cpu().numpy()
        _close_or_inf(got, want)
        safe = lib.lb_enhanced_varlen(rte, rtr, env, W, V, keogh=keogh, safe=True).cpu().numpy()
        fin = np.isfinite(want)
        assert np.all(safe[fin] <= want[fin]), kind
        np.testing.assert_array_equal(np.isinf(safe), ~fin)


# ---------------------------------------------------------------------- DTW

DTW_CASES = [(20, 60, 0), (20, 60, 1), (20, 60, 5), (100, 160, 13), (100, 160, 31),
             (100, 160, 40), (300, 420, 100), (300, 420, 300), (900, 1100, 1023),
             (1000, 1800, 1500), (2, 12, 3), (500, 520, 600)]


@pytest.mark.parametrize("lo,hi,W", DTW_CASES)
def test_dtw_varlen_parity(lib, orc, lo, hi, W):
    import torch
    tr = _series_set(lo * 3 + W, 24, lo, hi)
    te = _series_set(lo * 3 + W + 1, 16, lo, hi)
    ml = max(max(map(len, tr)), max(map(len, te)))
    Weff = min(W, ml - 1)
    pairs = np.array([(q, t) for q in range(len(te)) for t in range(len(tr))], np.int32)
    got = lib.dtw_windowed_varlen(lib.ragged(te), lib.ragged(tr),
                                  torch.from_numpy(pairs).cuda(), W).cpu().numpy()
    tv, to = _pack(tr)
    qv, qo = _pack(te)
    want = orc.dtw_matrix_var(qv, qo, tv, to, Weff).ravel()
    _close_or_inf(got, want)
    if W < hi - lo:
        assert np.isinf(want).any()   # the case has pairs without a warping path


# ------------------------------------------------------------------- search

def _labels(seed, n, k=4):
    return np.random.default_rng(seed).integers(0, k, n).astype(np.int32)


def _search(lib, tr, labels, te, W, V, flags=0, stats=False, max_len=None):
    import torch
    res = lib.nn_dtw_search_varlen(lib.ragged(tr), torch.from_numpy(labels).cuda(),
                                   lib.ragged(te), W, V, flags=flags, stats=stats,
                                   max_len=max_len)
    return (res.nn_idx.cpu().numpy(), res.nn_label.cpu().numpy(), res.nn_dist.cpu().numpy(),
            res.stats)


SEARCH_CASES = [(100, 160, 0, 5), (100, 160, 13, 1), (100, 160, 13, 5), (100, 160, 30, 5),
                (100, 160, 200, 5), (2, 9, 2, 2), (448, 576, 102, 5)]


@pytest.mark.parametrize("lo,hi,W,V", SEARCH_CASES)
def test_search_varlen_matches_oracle(lib, orc, lo, hi, W, V):
    tr = _series_set(lo + W + V, 300, lo, hi)
    # (the last query is 5 points longer than every training series: it has
    # no warping path inside windows below 5)
    te = _series_set(lo + W + V + 1, 80, lo, hi) + _series_set(lo + W + V + 2, 1, hi + 5, hi + 5)
    labels = _labels(lo + W, len(tr))
    ml = max(max(map(len, tr)), max(map(len, te)))
    tv, to = _pack(tr)
    qv, qo = _pack(te)
    bi, bl, bd = orc.nn_brute_var(tv, to, labels, qv, qo, min(W, ml - 1))
    for flags in (0, lib.NO_PRUNE, lib.KEOGH_BOUND, lib.NO_ABANDON, lib.EXACT_DIST):
        idx, lab, dist, _ = _search(lib, tr, labels, te, W, V, flags=flags)
        np.testing.assert_array_equal(idx, bi, err_msg=f"flags {flags}")
        np.testing.assert_array_equal(lab, bl, err_msg=f"flags {flags}")
        if flags == lib.EXACT_DIST:
            np.testing.assert_array_equal(dist, bd)
        else:
            _close_or_inf(dist, bd)
    assert (bi[-1] == -1) == (W < 5)


def test_search_varlen_equal_lengths_is_the_equal_length_search(lib):
    import torch
    xs = synth.random_series(71, 200, 128)
    qs = synth.random_series(72, 60, 128)
    labels = _labels(73, 200)
    for W, V in ((13, 5), (0, 1), (127, 3)):
        a = lib.nn_dtw_search(torch.from_numpy(xs).cuda(), torch.from_numpy(labels).cuda(),
                              torch.from_numpy(qs).cuda(), W, V, flags=lib.EXACT_DIST)
        b = _search(lib, list(xs), labels, list(qs), W, V, flags=lib.EXACT_DIST)
        np.testing.assert_array_equal(a.nn_idx.cpu().numpy(), b[0])
        np.testing.assert_array_equal(a.nn_label.cpu().numpy(), b[1])
        np.testing.assert_array_equal(a.nn_dist.cpu().numpy(), b[2])


def test_search_varlen_ties_and_recheck(lib, orc):
    """Exact duplicates at higher indices and queries that are training
    series: distances tie, the FP64 recheck runs without NNDTW_EXACT_DIST and
    the lowest index wins."""
    tr = _series_set(81, 120, 60, 90)
    tr = tr + [x.copy() for x in tr[:40]]
    te = [tr[k].copy() for k in range(0, 40, 3)] + _series_set(82, 20, 60, 90)
    labels = np.arange(len(tr), dtype=np.int32) % 7
    idx, lab, dist, st = _search(lib, tr, labels, te, 9, 4, stats=True)
    tv, to = _pack(tr)
    qv, qo = _pack(te)
    bi, bl, bd = orc.nn_brute_var(tv, to, labels, qv, qo, 9)
    np.testing.assert_array_equal(idx, bi)
    np.testing.assert_array_equal(lab, bl)
    assert np.all(idx < 120)
    assert st["rechecked"] > 0
    assert np.all(dist[:14] == 0.0)


def test_search_varlen_bad_lengths(lib):
    """A series whose length lies outside [2, max_len] matches nothing; with
    NNDTW_CHECK_FINITE the call reports it."""
    tr = _series_set(91, 30, 40, 60)
    tr[3] = tr[3][:1]                           # length 1
    te = _series_set(92, 10, 40, 60)
    te[2] = _series_set(93, 1, 75, 75)[0]       # longer than max_len below
    labels = _labels(94, len(tr))
    idx, lab, dist, _ = _search(lib, tr, labels, te, 20, 3, max_len=70)
    assert idx[2] == -1 and lab[2] == -1 and math.isinf(dist[2])
    assert not (idx == 3).any()
    with pytest.raises(lib.NnDtwError):
        _search(lib, tr, labels, te, 20, 3, flags=lib.CHECK_FINITE, max_len=70)


def test_search_varlen_chunks(lib, orc):
    """Q x N above one query chunk (NNDTW_CHUNK_PAIRS pairs): sampled queries
    against the oracle."""
    tr = _series_set(101, 20000, 8, 12)
    te = _series_set(102, 3500, 8, 12)
    labels = _labels(103, len(tr), 5)
    assert len(tr) * len(te) > (1 << 26)
    idx, lab, dist, _ = _search(lib, tr, labels, te, 2, 2)
    sample = np.random.default_rng(104).choice(len(te), 40, replace=False)
    tv, to = _pack(tr)
    qv, qo = _pack([te[k] for k in sample])
    bi, bl, bd = orc.nn_brute_var(tv, to, labels, qv, qo, 2)
    np.testing.assert_array_equal(idx[sample], bi)
    np.testing.assert_array_equal(lab[sample], bl)
    _close_or_inf(dist[sample], bd)


def test_search_varlen_full_workload_every_query(lib):
    """The unequal-length workload at full size (8,000 x 2,000, lengths
    448..576, W = 102): every query against the stored oracle results."""
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_full_golden as g
    rows = g.read(g.VARLEN_PATH)
    ds = synth.make_varlen()
    idx, lab, dist, st = _search(lib, ds.train, ds.train_labels, ds.test, ds.W, ds.V,
                                 stats=True)
    want = np.array([r[1] for r in rows]), np.array([r[2] for r in rows])
    wd = np.array([r[3] for r in rows])
    np.testing.assert_array_equal(idx, want[0])
    np.testing.assert_array_equal(lab, want[1])
    _close_or_inf(dist, wd)
    # (the compaction prunes against each query's first candidate, the
    # DTW kernel further against the live best)
    assert st["lb_pruned"] > 0.25 * st["pairs"]
    assert st["lb_pruned"] + st["lb_pruned_live"] > 0.5 * st["pairs"]


def test_search_varlen_host_buffers(lib, orc):
    """The host-buffer entry point (copies in, search, copies out) returns
    the device search's results."""
    tr = _series_set(111, 150, 40, 70)
    te = _series_set(112, 40, 40, 70)
    labels = _labels(113, len(tr))
    tv, to = _pack(tr)
    qv, qo = _pack(te)
    hs = lib.VarlenHostSearch(tv, to, labels, qv, qo, 12, 4, max_len=70)
    for _ in range(2):
        idx, lab, dist = hs()
        d_idx, d_lab, d_dist, _ = _search(lib, tr, labels, te, 12, 4, max_len=70)
        np.testing.assert_array_equal(idx, d_idx)
        np.testing.assert_array_equal(lab, d_lab)
        np.testing.assert_array_equal(dist, d_dist)
    bi, bl, _ = orc.nn_brute_var(tv, to, labels, qv, qo, 12)
    np.testing.assert_array_equal(idx, bi)
    np.testing.assert_array_equal(lab, bl)
    h2d, d2h = hs.bytes_per_call()
    assert h2d == tv.nbytes + to.nbytes + qv.nbytes + qo.nbytes + labels.nbytes
    assert d2h == len(te) * 16
