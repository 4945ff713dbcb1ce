"""Batched search over the 64 heterogeneous datasets of the batching workload
(L 24..2048, N 16..8000, W 0..L, V 1..8): equal to separate searches, equal
when replayed from a CUDA graph, and equal to the FP64 oracle on sampled
queries of every dataset."""
import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


@pytest.fixture(scope="module")
def batch():
    dsets = synth.make_batched(64)
    sets = [dict(train=_t(d.train), labels=_t(d.train_labels), test=_t(d.test), W=d.W, V=d.V)
            for d in dsets]
    return dsets, sets


def _np(r):
    return r.nn_idx.cpu().numpy(), r.nn_label.cpu().numpy(), r.nn_dist.cpu().numpy()


def test_batched_equals_separate_searches(lib, batch):
    dsets, sets = batch
    res = lib.nn_dtw_search_batched(sets)
    for d, s, r in zip(dsets, sets, res):
        single = lib.nn_dtw_search(s["train"], s["labels"], s["test"], s["W"], s["V"])
        for a, b in zip(_np(r), _np(single)):
            np.testing.assert_array_equal(a, b, err_msg=d.name)


def test_batched_graph_replay(lib, batch):
    dsets, sets = batch
    bs = lib.BatchedSearch(sets, graph=True)
    first = [_np(r) for r in bs.run()]
    second = [_np(r) for r in bs.run()]
    eager = [_np(r) for r in lib.nn_dtw_search_batched(sets)]
    for x, y, z in zip(first, second, eager):
        for a, b, c in zip(x, y, z):
            np.testing.assert_array_equal(a, b)
            np.testing.assert_array_equal(a, c)


@pytest.fixture(scope="module")
def golden_batched():
    """The oracle's 1-NN of every query of the 64 datasets, stored by
    tests/golden/make_full_golden.py: {dataset: (idx, label, dist)}."""
    from golden import make_full_golden as fg
    rows = fg.read(fg.BATCHED_PATH)
    out = {}
    for d in sorted({r[0] for r in rows}):
        rs = [r for r in rows if r[0] == d]
        out[d] = (np.array([r[2] for r in rs], np.int32), np.array([r[3] for r in rs], np.int32),
                  np.array([r[4] for r in rs], np.float64))
    return out


def _check_every_query(dsets, results, golden):
    assert len(golden) == len(dsets)
    for k, (d, r) in enumerate(zip(dsets, results)):
        idx, lab, dist = r
        gi, gl, gd = golden[k]
        assert gi.shape[0] == d.Q, d.name
        np.testing.assert_array_equal(idx, gi, err_msg=d.name)
        np.testing.assert_array_equal(lab, gl, err_msg=d.name)
        np.testing.assert_allclose(dist, gd, rtol=1e-4, atol=0, err_msg=d.name)


def test_batched_matches_oracle_every_query(lib, batch, golden_batched):
    """All 35,843 queries of the 64 datasets, in one batched call and in the
    CUDA-graph replay the bench times, against the oracle's stored results."""
    dsets, sets = batch
    _check_every_query(dsets, [_np(r) for r in lib.nn_dtw_search_batched(sets)], golden_batched)
    bs = lib.BatchedSearch(sets, graph=True)
    bs.run()
    _check_every_query(dsets, [_np(r) for r in bs.run()], golden_batched)


def test_batched_other_flags_match_oracle(lib, batch, golden_batched):
    """Every dataset with search flags the bench's tuner may choose (the
    cascade's second stage and every admissible DTW layout, dealt out in
    turn): still the oracle's results for every query."""
    from paper_1808_09617_gb300 import autotune
    dsets, sets = batch
    cascade = (0, lib.REVERSE, lib.IMPROVED, lib.REVERSE | lib.IMPROVED)
    other = []
    for k, (d, s) in enumerate(zip(dsets, sets)):
        groups = autotune.admissible_groups(min(d.W, d.L - 1), d.L)
        g = groups[(k // 4) % len(groups)] if groups else 0
        t = dict(s)
        t["flags"] = cascade[k % 4] | (lib.DTW_GROUP(g) if g else 0)
        other.append(t)
    _check_every_query(dsets, [_np(r) for r in lib.nn_dtw_search_batched(other)],
                       golden_batched)


def test_batched_order_and_groups_of_64(lib, batch, golden_batched):
    """The datasets in another order and more than 64 of them (the 64 in
    reverse, then the first 16 again: two groups of at most 64, and every
    stage reorders its datasets by their cost): each dataset's results are
    still the oracle's."""
    dsets, sets = batch
    order = list(range(63, -1, -1)) + list(range(16))
    res = lib.nn_dtw_search_batched([sets[k] for k in order])
    assert len(res) == len(order)
    for k, r in zip(order, res):
        _check_every_query([dsets[k]], [_np(r)], {0: golden_batched[k]})


def test_batched_rejects_bad_descriptors(lib, batch):
    _, sets = batch
    bad = [dict(sets[0]), dict(sets[1])]
    bad[1]["V"] = 0
    with pytest.raises(lib.NnDtwError) as e:
        lib.nn_dtw_search_batched(bad)
    assert e.value.code == lib.EINVAL
