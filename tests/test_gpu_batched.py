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


def test_batched_matches_oracle_on_samples(lib, orc, batch):
    dsets, sets = batch
    res = lib.nn_dtw_search_batched(sets)
    rng = np.random.default_rng(64)
    for d, r in zip(dsets, res):
        idx, lab, dist = _np(r)
        k = min(2, d.Q)
        sample = np.sort(rng.choice(d.Q, k, replace=False))
        ri, rl, rd, _ = orc.nn_pruned(d.train, d.train_labels, d.test[sample], d.W, d.V)
        np.testing.assert_array_equal(idx[sample], ri, err_msg=d.name)
        np.testing.assert_array_equal(lab[sample], rl, err_msg=d.name)
        np.testing.assert_allclose(dist[sample], rd, rtol=1e-4, atol=0, err_msg=d.name)


def test_batched_rejects_bad_descriptors(lib, batch):
    _, sets = batch
    bad = [dict(sets[0]), dict(sets[1])]
    bad[1]["V"] = 0
    with pytest.raises(lib.NnDtwError) as e:
        lib.nn_dtw_search_batched(bad)
    assert e.value.code == lib.EINVAL
