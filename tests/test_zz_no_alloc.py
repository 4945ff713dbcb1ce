"""The allocation-free search entry point (nn_dtw_search_noalloc) against the
regular one (nn_dtw_search), through the C ABI.

nn_dtw_search_noalloc serves callers that cannot allocate device memory (for
instance next to another framework's caching allocator that owns the device
memory, or on a path that must not risk cudaMalloc's device synchronization):
its scratch is a fixed 16 MiB array inside the library, shared by all calls.
Two calls in a row on different inputs check that the second call is not
disturbed by what the first left in that array.  This file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL32 = 1e-4


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _np(r):
    return r.nn_idx.cpu().numpy(), r.nn_label.cpu().numpy(), r.nn_dist.cpu().numpy()


def _inputs():
    ds = synth.make_pairs(5)
    first = (ds.train, ds.train_labels, ds.test, ds.W, 5)
    rng = np.random.default_rng(4242)
    train2 = synth.random_series(4243, 300, 100)
    test2 = synth.random_series(4244, 77, 100)
    labels2 = rng.integers(0, 6, 300).astype(np.int32)
    second = (train2, labels2, test2, 9, 3)
    return first, second


def test_noalloc_matches_regular_search_on_two_calls_in_a_row(lib):
    first, second = _inputs()
    results = []
    for train, labels, test, W, V in (first, second):
        r = lib.nn_dtw_search_noalloc(_t(train), _t(labels), _t(test), W, V, stats=True)
        results.append((_np(r), r.stats))
    for (got, st), (train, labels, test, W, V) in zip(results, (first, second)):
        ref = lib.nn_dtw_search(_t(train), _t(labels), _t(test), W, V, stats=True)
        ri, rl, rd = _np(ref)
        gi, gl, gd = got
        np.testing.assert_array_equal(gi, ri)
        np.testing.assert_array_equal(gl, rl)
        np.testing.assert_allclose(gd, rd, rtol=RTOL32, atol=0)
        assert st["pairs"] == ref.stats["pairs"]
        assert st["lb_pruned"] == ref.stats["lb_pruned"]


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    train = _t(synth.random_series(4245, 4000, 256))
    test = _t(synth.random_series(4246, 2000, 256))
    labels = _t(np.zeros(4000, np.int32))
    assert lib.nn_dtw_workspace_size(4000, 2000, 256, 26, 5) > 16 << 20
    with pytest.raises(lib.NnDtwError) as e:
        lib.nn_dtw_search_noalloc(train, labels, test, 26, 5)
    assert e.value.code == lib.ENOSPACE
