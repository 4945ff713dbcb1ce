"""Searches beyond the chunk size: Q x N above 2^31 (queries run in chunks
of NNDTW_CHUNK_PAIRS pairs over one bounded workspace), against the oracle's
stored results for sampled queries; leave-one-out across chunks against
brute force with the query removed; a chunked dataset inside a batch."""
import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL32 = 1e-4


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def test_search_above_2_31_pairs(lib):
    from golden import make_full_golden as fg
    train, labels, test, sample = fg.large_inputs()
    N, Q = train.shape[0], test.shape[0]
    assert N * Q > 2 ** 31
    ws_bytes = lib.nn_dtw_workspace_size(N, Q, fg.LARGE_L, fg.LARGE_W, fg.LARGE_V)
    # the workspace holds one chunk, not Q x N pairs
    assert ws_bytes < 64 * (1 << 26) + 64 * N * fg.LARGE_L
    r = lib.nn_dtw_search(_t(train), _t(labels), _t(test), fg.LARGE_W, fg.LARGE_V, stats=True)
    idx, lab, dist = r.nn_idx.cpu().numpy(), r.nn_label.cpu().numpy(), r.nn_dist.cpu().numpy()
    assert r.stats["pairs"] == N * Q
    rows = np.array(fg.read(fg.LARGE_PATH), dtype=object)
    q = rows[:, 0].astype(np.int64)
    assert np.array_equal(q, sample)
    np.testing.assert_array_equal(idx[q], rows[:, 1].astype(np.int32))
    np.testing.assert_array_equal(lab[q], rows[:, 2].astype(np.int32))
    np.testing.assert_allclose(dist[q], rows[:, 3].astype(np.float64), rtol=RTOL32, atol=0)
    # every query's neighbour is a valid training index
    assert idx.min() >= 0 and idx.max() < N


def test_leave_one_out_across_chunks(lib, orc):
    """Leave-one-out with N x N above the chunk size: queries of later chunks
    still never match themselves; sampled queries of the second chunk equal
    brute force over the training set with that series removed."""
    N, L, W, V = 9000, 12, 2, 2
    assert N * N > (1 << 26)
    train = synth.random_series(7201, N, L)
    labels = np.random.default_rng(7202).integers(0, 4, N).astype(np.int32)
    r = lib.nn_dtw_search(_t(train), _t(labels), _t(train), W, V, flags=lib.LEAVE_ONE_OUT)
    idx = r.nn_idx.cpu().numpy()
    dist = r.nn_dist.cpu().numpy()
    assert np.all(idx != np.arange(N))
    qc = (1 << 26) // N
    for i in (qc, qc + 1, N - 1, 3 * N // 4):
        keep = np.arange(N) != i
        bi, _, bd = orc.nn_brute(train[keep], labels[keep], train[i:i + 1], W)
        want = int(np.arange(N)[keep][bi[0]])
        assert idx[i] == want, i
        assert abs(dist[i] - bd[0]) <= RTOL32 * bd[0]


def test_batch_with_a_chunked_dataset(lib):
    """A batch with one dataset above the chunk size (its chunks run in
    successive rounds) gives the same results as separate searches."""
    big_tr = synth.random_series(7301, 20000, 16)
    big_te = synth.random_series(7302, 4000, 16)
    assert big_tr.shape[0] * big_te.shape[0] > (1 << 26)
    small_tr = synth.random_series(7303, 300, 40)
    small_te = synth.random_series(7304, 77, 40)
    rng = np.random.default_rng(7305)
    sets = [dict(train=_t(big_tr), labels=_t(rng.integers(0, 3, 20000).astype(np.int32)),
                 test=_t(big_te), W=1, V=2),
            dict(train=_t(small_tr), labels=_t(rng.integers(0, 3, 300).astype(np.int32)),
                 test=_t(small_te), W=4, V=3)]
    res = lib.nn_dtw_search_batched(sets)
    for s, r in zip(sets, res):
        one = lib.nn_dtw_search(s["train"], s["labels"], s["test"], s["W"], s["V"])
        np.testing.assert_array_equal(r.nn_idx.cpu().numpy(), one.nn_idx.cpu().numpy())
        np.testing.assert_array_equal(r.nn_dist.cpu().numpy(), one.nn_dist.cpu().numpy())
