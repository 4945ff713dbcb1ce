"""Leave-one-out search and window learning (Sec. 1 and Sec. 4: W is chosen
by leave-one-out 1-NN accuracy on the training set) against the oracle's
brute-force leave-one-out neighbours."""
import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _set(seed, N, L, dup=True):
    rng = np.random.default_rng(seed)
    x = synth.znormed_walks(rng, N, L)
    if dup:
        x[N - 1] = x[0]          # an exact duplicate: each finds the other at distance 0
        x[N - 2] = x[1]
    lab = rng.integers(0, 4, N).astype(np.int32)
    return x, lab


@pytest.mark.parametrize("fp64", [False, True])
@pytest.mark.parametrize("N,L,W,V", [(90, 64, 6, 3), (61, 150, 149, 5), (40, 33, 0, 1), (2, 20, 4, 2)])
def test_loo_search_matches_oracle(lib, orc, fp64, N, L, W, V):
    x, lab = _set(N + L, N, L, dup=N > 3)
    x = x if fp64 else x.astype(np.float32)
    ri, rl, rd = orc.nn_loo(x, lab, W)
    r = lib.nn_dtw_search(_t(x), _t(lab), _t(x), W, V, flags=lib.LEAVE_ONE_OUT, stats=True)
    idx, labr, dist = (r.nn_idx.cpu().numpy(), r.nn_label.cpu().numpy(), r.nn_dist.cpu().numpy())
    np.testing.assert_array_equal(idx, ri)
    np.testing.assert_array_equal(labr, rl)
    assert (idx != np.arange(N)).all()
    if fp64:
        np.testing.assert_array_equal(dist, rd)
    else:
        np.testing.assert_allclose(dist, rd, rtol=1e-4, atol=0)
    if N > 3:
        assert idx[0] == N - 1 and idx[N - 1] == 0 and dist[0] == 0.0


@pytest.mark.parametrize("extra", ["NO_PRUNE", "NO_ABANDON", "REVERSE"])
def test_loo_search_with_flags(lib, orc, extra):
    """Leave-one-out with the bound or the abandoning switched off, or the
    reverse bound on: the same neighbours, never the query itself."""
    x, lab = _set(5, 70, 48)
    x = x.astype(np.float32)
    ri, rl, rd = orc.nn_loo(x, lab, 9)
    r = lib.nn_dtw_search(_t(x), _t(lab), _t(x), 9, 3,
                          flags=lib.LEAVE_ONE_OUT | getattr(lib, extra))
    np.testing.assert_array_equal(r.nn_idx.cpu().numpy(), ri)
    np.testing.assert_array_equal(r.nn_label.cpu().numpy(), rl)


def test_loo_needs_a_square_set(lib):
    x, lab = _set(3, 20, 16)
    x = x.astype(np.float32)
    with pytest.raises(lib.NnDtwError):
        lib.nn_dtw_search(_t(x), _t(lab), _t(x[:10]), 3, 2, flags=lib.LEAVE_ONE_OUT)


@pytest.mark.parametrize("N,L,V", [(150, 96, 4), (64, 200, 2)])
def test_learn_window_matches_oracle(lib, orc, N, L, V):
    x, lab = _set(7 * N, N, L)
    # class shapes, so that accuracy depends on W
    rng = np.random.default_rng(N)
    lab = rng.integers(0, 3, N).astype(np.int32)
    for c in range(3):
        m = lab == c
        x[m] += np.sin(np.linspace(0, (2 + c) * np.pi, L))[None, :]
    x = x.astype(np.float32)
    windows = [0, 1, 2, L // 20, L // 10, L // 4, L - 1]
    correct = lib.nn_dtw_learn_window(_t(x), _t(lab), windows, V).cpu().numpy()
    ref = orc.loo_correct(x, lab, windows)
    np.testing.assert_array_equal(correct, ref)
    W, acc = lib.learn_window(_t(x), _t(lab), windows, V)
    best = max(range(len(windows)), key=lambda k: (ref[k], -windows[k]))
    assert W == windows[best]
    np.testing.assert_allclose(acc, ref / N)


def test_learn_window_equals_separate_loo_searches(lib):
    x, lab = _set(11, 120, 80)
    x = x.astype(np.float32)
    windows = [0, 4, 8, 79]
    correct = lib.nn_dtw_learn_window(_t(x), _t(lab), windows, 3).cpu().numpy()
    for k, W in enumerate(windows):
        r = lib.nn_dtw_search(_t(x), _t(lab), _t(x), W, 3, flags=lib.LEAVE_ONE_OUT)
        assert correct[k] == int((r.nn_label.cpu().numpy() == lab).sum())
