"""LB_Enhanced^V with the LB_Improved bridge (Sec. 5 with Sec. 2.2.4, Eq. 5)
through the C ABI, against the oracle: the second envelopes bit-exact, the
bound values within the FP32 tolerance (FP64: 1e-12), the safe values never
above the exact bound, and searches with the bound in the cascade giving
bit-identical neighbours."""
import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL32 = 1e-4


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _series(seed, n, L, dtype=np.float32):
    return synth.random_series(seed, n, L, dtype)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
@pytest.mark.parametrize("L,W", [(2, 0), (2, 1), (17, 3), (100, 13), (300, 33), (1024, 102),
                                 (1024, 1023), (4096, 409), (129, 5000), (8192, 700)])
def test_second_envelopes_bit_exact(lib, orc, dt, L, W):
    """(window max of Lo, window min of U), i.e. the oracle's envelope scan run
    on Lo and on U."""
    x = _series(L * 3 + W, 23, L, dt)
    env = lib.nn_dtw_build_envelopes(_t(x), W)
    env2 = lib.nn_dtw_build_second_envelopes(env, W).cpu().numpy()
    U, Lo = orc.envelopes(x, W)
    UoLo, _ = orc.envelopes(Lo, W)
    _, LoU = orc.envelopes(U, W)
    np.testing.assert_array_equal(env2[..., 0], UoLo.astype(dt))
    np.testing.assert_array_equal(env2[..., 1], LoU.astype(dt))


def _improved(lib, test, train, W, V, safe=False):
    env = lib.nn_dtw_build_envelopes(_t(train), W)
    tenv = lib.nn_dtw_build_envelopes(_t(test), W)
    env2 = lib.nn_dtw_build_second_envelopes(env, W)
    return lib.lb_enhanced_improved(_t(test), tenv, _t(train), env, env2, W, V,
                                    safe=safe).cpu().numpy()


CASES = [(256, 26, 5), (256, 26, 1), (100, 0, 3), (57, 56, 20), (200, 50, 64), (2, 1, 1),
         (3, 2, 1), (5, 2, 2), (1024, 102, 5), (130, 3, 7), (31, 30, 15), (600, 300, 4)]


@pytest.mark.parametrize("L,W,V", CASES)
def test_lb_improved_parity(lib, orc, L, W, V):
    test = _series(7000 + L, 37, L)
    train = _series(8000 + W, 70, L)
    lb = _improved(lib, test, train, W, V)
    safe = _improved(lib, test, train, W, V, safe=True)
    ref = orc.lb_matrix(test, train, W, V, "improved")
    np.testing.assert_allclose(lb, ref, rtol=RTOL32, atol=1e-6)
    assert np.all(safe.astype(np.float64) <= ref), "safe bound above the exact bound"
    assert np.all(safe <= lb)
    # never below LB_Enhanced, never above DTW
    enh = orc.lb_matrix(test, train, W, V, "enhanced")
    assert np.all(ref >= enh * (1 - 1e-12))
    if L <= 256:
        assert np.all(safe.astype(np.float64) <= orc.dtw_pairs(test, train, W))


@pytest.mark.parametrize("L,W,V", [(128, 13, 5), (33, 4, 16), (300, 299, 2), (64, 0, 2)])
def test_lb_improved_f64_parity(lib, orc, L, W, V):
    test = _series(9000 + L, 19, L, np.float64)
    train = _series(9500 + L, 65, L, np.float64)
    lb = _improved(lib, test, train, W, V)
    ref = orc.lb_matrix(test, train, W, V, "improved")
    np.testing.assert_allclose(lb, ref, rtol=1e-12, atol=1e-15)
    safe = _improved(lib, test, train, W, V, safe=True)
    assert np.all(safe <= ref)


def test_lb_enhanced_improved_rejects_lb_new_flag(lib):
    import ctypes
    L, W, V = 16, 2, 2
    x = _t(_series(1, 4, L))
    env = lib.nn_dtw_build_envelopes(x, W)
    env2 = lib.nn_dtw_build_second_envelopes(env, W)
    out = _t(np.zeros((4, 4), np.float32))
    raw = lib.load()
    rc = raw.lb_enhanced_improved(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(env.data_ptr()),
                                  4, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(env.data_ptr()),
                                  ctypes.c_void_p(env2.data_ptr()), 4, L, W, V, lib.LB_NEW,
                                  ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1   # NNDTW_EINVAL (NNDTW_LB_KEOGH selects LB_Improved itself)


def _search(lib, train, labels, test, W, V, flags):
    r = lib.nn_dtw_search(_t(train), _t(labels), _t(test), W, V, flags=flags, stats=True)
    return (r.nn_idx.cpu().numpy(), r.nn_label.cpu().numpy(), r.nn_dist.cpu().numpy(),
            r.stats)


def _expect(orc, train, labels, test, W, res, fp64):
    bi, bl, bd = orc.nn_brute(train, labels, test, W)
    idx, lab, dist, _ = res
    np.testing.assert_array_equal(idx, bi)
    np.testing.assert_array_equal(lab, bl)
    if fp64:
        np.testing.assert_array_equal(dist, bd)
    else:
        np.testing.assert_allclose(dist, bd, rtol=RTOL32, atol=0)


@pytest.mark.parametrize("fp64", [False, True])
def test_search_improved_bound(lib, orc, fp64):
    """The bound with the LB_Improved bridge drops survivors of LB_Enhanced
    without changing any result: every queue pair is dropped by it or has
    its DTW started."""
    ds = synth.make_pairs(5)
    dt = np.float64 if fp64 else np.float32
    train, labels = ds.train[:300].astype(dt), ds.train_labels[:300]
    test = ds.test[:150].astype(dt)
    base = lib.NO_REVERSE
    on = _search(lib, train, labels, test, ds.W, 5, base | lib.IMPROVED)
    off = _search(lib, train, labels, test, ds.W, 5, base)
    _expect(orc, train, labels, test, ds.W, on, fp64)
    _expect(orc, train, labels, test, ds.W, off, fp64)
    s_on, s_off = on[3], off[3]
    assert s_on["lb_pruned_improved"] > 0 and s_off["lb_pruned_improved"] == 0
    assert s_on["lb_pruned_reverse"] == 0
    assert s_on["lb_pruned"] == s_off["lb_pruned"]
    # every queued pair is dropped by the second stage, dropped unstarted by
    # its bound against the live best, or started
    assert (s_on["dtw_started"] + s_on["lb_pruned_live"] + s_on["lb_pruned_improved"]
            == s_off["dtw_started"] + s_off["lb_pruned_live"])


@pytest.mark.parametrize("fp64", [False, True])
def test_search_improved_with_reverse(lib, orc, fp64):
    """Both second-stage bounds at once: a pair is dropped by either, counted
    once, and nothing changes the neighbours."""
    ds = synth.make_pairs(5)
    dt = np.float64 if fp64 else np.float32
    train, labels = ds.train[:300].astype(dt), ds.train_labels[:300]
    test = ds.test[:150].astype(dt)
    both = _search(lib, train, labels, test, ds.W, 5, lib.IMPROVED | lib.REVERSE)
    off = _search(lib, train, labels, test, ds.W, 5, lib.NO_REVERSE)
    _expect(orc, train, labels, test, ds.W, both, fp64)
    s, s0 = both[3], off[3]
    dropped = s["lb_pruned_improved"] + s["lb_pruned_reverse"]
    assert s["lb_pruned_improved"] > 0
    assert (s["dtw_started"] + s["lb_pruned_live"] + dropped
            == s0["dtw_started"] + s0["lb_pruned_live"])


@pytest.mark.parametrize("L,W,V", [(160, 40, 4), (160, 159, 3), (96, 0, 2), (600, 60, 5),
                                   (1500, 150, 5)])
def test_search_improved_windows(lib, orc, L, W, V):
    """Narrow, full and zero windows, and long series, with the bound on."""
    rng = np.random.default_rng(L + W)
    N, Q = (300, 60) if L < 1000 else (120, 20)
    train = synth.znormed_walks(rng, N, L).astype(np.float32)
    test = synth.znormed_walks(rng, Q, L).astype(np.float32)
    labels = rng.integers(0, 4, N).astype(np.int32)
    res = _search(lib, train, labels, test, W, V, lib.IMPROVED)
    _expect(orc, train, labels, test, W, res, False)


def test_search_improved_leave_one_out(lib, orc):
    rng = np.random.default_rng(5)
    N, L, W = 120, 64, 6
    x = synth.znormed_walks(rng, N, L).astype(np.float32)
    x[N - 1] = x[0]
    lab = rng.integers(0, 3, N).astype(np.int32)
    ri, rl, _ = orc.nn_loo(x, lab, W)
    r = lib.nn_dtw_search(_t(x), _t(lab), _t(x), W, 3, flags=lib.LEAVE_ONE_OUT | lib.IMPROVED)
    np.testing.assert_array_equal(r.nn_idx.cpu().numpy(), ri)
    np.testing.assert_array_equal(r.nn_label.cpu().numpy(), rl)


def test_batched_with_improved(lib, orc):
    """The batched search with the bound asked for per dataset (descriptor
    flags) equals separate oracle searches."""
    import torch
    sets = []
    for k, (N, Q, L, W) in enumerate([(200, 50, 128, 13), (90, 30, 300, 299), (150, 40, 64, 0)]):
        rng = np.random.default_rng(100 + k)
        tr = synth.znormed_walks(rng, N, L).astype(np.float32)
        te = synth.znormed_walks(rng, Q, L).astype(np.float32)
        lb = rng.integers(0, 5, N).astype(np.int32)
        sets.append((tr, lb, te, W))
    descs = [dict(train=_t(tr), labels=_t(lb), test=_t(te), W=W, V=4, flags=lib.IMPROVED)
             for tr, lb, te, W in sets]
    out = lib.nn_dtw_search_batched(descs)
    torch.cuda.synchronize()
    for (tr, lb, te, W), r in zip(sets, out):
        bi, bl, _ = orc.nn_brute(tr, lb, te, W)
        np.testing.assert_array_equal(r.nn_idx.cpu().numpy(), bi)
        np.testing.assert_array_equal(r.nn_label.cpu().numpy(), bl)
