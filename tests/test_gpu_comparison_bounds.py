"""The paper's comparison bounds on the GPU against the FP64 oracle:
LB_Improved (Sec. 2.2.4, Eq. 5) and LB_New (Sec. 2.2.5), every pair of a
query set against a training set, FP32 within 1e-4 and FP64 within 1e-12;
rounding-safe values never above the exact bound; both never above DTW."""
import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL32 = 1e-4
CASES = [(256, 26), (2, 0), (2, 1), (3, 1), (100, 0), (57, 56), (200, 50), (130, 3),
         (31, 30), (1024, 102), (700, 2000), (8192, 40)]


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda")


def _improved(lib, test, train, W, safe=False):
    te, tr = _t(test), _t(train)
    env = lib.nn_dtw_build_envelopes(tr, W)
    tenv = lib.nn_dtw_build_envelopes(te, W)
    env2 = lib.nn_dtw_build_second_envelopes(env, W)
    return lib.lb_improved(te, tenv, tr, env, env2, W, safe=safe).cpu().numpy()


@pytest.mark.parametrize("L,W", CASES)
def test_lb_improved_parity(lib, orc, L, W):
    test = synth.random_series(6100 + L, 33, L)
    train = synth.random_series(6200 + W, 70, L)
    got = _improved(lib, test, train, W)
    safe = _improved(lib, test, train, W, safe=True)
    ref = orc.lb_matrix(test, train, W, 1, "lb_improved")
    np.testing.assert_allclose(got, ref, rtol=RTOL32, atol=1e-6)
    assert np.all(safe.astype(np.float64) <= ref)
    # never below LB_Keogh (its first pass)
    env = lib.nn_dtw_build_envelopes(_t(train), W)
    keo = lib.lb_enhanced(_t(test), _t(train), env, W, 1, keogh=True).cpu().numpy()
    assert np.all(got >= keo * (1 - 1e-6))


@pytest.mark.parametrize("L,W", CASES)
def test_lb_new_parity(lib, orc, L, W):
    test = synth.random_series(6300 + L, 33, L)
    train = synth.random_series(6400 + W, 70, L)
    got = lib.lb_new(_t(test), _t(train), W).cpu().numpy()
    safe = lib.lb_new(_t(test), _t(train), W, safe=True).cpu().numpy()
    ref = orc.lb_matrix(test, train, W, 1, "new")
    np.testing.assert_allclose(got, ref, rtol=RTOL32, atol=1e-6)
    assert np.all(safe.astype(np.float64) <= ref)


@pytest.mark.parametrize("L,W", [(128, 13), (33, 4), (300, 299), (2, 0)])
def test_comparison_bounds_f64(lib, orc, L, W):
    test = synth.random_series(6500 + L, 19, L, np.float64)
    train = synth.random_series(6600 + L, 41, L, np.float64)
    np.testing.assert_allclose(_improved(lib, test, train, W),
                               orc.lb_matrix(test, train, W, 1, "lb_improved"),
                               rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(lib.lb_new(_t(test), _t(train), W).cpu().numpy(),
                               orc.lb_matrix(test, train, W, 1, "new"), rtol=1e-12, atol=1e-15)


def test_comparison_bounds_never_exceed_dtw(lib, orc):
    L, W = 150, 15
    test = synth.random_series(6701, 16, L)
    train = synth.random_series(6702, 40, L)
    d = orc.dtw_pairs(test, train, W)
    assert np.all(_improved(lib, test, train, W, safe=True) <= d)
    assert np.all(lib.lb_new(_t(test), _t(train), W, safe=True).cpu().numpy() <= d)


def test_comparison_bound_flags_rejected(lib):
    import torch
    tr = _t(synth.random_series(6801, 5, 16))
    te = _t(synth.random_series(6802, 3, 16))
    env = lib.nn_dtw_build_envelopes(tr, 2)
    out = torch.empty((3, 5), dtype=torch.float32, device="cuda")
    lib_c = lib.load()
    import ctypes
    vp = ctypes.c_void_p
    rc = lib_c.lb_enhanced(vp(te.data_ptr()), 3, vp(tr.data_ptr()), vp(env.data_ptr()), 5, 16, 2,
                           1, lib.LB_NEW | lib.LB_KEOGH, vp(out.data_ptr()), None)
    assert rc == lib.EINVAL
