"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Tolerances: FP32 LB and DTW values within 1e-4 relative of the oracle (the
FP32 error bound of a sum of n non-negative terms is about n * 2^-24 in the
worst case and ~sqrt(n) * 2^-24 in practice); FP64 DTW and every FP64 search
result bit-identical; NN indices and labels bit-identical in every mode.
"""
import numpy as np
import pytest

from paper_1808_09617_gb300 import synth

pytestmark = pytest.mark.gpu

RTOL32 = 1e-4


def _t(x, dev="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev)


def _series(seed, n, L, dtype=np.float32):
    return synth.random_series(seed, n, L, dtype)


# ---------------------------------------------------------------- envelopes

ENV_CASES = [(2, 0), (2, 1), (3, 1), (5, 2), (17, 3), (100, 13), (256, 26), (300, 31),
             (300, 32), (300, 33), (129, 1), (24, 24), (1024, 102), (1024, 512), (1024, 1023),
             (1024, 5000), (4096, 409), (4096, 100), (4096, 4095), (33, 7), (8192, 819),
             (8192, 8191), (6000, 31), (5000, 2500)]


@pytest.mark.parametrize("L,W", ENV_CASES)
def test_envelopes_bit_exact(lib, orc, L, W):
    x = _series(L * 7 + W, 37, L)
    env = lib.nn_dtw_build_envelopes(_t(x), W).cpu().numpy()
    U, Lo = orc.envelopes(x, W)
    np.testing.assert_array_equal(env[..., 0], U.astype(np.float32))
    np.testing.assert_array_equal(env[..., 1], Lo.astype(np.float32))


@pytest.mark.parametrize("L,W", [(128, 13), (7, 3), (1000, 999), (8192, 100), (8192, 8191)])
def test_envelopes_f64_bit_exact(lib, orc, L, W):
    x = _series(L + W, 11, L, np.float64)
    env = lib.nn_dtw_build_envelopes(_t(x), W).cpu().numpy()
    U, Lo = orc.envelopes(x, W)
    np.testing.assert_array_equal(env[..., 0], U)
    np.testing.assert_array_equal(env[..., 1], Lo)


# ---------------------------------------------------------------- bounds

LB_CASES = [(256, 26, 1), (256, 26, 2), (256, 26, 5), (100, 0, 3), (57, 56, 20), (200, 50, 64),
            (2, 1, 1), (5, 2, 2), (1024, 102, 5), (130, 3, 7), (31, 30, 15), (8192, 819, 5)]


@pytest.mark.parametrize("L,W,V", LB_CASES)
def test_lb_enhanced_parity(lib, orc, L, W, V):
    test = _series(1000 + L, 37, L)
    train = _series(2000 + W, 70, L)
    env = lib.nn_dtw_build_envelopes(_t(train), W)
    lb = lib.lb_enhanced(_t(test), _t(train), env, W, V).cpu().numpy()
    safe = lib.lb_enhanced(_t(test), _t(train), env, W, V, safe=True).cpu().numpy()
    keo = lib.lb_enhanced(_t(test), _t(train), env, W, V, keogh=True).cpu().numpy()
    ref = orc.lb_matrix(test, train, W, V, "enhanced")
    refk = orc.lb_matrix(test, train, W, V, "keogh")
    np.testing.assert_allclose(lb, ref, rtol=RTOL32, atol=1e-6)
    np.testing.assert_allclose(keo, refk, rtol=RTOL32, atol=1e-6)
    assert np.all(safe.astype(np.float64) <= ref), "safe bound above the exact bound"
    assert np.all(safe <= lb)


@pytest.mark.parametrize("tile", [1, 2, 3])
@pytest.mark.parametrize("L,W,V", [(256, 26, 5), (77, 3, 2), (1000, 100, 8)])
def test_lb_every_tile_shape(lib, orc, L, W, V, tile):
    """Every tile shape of the bound pass (32 x 32, 64 x 64, 128 x 64) gives
    the oracle's bounds, ragged tiles included; the search with each tile
    shape gives the oracle's neighbours."""
    test = _series(1500 + L, 141, L)
    train = _series(1600 + W, 203, L)
    env = lib.nn_dtw_build_envelopes(_t(train), W)
    lb = lib.lb_enhanced(_t(test), _t(train), env, W, V, tile=tile).cpu().numpy()
    ref = orc.lb_matrix(test, train, W, V, "enhanced")
    np.testing.assert_allclose(lb, ref, rtol=RTOL32, atol=1e-6)
    keo = lib.lb_enhanced(_t(test), _t(train), env, W, V, keogh=True, tile=tile).cpu().numpy()
    np.testing.assert_allclose(keo, orc.lb_matrix(test, train, W, V, "keogh"), rtol=RTOL32,
                               atol=1e-6)
    labels = np.arange(train.shape[0], dtype=np.int32) % 5
    brute = orc.nn_brute(train, labels, test[:40], W)
    _check_search(lib, orc, train, labels, test[:40], W, V, flags=lib.LB_TILE(tile), brute=brute)


@pytest.mark.parametrize("L,W,V", [(128, 13, 5), (33, 4, 16), (300, 299, 2)])
def test_lb_enhanced_f64_parity(lib, orc, L, W, V):
    test = _series(3000 + L, 19, L, np.float64)
    train = _series(4000 + L, 65, L, np.float64)
    env = lib.nn_dtw_build_envelopes(_t(train), W)
    lb = lib.lb_enhanced(_t(test), _t(train), env, W, V).cpu().numpy()
    ref = orc.lb_matrix(test, train, W, V, "enhanced")
    np.testing.assert_allclose(lb, ref, rtol=1e-12, atol=1e-15)
    keo = lib.lb_enhanced(_t(test), _t(train), env, W, V, keogh=True).cpu().numpy()
    np.testing.assert_allclose(keo, orc.lb_matrix(test, train, W, V, "keogh"), rtol=1e-12,
                               atol=1e-15)


def test_lb_never_exceeds_dtw(lib, orc):
    L, W, V = 200, 20, 5
    test = _series(51, 16, L)
    train = _series(52, 40, L)
    env = lib.nn_dtw_build_envelopes(_t(train), W)
    safe = lib.lb_enhanced(_t(test), _t(train), env, W, V, safe=True).cpu().numpy()
    d = orc.dtw_pairs(test, train, W)
    assert np.all(safe <= d)


# ---------------------------------------------------------------- DTW values

# W spans every group width: G=1 (W<=31), 2 (32..63), 4, 8, 16, 32 (W<=1023)
DTW_CASES = [(2, 0), (2, 1), (3, 1), (3, 2), (40, 0), (40, 1), (64, 13), (256, 26), (256, 31),
             (256, 32), (256, 63), (300, 64), (300, 127), (600, 128), (600, 255), (1000, 256),
             (1024, 511), (1024, 512), (1024, 1023), (2048, 1023), (777, 776), (50, 49),
             (4096, 409), (129, 64), (128, 127), (2048, 1024), (2048, 2047), (1500, 1200),
             (4096, 4095)]


@pytest.mark.parametrize("L,W", DTW_CASES)
def test_dtw_parity(lib, orc, L, W):
    import torch
    nq, nt = 5, 9
    test = _series(5000 + L, nq, L)
    train = _series(6000 + W, nt, L)
    rng = np.random.default_rng(L * 31 + W)
    P = 23
    pairs = np.stack([rng.integers(0, nq, P), rng.integers(0, nt, P)], 1).astype(np.int32)
    pairs[0] = (0, 0)
    got = lib.dtw_windowed(_t(test), _t(train), _t(pairs), W).cpu().numpy()
    ref = orc.dtw_pairs(test, train, W, pairs=pairs)
    np.testing.assert_allclose(got, ref, rtol=RTOL32, atol=0)
    got64 = lib.dtw_windowed(_t(test.astype(np.float64)), _t(train.astype(np.float64)),
                             _t(pairs), W).cpu().numpy()
    np.testing.assert_array_equal(got64, ref)
    # identical series: distance exactly 0
    z = lib.dtw_windowed(_t(train), _t(train), _t(np.array([[1, 1]], np.int32)), W)
    assert float(z.cpu()[0]) == 0.0
    torch.cuda.synchronize()


# ---------------------------------------------------------------- search

def _search(lib, train, labels, test, W, V, **kw):
    r = lib.nn_dtw_search(_t(train), _t(labels), _t(test), W, V, **kw)
    return r.nn_idx.cpu().numpy(), r.nn_label.cpu().numpy(), r.nn_dist.cpu().numpy(), r.stats


def _check_search(lib, orc, train, labels, test, W, V, flags=0, brute=None):
    idx, lab, dist, st = _search(lib, train, labels, test, W, V, flags=flags, stats=True)
    bi, bl, bd = brute if brute is not None else orc.nn_brute(train, labels, test, W)
    np.testing.assert_array_equal(idx, bi)
    np.testing.assert_array_equal(lab, bl)
    if train.dtype == np.float64 or (flags & lib.EXACT_DIST):
        np.testing.assert_array_equal(dist, bd)
    else:
        np.testing.assert_allclose(dist, bd, rtol=RTOL32, atol=0)
    Q, N = test.shape[0], train.shape[0]
    assert st["pairs"] == Q * N
    assert 0 <= st["lb_pruned"] <= Q * N - Q
    assert st["dtw_started"] >= Q
    return st


def test_search_tiny_golden(lib, orc):
    import os
    ds = synth.make_tiny()
    rows = [l.split() for l in open(os.path.join(os.path.dirname(__file__), "golden",
                                                 "tiny_nn.txt")) if not l.startswith("#")]
    gi = np.array([int(r[1]) for r in rows], np.int32)
    gl = np.array([int(r[2]) for r in rows], np.int32)
    gd = np.array([float.fromhex(r[3]) for r in rows])
    # FP64 form on the FP64 data: everything bit-exact
    idx, lab, dist, _ = _search(lib, ds.train, ds.train_labels, ds.test, ds.W, ds.V)
    np.testing.assert_array_equal(idx, gi)
    np.testing.assert_array_equal(lab, gl)
    np.testing.assert_array_equal(dist, gd)


@pytest.mark.parametrize("V", [1, 2, 5])
def test_search_pairs_workload(lib, orc, V):
    ds = synth.make_pairs(V)
    brute = orc.nn_brute(ds.train, ds.train_labels, ds.test, ds.W)
    st = _check_search(lib, orc, ds.train, ds.train_labels, ds.test, ds.W, V, brute=brute)
    assert st["lb_pruned"] > 0
    _check_search(lib, orc, ds.train, ds.train_labels, ds.test, ds.W, V,
                  flags=lib.EXACT_DIST, brute=brute)


SEARCH_CASES = [
    # N, Q, L, W, V
    (1, 1, 16, 3, 2), (3, 100, 40, 5, 3), (70, 65, 2, 1, 1), (70, 65, 3, 0, 1),
    (130, 33, 64, 0, 5), (130, 33, 64, 63, 5), (130, 33, 64, 100, 5), (129, 67, 77, 7, 40), (150, 40, 300, 299, 5), (60, 25, 1500, 1499, 3), (90, 30, 33, 40, 2),
    (200, 50, 150, 40, 5), (100, 20, 300, 130, 8), (64, 10, 1024, 300, 5),
    (40, 8, 1024, 1023, 5), (257, 31, 101, 10, 4),
]


@pytest.mark.parametrize("N,Q,L,W,V", SEARCH_CASES)
def test_search_parity(lib, orc, N, Q, L, W, V):
    rng = np.random.default_rng(N * 1000 + Q * 10 + L)
    train = _series(7000 + N + L, N, L)
    test = _series(8000 + Q + W, Q, L)
    labels = rng.integers(0, 5, N).astype(np.int32)
    brute = orc.nn_brute(train, labels, test, W)
    _check_search(lib, orc, train, labels, test, W, V, brute=brute)
    _check_search(lib, orc, train.astype(np.float64), labels, test.astype(np.float64), W, V)


def test_search_ties_lowest_index(lib, orc):
    L, W, V = 60, 6, 3
    base = _series(9001, 40, L)
    train = np.concatenate([base, base[:20], base[5:15]], axis=0)  # exact duplicates later
    train = np.concatenate([train[30:40], train], axis=0)          # and some earlier
    labels = np.arange(train.shape[0], dtype=np.int32) % 7
    test = np.concatenate([_series(9002, 30, L), base[:10]], axis=0)  # some queries equal a series
    brute = orc.nn_brute(train, labels, test, W)
    st = _check_search(lib, orc, train, labels, test, W, V, brute=brute)
    # the queries equal to a duplicated series have two candidates at the same
    # FP32 distance: the FP64 recheck must have run for them
    assert st["rechecked"] >= 20 and st["recheck_queries"] >= 10
    _check_search(lib, orc, train, labels, test, W, V, flags=lib.EXACT_DIST, brute=brute)
    # all training series identical: every query's NN is index 0
    same = np.repeat(base[:1], 50, axis=0)
    idx, _, _, _ = _search(lib, same, labels[:50], test, W, V)
    assert np.all(idx == 0)


def test_search_near_ties_recheck_fires(lib, orc):
    """Planted near ties: each query has two training series whose DTW
    distances differ by far less than the FP32 rounding margin (one is the
    other with a few elements moved by one FP32 ulp).  Without EXACT_DIST the
    search must re-evaluate both in FP64 and return the oracle's index, which
    is the nudged copy for some queries and the original for others."""
    L, W, V = 200, 20, 4
    rng = np.random.default_rng(77)
    test = _series(9101, 24, L)
    train = [_series(9102, 150, L)]
    for q in range(test.shape[0]):
        near = (test[q] + 0.05 * rng.standard_normal(L)).astype(np.float32)
        nudged = near.copy()
        pos = rng.choice(L, 6, replace=False)
        direction = np.inf if q % 2 else -np.inf
        nudged[pos] = np.nextafter(nudged[pos], np.float32(direction))
        # the nudged copy first for half of the queries: the lower index is
        # not always the answer
        train.append(np.stack([nudged, near] if q % 3 == 0 else [near, nudged]))
    train = np.concatenate(train, axis=0)
    labels = (np.arange(train.shape[0]) % 5).astype(np.int32)
    brute = orc.nn_brute(train, labels, test, W)
    assert np.all(brute[0] >= 150)
    st = _check_search(lib, orc, train, labels, test, W, V, brute=brute)
    assert st["rechecked"] >= 2 * test.shape[0] - 4
    assert st["recheck_queries"] >= test.shape[0] - 2


def test_search_w0_bound_near_ties(lib, orc):
    """W = 0, where the search takes the bound from |a|^2 + |b|^2 - 2 a.b less
    its rounding margin: planted near ties (elements one FP32 ulp apart),
    also on series far from zero (offset 1000, where that form cancels most
    of its digits), still give the oracle's index, label and distance."""
    L, W, V = 300, 0, 5
    rng = np.random.default_rng(78)
    for offset in (0.0, 1000.0):
        test = (_series(9201, 20, L) + offset).astype(np.float32)
        train = [(_series(9202, 100, L) + offset).astype(np.float32)]
        for q in range(test.shape[0]):
            near = (test[q] + 0.05 * rng.standard_normal(L)).astype(np.float32)
            nudged = near.copy()
            pos = rng.choice(L, 6, replace=False)
            nudged[pos] = np.nextafter(nudged[pos], np.float32(np.inf if q % 2 else -np.inf))
            train.append(np.stack([nudged, near] if q % 3 == 0 else [near, nudged]))
        train = np.concatenate(train, axis=0)
        labels = (np.arange(train.shape[0]) % 5).astype(np.int32)
        brute = orc.nn_brute(train, labels, test, W)
        assert np.all(brute[0] >= 100)
        _check_search(lib, orc, train, labels, test, W, V, brute=brute)
        _check_search(lib, orc, train, labels, test, W, V, flags=lib.EXACT_DIST, brute=brute)


@pytest.mark.parametrize("flag", ["NO_PRUNE", "NO_ABANDON", "EXACT_DIST", "CHECK_FINITE"])
def test_search_flags(lib, orc, flag):
    ds = synth.make_pairs(5)
    train, test = ds.train[:300], ds.test[:120]
    labels = ds.train_labels[:300]
    brute = orc.nn_brute(train, labels, test, ds.W)
    _check_search(lib, orc, train, labels, test, ds.W, 5, flags=getattr(lib, flag), brute=brute)


def test_search_rejects_nonfinite(lib):
    train = _series(11, 20, 32)
    train[3, 5] = np.inf
    test = _series(12, 4, 32)
    with pytest.raises(lib.NnDtwError) as e:
        _search(lib, train, np.zeros(20, np.int32), test, 3, 2, flags=lib.CHECK_FINITE)
    assert e.value.code == lib.ENONFINITE


def test_search_host_entry_matches(lib, orc):
    ds = synth.make_pairs(5)
    r = lib.nn_dtw_search_host(ds.train, ds.train_labels, ds.test, ds.W, 5, stats=True)
    idx, lab, dist, _ = _search(lib, ds.train, ds.train_labels, ds.test, ds.W, 5)
    np.testing.assert_array_equal(r.nn_idx, idx)
    np.testing.assert_array_equal(r.nn_label, lab)
    np.testing.assert_array_equal(r.nn_dist, dist)


def test_search_workspace_too_small(lib):
    import torch
    train = _t(_series(13, 10, 32))
    test = _t(_series(14, 3, 32))
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(lib.NnDtwError) as e:
        lib.nn_dtw_search(train, _t(np.zeros(10, np.int32)), test, 3, 2, workspace=ws)
    assert e.value.code == lib.ENOSPACE


@pytest.mark.parametrize("W_ratio", [0.1, 0.5, 1.0])
def test_search_precision_workload_every_query(lib, orc, W_ratio):
    """The full-size precision workload (10,000 x 2,000, L=1024, W = 102, 512
    and 1023) on the GPU: every query's index and label equal the oracle's
    stored results (tests/golden/make_full_golden.py), distances within
    1e-4, and the same with the cascade's second stage (LB_Improved bridge)."""
    from golden import make_full_golden as fg
    ds = synth.make_precision(W_ratio)
    rows = np.array(fg.read(fg.precision_path(W_ratio)), dtype=object)
    assert rows.shape[0] == ds.Q
    gi = rows[:, 1].astype(np.int32)
    gl = rows[:, 2].astype(np.int32)
    gd = rows[:, 3].astype(np.float64)
    for flags in (0, lib.IMPROVED):
        idx, lab, dist, st = _search(lib, ds.train, ds.train_labels, ds.test, ds.W, ds.V,
                                     flags=flags, stats=True)
        np.testing.assert_array_equal(idx, gi)
        np.testing.assert_array_equal(lab, gl)
        np.testing.assert_allclose(dist, gd, rtol=RTOL32, atol=0)


@pytest.mark.parametrize("L,W", [(300, 26), (257, 63), (600, 200), (1024, 511), (64, 3), (90, 89)])
def test_dtw_every_group_width_same_values(lib, orc, L, W):
    """Every admissible lanes-per-pair choice computes the same DTW values."""
    test = _series(777 + L, 6, L)
    train = _series(778 + W, 11, L)
    rng = np.random.default_rng(W)
    pairs = np.stack([rng.integers(0, 6, 40), rng.integers(0, 11, 40)], 1).astype(np.int32)
    ref = orc.dtw_pairs(test, train, W, pairs=pairs)
    for g in (1, 2, 4, 8, 16, 32, lib.ROWS_GROUP, lib.ROWS16_GROUP, lib.ROWS8_GROUP):
        got = lib.dtw_windowed(_t(test), _t(train), _t(pairs), W,
                               flags=lib.DTW_GROUP(g)).cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=RTOL32, atol=0, err_msg=f"G={g}")


@pytest.mark.parametrize("L", [1, 2, 5, 31, 32, 33, 64, 100, 1000, 2047, 2048, 2049, 2600, 3001,
                               4095, 4096, 4097, 6000, 8192])
def test_dtw_full_window_row_layout(lib, orc, L):
    """Full windows (W >= L-1) use the row layout by default; the diagonal layout
    (forced by a group width) must agree."""
    W = L - 1 if L > 1 else 0
    test = _series(900 + L, 4, L)
    train = _series(901 + L, 7, L)
    pairs = np.array([[q, t] for q in range(4) for t in range(7)], np.int32)
    ref = orc.dtw_pairs(test, train, W, pairs=pairs)
    got = lib.dtw_windowed(_t(test), _t(train), _t(pairs), W).cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=RTOL32, atol=0)
    big = lib.dtw_windowed(_t(test), _t(train), _t(pairs), W + 1000).cpu().numpy()
    np.testing.assert_array_equal(big, got)


@pytest.mark.parametrize("L", [1, 3, 4, 7, 8, 9, 16, 17, 100, 128, 129, 300, 512, 513, 1000, 1024])
def test_dtw_full_window_grouped_rows(lib, orc, L):
    """The row layout with 16 or 8 lanes per pair (L <= 64 G) gives the oracle's
    values; longer series fall back to the one-pair-per-warp kernel."""
    W = L - 1 if L > 1 else 0
    test = _series(1900 + L, 5, L)
    train = _series(1901 + L, 9, L)
    rng = np.random.default_rng(L)
    pairs = np.stack([rng.integers(0, 5, 70), rng.integers(0, 9, 70)], 1).astype(np.int32)
    ref = orc.dtw_pairs(test, train, W, pairs=pairs)
    for g in (lib.ROWS16_GROUP, lib.ROWS8_GROUP):
        got = lib.dtw_windowed(_t(test), _t(train), _t(pairs), W,
                               flags=lib.DTW_GROUP(g)).cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=RTOL32, atol=0, err_msg=f"G={g}")


@pytest.mark.parametrize("g", ["rows16", "rows8"])
@pytest.mark.parametrize("L,N,Q", [(200, 300, 120), (37, 500, 200), (500, 90, 40)])
def test_search_grouped_rows(lib, orc, g, L, N, Q):
    """Full-window searches with the grouped row layout (seeds, abandoning, best
    updates, ties) return the exhaustive FP64 nearest neighbours."""
    rng = np.random.default_rng(L + N)
    train = synth.znormed_walks(rng, N, L).astype(np.float32)
    test = synth.znormed_walks(rng, Q, L).astype(np.float32)
    test[:3] = train[:3]                       # exact matches, distance 0
    labels = rng.integers(0, 5, N).astype(np.int32)
    brute = orc.nn_brute(train, labels, test, L - 1)
    grp = lib.ROWS16_GROUP if g == "rows16" else lib.ROWS8_GROUP
    _check_search(lib, orc, train, labels, test, L - 1, 3, flags=lib.DTW_GROUP(grp), brute=brute)


@pytest.mark.parametrize("fp64", [False, True])
def test_search_reverse_bound(lib, orc, fp64):
    """The cascade's reverse bound drops survivors without changing any
    result: every queue pair is either dropped by it or has its DTW started,
    and with NNDTW_NO_REVERSE every one is started."""
    ds = synth.make_pairs(5)
    dt = np.float64 if fp64 else np.float32
    train, labels, test = ds.train[:300].astype(dt), ds.train_labels[:300], ds.test[:150].astype(dt)
    brute = orc.nn_brute(train, labels, test, ds.W)
    on = _check_search(lib, orc, train, labels, test, ds.W, 5, flags=lib.REVERSE, brute=brute)
    off = _check_search(lib, orc, train, labels, test, ds.W, 5, flags=lib.NO_REVERSE, brute=brute)
    assert on["lb_pruned_reverse"] > 0 and off["lb_pruned_reverse"] == 0
    assert on["lb_pruned"] == off["lb_pruned"]
    assert (on["dtw_started"] + on["lb_pruned_live"] + on["lb_pruned_reverse"]
            == off["dtw_started"] + off["lb_pruned_live"])


@pytest.mark.parametrize("g", [2, 8, 32, "rows", "rows16", "rows8"])
def test_search_reverse_bound_layouts(lib, orc, g):
    """The reverse bound in every DTW layout (diagonal groups, rows with 32, 16
    and 8 lanes) on a full-window search."""
    rng = np.random.default_rng(77)
    L, N, Q = 160, 400, 120
    train = synth.znormed_walks(rng, N, L).astype(np.float32)
    test = synth.znormed_walks(rng, Q, L).astype(np.float32)
    labels = rng.integers(0, 4, N).astype(np.int32)
    W = L - 1 if isinstance(g, str) else 40
    brute = orc.nn_brute(train, labels, test, W)
    grp = {"rows": lib.ROWS_GROUP, "rows16": lib.ROWS16_GROUP, "rows8": lib.ROWS8_GROUP}.get(g, g)
    on = _check_search(lib, orc, train, labels, test, W, 4, flags=lib.DTW_GROUP(grp) | lib.REVERSE,
                       brute=brute)
    off = _check_search(lib, orc, train, labels, test, W, 4, flags=lib.DTW_GROUP(grp) | lib.NO_REVERSE,
                        brute=brute)
    assert on["lb_pruned_reverse"] > 0 and off["lb_pruned_reverse"] == 0
    assert (on["dtw_started"] + on["lb_pruned_live"] + on["lb_pruned_reverse"]
            == off["dtw_started"] + off["lb_pruned_live"])


def test_search_reverse_bound_defaults(lib, orc):
    """The FP64 form tests the reverse bound by default, the FP32 form only
    when asked (NNDTW_REVERSE)."""
    rng = np.random.default_rng(78)
    L, N, Q = 200, 300, 80
    train = synth.znormed_walks(rng, N, L)
    test = synth.znormed_walks(rng, Q, L)
    labels = rng.integers(0, 4, N).astype(np.int32)
    brute = orc.nn_brute(train, labels, test, 30)
    f64 = _check_search(lib, orc, train, labels, test, 30, 4, brute=brute)
    f32 = _check_search(lib, orc, train.astype(np.float32), labels, test.astype(np.float32), 30, 4)
    assert f64["lb_pruned_reverse"] > 0 and f32["lb_pruned_reverse"] == 0


@pytest.mark.parametrize("L,N,Q", [(3000, 40, 12), (4096, 20, 6), (8192, 8, 3)])
def test_search_long_full_window(lib, orc, L, N, Q):
    """Full windows of series longer than 2048 (a CTA per pair in the row
    layout; the FP64 recheck of the tie on FP32 series staged as FP32): the
    exhaustive FP64 nearest neighbours, ties included."""
    rng = np.random.default_rng(L)
    train = synth.znormed_walks(rng, N, L).astype(np.float32)
    test = synth.znormed_walks(rng, Q, L).astype(np.float32)
    test[0] = train[5]
    labels = rng.integers(0, 3, N).astype(np.int32)
    _check_search(lib, orc, train, labels, test, L - 1, 4)


@pytest.mark.parametrize("L,W,N,Q,improved", [(8192, 8191, 6, 2, False), (6000, 600, 10, 3, False),
                                               (8192, 5000, 5, 2, False), (6000, 600, 10, 3, True),
                                               (8192, 8191, 6, 2, True)])
def test_search_f64_long_series(lib, orc, L, W, N, Q, improved):
    """The FP64 form on series up to 8192: the FP64 kernel reads the series
    from global memory when the two series and the band do not fit in shared
    memory (L = 8192, W = 8191); results bit-identical to the oracle."""
    rng = np.random.default_rng(L + W)
    train = synth.znormed_walks(rng, N, L)
    test = synth.znormed_walks(rng, Q, L)
    test[0] = train[N - 1]
    labels = rng.integers(0, 3, N).astype(np.int32)
    _check_search(lib, orc, train, labels, test, W, 3, flags=lib.IMPROVED if improved else 0)
    if improved:   # and the FP32 form on the same series
        _check_search(lib, orc, train.astype(np.float32), labels, test.astype(np.float32), W, 3,
                      flags=lib.IMPROVED | lib.REVERSE)


@pytest.mark.parametrize("g", [1, 2, 4, 8])
def test_search_group_override(lib, orc, g):
    ds = synth.make_pairs(5)
    brute = orc.nn_brute(ds.train[:200], ds.train_labels[:200], ds.test[:100], ds.W)
    _check_search(lib, orc, ds.train[:200], ds.train_labels[:200], ds.test[:100], ds.W, 5,
                  flags=lib.DTW_GROUP(g), brute=brute)


@pytest.mark.parametrize("N,Q,L,W", [(12, 5, 2048, 1500), (9, 4, 1100, 1099), (7, 3, 2048, 1024),
                                     (5, 2, 8192, 5000), (6, 3, 6000, 1023)])
def test_search_wide_windows(lib, orc, N, Q, L, W):
    """Windows beyond the register kernel (W >= 1024) use the shared-memory band kernel."""
    train = _series(31 + L, N, L)
    test = _series(32 + W, Q, L)
    labels = np.arange(N, dtype=np.int32) % 3
    brute = orc.nn_brute(train, labels, test, W)
    _check_search(lib, orc, train, labels, test, W, 5, brute=brute)
    _check_search(lib, orc, train, labels, test, W, 5, flags=lib.EXACT_DIST, brute=brute)


@pytest.mark.parametrize("fp64", [False, True])
def test_search_keogh_bound(lib, orc, fp64):
    """LB_Keogh as the pruning bound (the baseline of the paper's V study):
    the same neighbours, and never more pruning than LB_Enhanced^1, which is
    at least LB_Keogh for every pair (same first candidates, same upper
    bounds)."""
    ds = synth.make_pairs(5)
    dt = np.float64 if fp64 else np.float32
    train, labels, test = ds.train[:300].astype(dt), ds.train_labels[:300], ds.test[:120].astype(dt)
    brute = orc.nn_brute(train, labels, test, ds.W)
    k = _check_search(lib, orc, train, labels, test, ds.W, 1,
                      flags=lib.KEOGH_BOUND | lib.REVERSE | lib.IMPROVED, brute=brute)
    e = _check_search(lib, orc, train, labels, test, ds.W, 1, flags=lib.NO_REVERSE, brute=brute)
    assert k["lb_pruned_reverse"] == 0 and k["lb_pruned_improved"] == 0
    assert 0 < k["lb_pruned"] <= e["lb_pruned"]


def test_binding_rejects_mismatched_shapes(lib):
    """The binding checks every device buffer's shape against the sizes it
    passes, so that no kernel reads or writes past a caller's tensor."""
    L, W = 32, 3
    train = _t(_series(1, 10, L))
    test = _t(_series(2, 4, L))
    labels = _t(np.zeros(10, np.int32))
    env = lib.nn_dtw_build_envelopes(train, W)
    with pytest.raises(ValueError, match="env"):
        lib.lb_enhanced(test, train, env[:9], W, 2)
    with pytest.raises(ValueError, match="train"):
        lib.lb_enhanced(test, _t(_series(3, 10, L + 1)), env, W, 2)
    with pytest.raises(ValueError, match="labels"):
        lib.nn_dtw_search(train, _t(np.zeros(9, np.int32)), test, W, 2)
    with pytest.raises(ValueError, match="env"):
        lib.nn_dtw_search(train, labels, test, W, 2, env=env[:, :16].contiguous())
    with pytest.raises(ValueError, match="pairs"):
        lib.dtw_windowed(test, train, _t(np.zeros((5, 3), np.int32)), W)
    with pytest.raises(ValueError, match="test_env"):
        env2 = lib.nn_dtw_build_second_envelopes(env, W)
        lib.lb_enhanced_improved(test, env, train, env, env2, W, 2)
