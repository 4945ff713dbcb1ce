"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each ``pin_*`` takes an ``oracle.Oracle`` and raises AssertionError on a
mismatch.  They are run against the real oracle (test_oracle_pins.py) and
against deliberately broken copies of it (test_oracle_mutants.py), which shows
that a plausible mistake anywhere in the oracle fails at least one of them.

None of the expected values below comes from the oracle's own recurrences:
they come from closed forms, exhaustive enumeration of warping paths,
explicit band sets, scipy's sliding-window filters, or inequalities that the
paper proves (Theorems 1 and 2).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.ndimage import maximum_filter1d, minimum_filter1d

from oracle import paths


def _rng(seed):
    return np.random.default_rng(seed)


def _rel_close(x, y, rtol):
    return abs(x - y) <= rtol * max(abs(x), abs(y), 1e-300)


def _series(rng, L):
    return rng.standard_normal(L)


# --------------------------------------------------------------------- DTW ---

def pin_dtw_w0_is_squared_euclidean(orc, trials=40):
    """DTW_0 is the (squared) Euclidean distance (Sec. 2.1)."""
    rng = _rng(1)
    for _ in range(trials):
        L = int(rng.integers(1, 80))
        a, b = _series(rng, L), _series(rng, L)
        exact = math.fsum((a - b) ** 2)
        got = orc.dtw(a, b, 0)
        assert _rel_close(got, exact, 1e-13), (L, got, exact)


def pin_dtw_equals_min_over_all_paths(orc, max_L=6):
    """DTW_W is the minimum cost over all warping paths inside the window
    (boundary, continuity and monotonicity constraints of Sec. 2.1)."""
    rng = _rng(2)
    for L in range(1, max_L + 1):
        for W in range(0, L + 1):
            for _ in range(3):
                a, b = _series(rng, L), _series(rng, L)
                exact = paths.dtw_by_paths(a, b, W)
                got = orc.dtw(a, b, W)
                assert _rel_close(got, exact, 1e-12), (L, W, got, exact)


def pin_dtw_symmetric_and_monotone(orc, trials=20):
    """DTW_W(A,B) = DTW_W(B,A); DTW_W is non-increasing in W; every W >= L-1
    gives the unconstrained DTW (Sec. 2.1)."""
    rng = _rng(3)
    for _ in range(trials):
        L = int(rng.integers(2, 40))
        a, b = _series(rng, L), _series(rng, L)
        vals = [orc.dtw(a, b, W) for W in range(0, L + 2)]
        for W in range(0, L + 2):
            assert orc.dtw(b, a, W) == vals[W]
        for W in range(1, L + 2):
            assert vals[W] <= vals[W - 1], (W, vals[W], vals[W - 1])
        assert vals[L - 1] == vals[L] == vals[L + 1] == orc.dtw(a, b, 10 * L)


def pin_dtw_early_abandon(orc, trials=30):
    """Early abandoning never changes a distance that is within the cutoff,
    and only ever answers +inf for distances above it."""
    rng = _rng(4)
    for _ in range(trials):
        L = int(rng.integers(2, 50))
        W = int(rng.integers(0, L))
        a, b = _series(rng, L), _series(rng, L)
        d = orc.dtw(a, b, W)
        assert orc.dtw(a, b, W, cutoff=d) == d
        assert orc.dtw(a, b, W, cutoff=d * 1.5) == d
        r = orc.dtw(a, b, W, cutoff=d * 0.5)
        assert r == d or math.isinf(r)


# -------------------------------------------------------------- envelopes ---

def pin_envelope_is_sliding_max_min(orc, trials=30):
    """U and Lo (Eq. 3-4) are the sliding max / min over the clipped window;
    scipy's filters with edge replication compute the same thing."""
    rng = _rng(5)
    for _ in range(trials):
        L = int(rng.integers(1, 120))
        W = int(rng.integers(0, L + 3))
        b = _series(rng, L)
        U, Lo = orc.envelope(b, W)
        size = 2 * W + 1
        np.testing.assert_array_equal(U, maximum_filter1d(b, size=size, mode="nearest"))
        np.testing.assert_array_equal(Lo, minimum_filter1d(b, size=size, mode="nearest"))
    b = _series(rng, 33)
    U, Lo = orc.envelope(b, 0)
    np.testing.assert_array_equal(U, b)
    np.testing.assert_array_equal(Lo, b)
    U, Lo = orc.envelope(b, 32)
    assert np.all(U == b.max()) and np.all(Lo == b.min())


# ---------------------------------------------------------------- LB_Keogh ---

def pin_lb_keogh(orc, trials=40):
    """LB_Keogh at W=0 is the Euclidean distance; LB_Keogh <= DTW_W."""
    rng = _rng(6)
    for _ in range(trials):
        L = int(rng.integers(2, 60))
        a, b = _series(rng, L), _series(rng, L)
        U, Lo = orc.envelope(b, 0)
        assert _rel_close(orc.lb_keogh(a, U, Lo), math.fsum((a - b) ** 2), 1e-13)
        W = int(rng.integers(0, L + 1))
        U, Lo = orc.envelope(b, W)
        assert orc.lb_keogh(a, U, Lo) <= orc.dtw(a, b, W) * (1 + 1e-12)


# ------------------------------------------------------------- LB_Enhanced ---

def pin_lb_enhanced_matches_band_sets(orc, max_L=12):
    """Algorithm 1 (with D = +inf) equals Eq. 7 summed from explicit band sets."""
    rng = _rng(7)
    for L in range(2, max_L + 1):
        for W in range(0, L + 1):
            for V in range(1, L // 2 + 1):
                a, b = _series(rng, L), _series(rng, L)
                U, Lo = orc.envelope(b, W)
                got = orc.lb_enhanced(a, b, U, Lo, W, V)
                exact = paths.lb_enhanced_by_sets(a, b, W, V)
                assert _rel_close(got, exact, 1e-12), (L, W, V, got, exact)


def pin_theorems_1_and_2(orc, trials=60):
    """Theorem 1 (left bands), its right-band analogue and Theorem 2
    (LB_Enhanced^V <= the proof's intermediate sum <= DTW_W)."""
    rng = _rng(8)
    for _ in range(trials):
        L = int(rng.integers(2, 14))
        W = int(rng.integers(0, L + 1))
        V = int(rng.integers(1, L // 2 + 1))
        a, b = _series(rng, L), _series(rng, L)
        d = orc.dtw(a, b, W)
        tol = 1 + 1e-12
        assert paths.full_left_band_bound(a, b, W) <= d * tol
        assert paths.full_right_band_bound(a, b, W) <= d * tol
        U, Lo = orc.envelope(b, W)
        lb = orc.lb_enhanced(a, b, U, Lo, W, V)
        mid = paths.theorem2_intermediate(a, b, W, V)
        assert lb <= mid * tol and mid <= d * tol, (L, W, V, lb, mid, d)


def pin_lb_enhanced_bounds_dtw_larger(orc, trials=40):
    """Theorem 2 on longer series, with LB_Keogh alongside; LB_Enhanced^1 is
    at least LB_Keogh (its first and last terms replace envelope distances
    by point distances of cells inside the envelope's window)."""
    rng = _rng(9)
    for _ in range(trials):
        L = int(rng.integers(16, 200))
        W = int(rng.integers(0, L))
        V = int(rng.integers(1, min(20, L // 2) + 1))
        a, b = _series(rng, L), _series(rng, L)
        U, Lo = orc.envelope(b, W)
        d = orc.dtw(a, b, W)
        lbe = orc.lb_enhanced(a, b, U, Lo, W, V)
        lbk = orc.lb_keogh(a, U, Lo)
        assert lbe <= d * (1 + 1e-12)
        assert orc.lb_enhanced(a, b, U, Lo, W, 1) >= lbk * (1 - 1e-12)


def pin_reverse_bound(orc, trials=40):
    """The cascade's reverse bound: LB_Enhanced^V(B, A), computed over A's
    envelope, bounds DTW_W(A, B) as well (DTW_W is symmetric); its two ends
    and its bands equal those of LB_Enhanced^V(A, B) (each band takes the
    minimum over the cells (i, j) and (j, i)), so the two bounds differ only
    in their LB_Keogh bridges over [n_b, L - n_b)."""
    rng = _rng(12)
    for _ in range(trials):
        L = int(rng.integers(4, 120))
        W = int(rng.integers(0, L))
        V = int(rng.integers(1, min(12, L // 2) + 1))
        a, b = _series(rng, L), _series(rng, L)
        Ub, Lb = orc.envelope(b, W)
        Ua, La = orc.envelope(a, W)
        ab = orc.lb_enhanced(a, b, Ub, Lb, W, V)
        ba = orc.lb_enhanced(b, a, Ua, La, W, V)
        d = orc.dtw(a, b, W)
        assert max(ab, ba) <= d * (1 + 1e-12), (L, W, V, ab, ba, d)
        nb = min(L // 2, V)
        mid = slice(nb, L - nb)
        bridge_ab = math.fsum((a[mid] - np.clip(a[mid], Lb[mid], Ub[mid])) ** 2)
        bridge_ba = math.fsum((b[mid] - np.clip(b[mid], La[mid], Ua[mid])) ** 2)
        assert abs((ab - bridge_ab) - (ba - bridge_ba)) <= 1e-12 * max(ab, ba, 1.0), (L, W, V)


def pin_lb_improved_bridge_bounds_dtw(orc, max_L=8):
    """LB_Enhanced^V with the LB_Improved bridge (Sec. 5, Sec. 2.2.4) never
    exceeds DTW_W, taken here as the minimum over every warping path, and never
    falls below LB_Enhanced^V; at W = 0 it is the Euclidean distance (B's
    envelope is B, so A' = B and the second pass adds nothing); with
    2 n_b = L (even L) its bridge is empty and it equals LB_Enhanced^V.  Integer-valued
    series give ties between cells and envelope values."""
    rng = _rng(13)
    tol = 1 + 1e-12
    for L in range(2, max_L + 1):
        for W in range(0, L + 1):
            for V in range(1, L // 2 + 1):
                for kind in range(2):
                    if kind:
                        a = rng.integers(-2, 3, L).astype(float)
                        b = rng.integers(-2, 3, L).astype(float)
                    else:
                        a, b = _series(rng, L), _series(rng, L)
                    U, Lo = orc.envelope(b, W)
                    lbi = orc.lb_enhanced_improved(a, b, U, Lo, W, V)
                    lbe = orc.lb_enhanced(a, b, U, Lo, W, V)
                    d = paths.dtw_by_paths(a, b, W)
                    assert lbe <= lbi * tol and lbi <= d * tol, (L, W, V, lbe, lbi, d)
                    if W == 0:
                        assert _rel_close(lbi, math.fsum((a - b) ** 2), 1e-13)
                    if 2 * min(L // 2, V) >= L:
                        assert lbi == lbe, (L, W, V)
                    assert orc.lb_enhanced_improved(a, a, *orc.envelope(a, W), W, V) == 0.0


def pin_lb_improved_bridge_closed_form(orc, trials=60):
    """The second pass of the LB_Improved bridge in closed form.  For |i - j|
    <= W the envelope of B satisfies Lo_i <= B_j <= U_i, so the projection A'
    (Eq. 5) exceeds B_j somewhere in j's window exactly when max(A_i, Lo_i)
    does, and otherwise its window maximum is max(U^A_j, max_i Lo_i), with
    U^A the envelope of A; the lower side mirrors this.  The term of B_j is
    therefore its distance to [min(L^A_j, min_i U_i), max(U^A_j, max_i Lo_i)]
    (window minima and maxima by scipy's filters), summed over the bridge
    n_b < j <= L - n_b."""
    rng = _rng(14)
    for _ in range(trials):
        L = int(rng.integers(2, 150))
        W = int(rng.integers(0, L + 2))
        V = int(rng.integers(1, max(1, min(10, L // 2)) + 1))
        a, b = _series(rng, L), _series(rng, L)
        size = 2 * W + 1
        f_max = lambda x: maximum_filter1d(x, size=size, mode="nearest")
        f_min = lambda x: minimum_filter1d(x, size=size, mode="nearest")
        Ub, Lb = f_max(b), f_min(b)
        Ua, La = f_max(a), f_min(a)
        hi = np.maximum(Ua, f_max(Lb))
        lo = np.minimum(La, f_min(Ub))
        nb = min(L // 2, V)
        mid = slice(nb, L - nb)
        second = math.fsum((b[mid] - np.clip(b[mid], lo[mid], hi[mid])) ** 2)
        U, Lo = orc.envelope(b, W)
        got = orc.lb_enhanced_improved(a, b, U, Lo, W, V) - orc.lb_enhanced(a, b, U, Lo, W, V)
        assert abs(got - second) <= 1e-12 * max(abs(second), 1.0), (L, W, V, got, second)


def pin_lb_improved_standalone(orc, max_L=8, trials=60):
    """LB_Improved (Sec. 2.2.4): never above DTW_W (minimum over every warping
    path), never below LB_Keogh, the Euclidean distance at W = 0 (A' = B), zero
    for A = B; and equal to LB_Keogh plus its second pass in closed form:
    B_j's distance to [min(L^A_j, min_i U_i), max(U^A_j, max_i Lo_i)] with
    window extremes from scipy's filters, summed over all of j = 1..L (the
    identity of the bridge pin above with an empty band set)."""
    rng = _rng(15)
    tol = 1 + 1e-12
    for L in range(1, max_L + 1):
        for W in range(0, L + 1):
            for kind in range(2):
                if kind:
                    a = rng.integers(-2, 3, L).astype(float)
                    b = rng.integers(-2, 3, L).astype(float)
                else:
                    a, b = _series(rng, L), _series(rng, L)
                U, Lo = orc.envelope(b, W)
                lbi = orc.lb_improved(a, b, U, Lo, W)
                d = paths.dtw_by_paths(a, b, W)
                assert orc.lb_keogh(a, U, Lo) <= lbi * tol and lbi <= d * tol, (L, W, lbi, d)
                if W == 0:
                    assert _rel_close(lbi, math.fsum((a - b) ** 2), 1e-13)
                assert orc.lb_improved(a, a, *orc.envelope(a, W), W) == 0.0
    for _ in range(trials):
        L = int(rng.integers(2, 150))
        W = int(rng.integers(0, L + 2))
        a, b = _series(rng, L), _series(rng, L)
        size = 2 * W + 1
        f_max = lambda x: maximum_filter1d(x, size=size, mode="nearest")
        f_min = lambda x: minimum_filter1d(x, size=size, mode="nearest")
        Ub, Lb = f_max(b), f_min(b)
        hi = np.maximum(f_max(a), f_max(Lb))
        lo = np.minimum(f_min(a), f_min(Ub))
        first = math.fsum((a - np.clip(a, Lb, Ub)) ** 2)
        second = math.fsum((b - np.clip(b, lo, hi)) ** 2)
        U, Lo = orc.envelope(b, W)
        got = orc.lb_improved(a, b, U, Lo, W)
        assert abs(got - (first + second)) <= 1e-12 * max(first + second, 1.0), (L, W)


def pin_lb_new(orc, max_L=8, trials=60):
    """LB_New (Sec. 2.2.5): never above DTW_W (every warping path), never below
    LB_Keogh nor LB_Enhanced^1 (its interior terms are distances to points of
    the window, the Keogh terms distances to the window's range), the
    Euclidean distance at W = 0, zero for A = B; with W >= L-1 every interior
    term is A_i's squared distance to the nearest value of all of B (a 1-D
    nearest-neighbour query on sorted B), and for any W the window minima by
    numpy's sliding windows."""
    rng = _rng(16)
    tol = 1 + 1e-12
    for L in range(2, max_L + 1):
        for W in range(0, L + 1):
            for kind in range(2):
                if kind:
                    a = rng.integers(-2, 3, L).astype(float)
                    b = rng.integers(-2, 3, L).astype(float)
                else:
                    a, b = _series(rng, L), _series(rng, L)
                U, Lo = orc.envelope(b, W)
                lbn = orc.lb_new(a, b, W)
                d = paths.dtw_by_paths(a, b, W)
                assert lbn <= d * tol, (L, W, lbn, d)
                assert orc.lb_keogh(a, U, Lo) <= lbn * tol
                assert orc.lb_enhanced(a, b, U, Lo, W, 1) <= lbn * tol
                if W == 0:
                    assert _rel_close(lbn, math.fsum((a - b) ** 2), 1e-13)
                assert orc.lb_new(a, a, W) == 0.0
    from numpy.lib.stride_tricks import sliding_window_view
    for _ in range(trials):
        L = int(rng.integers(2, 200))
        W = int(rng.integers(0, L + 2))
        a, b = _series(rng, L), _series(rng, L)
        ends = (a[0] - b[0]) ** 2 + (a[-1] - b[-1]) ** 2
        if W >= L - 1:
            sb = np.sort(b)
            k = np.clip(np.searchsorted(sb, a[1:-1]), 1, L - 1)
            near = np.minimum(np.abs(a[1:-1] - sb[k - 1]), np.abs(a[1:-1] - sb[k]))
        else:
            padded = np.concatenate([np.full(W, np.inf), b, np.full(W, np.inf)])
            win = sliding_window_view(padded, 2 * W + 1)[1:-1]
            near = np.min(np.abs(win - a[1:-1, None]), axis=1)
        exact = ends + math.fsum(near ** 2)
        got = orc.lb_new(a, b, W)
        assert _rel_close(got, exact, 1e-12), (L, W, got, exact)


def pin_lb_enhanced_w0_is_euclidean(orc, trials=30):
    """At W=0 every band is the single diagonal cell and U = Lo = B, so
    LB_Enhanced^V = DTW_0 = the Euclidean distance for every V."""
    rng = _rng(10)
    for _ in range(trials):
        L = int(rng.integers(2, 64))
        a, b = _series(rng, L), _series(rng, L)
        U, Lo = orc.envelope(b, 0)
        exact = math.fsum((a - b) ** 2)
        for V in (1, 2, max(1, L // 2)):
            assert _rel_close(orc.lb_enhanced(a, b, U, Lo, 0, V), exact, 1e-13)


def pin_algorithm1_abandon(orc, trials=30):
    """Algorithm 1 returns +inf exactly when the band sum reaches D."""
    rng = _rng(11)
    for _ in range(trials):
        L = int(rng.integers(4, 20))
        W = int(rng.integers(1, L))
        V = int(rng.integers(1, L // 2 + 1))
        a, b = _series(rng, L), _series(rng, L)
        U, Lo = orc.envelope(b, W)
        nb = min(L // 2, V)
        band = math.fsum([paths.band_min(a, b, paths.left_band(i, L, W)) for i in range(1, nb + 1)]
                         + [paths.band_min(a, b, paths.right_band(i, L, W))
                            for i in range(L - nb + 1, L + 1)])
        full = orc.lb_enhanced(a, b, U, Lo, W, V)
        assert math.isinf(orc.lb_enhanced(a, b, U, Lo, W, V, D=band * (1 - 1e-9)))
        assert orc.lb_enhanced(a, b, U, Lo, W, V, D=band * (1 + 1e-9)) == full
        assert math.isinf(orc.lb_enhanced(a, b, U, Lo, W, V, D=0.0))


# ------------------------------------------------------------------ 1-NN ---

def _small_set(seed, N, Q, L, classes=3):
    rng = _rng(seed)
    train = rng.standard_normal((N, L)).cumsum(axis=1)
    test = rng.standard_normal((Q, L)).cumsum(axis=1)
    labels = rng.integers(0, classes, N).astype(np.int32)
    return train, labels, test


def pin_nn_brute_by_paths(orc):
    """1-NN by the oracle equals the argmin (lowest index on ties) of the
    path-enumeration DTW on tiny series."""
    train, labels, test = _small_set(12, 7, 4, 5)
    for W in (0, 1, 2, 4):
        idx, lab, dist = orc.nn_brute(train, labels, test, W)
        for q in range(test.shape[0]):
            ds = [paths.dtw_by_paths(test[q], train[t], W) for t in range(train.shape[0])]
            best = int(np.argmin(ds))
            assert idx[q] == best and lab[q] == labels[best]
            assert _rel_close(dist[q], ds[best], 1e-12)


def pin_nn_w0_is_euclidean_nn(orc):
    """At W=0 the 1-NN is the Euclidean nearest neighbour."""
    train, labels, test = _small_set(13, 40, 10, 30)
    idx, _, _ = orc.nn_brute(train, labels, test, 0)
    for q in range(test.shape[0]):
        ed = [math.fsum((test[q] - t) ** 2) for t in train]
        assert idx[q] == int(np.argmin(ed))


def pin_nn_pruned_equals_brute(orc):
    """The paper's lower-bound search (Sec. 4) gives exactly the brute-force
    result, ties included: duplicated training series resolve to the lowest
    index in both."""
    train, labels, test = _small_set(14, 60, 12, 40)
    dup = np.concatenate([train, train[:20]], axis=0)   # exact duplicates at higher indices
    dlab = np.concatenate([labels, labels[:20]])
    front = np.concatenate([train[20:40], train], axis=0)  # duplicates at lower indices
    flab = np.concatenate([labels[20:40], labels])
    for tr, lb in ((train, labels), (dup, dlab), (front, flab)):
        for W in (0, 3, 8, 39):
            for V in (1, 2, 5):
                bi, bl, bd = orc.nn_brute(tr, lb, test, W)
                pi, pl, pd, _ = orc.nn_pruned(tr, lb, test, W, V)
                np.testing.assert_array_equal(bi, pi)
                np.testing.assert_array_equal(bl, pl)
                np.testing.assert_array_equal(bd, pd)
    # exact duplicate at a higher index never wins; at a lower index it always does
    bi, _, _ = orc.nn_brute(dup, dlab, test, 5)
    assert np.all(bi < 60)
    fi, _, _ = orc.nn_brute(front, flab, test, 5)
    assert not np.any((fi >= 40) & (fi < 60))
    # A tie that the Euclidean ordering visits in the "wrong" order: train 0 is
    # the query shifted by one step (DTW_1 = 0, ED = 2), train 1 is the query
    # itself (DTW = ED = 0).  Both are at distance 0, so index 0 must win,
    # although the search meets index 1 first.
    q = np.array([[0.0, 1.0, 0.0, 0.0]])
    tr = np.array([[0.0, 0.0, 1.0, 0.0], [0.0, 1.0, 0.0, 0.0], [3.0, 3.0, 3.0, 3.0]])
    lb = np.array([7, 8, 9], np.int32)
    for V in (1, 2):
        bi, bl, bd = orc.nn_brute(tr, lb, q, 1)
        pi, pl, pd, _ = orc.nn_pruned(tr, lb, q, 1, V)
        assert bi[0] == 0 and bl[0] == 7 and bd[0] == 0.0
        assert pi[0] == 0 and pl[0] == 7 and pd[0] == 0.0


def pin_nn_loo_equals_removal(orc):
    """Leave-one-out 1-NN (window learning): the neighbour of series q among
    the others is the brute-force neighbour in the set with q removed; exact
    duplicates find each other at distance 0."""
    rng = _rng(13)
    for trial in range(6):
        N, L = int(rng.integers(3, 12)), int(rng.integers(4, 30))
        W = int(rng.integers(0, L))
        tr = rng.standard_normal((N, L))
        if trial % 2:
            tr[N - 1] = tr[0]                       # a duplicate pair
        lab = rng.integers(0, 3, N).astype(np.int32)
        li, ll, ld = orc.nn_loo(tr, lab, W)
        for q in range(N):
            keep = np.array([t for t in range(N) if t != q])
            bi, bl, bd = orc.nn_brute(tr[keep], lab[keep], tr[q:q + 1], W)
            assert li[q] == keep[bi[0]] and ll[q] == bl[0] and ld[q] == bd[0], (trial, q)
        if trial % 2:
            assert li[0] == N - 1 and ld[0] == 0.0 and li[N - 1] == 0 and ld[N - 1] == 0.0
    # the counts of window learning follow from the neighbours' labels
    tr = rng.standard_normal((8, 16))
    lab = np.array([0, 0, 1, 1, 2, 2, 0, 1], np.int32)
    c = orc.loo_correct(tr, lab, [0, 3, 15])
    for k, W in enumerate([0, 3, 15]):
        assert c[k] == int((orc.nn_loo(tr, lab, W)[1] == lab).sum())


# -------------------------------------------------------- unequal lengths ---

def _lengths(rng, lo, hi):
    return int(rng.integers(lo, hi + 1)), int(rng.integers(lo, hi + 1))


def pin_dtw_var_equals_min_over_all_paths(orc, max_L=6):
    """DTW_W on an L_A x L_B grid is the minimum cost over every warping path
    from (1, 1) to (L_A, L_B) inside the window, +inf when none fits."""
    rng = _rng(31)
    for LA in range(1, max_L + 1):
        for LB in range(1, max_L + 1):
            for W in range(0, max(LA, LB) + 1):
                a, b = _series(rng, LA), _series(rng, LB)
                exact = paths.dtw_by_paths_var(a, b, W)
                got = orc.dtw_var(a, b, W)
                if math.isinf(exact):
                    assert math.isinf(got) and abs(LA - LB) > W, (LA, LB, W, got)
                else:
                    assert _rel_close(got, exact, 1e-12), (LA, LB, W, got, exact)


def pin_dtw_var_symmetric_and_reduces(orc, trials=30):
    """DTW_W(A, B) = DTW_W(B, A) bit for bit; with equal lengths it is the
    equal-length DTW; it is +inf exactly when |L_A - L_B| > W; every W at or
    above max(L_A, L_B) - 1 gives the same value; early abandoning only ever
    answers +inf above the cutoff."""
    rng = _rng(32)
    for _ in range(trials):
        LA, LB = _lengths(rng, 2, 40)
        a, b = _series(rng, LA), _series(rng, LB)
        for W in (0, abs(LA - LB), abs(LA - LB) + 3, max(LA, LB) - 1, 2 * max(LA, LB)):
            d = orc.dtw_var(a, b, W)
            assert orc.dtw_var(b, a, W) == d
            assert math.isinf(d) == (abs(LA - LB) > W)
            if not math.isinf(d):
                assert orc.dtw_var(a, b, W, cutoff=d) == d
                r = orc.dtw_var(a, b, W, cutoff=d * 0.5)
                assert r == d or math.isinf(r)
                # a cutoff below the first row's smallest cell abandons at once
                assert math.isinf(orc.dtw_var(a, b, W, cutoff=-1.0))
        assert orc.dtw_var(a, b, max(LA, LB) - 1) == orc.dtw_var(a, b, 10 * max(LA, LB))
        c = _series(rng, LA)
        for W in (0, 3, LA):
            assert orc.dtw_var(a, c, W) == orc.dtw(a, c, W)


def pin_envelope_var(orc, trials=30):
    """B's envelope for the rows of a longer or shorter series: rows up to
    L_B are scipy's sliding max / min, rows beyond L_B the max / min of B's
    tail from i-W on."""
    rng = _rng(33)
    for _ in range(trials):
        LB = int(rng.integers(1, 90))
        W = int(rng.integers(0, LB + 3))
        b = _series(rng, LB)
        U, Lo = orc.envelope_var(b, W)
        assert U.shape[0] == LB + W
        size = 2 * W + 1
        np.testing.assert_array_equal(U[:LB], maximum_filter1d(b, size=size, mode="nearest"))
        np.testing.assert_array_equal(Lo[:LB], minimum_filter1d(b, size=size, mode="nearest"))
        for i in range(LB + 1, LB + W + 1):
            tail = b[max(1, i - W) - 1:]
            assert U[i - 1] == tail.max() and Lo[i - 1] == tail.min(), (LB, W, i)
        U0, Lo0 = orc.envelope(b, W)
        np.testing.assert_array_equal(orc.envelope_var(b, W, E=LB)[0], U0)
        np.testing.assert_array_equal(orc.envelope_var(b, W, E=LB)[1], Lo0)


def pin_lb_enhanced_var_matches_band_sets(orc, max_L=10):
    """LB_Enhanced^V for unequal lengths equals its sum from explicit cell
    sets (start- and end-corner L-shapes inside the window, Keogh terms of
    the bridge rows), and is +inf with no path."""
    rng = _rng(34)
    for LA in range(2, max_L + 1):
        for LB in range(2, max_L + 1):
            for W in range(0, max(LA, LB) + 1):
                for V in (1, 2, 3, 5):
                    a, b = _series(rng, LA), _series(rng, LB)
                    got = orc.lb_enhanced_var(a, b, W, V)
                    exact = paths.lb_enhanced_by_sets_var(a, b, W, V)
                    if math.isinf(exact):
                        assert math.isinf(got), (LA, LB, W, V, got)
                    else:
                        assert _rel_close(got, exact, 1e-12), (LA, LB, W, V, got, exact)


def pin_lb_var_bounds_dtw(orc, trials=80):
    """The unequal-length bounds stay below DTW: LB_Enhanced^V <= the proof's
    intermediate sum (row minima over whole windows) <= DTW_W, checked by
    path enumeration on small grids and by the oracle's DTW on longer ones;
    LB_Keogh <= DTW_W; LB_Enhanced^1 >= LB_Keogh; Algorithm 1's abandon."""
    rng = _rng(35)
    for k in range(trials):
        small = k % 2 == 0
        LA, LB = _lengths(rng, 2, 7) if small else _lengths(rng, 8, 120)
        W = int(rng.integers(abs(LA - LB), max(LA, LB) + 1))
        V = int(rng.integers(1, min(LA, LB) // 2 + 2))
        a, b = _series(rng, LA), _series(rng, LB)
        d = paths.dtw_by_paths_var(a, b, W) if small else orc.dtw_var(a, b, W)
        tol = 1 + 1e-12
        lbe = orc.lb_enhanced_var(a, b, W, V)
        mid = paths.theorem2_intermediate_var(a, b, W, V)
        assert lbe <= mid * tol and mid <= d * tol, (LA, LB, W, V, lbe, mid, d)
        lbk = orc.lb_keogh_var(a, b, W)
        assert lbk <= d * tol
        assert orc.lb_enhanced_var(a, b, W, 1) >= lbk * (1 - 1e-12)
        assert math.isinf(orc.lb_enhanced_var(a, b, W, V, D=0.0))
        assert orc.lb_enhanced_var(a, b, W, V, D=lbe * 2 + 1) == lbe
    a, b = _series(rng, 10), _series(rng, 4)
    assert math.isinf(orc.lb_enhanced_var(a, b, 5, 2)) and math.isinf(orc.lb_keogh_var(a, b, 5))


def pin_lb_var_reduces_to_equal_length(orc, trials=30):
    """With L_A = L_B the unequal-length bounds are the equal-length ones,
    bit for bit."""
    rng = _rng(36)
    for _ in range(trials):
        L = int(rng.integers(2, 60))
        W = int(rng.integers(0, L + 2))
        V = int(rng.integers(1, L // 2 + 2))
        a, b = _series(rng, L), _series(rng, L)
        U, Lo = orc.envelope(b, W)
        assert orc.lb_enhanced_var(a, b, W, V) == orc.lb_enhanced(a, b, U, Lo, W, V)
        assert orc.lb_keogh_var(a, b, W) == orc.lb_keogh(a, U, Lo)


def _ragged_set(rng, n, lo, hi, dup_of=None):
    lens = rng.integers(lo, hi + 1, n)
    xs = [rng.standard_normal(int(m)).cumsum() for m in lens]
    return xs


def _pack(xs):
    off = np.zeros(len(xs) + 1, np.int64)
    off[1:] = np.cumsum([len(x) for x in xs])
    return np.concatenate(xs), off


def pin_nn_var(orc):
    """1-NN over ragged sets: the brute force equals the argmin of the
    path-enumeration DTW on tiny series (index -1 and label -1 when no
    series fits the window), the lower-bound search equals the brute force
    (ties to the lowest index, duplicates included), and the matrix drivers
    equal the single-pair routines."""
    rng = _rng(37)
    tr = _ragged_set(rng, 8, 2, 6)
    te = _ragged_set(rng, 5, 2, 6)
    labels = rng.integers(0, 3, len(tr)).astype(np.int32)
    trv, tro = _pack(tr)
    tev, teo = _pack(te)
    for W in (0, 1, 2, 5):
        idx, lab, dist = orc.nn_brute_var(trv, tro, labels, tev, teo, W)
        for q in range(len(te)):
            ds = [paths.dtw_by_paths_var(te[q], tr[t], W) for t in range(len(tr))]
            if all(math.isinf(x) for x in ds):
                assert idx[q] == -1 and lab[q] == -1 and math.isinf(dist[q])
            else:
                best = int(np.argmin(ds))
                assert idx[q] == best and lab[q] == labels[best]
                assert _rel_close(dist[q], ds[best], 1e-12)
    assert (orc.nn_brute_var(trv, tro, labels, tev, teo, 0)[0] == -1).any()
    tr = _ragged_set(rng, 50, 20, 40)
    tr += [x.copy() for x in tr[:10]]                  # duplicates at higher indices
    te = _ragged_set(rng, 12, 18, 44)
    labels = rng.integers(0, 4, len(tr)).astype(np.int32)
    trv, tro = _pack(tr)
    tev, teo = _pack(te)
    for W in (0, 3, 12, 50):
        bi, bl, bd = orc.nn_brute_var(trv, tro, labels, tev, teo, W)
        for V in (1, 2, 5):
            pi, pl, pd, _ = orc.nn_pruned_var(trv, tro, labels, tev, teo, W, V)
            np.testing.assert_array_equal(bi, pi)
            np.testing.assert_array_equal(bl, pl)
            np.testing.assert_array_equal(bd, pd)
        assert np.all(bi < 50)
        dm = orc.dtw_matrix_var(tev, teo, trv, tro, W)
        lm = orc.lb_matrix_var(tev, teo, trv, tro, W, 3)
        km = orc.lb_matrix_var(tev, teo, trv, tro, W, 3, kind="keogh")
        for q in (0, 5, 11):
            for t in (0, 17, 59):
                assert dm[q, t] == orc.dtw_var(te[q], tr[t], W)
                assert lm[q, t] == orc.lb_enhanced_var(te[q], tr[t], W, 3)
                assert km[q, t] == orc.lb_keogh_var(te[q], tr[t], W)
    # integer-valued series: exact distance ties are common, and the search
    # meets them in bound order, not index order
    tr = [rng.integers(0, 3, int(m)).astype(float) for m in rng.integers(3, 7, 60)]
    te = [rng.integers(0, 3, int(m)).astype(float) for m in rng.integers(3, 7, 30)]
    labels = np.arange(len(tr), dtype=np.int32)
    trv, tro = _pack(tr)
    tev, teo = _pack(te)
    for W in (1, 2, 4):
        bi, _, bd = orc.nn_brute_var(trv, tro, labels, tev, teo, W)
        for V in (1, 2):
            pi, _, pd, _ = orc.nn_pruned_var(trv, tro, labels, tev, teo, W, V)
            np.testing.assert_array_equal(bi, pi)
            np.testing.assert_array_equal(bd, pd)


ALL_PINS = [
    pin_dtw_w0_is_squared_euclidean,
    pin_dtw_equals_min_over_all_paths,
    pin_dtw_symmetric_and_monotone,
    pin_dtw_early_abandon,
    pin_envelope_is_sliding_max_min,
    pin_lb_keogh,
    pin_lb_enhanced_matches_band_sets,
    pin_theorems_1_and_2,
    pin_lb_enhanced_bounds_dtw_larger,
    pin_lb_enhanced_w0_is_euclidean,
    pin_reverse_bound,
    pin_lb_improved_bridge_bounds_dtw,
    pin_lb_improved_bridge_closed_form,
    pin_lb_improved_standalone,
    pin_lb_new,
    pin_algorithm1_abandon,
    pin_nn_brute_by_paths,
    pin_nn_w0_is_euclidean_nn,
    pin_nn_pruned_equals_brute,
    pin_nn_loo_equals_removal,
    pin_dtw_var_equals_min_over_all_paths,
    pin_dtw_var_symmetric_and_reduces,
    pin_envelope_var,
    pin_lb_enhanced_var_matches_band_sets,
    pin_lb_var_bounds_dtw,
    pin_lb_var_reduces_to_equal_length,
    pin_nn_var,
]
