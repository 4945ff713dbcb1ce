"""The arithmetic behind the FP32 cascade filter's LB_Improved term, checked
on the host against the oracle (CPU only).

The filter reads, per training element, B_j and its two gaps to the second
envelopes, gap_up = B_j - max Lo and gap_dn = min U - B_j over j's window,
rounded down to half precision, and takes the term min(B_j - U^A_j, gap_up)^2
above the query's envelope and min(Lo^A_j - B_j, gap_dn)^2 below it.  Exact
gaps give exactly the oracle's second pass (Sec. 2.2.4, Eq. 5); gaps rounded
down give terms that are never larger, so the bound stays a lower bound, and
only slightly smaller."""
import math

import numpy as np
from scipy.ndimage import maximum_filter1d, minimum_filter1d


def _f16_down(x):
    """x rounded down to half precision (the largest half value <= x), as
    float64; values beyond the half range saturate to its largest finite."""
    with np.errstate(over="ignore"):    # beyond the half range: +inf, stepped down below
        h = x.astype(np.float16).astype(np.float64)
        over = h > x
        h[over] = np.nextafter(x[over].astype(np.float16), np.float16(-np.inf)).astype(np.float64)
    big = ~np.isfinite(h)
    h[big] = float(np.finfo(np.float16).max)
    return h


def _terms(a, b, W, nb, round_gaps):
    L = a.shape[0]
    size = 2 * W + 1
    U = maximum_filter1d(b, size=size, mode="nearest")
    Lo = minimum_filter1d(b, size=size, mode="nearest")
    Ua = maximum_filter1d(a, size=size, mode="nearest")
    La = minimum_filter1d(a, size=size, mode="nearest")
    gap_up = b - maximum_filter1d(Lo, size=size, mode="nearest")
    gap_dn = minimum_filter1d(U, size=size, mode="nearest") - b
    assert (gap_up >= 0).all() and (gap_dn >= 0).all()
    if round_gaps:
        gap_up, gap_dn = _f16_down(gap_up), _f16_down(gap_dn)
    up, dn = b - Ua, La - b
    d = np.maximum(np.maximum(np.minimum(up, gap_up), np.minimum(dn, gap_dn)), 0.0)
    mid = slice(nb, L - nb)
    return d[mid] ** 2


def test_packed_gaps_never_raise_a_term(orc):
    rng = np.random.default_rng(21)
    for _ in range(60):
        L = int(rng.integers(2, 300))
        W = int(rng.integers(0, L + 2))
        V = int(rng.integers(1, max(1, min(10, L // 2)) + 1))
        nb = min(L // 2, V)
        scale = 10.0 ** rng.uniform(-3, 5)      # includes gaps beyond the half range
        a, b = scale * rng.standard_normal(L), scale * rng.standard_normal(L)
        exact = _terms(a, b, W, nb, False)
        packed = _terms(a, b, W, nb, True)
        assert (packed <= exact).all()
        # the exact closed form is the oracle's second pass
        Ub, Lb = orc.envelope(b, W)
        second = orc.lb_enhanced_improved(a, b, Ub, Lb, W, V) - orc.lb_enhanced(a, b, Ub, Lb, W, V)
        assert abs(math.fsum(exact) - second) <= 1e-9 * max(abs(second), 1e-300) + 1e-12 * scale ** 2
        # and rounding the gaps down costs little of it while they fit half precision
        if scale < 1e3 and math.fsum(exact) > 0:
            assert math.fsum(packed) >= (1 - 2e-3) ** 2 * math.fsum(exact) - 1e-9 * scale ** 2
