"""Brute-force checks that share nothing with the oracle's recurrences.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``all_warping_paths`` enumerates every warping path of Sec. 2.1 directly from
  its constraints (boundary: starts at (1,1) and ends at (L,L); continuity and
  monotonicity: each link advances i, j or both by one), restricted to the
  window |i - j| <= W.  ``dtw_by_paths`` takes the minimum path cost, which is
  DTW_W by definition (Eq. 2 without the square root).
* ``left_band`` / ``right_band`` build the cell sets of Sec. 3 (Theorem 1 and
  the right-band analogue) as explicit sets, and ``lb_enhanced_by_sets`` sums
  Eq. 7 term by term from them: a second route to LB_Enhanced that does not
  follow Algorithm 1's loops.

Indices here are 1-based as in the paper; arrays are 0-based.
"""
from __future__ import annotations

import math


def all_warping_paths(L: int, W: int):
    """Yield every warping path (list of 1-based (i, j) links) inside the window."""
    out = []

    def rec(i, j, path):
        if (i, j) == (L, L):
            out.append(list(path))
            return
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            ni, nj = i + di, j + dj
            if ni <= L and nj <= L and abs(ni - nj) <= W:
                path.append((ni, nj))
                rec(ni, nj, path)
                path.pop()

    rec(1, 1, [(1, 1)])
    return out


def path_cost(a, b, path) -> float:
    """Sum of delta(A_i, B_j) = (A_i - B_j)^2 over the links, summed exactly."""
    return math.fsum((float(a[i - 1]) - float(b[j - 1])) ** 2 for i, j in path)


def dtw_by_paths(a, b, W: int) -> float:
    L = len(a)
    return min(path_cost(a, b, p) for p in all_warping_paths(L, W))


def left_band(i: int, L: int, W: int):
    """L^W_i = {(j, i), (i, j) : max(1, i-W) <= j <= i} (Sec. 3)."""
    cells = set()
    for j in range(max(1, i - W), i + 1):
        cells.add((j, i))
        cells.add((i, j))
    return cells


def right_band(i: int, L: int, W: int):
    """R^W_i = {(j, i), (i, j) : i <= j <= min(L, i+W)} (Sec. 3, read from the
    right-band loop of Algorithm 1; the printed set is garbled)."""
    cells = set()
    for j in range(i, min(L, i + W) + 1):
        cells.add((j, i))
        cells.add((i, j))
    return cells


def vertical_band(i: int, L: int, W: int):
    """V_i = {(i, j) : max(1, i-W) <= j <= min(L, i+W)} (proof of Theorem 2)."""
    return {(i, j) for j in range(max(1, i - W), min(L, i + W) + 1)}


def band_min(a, b, cells) -> float:
    return min((float(a[j - 1]) - float(b[k - 1])) ** 2 for j, k in cells)


def keogh_term(a, b, i: int, W: int) -> float:
    """The bridge term of Eq. 7 for index i: the squared distance from A_i to
    the interval spanned by B over A_i's window (zero inside it).  The window
    extremes are taken here with Python's max/min over the window's values, not
    from envelope arrays."""
    L = len(a)
    window = [float(b[j - 1]) for j in range(max(1, i - W), min(L, i + W) + 1)]
    lo, hi = min(window), max(window)
    x = float(a[i - 1])
    if x > hi:
        return (x - hi) ** 2
    if x < lo:
        return (x - lo) ** 2
    return 0.0


def lb_enhanced_by_sets(a, b, W: int, V: int) -> float:
    """Eq. 7 summed term by term: left-band minima for i <= V, right-band
    minima for i > L - V, the Keogh bridge term otherwise."""
    L = len(a)
    terms = []
    for i in range(1, L + 1):
        if i <= V:
            terms.append(band_min(a, b, left_band(i, L, W)))
        elif i > L - V:
            terms.append(band_min(a, b, right_band(i, L, W)))
        else:
            terms.append(keogh_term(a, b, i, W))
    return math.fsum(terms)


def theorem2_intermediate(a, b, W: int, V: int) -> float:
    """The middle line of the proof of Theorem 2: left-band minima for i <= V,
    the minimum over the vertical band V_i for the bridge, right-band minima for
    i > L - V.  The proof places it between LB_Enhanced^V and DTW_W."""
    L = len(a)
    terms = []
    for i in range(1, L + 1):
        if i <= V:
            terms.append(band_min(a, b, left_band(i, L, W)))
        elif i > L - V:
            terms.append(band_min(a, b, right_band(i, L, W)))
        else:
            terms.append(band_min(a, b, vertical_band(i, L, W)))
    return math.fsum(terms)


def full_left_band_bound(a, b, W: int) -> float:
    """Theorem 1: sum over all i of the left-band minima."""
    L = len(a)
    return math.fsum(band_min(a, b, left_band(i, L, W)) for i in range(1, L + 1))


def full_right_band_bound(a, b, W: int) -> float:
    """Right-band analogue of Theorem 1."""
    L = len(a)
    return math.fsum(band_min(a, b, right_band(i, L, W)) for i in range(1, L + 1))
