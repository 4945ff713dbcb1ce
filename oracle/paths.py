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

import functools
import math

import numpy as np


def all_warping_paths(L: int, W: int):
    """Every warping path (list of 1-based (i, j) links) inside the window."""
    return all_warping_paths_var(L, L, W)


def path_cost(a, b, path) -> float:
    """Sum of delta(A_i, B_j) = (A_i - B_j)^2 over the links, summed exactly."""
    return math.fsum((float(a[i - 1]) - float(b[j - 1])) ** 2 for i, j in path)


@functools.lru_cache(maxsize=None)
def _incidence(LA: int, LB: int, W: int):
    """Row k marks the cells of the k-th warping path of an LA x LB grid
    (0/1 entries, cells in row-major order); None when no path fits."""
    ps = all_warping_paths_var(LA, LB, W)
    if not ps:
        return None
    M = np.zeros((len(ps), LA * LB))
    for k, p in enumerate(ps):
        for i, j in p:
            M[k, (i - 1) * LB + (j - 1)] = 1.0
    return M


def _min_path_cost(a, b, W: int) -> float:
    """Minimum over every warping path of the sum of its cells' deltas: all
    path costs at once as the incidence matrix times the cell costs (each a
    sum of at most LA + LB - 1 terms, exact for small integers)."""
    a = np.asarray(a, dtype=float)
    b = np.asarray(b, dtype=float)
    M = _incidence(len(a), len(b), int(W))
    if M is None:
        return math.inf
    cost = ((a[:, None] - b[None, :]) ** 2).ravel()
    return float((M @ cost).min())


def dtw_by_paths(a, b, W: int) -> float:
    assert len(a) == len(b)
    return _min_path_cost(a, b, W)


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


# ------------------------------------------------------- unequal lengths ---
# A has L_A points and B has L_B.  A warping path runs from (1, 1) to
# (L_A, L_B) with the same three kinds of links, inside |i - j| <= W.

def all_warping_paths_var(LA: int, LB: int, W: int):
    out = []

    def rec(i, j, path):
        if (i, j) == (LA, LB):
            out.append(list(path))
            return
        for di, dj in ((1, 0), (0, 1), (1, 1)):
            ni, nj = i + di, j + dj
            if ni <= LA and nj <= LB and abs(ni - nj) <= W:
                path.append((ni, nj))
                rec(ni, nj, path)
                path.pop()

    rec(1, 1, [(1, 1)])
    return out


def dtw_by_paths_var(a, b, W: int) -> float:
    """Minimum path cost over every warping path of the L_A x L_B grid inside
    the window; +inf when there is none."""
    return _min_path_cost(a, b, W)


def left_band_var(i: int, W: int):
    """The start corner's L-shape of index i: (i, j) and (j, i), j <= i,
    inside the window."""
    return {c for j in range(1, i + 1) for c in ((i, j), (j, i)) if abs(c[0] - c[1]) <= W}


def right_band_var(i: int, LA: int, LB: int, W: int):
    """The end corner's L-shape of index i: (L_A-i+1, L_B-j+1) and
    (L_A-j+1, L_B-i+1), j <= i, inside the window."""
    cells = set()
    for j in range(1, i + 1):
        for c in ((LA - i + 1, LB - j + 1), (LA - j + 1, LB - i + 1)):
            if abs(c[0] - c[1]) <= W:
                cells.add(c)
    return cells


def keogh_term_var(a, b, i: int, W: int) -> float:
    """Distance from A_i to the interval spanned by B over row i's window
    max(1, i-W) .. min(L_B, i+W), window extremes by Python's max/min."""
    window = [float(b[j - 1]) for j in range(max(1, i - W), min(len(b), i + W) + 1)]
    lo, hi = min(window), max(window)
    x = float(a[i - 1])
    if x > hi:
        return (x - hi) ** 2
    if x < lo:
        return (x - lo) ** 2
    return 0.0


def lb_enhanced_by_sets_var(a, b, W: int, V: int) -> float:
    """LB_Enhanced^V for unequal lengths summed from explicit cell sets:
    n_b start-corner bands, n_b end-corner bands, and the Keogh terms of
    rows n_b+1 .. L_A-n_b; +inf when |L_A - L_B| > W."""
    LA, LB = len(a), len(b)
    if abs(LA - LB) > W:
        return math.inf
    nb = min(min(LA, LB) // 2, V)
    terms = [band_min(a, b, left_band_var(i, W)) for i in range(1, nb + 1)]
    terms += [band_min(a, b, right_band_var(i, LA, LB, W)) for i in range(1, nb + 1)]
    terms += [keogh_term_var(a, b, i, W) for i in range(nb + 1, LA - nb + 1)]
    return math.fsum(terms)


def theorem2_intermediate_var(a, b, W: int, V: int) -> float:
    """The bands as above with the minimum over each bridge row's whole
    window instead of its Keogh term: between the bound and DTW."""
    LA, LB = len(a), len(b)
    nb = min(min(LA, LB) // 2, V)
    terms = [band_min(a, b, left_band_var(i, W)) for i in range(1, nb + 1)]
    terms += [band_min(a, b, right_band_var(i, LA, LB, W)) for i in range(1, nb + 1)]
    terms += [band_min(a, b, {(i, j) for j in range(max(1, i - W), min(LB, i + W) + 1)})
              for i in range(nb + 1, LA - nb + 1)]
    return math.fsum(terms)
