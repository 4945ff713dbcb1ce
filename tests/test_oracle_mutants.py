"""Plant plausible mistakes in copies of the oracle and check that the pins
catch each one (CPU only; the real oracle source is never modified)."""
import os

import pytest

import oracle
import oracle_pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "nndtw_oracle.c")

# name: (site, replacement) or (site, replacement, 0) for the first of two
# occurrences
MUTANTS = {
    "dtw_drops_diagonal_predecessor": (
        "jhi = imin(L, i + W);\n        cur[jlo - 1] = INF;\n        double rowmin = INF;\n"
        "        for (int j = jlo; j <= jhi; j++) {\n"
        "            double m = dmin(dmin(prev[j - 1], cur[j - 1]), prev[j]);",
        "jhi = imin(L, i + W);\n        cur[jlo - 1] = INF;\n        double rowmin = INF;\n"
        "        for (int j = jlo; j <= jhi; j++) {\n"
        "            double m = dmin(cur[j - 1], prev[j]);"),
    "dtw_window_one_short": (
        "int jlo = imax(1, i - W), jhi = imin(L, i + W);\n        cur[jlo - 1] = INF;",
        "int jlo = imax(1, i - W), jhi = imin(L, i + W - 1 < i ? i : i + W - 1);\n        cur[jlo - 1] = INF;"),
    "delta_not_squared": ("double t = d * d;", "double t = d < 0 ? -d : d;"),
    "envelope_window_one_short": (
        "int jlo = imax(1, i - W), jhi = imin(L, i + W);\n        double u",
        "int jlo = imax(1, i - W + (W > 0)), jhi = imin(L, i + W);\n        double u"),
    "envelope_max_min_swapped": ("if (B[j - 1] > u) u = B[j - 1];", "if (B[j - 1] < u) u = B[j - 1];", 0),
    "keogh_lower_uses_upper": (
        "else if (A[i] < Lo[i]) res = res + delta(A[i], Lo[i]);",
        "else if (A[i] < Lo[i]) res = res + delta(A[i], U[i]);"),
    "lbenh_drops_last_end": (
        "double res = delta(a(1), b(1)) + delta(a(L), b(L));",
        "double res = delta(a(1), b(1));"),
    "lbenh_right_band_index_off": (
        "minR = dmin(minR, delta(a(L - i + 1), b(L - j + 1)));",
        "minR = dmin(minR, delta(a(L - i + 1), b(L - j)));"),
    "lbenh_left_band_transposed": (
        "\n            minL = dmin(minL, delta(a(j), b(i)));",
        "\n            minL = dmin(minL, delta(a(j), b(j)));"),
    "lbenh_n_bands_plus_one": ("int n_bands = imin(L / 2, V);", "int n_bands = imin(L / 2, V + 1);"),
    "lbenh_keogh_bridge_overlaps_bands": (
        "for (int i = n_bands + 1; i <= L - n_bands; i++) {\n        if (a(i) > U[i - 1])",
        "for (int i = n_bands; i <= L - n_bands; i++) {\n        if (a(i) > U[i - 1])"),
    "lbenh_abandon_wrong_way": ("if (res >= D) return INFINITY;", "if (res < D) return INFINITY;", 0),
    "lbimp_second_pass_without_projection": (
        "        else Ap[i] = A[i];\n    }\n    oracle_envelope(Ap, L, W, Up, Lp);\n    for (int j = nb + 1;",
        "        Ap[i] = A[i];\n    }\n    oracle_envelope(Ap, L, W, Up, Lp);\n    for (int j = nb + 1;"),
    "lbimproved_without_projection": (
        "        else Ap[i] = A[i];\n    }\n    oracle_envelope(Ap, L, W, Up, Lp);\n    res = res +",
        "        Ap[i] = A[i];\n    }\n    oracle_envelope(Ap, L, W, Up, Lp);\n    res = res +"),
    "lbimp_second_pass_overlaps_bands": (
        "for (int j = nb + 1; j <= L - nb; j++) {",
        "for (int j = nb; j <= L - nb; j++) {"),
    "lbimp_second_pass_lower_uses_upper": (
        "else if (B[j - 1] < Lp[j - 1]) res = res + delta(B[j - 1], Lp[j - 1]);",
        "else if (B[j - 1] < Lp[j - 1]) res = res + delta(B[j - 1], Up[j - 1]);"),
    "lbimproved_skips_second_pass": (
        "    res = res + oracle_lb_keogh(B, Up, Lp, L);\n", "\n"),
    "lbimproved_second_pass_against_b_envelope": (
        "    oracle_envelope(Ap, L, W, Up, Lp);\n    res = res + oracle_lb_keogh(B, Up, Lp, L);",
        "    oracle_envelope(Ap, L, W, Up, Lp);\n    res = res + oracle_lb_keogh(B, U, Lo, L);"),
    "lbnew_window_one_short": (
        "        int jlo = imax(1, i - W), jhi = imin(L, i + W);\n        double m = INFINITY;",
        "        int jlo = imax(1, i - W), jhi = imin(L, i + W - (W > 0));\n        double m = INFINITY;"),
    "lbnew_drops_an_end": (
        "    double res = delta(A[0], B[0]) + delta(A[L - 1], B[L - 1]);\n    for (int i = 2; i <= L - 1; i++) {",
        "    double res = delta(A[0], B[0]);\n    for (int i = 2; i <= L - 1; i++) {"),
    "lbnew_interior_runs_to_the_end": (
        "    for (int i = 2; i <= L - 1; i++) {\n        int jlo",
        "    for (int i = 2; i <= L; i++) {\n        int jlo"),
    "nn_ties_to_highest_index": ("if (d < best) { best = d; bi = t; }", "if (d <= best) { best = d; bi = t; }", 0),
    "loo_keeps_the_query_itself": ("if (j->exclude_self && t == q) continue;", ""),
    "var_dtw_window_one_short": (
        "int jlo = imax(1, i - W), jhi = imin(LB, i + W);\n        cur[jlo - 1] = INF;",
        "int jlo = imax(1, i - W), jhi = imin(LB, i + W - 1 < i ? i : i + W - 1);\n        cur[jlo - 1] = INF;"),
    "var_envelope_window_one_short": (
        "int jlo = imax(1, i - W), jhi = imin(LB, i + W);\n        double u",
        "int jlo = imax(1, i - W), jhi = imin(LB, i + W - (W > 0));\n        double u"),
    "var_end_term_at_equal_length_corner": (
        "double res = delta(a(1), b(1)) + delta(a(LA), b(LB));",
        "double res = delta(a(1), b(1)) + delta(a(LA), b(LA < LB ? LA : LB));"),
    "var_right_band_ignores_window": (
        "            if (in_window(LA - i + 1, LB - j + 1, W))\n", ""),
    "var_left_band_ignores_window": (
        "            if (in_window(i, j, W)) {\n                minL = dmin(minL, delta(a(i), b(j)));",
        "            {\n                minL = dmin(minL, delta(a(i), b(j)));"),
    "var_right_band_arm_collapsed": (
        "minR = dmin(minR, delta(a(LA - j + 1), b(LB - i + 1)));",
        "minR = dmin(minR, delta(a(LA - i + 1), b(LB - i + 1)));"),
    "var_n_bands_ignores_short_series": (
        "int n_bands = imin(imin(LA, LB) / 2, V);", "int n_bands = V;"),
    "var_pruned_drops_tie_update": (
        "            double d = dtw_rows_var(A, LA, B, LB, j->W, D, rows, rows + (LB + 1));\n"
        "            if (isinf(d)) { j->stats[1]++; continue; }\n"
        "            j->stats[2]++;\n"
        "            if (d < D || (d == D && t < bi)) { D = d; bi = t; }",
        "            double d = dtw_rows_var(A, LA, B, LB, j->W, D, rows, rows + (LB + 1));\n"
        "            if (isinf(d)) { j->stats[1]++; continue; }\n"
        "            j->stats[2]++;\n"
        "            if (d < D) { D = d; bi = t; }"),
    "var_brute_keeps_last_minimum": (
        "                                      INFINITY);\n            if (d < best) { best = d; bi = t; }",
        "                                      INFINITY);\n            if (d <= best) { best = d; bi = t; }"),
    "pruned_search_drops_tie_update": (
        "if (d < D || (d == D && t < bi)) { D = d; bi = t; }",
        "if (d < D) { D = d; bi = t; }", 0),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new, *nth = MUTANTS[name]
    src = open(SRC).read()
    if nth:
        # a site that the unequal-length routines repeat: the equal-length
        # routine's copy comes first in the file
        assert src.count(old) == 2, f"mutation site for {name} not found exactly twice"
        at = src.index(old)
        mutated = src[:at] + new + src[at + len(old):]
    else:
        assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
        mutated = src.replace(old, new)
    path = tmp_path / "mut.c"
    path.write_text(mutated)
    so = oracle.compile_oracle(str(path), str(tmp_path / "libmut.so"))
    orc = oracle.Oracle(oracle.load(so))
    for pin in oracle_pins.ALL_PINS:
        try:
            pin(orc)
        except AssertionError:
            return              # caught
    pytest.fail(f"mutant {name} passed every pin")
