"""The pins must catch plausible mistakes in the oracle.

Each case copies oracle.c to a temporary directory, plants one mistake by a
literal text substitution, builds it, and runs the pin suite against the
broken copy (through MS_ORACLE_SO). The suite must fail for every mutant.
Nothing here touches a GPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

MUTANTS = {
    "window_exclusive": ("        if (cs >= c) {\n            for", "        if (cs > c) {\n            for"),
    "mean_not_renormalised": ("x_new[k] = y[k] / yn;", "x_new[k] = y[k] / (double)cnt;"),
    "update_drops_first_dim": ("            for (int32_t k = 0; k < dim; ++k) y[k] += p[k];",
                               "            for (int32_t k = 1; k < dim; ++k) y[k] += p[k];"),
    "merge_support_ascending": ("return a->support > b->support ? -1 : 1;", "return a->support > b->support ? 1 : -1;"),
    "merge_tie_latest_first": ("return a->order < b->order ? -1 : 1;", "return a->order < b->order ? 1 : -1;"),
    "merge_inclusive_keep": ("if (n_kept == 0 || best < merge_cos) {", "if (n_kept == 0 || best <= merge_cos + 0.05) {"),
    "early_stop_at_gamma": ("if ((double)nconv > gamma * (double)m || nmove == 0) break;",
                            "if ((double)nconv >= gamma * (double)m || nmove == 0) break;"),
    "schedule_floor": ("nn = N - (int64_t)ceil(nmin);", "nn = N - (int64_t)floor(nmin);"),
    "schedule_no_doubling": ("nn = 2 * N;", "nn = N + N / 2;"),
    "eq19_uses_eq15_base": ("return log(1.0 - exp(log(P) / I)) / log(1.0 - r / I);",
                            "return log(1.0 - exp(log(P) / I)) / log(1.0 - 1.0 / (2.0 * I));"),
    "eq14_missing_power_I": ("return pow(1.0 - pow(1.0 - r / I, N), I);", "return 1.0 - pow(1.0 - r / I, N);"),
    "cover_exclusive": ("            if (best >= c) {", "            if (best > c) {"),
    "label_ties_highest": ("            if (cs > b1) {", "            if (cs >= b1) {"),
    "seeds_ignore_coverage": ("            if (covered[i]) continue;\n            covered[i] = 1;",
                              "            covered[i] = 1;"),
    "perm_offset_ignored": ("return (int64_t)((aj + (uint64_t)b) % (uint64_t)n);", "return (int64_t)(aj % (uint64_t)n);"),
    "merge_keep_at_threshold": ("if (n_kept == 0 || best < merge_cos) {", "if (n_kept == 0 || best <= merge_cos) {"),
    "schedule_double_at_edge": ("if ((double)N < L * nmin)", "if ((double)N <= L * nmin)"),
    "schedule_shrink_at_edge": ("else if ((double)N > H * nmin)", "else if ((double)N >= H * nmin)"),
    "schedule_no_clamp": ("    if (nn > hi) nn = hi;\n", ""),
    "background_zero": ("for (int64_t i = 0; i < n_pixels; ++i) labels[i] = -1;",
                        "for (int64_t i = 0; i < n_pixels; ++i) labels[i] = 0;"),
    "merge_least_similar": ("            if (cs > best) best = cs;\n        }\n        if (n_kept > 0) {",
                            "            if (best == -INFINITY || cs < best) best = cs;\n        }\n        if (n_kept > 0) {"),
    "perm_tie_upper_first": ("        if (lo >= 1 && lo <= n - 1 && gcd64(lo, n) == 1) { pick = lo; break; }\n"
                             "        if (hi >= 1 && hi <= n - 1 && gcd64(hi, n) == 1) { pick = hi; break; }",
                             "        if (hi >= 1 && hi <= n - 1 && gcd64(hi, n) == 1) { pick = hi; break; }\n"
                             "        if (lo >= 1 && lo <= n - 1 && gcd64(lo, n) == 1) { pick = lo; break; }"),
    "perm_golden_truncated": ("floor(0.6180339887 * (double)n + 0.5)", "floor(0.6180339887 * (double)n)"),
    "seed_iters_count_idle_seeds": ("        si += active;", "        si += m;"),
    "no_stop_when_none_moving": ("if ((double)nconv > gamma * (double)m || nmove == 0) break;",
                                 "if ((double)nconv > gamma * (double)m) break;"),
    "moving_seeds_offered": ("            if (sstate[s] != 1) {", "            if (sstate[s] == 2) {"),
    "schedule_uses_round_modes": ("        N = or_next_n(N, n_kept, 1.0, cfg->P_target, L, cfg->H, uncovered);",
                                  "        N = or_next_n(N, n_kept - k0, 1.0, cfg->P_target, L, cfg->H, uncovered);"),
    "carry_unbounded": ("st.n_carry = n_free < max_draw ? n_free : max_draw;", "st.n_carry = n_free;"),
    "all_seeds_keeps_gamma": ("const double gamma = cfg->all_seeds ? 1.0 : cfg->gamma;", "const double gamma = cfg->gamma;"),
    "mask_inverted": ("if (mask != NULL && mask[i] == 0) continue;", "if (mask != NULL && mask[i] != 0) continue;"),
    "label_margin_stale_second": ("            if (cs > b1) {\n                b2 = b1;\n", "            if (cs > b1) {\n"),
    "schedule_no_floor": ("    if (nn < 1) nn = 1;\n", ""),
    "window_margin_ignored": ("            if (m < mm) mm = m;\n        }\n        if (cs >= c) {",
                              "        }\n        if (cs >= c) {"),
    "cover_margin_ignored": ("            double marg = fabs(best - c);\n            if (marg < mm) mm = marg;\n"
                             "            if (best >= c) {", "            if (best >= c) {"),
    "normalise_skipped": ("for (int32_t k = 0; k < dim; ++k) p[k] = (double)e[k] / nrm;",
                          "for (int32_t k = 0; k < dim; ++k) p[k] = (double)e[k];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.h"), tmp_path / "oracle.h")
    (tmp_path / "oracle.c").write_text(src.replace(old, new))
    so = str(tmp_path / "liboracle_mut.so")
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                    str(tmp_path / "oracle.c"), "-o", so, "-lm"], check=True, capture_output=True)
    env = dict(os.environ, MS_ORACLE_SO=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"pins did not catch mutant {name}:\n{r.stdout[-2000:]}"
