"""The oracle's pins have teeth: each plausible mistake planted in a copy of the
oracle (a flipped comparison, a dropped term, a transposed operand, a wrong
range end) must make at least one pin of test_oracle_pins fail.  Mutants are
compiled from text-substituted copies of oracle/bp_oracle.c in a temporary
directory; the oracle itself is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

import oracle as O
from test_oracle_pins import (check_bruteforce_opt, check_dual_feasible_dp, check_fig3,
                              check_full_maximum, check_l1_special_cases, check_l2,
                              check_param_counts, check_reduction, check_vb2_cap,
                              check_vb2_cap_golden)
from test_oracle_reduction import (check_closing_grows, check_examples, check_plain_variant,
                                   check_variants_valid)

SRC = os.path.join(os.path.dirname(O.__file__), "bp_oracle.c")

# (name, exact snippet of bp_oracle.c, replacement)
MUTANTS = [
    ("mt_strict", "if (c - l < w) return c;", "if (c - l <= w) return c;"),
    ("mt_lower", "if (l <= w && w <= c - l) return w;", "if (l < w && w <= c - l) return w;"),
    ("rad2_swap_floors", "return c / 3;", "return c / 2;"),
    ("rad2_mirror_off_by_one", "return c - f_rad2(c - w, l, c);", "return c - f_rad2(c - w + 1, l, c);"),
    ("rad2_case2_strict", "if (l <= w && w <= c - 2 * l) return c / 3;",
     "if (l <= w && w < c - 2 * l) return c / 3;"),
    ("fs1_divisible_value", "if ((w * (l + 1)) % c == 0) return w * l;",
     "if ((w * (l + 1)) % c == 0) return w * (l + 1);"),
    ("fs1_no_divisible_case", "if ((w * (l + 1)) % c == 0) return w * l;", ""),
    ("ccm1_half_doubled", "if (2 * w == c) return c / l;", "if (2 * w == c) return 2 * (c / l);"),
    ("ccm1_transposed", "return 2 * (c / l) - 2 * ((c - w) / l);", "return 2 * (c / l) - 2 * (w / l);"),
    ("vb2_big_operand", "- 2 * max64(0, ceil_div(c * l - w * l, c) - 1);",
     "- 2 * max64(0, ceil_div(w * l, c) - 1);"),
    ("vb2_small_no_minus_one", "return 2 * max64(0, ceil_div(w * l, c) - 1); /* 2w < c */",
     "return 2 * max64(0, ceil_div(w * l, c)); /* 2w < c */"),
    ("vb2_half_doubled", "if (2 * w == c) return max64(0, ceil_div(c * l, c) - 1);",
     "if (2 * w == c) return 2 * max64(0, ceil_div(c * l, c) - 1);"),
    ("bj1_dropped_term", "return (w / l) * (l - c % l) + w % l - c % l;",
     "return (w / l) * (l - c % l) + w % l;"),
    ("bj1_sign", "if (w % l <= c % l) return (w / l) * (l - c % l);",
     "if (w % l <= c % l) return (w / l) * (l + c % l);"),
    ("range_rad2_lo", "*lo = c / 4 + 1; *hi = c / 3;", "*lo = c / 4;     *hi = c / 3;"),
    ("range_mt_hi", "case ORC_MT:   *lo = 0;         *hi = c / 2;", "case ORC_MT:   *lo = 0;         *hi = c / 2 + 1;"),
    ("range_vb2_lo", "case ORC_VB2:  *lo = 2;", "case ORC_VB2:  *lo = 1;"),
    ("range_fs1_hi", "*lo = 1;         *hi = 100;", "*lo = 1;         *hi = 99; "),
    ("floor_not_ceil", "static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }",
     "static int64_t ceil_div(int64_t a, int64_t b) { return a / b; }"),
    ("tie_break_last_lambda", "if (lb > best) { best = lb; best_l = l; }",
     "if (lb >= best) { best = lb; best_l = l; }"),
    ("tie_break_last_dff", "if (lf > best) { best = lf; best_d = d; best_l = l; }",
     "if (lf >= best) { best = lf; best_d = d; best_l = l; }"),
    ("reduce_residual_not_load", "if (load[j] > 0) out[r++] = load[j];",
     "if (load[j] > 0) out[r++] = c - load[j];"),
    ("reduce_keeps_packed", "if (assign[i] == -1) out[r++] = w[i];",
     "if (assign[i] >= -1) out[r++] = w[i];"),
    ("l2_medium_bound", "else if (2 * w[i] > c && w[i] <= c - l) { n2++; s2 += w[i]; }",
     "else if (2 * w[i] >= c && w[i] <= c - l) { n2++; s2 += w[i]; }"),
    ("reduce_ex_filler_sign", "int64_t v = load[j] + (c - cap);", "int64_t v = load[j] - (c - cap);"),
    ("reduce_ex_close_when_equal", "if (mode == 1 && v > 0 && (minw < 0 || c - v < minw)) v = c;",
     "if (mode == 1 && v > 0 && (minw < 0 || c - v <= minw)) v = c;"),
    ("reduce_ex_close_empty_bins", "if (mode == 1 && v > 0 && (minw < 0 || c - v < minw)) v = c;",
     "if (mode == 1 && v >= 0 && (minw < 0 || c - v < minw)) v = c;"),
    ("reduce_ex_cap_ignored", "int64_t cap = bin_max ? bin_max[j] : c;", "int64_t cap = c;"),
    # the VB2 cap of Sec. 4: floor(UINT_MAX / (r max w')), at most c
    ("vb2_cap_no_r", "int64_t cap = (int64_t)4294967295LL / (r * wmax);",
     "int64_t cap = (int64_t)4294967295LL / wmax;"),
    ("vb2_cap_sum_not_max", "if (wr[i] > wmax) wmax = wr[i];", "wmax += wr[i];"),
    ("vb2_cap_signed_limit", "int64_t cap = (int64_t)4294967295LL / (r * wmax);",
     "int64_t cap = (int64_t)2147483647LL / (r * wmax);"),
    ("vb2_cap_ceil", "int64_t cap = (int64_t)4294967295LL / (r * wmax);",
     "int64_t cap = ((int64_t)4294967295LL + r * wmax - 1) / (r * wmax);"),
    ("vb2_cap_not_min_c", "return cap < c ? cap : c;", "return cap;"),
]

BATTERY = (
    lambda o: check_param_counts(o),
    lambda o: check_fig3(o),
    lambda o: check_dual_feasible_dp(o, cmax=24),
    lambda o: check_bruteforce_opt(o, trials=60),
    lambda o: check_l2(o, trials=150),
    lambda o: check_l1_special_cases(o, trials=60),
    lambda o: check_vb2_cap(o, trials=60),
    lambda o: check_vb2_cap_golden(o),
    lambda o: check_reduction(o, trials=80),
    lambda o: check_full_maximum(o),
    lambda o: check_plain_variant(o, trials=100),
    lambda o: check_variants_valid(o, 1, True, trials=160),
    lambda o: check_variants_valid(o, 1, False, trials=160),
    lambda o: check_closing_grows(o),
    lambda o: check_examples(o),
)


def test_snippets_present():
    src = open(SRC).read()
    for name, old, _ in MUTANTS:
        assert src.count(old) == 1, name


_RUNNER = """
import sys
sys.path[:0] = [{root!r}, {tests!r}]
import oracle as O
from test_oracle_mutants import BATTERY
mut = O.Oracle({lib!r})
caught = 0
for check in BATTERY:
    try:
        check(mut)
    except (AssertionError, ValueError):
        caught += 1
sys.exit(10 if caught else 0)
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="gcc missing")
@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(tmp_path, name, old, new):
    """A mutant is caught when a pin fails, or when the mutant crashes or hangs
    (e.g. a recursion that no longer terminates) -- each run is a subprocess
    with a time limit."""
    src = open(SRC).read()
    assert src.count(old) == 1
    mpath = tmp_path / "mutant.c"
    mpath.write_text(src.replace(old, new))
    lib = str(tmp_path / "libmutant.so")
    O.build(str(mpath), lib)
    here = os.path.dirname(os.path.abspath(__file__))
    code = _RUNNER.format(root=os.path.dirname(here), tests=here, lib=lib)
    try:
        rc = subprocess.run([sys.executable, "-c", code], timeout=60,
                            capture_output=True).returncode
    except subprocess.TimeoutExpired:
        rc = -1
    assert rc != 0, f"mutant {name} survived every pin"
