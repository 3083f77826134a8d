"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself or with the CUDA path.  The pins:
  (p1) dual feasibility (Sec. 3.1): for every DFF and integer lambda of its
       range, sum f(x_i) <= f(c) over every multiset with sum x_i <= c, and
       f(0) = 0 -- by exact knapsack DP for c <= 40, cross-checked by literal
       multiset enumeration for c <= 14;
  (p2) brute-force optimum: L1 <= every DFF bound <= OPT on tiny instances;
  (p3) L2 from its definition (Sec. 3.1): L2 = max(L_MT, #{w > c/2}),
       L_MT = L2 for even c, and the collection bound >= L2;
  (p4) special cases that reduce to L1: MT at lambda 0, BJ1 at lambda 1, at
       lambda = c and at every divisor of c;
  (p5) the worked example of Fig. 3 (tests/golden/fig3_partial_packing.txt)
       and the hand-derived parameter counts (tests/golden/param_counts.txt);
  (p6) the VB2 overflow cap of Sec. 4 only removes parameters, and on the
       hand-derived cases of tests/golden/vb2_cap.txt (the cap cuts VB2's
       range below c, stops at c, or empties it) it gives the hand-derived
       L_VB2 and excludes a better parameter;
  plus reduction invariants (Sec. 3 "Feasibility check").
Each check is a plain function so that the mutation test can run the whole
battery against deliberately broken copies of the oracle.
"""
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------------------
# fixtures as data
# ---------------------------------------------------------------------------
def load_fig3():
    items, assign, params = [], [], []
    out = {}
    with open(os.path.join(GOLDEN, "fig3_partial_packing.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            tok = line.split()
            if tok[0] == "item":
                items.append(int(tok[1]))
                assign.append(int(tok[2]))
            elif tok[0] == "param":
                params.append((O.NAMES.index(tok[1]), int(tok[2]), int(tok[3]), int(tok[4]),
                               int(tok[5])))
            elif tok[0] == "reduced_multiset":
                out["reduced"] = sorted(int(x) for x in tok[1:])
            else:
                out[tok[0]] = int(tok[1])
    out["items"], out["assign"], out["params"] = items, assign, params
    return out


def load_vb2_cap():
    cases = []
    with open(os.path.join(GOLDEN, "vb2_cap.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            name, c, items, cap, bnd, lam, wl, wlb = line.split()
            sizes = []
            for part in items.split(","):
                cnt, size = part.split("x")
                sizes += [int(size)] * int(cnt)
            cases.append(dict(name=name, c=int(c), items=sizes, cap=int(cap),
                              capped=(int(bnd), int(lam)),
                              witness=None if wl == "-" else (int(wl), int(wlb))))
    return cases


def load_param_counts():
    rows = []
    with open(os.path.join(GOLDEN, "param_counts.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(x) for x in line.split()])
    return rows


# ---------------------------------------------------------------------------
# checks (each raises AssertionError on failure)
# ---------------------------------------------------------------------------
def check_param_counts(orc):
    for row in load_param_counts():
        c, counts = row[0], row[1:]
        for d in range(6):
            assert orc.param_range(d, c)[2] == counts[d], (O.NAMES[d], c)


def check_dual_feasible_dp(orc, cmax=40):
    for c in range(1, cmax + 1):
        for d in range(6):
            lo, hi, _ = orc.param_range(d, c)
            for lam in range(lo, hi + 1):
                assert orc.dff(d, 0, lam, c) == 0, (O.NAMES[d], lam, c, "f(0)")
                fc = orc.dff(d, c, lam, c)
                assert fc > 0, (O.NAMES[d], lam, c, "f(c) > 0")
                assert orc.dff_knapsack_max(d, lam, c) <= fc, (O.NAMES[d], lam, c)


def _multisets(total_max):
    """All multisets of positive integers with sum <= total_max (non-increasing tuples)."""
    out = [()]

    def rec(prefix, remaining, largest):
        for x in range(min(largest, remaining), 0, -1):
            t = prefix + (x,)
            out.append(t)
            rec(t, remaining - x, x)

    rec((), total_max, total_max)
    return out


def check_dual_feasible_enum(orc, cmax=14):
    for c in range(1, cmax + 1):
        ms = _multisets(c)
        for d in range(6):
            lo, hi, _ = orc.param_range(d, c)
            for lam in range(lo, hi + 1):
                f = [orc.dff(d, x, lam, c) for x in range(c + 1)]
                best = max(sum(f[x] for x in m) for m in ms)
                assert best <= f[c], (O.NAMES[d], lam, c)
                assert best == orc.dff_knapsack_max(d, lam, c), (O.NAMES[d], lam, c, "dp")


def check_bruteforce_opt(orc, trials=150, seed=11):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        c = int(rng.integers(1, 21))
        n = int(rng.integers(0, 11))
        w = rng.integers(0, c + 1, size=n)
        opt = orc.opt_bins(w, c)
        l1 = orc.l1(w, c)
        lb, _, _, _ = orc.lb(w, c, opt)
        assert l1 <= lb <= opt, (list(w), c, l1, lb, opt)
        for d in range(6):
            lo, hi, _ = orc.param_range(d, c)
            for lam in range(lo, hi + 1):
                v = orc.lb_param(d, lam, w, c)
                assert v <= lb, (O.NAMES[d], lam, list(w), c)
                assert v <= opt, (O.NAMES[d], lam, list(w), c, v, opt)


def _l_mt(orc, w, c):
    lo, hi, _ = orc.param_range(O.MT, c)
    return max(orc.lb_param(O.MT, lam, w, c) for lam in range(lo, hi + 1))


def check_l2(orc, trials=300, seed=12):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        c = int(rng.integers(1, 41))
        n = int(rng.integers(0, 16))
        w = rng.integers(0, c + 1, size=n)
        l2 = orc.l2(w, c)
        lmt = _l_mt(orc, w, c)
        nbig = int(np.sum(2 * w > c))
        assert l2 == max(lmt, nbig), (list(w), c, l2, lmt, nbig)
        if c % 2 == 0:
            assert lmt == l2, (list(w), c)
        lb, _, _, _ = orc.lb(w, c, 0)
        assert lb >= l2, (list(w), c)
    # the odd-capacity case where the two differ: three items of 3 in bins of 5
    assert orc.l2([3, 3, 3], 5) == 3 and _l_mt(orc, [3, 3, 3], 5) == 2


def check_l1_special_cases(orc, trials=200, seed=13):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        c = int(rng.integers(1, 200))
        n = int(rng.integers(0, 30))
        w = rng.integers(0, c + 1, size=n)
        l1 = -(-int(w.sum()) // c)
        assert orc.l1(w, c) == l1
        assert orc.lb_param(O.MT, 0, w, c) == l1
        assert orc.lb_param(O.BJ1, 1, w, c) == l1
        assert orc.lb_param(O.BJ1, c, w, c) == l1
        for lam in range(1, c + 1):
            if c % lam == 0:
                assert orc.lb_param(O.BJ1, lam, w, c) == l1, (lam, c)


def check_fig3(orc):
    g = load_fig3()
    c, k = g["capacity"], g["bins"]
    wr = orc.reduce(g["items"], g["assign"], k, c)
    assert sorted(wr.tolist()) == g["reduced"]
    for d, lam, s, fc, bound in g["params"]:
        assert orc.dff(d, c, lam, c) == fc, (O.NAMES[d], lam)
        assert sum(orc.dff(d, int(x), lam, c) for x in wr) == s, (O.NAMES[d], lam)
        assert orc.lb_param(d, lam, wr, c) == bound, (O.NAMES[d], lam)
    b, d, lam, feas = orc.lb(wr, c, k)
    assert b == g["bound"] and feas == bool(g["feasible"])
    # first attaining parameter in paper order is MT at lambda = 0 (= L1)
    assert (d, lam) == (O.MT, 0)


def check_vb2_cap(orc, trials=100, seed=14):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        c = int(rng.integers(2, 3000))
        n = int(rng.integers(1, 40))
        w = rng.integers(0, c + 1, size=n)
        full = orc.lb(w, c, 0)[0]
        cap = orc.lb(w, c, 0, vb2_cap=True)[0]
        assert cap <= full
        wmax = int(w.max())
        if wmax == 0 or 4294967295 // (n * wmax) >= c:
            assert cap == full


def check_vb2_cap_golden(orc):
    """The cap of Sec. 4 on hand-derived cases: L_VB2 over the capped range
    is the hand-derived (bound, first lambda); a witness parameter just past
    the cap (or past c, where the cap stops) has the hand-derived, larger
    bound, so the capped range really ends where the golden file says."""
    for g in load_vb2_cap():
        c, items = g["c"], g["items"]
        assert orc.lb_dff(O.VB2, items, c, vb2_cap=True) == g["capped"], g["name"]
        if g["witness"] is not None:
            wl, wlb = g["witness"]
            assert wl > g["cap"] and wlb > g["capped"][0]
            assert orc.lb_param(O.VB2, wl, items, c) == wlb, g["name"]
        if g["cap"] >= 2:
            # the last parameter of the capped range is evaluated: its bound
            # is at most the capped maximum
            assert orc.lb_param(O.VB2, g["cap"], items, c) <= g["capped"][0], g["name"]
        if c <= 4096:  # cap >= c: the capped bound is the uncapped one
            assert g["cap"] == c
            assert orc.lb_dff(O.VB2, items, c) == g["capped"], g["name"]


def check_reduction(orc, trials=200, seed=15):
    rng = np.random.default_rng(seed)
    for _ in range(trials):
        c = int(rng.integers(1, 100))
        n = int(rng.integers(0, 40))
        k = int(rng.integers(0, 12))
        w = rng.integers(0, c + 1, size=n)
        load = np.zeros(k, dtype=np.int64)
        a = np.full(n, -1, dtype=np.int32)
        for i in range(n):
            if k and rng.random() < 0.5:
                j = int(rng.integers(0, k))
                if load[j] + w[i] <= c:
                    load[j] += w[i]
                    a[i] = j
        wr = orc.reduce(w, a, k, c)
        assert int(wr.sum()) == int(w.sum())
        assert len(wr) == int(np.sum(a == -1)) + int(np.sum(load > 0))
        assert np.all(wr[: int(np.sum(a == -1))] == w[a == -1])
        # every packed bin becomes one item of its load, in bin order
        assert np.all(wr[int(np.sum(a == -1)):] == load[load > 0])


def printed_range(d, c):
    """The integer parameter ranges as printed in Sec. 3.1 (0 <= l <= c/2; c/4 < l <= c/3;
    1 <= l <= 100; 1 <= l <= c/2; 2 <= l <= c; 1 <= l <= c)."""
    return [l for l in range(0, max(c, 100) + 1)
            if ((d == O.MT and 2 * l <= c) or (d == O.RAD2 and 4 * l > c and 3 * l <= c)
                or (d == O.FS1 and 1 <= l <= 100) or (d == O.CCM1 and 1 <= l and 2 * l <= c)
                or (d == O.VB2 and 2 <= l <= c) or (d == O.BJ1 and 1 <= l <= c))]


def check_full_maximum(orc, trials=40, seed=16):
    """Alg. 2 without early exit: L_f is the maximum of the per-parameter bounds over
    the printed range (first attaining lambda), and the collection is the maximum of
    the L_f (first attaining DFF in the order MT, RAD2, FS1, CCM1, VB2, BJ1)."""
    rng = np.random.default_rng(seed)
    for t in range(trials):
        c = int(rng.integers(1, 130))
        n = int(rng.integers(0, 25))
        w = rng.integers(0, c + 1, size=n)
        best, arg = -1, None
        for d in range(6):
            vals = [(orc.lb_param(d, l, w, c), l) for l in printed_range(d, c)]
            if vals:
                m = max(v for v, _ in vals)
                first = next(l for v, l in vals if v == m)
                assert orc.lb_dff(d, w, c) == (m, first), (O.NAMES[d], list(w), c)
                if m > best:
                    best, arg = m, (d, first)
            else:
                assert orc.lb_dff(d, w, c)[0] == -1
        b, d, l, _ = orc.lb(w, c, 0)
        assert (b, (d, l)) == (best, arg), (list(w), c)


ALL_CHECKS = (check_param_counts, check_fig3, check_dual_feasible_dp, check_bruteforce_opt,
              check_l2, check_l1_special_cases, check_vb2_cap, check_reduction, check_full_maximum)


# ---------------------------------------------------------------------------
# tests
# ---------------------------------------------------------------------------
def test_param_counts(orc):
    check_param_counts(orc)


def test_fig3_worked_example(orc):
    check_fig3(orc)


def test_dual_feasible_dp(orc):
    check_dual_feasible_dp(orc, cmax=40)


def test_dual_feasible_enum(orc):
    check_dual_feasible_enum(orc, cmax=14)


def test_bruteforce_opt(orc):
    check_bruteforce_opt(orc)


def test_l2_closed_form(orc):
    check_l2(orc)


def test_l1_special_cases(orc):
    check_l1_special_cases(orc)


def test_vb2_cap(orc):
    check_vb2_cap(orc)


def test_vb2_cap_golden(orc):
    check_vb2_cap_golden(orc)


def test_full_maximum(orc):
    check_full_maximum(orc)


def test_reduction(orc):
    check_reduction(orc)


def test_invalid_inputs(orc):
    with pytest.raises(ValueError):
        orc.lb([7], 6, 1)
    with pytest.raises(ValueError):
        orc.lb([-1], 6, 1)
    with pytest.raises(ValueError):
        orc.reduce([4, 4], [0, 0], 1, 6)          # overfull bin
    with pytest.raises(ValueError):
        orc.reduce([1], [3], 2, 6)                # bin index out of range
    # empty instance: bound 0, first parameter (MT, 0)
    assert orc.lb([], 10, 0) == (0, O.MT, 0, True)
