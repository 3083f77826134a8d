"""Pins of the oracle's reduction variants (orc_reduce_ex).  The paper does
not define them (they are next steps after its Fig. 3 reduction), so they
are pinned by what must hold for any valid reduction: whenever the partial
packing can be completed, the reduced instance packs into the k bins (brute
force over every completion of tiny instances); closing bins only grows the
virtual items; with neither option the variant is the paper's reduction."""
import itertools

import numpy as np
import pytest


def completions_exist(w, assign, k, c, cap):
    """Brute force: can the unpacked items be placed into the k bins without
    exceeding any bin's capacity cap[j]?"""
    load = [0] * k
    free = []
    for wi, ai in zip(w, assign):
        if ai >= 0:
            load[ai] += wi
        else:
            free.append(wi)
    if any(load[j] > cap[j] for j in range(k)):
        return False
    for choice in itertools.product(range(k), repeat=len(free)):
        lj = list(load)
        for wi, j in zip(free, choice):
            lj[j] += wi
        if all(lj[j] <= cap[j] for j in range(k)):
            return True
    return False


def random_case(rng, with_cap):
    c = int(rng.integers(2, 13))
    k = int(rng.integers(1, 4))
    n = int(rng.integers(0, 7))
    w = [int(x) for x in rng.integers(0, c + 1, size=n)]
    cap = [int(x) for x in rng.integers(c // 2, c + 1, size=k)] if with_cap else [c] * k
    assign, load = [], [0] * k
    for wi in w:
        j = int(rng.integers(-1, k))
        if j >= 0 and load[j] + wi <= cap[j] and rng.random() < 0.6:
            load[j] += wi
            assign.append(j)
        else:
            assign.append(-1)
    return w, assign, k, c, cap


def check_plain_variant(orc, trials=300):
    rng = np.random.default_rng(3)
    for _ in range(trials):
        w, assign, k, c, _ = random_case(rng, False)
        want = orc.reduce(w, assign, k, c)
        assert np.array_equal(orc.reduce_ex(w, assign, k, c, 0, None), want)
        assert np.array_equal(orc.reduce_ex(w, assign, k, c, 0, [c] * k), want)


def check_variants_valid(orc, mode, with_cap, trials=400):
    """Completable partial packing => the reduced instance fits in k bins of
    size c (so every DFF bound of it is <= k)."""
    rng = np.random.default_rng(10 + 2 * mode + with_cap)
    seen = 0
    for _ in range(trials):
        w, assign, k, c, cap = random_case(rng, with_cap)
        if not completions_exist(w, assign, k, c, cap):
            continue
        seen += 1
        red = orc.reduce_ex(w, assign, k, c, mode, cap if with_cap else None)
        assert orc.opt_bins(red, c) <= k, (w, assign, k, c, cap, list(red))
        assert orc.lb(red, c, k)[0] <= k
    assert seen > trials // 4


def check_closing_grows(orc):
    rng = np.random.default_rng(21)
    grew = 0
    for _ in range(500):
        w, assign, k, c, cap = random_case(rng, True)
        try:
            r0 = orc.reduce_ex(w, assign, k, c, 0, cap)
        except ValueError:
            continue
        r1 = orc.reduce_ex(w, assign, k, c, 1, cap)
        assert len(r0) == len(r1)
        assert np.all(r1 >= r0)
        grew += int(np.any(r1 > r0))
        assert orc.lb(r1, c, k)[0] >= orc.lb(r0, c, k)[0]
    assert grew > 20


def check_examples(orc):
    # a bin whose cap equals its load has no free space: its item is c
    assert list(orc.reduce_ex([3, 4, 2], [0, 1, -1], 2, 10, 0, [3, 10])) == [2, 10, 4]
    # closing: free space 3 of bin 0 is below the smallest unpacked item (4)
    assert list(orc.reduce_ex([7, 4, 4], [0, -1, -1], 2, 10, 1, None)) == [4, 4, 10]
    # no unpacked item: every non-empty bin is closed, empty ones dropped
    assert list(orc.reduce_ex([7, 2], [0, 0], 3, 10, 1, None)) == [10]
    with pytest.raises(ValueError):
        orc.reduce_ex([5], [0], 1, 10, 0, [4])      # load above the cap
    with pytest.raises(ValueError):
        orc.reduce_ex([5], [0], 1, 10, 0, [11])     # cap above c


def test_plain_variant_is_the_papers_reduction(orc):
    check_plain_variant(orc)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("with_cap", [False, True])
def test_reduction_variants_are_valid(orc, mode, with_cap):
    check_variants_valid(orc, mode, with_cap)


def test_closing_only_grows_items(orc):
    check_closing_grows(orc)


def test_full_cap_bin_and_errors(orc):
    check_examples(orc)
