"""VB2's parameter cap of Sec. 4 on the device (bp_lb_set_vb2_cap): with the
cap on, bound, argmax and verdict equal the oracle's with the cap
(orc.lb(..., vb2_cap=True), orc.lb_dff(VB2, ..., vb2_cap=True)) on every path
that evaluates VB2 -- the VB2 kernel (fixed point, c <= 65535), the generic
kernel (fp32-corrected and 64-bit paths), VB2 from the prefix kernel's count
table on search nodes -- on the batched, search-node and plain calls, and on
instances built so that the cap removes VB2's best parameter.  With the cap
off the results are the uncapped ones (every other GPU test)."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I
from test_gpu_parity import assert_same, run_batch, run_nodes

pytestmark = pytest.mark.gpu

VB2 = 4


def oracle_batch(orc, rg, cap=True):
    out = [orc.lb(rg.instance(b), int(rg.capacity[b]), int(rg.bins[b]), vb2_cap=cap)
           for b in range(rg.count)]
    return tuple(np.array([o[i] for o in out]) for i in range(4))


def oracle_vb2_only(orc, instances, caps, bins):
    """L_VB2 with the cap, in the device's convention for a single-DFF mask
    whose range is empty: bound 0, argmax (-1, -1)."""
    b, d, l, f = [], [], [], []
    for w, c, k in zip(instances, caps, bins):
        v, lam = orc.lb_dff(VB2, w, c, vb2_cap=True)
        if v < 0:
            b.append(0), d.append(-1), l.append(-1)
        else:
            b.append(v), d.append(VB2), l.append(lam)
        f.append(b[-1] <= k)
    return np.array(b), np.array(d), np.array(l), np.array(f)


@pytest.fixture
def caph(cudalib):
    h = cudalib.bp_lb_create(10_000, 1 << 17)
    cudalib.bp_lb_set_vb2_cap(h, True)
    assert cudalib.bp_lb_get_vb2_cap(h) == 1
    yield h
    cudalib.bp_lb_destroy(h)


def capped_instances(seed=41):
    """Instances on every VB2 path whose cap floor(UINT_MAX / (r max w)) lies
    below c (c >= 10^4), plus small capacities where it does not."""
    rng = np.random.default_rng(seed)
    inst, caps = [], []
    for c, n in ((150, 40), (1000, 200), (10_000, 120), (10_000, 700), (60_000, 30),
                 (65_535, 50), (65_536, 40), (100_000, 25), (200_000, 12)):
        for _ in range(3):
            inst.append(rng.integers(1, c + 1, size=n))
            caps.append(c)
    return inst, caps


def test_cap_collection_batch(cudalib, caph, orc):
    inst, caps = capped_instances()
    rg = I.ragged_from_list(inst, caps)
    cut = [4294967295 // (len(w) * int(w.max())) < c for w, c in zip(inst, caps)]
    assert sum(cut) >= 15  # the cap bites on most of these
    want = oracle_batch(orc, rg)
    for algo in (cudalib.ALGO_PREFIX, cudalib.ALGO_DIRECT):
        for prune in (True, False):
            cudalib.bp_lb_set_algorithm(caph, algo)
            cudalib.bp_lb_set_pruning(caph, prune)
            assert_same(run_batch(cudalib, caph, rg), want, f"algo {algo} prune {prune}")
            assert_same(run_batch(cudalib, caph, rg, i64=True), want, f"i64 algo {algo}")
    cudalib.bp_lb_set_pruning(caph, True)
    cudalib.bp_lb_set_algorithm(caph, cudalib.ALGO_PREFIX)


def test_cap_vb2_only_batch(cudalib, caph, orc):
    """VB2 alone: the capped L_VB2 and its first parameter, where the cap cuts."""
    inst, caps = capped_instances(seed=42)
    rg = I.ragged_from_list(inst, caps)
    cudalib.bp_lb_set_dff_mask(caph, 1 << VB2)
    try:
        assert_same(run_batch(cudalib, caph, rg),
                    oracle_vb2_only(orc, inst, caps, rg.bins), "VB2 only")
    finally:
        cudalib.bp_lb_set_dff_mask(caph, 63)


def constructed():
    """Instances whose VB2 maximum lies above the cap (items of size c / 8 + 1:
    every VB2 bound is 0 for l < 8 and large at l = 8), on the VB2 kernel's
    fixed-point path (c = 60000, long lists over many staging chunks), the
    fp32-corrected path (c = 10^6) and the 64-bit path (c = 2^30); the hand
    cases of tests/golden/vb2_cap.txt; zero sizes counted in r."""
    out = []
    w = 60_000 // 8 + 1
    out += [([w] * 80_000, 60_000), ([w] * 40_000, 60_000), ([w] * 71_000, 60_000)]
    w = 10 ** 6 // 8 + 1
    out += [([w] * 4500, 10 ** 6), ([w] * 4000, 10 ** 6)]
    c = 1 << 30
    out += [([1 << 20] * 1000, c), ([(1 << 27) + 1] * 4, c), ([(1 << 27) + 1] * 2, c),
            ([2000] + [1] * 1021, 2000), ([c - 1] * 3, c),
            ([(1 << 27) + 1] * 4 + [0] * 4, c)]
    return out


def test_cap_cuts_vb2_maximum(cudalib, caph, orc):
    cases = constructed()
    inst = [np.asarray(w, np.int64) for w, _ in cases]
    caps = [c for _, c in cases]
    rg = I.ragged_from_list(inst, caps)
    want = oracle_vb2_only(orc, inst, caps, rg.bins)
    # the cap removed a larger bound: l = 8 would give far more on the first five
    for j in range(5):
        assert orc.lb_param(VB2, 8, inst[j], caps[j]) > want[0][j] or want[2][j] == 8
    cudalib.bp_lb_set_dff_mask(caph, 1 << VB2)
    try:
        for prune in (True, False):
            cudalib.bp_lb_set_pruning(caph, prune)
            assert_same(run_batch(cudalib, caph, rg), want, f"constructed, prune {prune}")
    finally:
        cudalib.bp_lb_set_pruning(caph, True)
        cudalib.bp_lb_set_dff_mask(caph, 63)


def test_cap_search_nodes(cudalib, caph, orc):
    """Search nodes: r counts the unpacked items and the non-empty bins; the
    u group's count-table VB2 (prefix kernel) and the VB2 kernel both clip."""
    for n, nodes, seed in ((500, 24, 51), (2000, 6, 52)):
        nd = I.search_nodes(seed=seed, n=n, c=10_000, nodes=nodes)
        want_b, want_d, want_l, want_f = [], [], [], []
        vb = []
        for j in range(nd.count):
            w, a, c, k = nd.node(j)
            red = orc.reduce(w, a, k, c)
            want = orc.lb(red, c, k, vb2_cap=True)
            want_b.append(want[0]), want_d.append(want[1]), want_l.append(want[2])
            want_f.append(want[3])
            vb.append((red, c, k))
        want = tuple(np.array(x) for x in (want_b, want_d, want_l, want_f))
        for prune in (True, False):
            cudalib.bp_lb_set_pruning(caph, prune)
            assert_same(run_nodes(cudalib, caph, nd), want, f"nodes n={n} prune {prune}")
        cudalib.bp_lb_set_pruning(caph, True)
        cudalib.bp_lb_set_dff_mask(caph, 1 << VB2)
        try:
            assert_same(run_nodes(cudalib, caph, nd),
                        oracle_vb2_only(orc, [x[0] for x in vb], [x[1] for x in vb],
                                        [x[2] for x in vb]), f"nodes VB2 only n={n}")
        finally:
            cudalib.bp_lb_set_dff_mask(caph, 63)


def test_cap_close_reduction(cudalib, caph, orc):
    """Under the closing reduction variant a closed bin is an item of size c,
    which is then max w' of the cap."""
    nd = I.search_nodes(seed=53, n=300, c=10_000, nodes=12)
    cudalib.bp_lb_set_reduction(caph, cudalib.REDUCE_CLOSE)
    try:
        want = []
        for j in range(nd.count):
            w, a, c, k = nd.node(j)
            want.append(orc.lb(orc.reduce_ex(w, a, k, c, mode=1), c, k, vb2_cap=True))
        want = tuple(np.array([x[i] for x in want]) for i in range(4))
        assert_same(run_nodes(cudalib, caph, nd), want, "close")
    finally:
        cudalib.bp_lb_set_reduction(caph, cudalib.REDUCE_LOADS)


def test_cap_plain_and_verdict(cudalib, orc):
    rng = np.random.default_rng(54)
    for c in (10_000, 100_000):
        h = cudalib.bp_lb_create(c, 1 << 12)
        try:
            cudalib.bp_lb_set_vb2_cap(h, True)
            for _ in range(4):
                w = rng.integers(1, c + 1, size=int(rng.integers(20, 200)))
                k = -(-int(w.sum()) // c) + int(rng.integers(0, 3))
                assert cudalib.bp_lb_eval(h, w, k) == orc.lb(w, c, k, vb2_cap=True)[:3]
                a = np.full(len(w), -1, np.int32)
                kb = len(w)
                a[: len(w) // 3] = np.arange(len(w) // 3)  # one item per bin
                red = orc.reduce(w, a, kb, c)
                assert cudalib.bp_lb_eval_node(h, w, a, kb) == orc.lb(red, c, kb, vb2_cap=True)[:3]
            # verdict mode with the cap: verdicts exact
            inst = [rng.integers(1, c + 1, size=60) for _ in range(16)]
            ks = [-(-int(x.sum()) // c) + int(rng.integers(-1, 2)) for x in inst]
            rg = I.ragged_from_list(inst, [c] * 16, bins=[max(0, k) for k in ks])
            cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_VERDICT)
            got = run_batch(cudalib, h, rg)
            want = oracle_batch(orc, rg)
            assert np.array_equal(got[3], want[3])
        finally:
            cudalib.bp_lb_destroy(h)
