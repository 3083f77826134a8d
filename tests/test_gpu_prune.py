"""VB2 pruning (exact): a VB2 parameter whose upper bound, from the
instance's sums, cannot beat the instance's best key so far is skipped.  The
results -- bound, first argmax, verdict -- are identical with pruning on and
off and equal the oracle's, including ties between VB2 and the DFFs on either
side of it in paper order, capacities past VB2's fixed-point range (128-bit
test), and verdict mode with k far above every bound."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

from test_gpu_parity import oracle_batch, oracle_node, run_batch, run_nodes

pytestmark = pytest.mark.gpu


def mixed(seed, caps, count, n_hi):
    rng = np.random.default_rng(seed)
    inst, cs = [], []
    for _ in range(count):
        c = int(rng.choice(caps))
        n = int(rng.integers(0, n_hi))
        kind = rng.integers(0, 3)
        if kind == 0:
            w = I.uniform_sizes(rng, n, 1, c)
        elif kind == 1:                      # many items just above c / 2: VB2 territory
            w = rng.integers(c // 2 - c // 20, c // 2 + c // 10 + 1, size=n)
        else:                                # small items only: loose upper bounds
            w = rng.integers(1, max(2, c // 6), size=n)
        inst.append(np.clip(w, 0, c))
        cs.append(c)
    return I.ragged_from_list(inst, cs)


def both(cudalib, h, rg):
    out = []
    for on in (1, 0):
        cudalib.bp_lb_set_pruning(h, on)
        assert cudalib.bp_lb_get_pruning(h) == on
        out.append(run_batch(cudalib, h, rg))
    cudalib.bp_lb_set_pruning(h, 1)
    return out


@pytest.mark.parametrize("algo", [1, 0])
def test_prune_identical_and_exact(cudalib, orc, algo):
    rg = mixed(61, (7, 150, 1000, 9999, 65535, 65536, 90_001), 90, 150)
    want = oracle_batch(orc, rg)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_algorithm(h, algo)
        on, off = both(cudalib, h, rg)
        for x, y, z in zip(on, off, want):
            assert np.array_equal(np.asarray(x), np.asarray(z))
            assert np.array_equal(np.asarray(y), np.asarray(z))
    finally:
        cudalib.bp_lb_destroy(h)


@pytest.mark.parametrize("mask", [(4,), (0, 4), (3, 4), (4, 5), (1, 2, 4), (0, 1, 2, 3, 4, 5)])
def test_prune_ties_under_masks(cudalib, orc, mask):
    """The slot's best key precedes VB2 (ties lose: cut B), follows it (BJ1:
    cut B - 1), or is VB2's own."""
    rg = mixed(62, (10, 150, 1000, 9999), 60, 120)
    rg.bins = np.zeros(rg.count, dtype=np.int64) + 1
    want = []
    for j in range(rg.count):
        w, c = rg.instance(j), int(rg.capacity[j])
        best = (0, -1, -1)
        for d in mask:
            lf, lam = orc.lb_dff(d, w, c)
            if lf >= 0 and (best[1] < 0 or lf > best[0]):
                best = (lf, d, lam)
        want.append(best)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_dff_mask(h, sum(1 << d for d in mask))
        for got in both(cudalib, h, rg):
            b, dd, ll, _ = got
            for j in range(rg.count):
                assert (b[j], dd[j], ll[j]) == want[j], (j, mask)
    finally:
        cudalib.bp_lb_destroy(h)


def test_prune_search_nodes(cudalib, orc):
    nd = I.search_nodes(seed=3, n=500, c=10_000, nodes=192)
    want = tuple(np.array(x) for x in zip(*[oracle_node(orc, nd, j) for j in range(nd.count)]))
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        for on in (1, 0):
            cudalib.bp_lb_set_pruning(h, on)
            got = run_nodes(cudalib, h, nd)
            for x, y in zip(got, want):
                assert np.array_equal(np.asarray(x), np.asarray(y)), on
    finally:
        cudalib.bp_lb_destroy(h)


def test_prune_plain_path(cudalib, orc):
    rng = np.random.default_rng(64)
    for c in (1000, 9999, 70_000):
        h = cudalib.bp_lb_create(c, 4096)
        try:
            for _ in range(3):
                w = I.uniform_sizes(rng, int(rng.integers(1, 300)), 1, c)
                want = orc.lb(w, c, 0)[:3]
                for on in (1, 0):
                    cudalib.bp_lb_set_pruning(h, on)
                    assert cudalib.bp_lb_eval(h, w, 0) == tuple(want), (c, on)
        finally:
            cudalib.bp_lb_destroy(h)


def test_verdict_huge_k_large_capacity(cudalib, orc):
    """k far above every bound (clamped to the stream length in the test),
    capacities on the 128-bit side: every instance feasible, witnesses real."""
    rng = np.random.default_rng(65)
    inst, caps = [], []
    for c in (65_536, 120_000, 300_001):
        for _ in range(2):
            inst.append(I.uniform_sizes(rng, int(rng.integers(1, 40)), 1, c))
            caps.append(c)
    rg = I.ragged_from_list(inst, caps)
    rg.bins = np.zeros(rg.count, dtype=np.int64) + (1 << 50)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_VERDICT)
        b, dd, ll, f = run_batch(cudalib, h, rg)
        assert bool(np.all(f))
        for j in range(rg.count):
            assert orc.lb_param(int(dd[j]), int(ll[j]), rg.instance(j), caps[j]) == b[j]
        # and k just below the maximum: infeasible, with a witness above k
        full = oracle_batch(orc, rg)[0]
        rg.bins = np.maximum(0, full - 1).astype(np.int64)
        b, dd, ll, f = run_batch(cudalib, h, rg)
        assert not bool(np.any(f))
        for j in range(rg.count):
            assert b[j] > rg.bins[j]
            assert orc.lb_param(int(dd[j]), int(ll[j]), rg.instance(j), caps[j]) == b[j]
    finally:
        cudalib.bp_lb_destroy(h)


def _vb2_table_mode(w, c, k):
    """The u-group tile's VB2 plan (vb2_table_plan in bp_lb_prefix.cuh),
    restated: 1 when VB2's parameters that can matter all lie in [2, lmax]
    with few enough count-table lookups."""
    w = np.asarray(w, dtype=np.int64)
    w = w[w > 0]
    small = w[2 * w < c]
    big = w[(2 * w > c) & (w < c)]
    nh, nf = int(np.sum(2 * w == c)), int(np.sum(w == c))
    ns, nb = len(small), len(big)
    L1 = -(-int(w.sum()) // c)
    kk = min(L1, len(w) + 0)
    K = 2 * nb + nh + 2 * nf
    D = int(small.sum()) - int((c - big).sum())
    alpha = 2 * D - c * (2 * kk - K)
    beta = 2 * ns * (c - 1) + c * (2 * kk - K) - c * (2 * ns - 2 * nb + 1) + 2
    if alpha >= 0 or 2 * alpha + beta <= 0:
        return 0
    lmax = min(c, (beta - 1) // (-alpha))
    U = (c - 1) // 2
    return 1 if U * lmax * lmax // (2 * c) + lmax <= (1 << 16) else 0


def vb2_strong_instances(orc, seed=67, tries=6000):
    """Random small instances (items above c / 2 mixed with small ones, and
    uniform ones), kept when VB2 is the argmax of the full bound, plus every
    tenth of the others."""
    rng = np.random.default_rng(seed)
    inst, caps = [], []
    for t in range(tries):
        c = int(rng.choice([60, 100, 150]))
        n = int(rng.integers(3, 60))
        if t % 2:
            w = rng.integers(1, c + 1, n)
        else:
            w = np.concatenate([rng.integers(c // 2 + 1, c, n // 2 + 1), rng.integers(1, c // 2, n // 2 + 1)])
        d = orc.lb([int(x) for x in w], c, 0)[1]
        if d == 4 or t % 10 == 0:
            inst.append(w)
            caps.append(c)
    return I.ragged_from_list(inst, caps)


def test_vb2_on_count_table(cudalib, orc):
    """VB2 evaluated from the u-group tile's count table (vb2_table_plan picks
    it for instances whose VB2 parameters that can matter are small): bound
    and argmax equal the oracle's, VB2 the argmax of several, with pruning
    on and off."""
    rg = vb2_strong_instances(orc)
    want = oracle_batch(orc, rg)
    modes = np.array([_vb2_table_mode(rg.instance(j), int(rg.capacity[j]), 0)
                      for j in range(rg.count)])
    assert int(np.sum((np.asarray(want[1]) == 4) & (modes == 1))) >= 2
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        for got in both(cudalib, h, rg):
            for x, y in zip(got, want):
                assert np.array_equal(np.asarray(x), np.asarray(y))
    finally:
        cudalib.bp_lb_destroy(h)


def _late_mode(w, c, cut):
    """The second VB2 plan of a cluster's u-group unit (late_vb2_plan),
    restated: the first plan's test with the cut of the keys already found."""
    w = np.asarray(w, dtype=np.int64)
    w = w[w > 0]
    small = w[2 * w < c]
    big = w[(2 * w > c) & (w < c)]
    nh, nf = int(np.sum(2 * w == c)), int(np.sum(w == c))
    ns, nb = len(small), len(big)
    kk = min(cut, len(w))
    K = 2 * nb + nh + 2 * nf
    D = int(small.sum()) - int((c - big).sum())
    alpha = 2 * D - c * (2 * kk - K)
    beta = 2 * ns * (c - 1) + c * (2 * kk - K) - c * (2 * ns - 2 * nb + 1) + 2
    if alpha >= 0:
        return 2 if alpha * c + beta <= 0 else 0
    if 2 * alpha + beta <= 0:
        return 2
    return 1


@pytest.mark.parametrize("cluster", [False, True])
def test_vb2_late_plan(cudalib, orc, cluster):
    """Instances whose MT / RAD2 / CCM1 bounds lie above L1, so that the
    u-group's first VB2 plan (cut L1) leaves VB2 to its kernel and a
    cluster unit's second plan (cut from the keys found) takes it on the
    count table: bound and argmax equal the oracle's with pruning on and
    off, with cluster tables on (c = 30000 and 100000 take clusters) and off
    (one plan), and with MT left out of the bound (no second plan)."""
    import concurrent.futures as cf
    rng = np.random.default_rng(91)
    inst, caps = [], []
    for c, n in ((3000, 800), (3000, 3000), (30000, 1500), (30000, 3000), (100000, 2000),
                 (100000, 3000)):
        inst.append(rng.integers(1, c + 1, size=n))
        caps.append(c)
    rg = I.ragged_from_list(inst, caps)
    rg.bins = np.zeros(rg.count, np.int64)
    with cf.ThreadPoolExecutor(6) as ex:
        want = list(ex.map(lambda j: orc.lb(inst[j], caps[j], 0), range(rg.count)))
        ucut = list(ex.map(lambda j: max(orc.lb_dff(d, inst[j], caps[j])[0] for d in (0, 1, 3)),
                           range(rg.count)))
    want = tuple(np.array(x) for x in zip(*want))
    late = [_late_mode(inst[j], caps[j], ucut[j]) for j in range(rg.count)]
    assert sum(m != 0 for m in late) >= 3, late
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_cluster_tables(h, cluster)
        for got in both(cudalib, h, rg):
            for x, y in zip(got, want):
                assert np.array_equal(np.asarray(x), np.asarray(y))
        cudalib.bp_lb_set_dff_mask(h, 0b111110)   # MT left out: VB2 planned once
        b, d, lam, _ = run_batch(cudalib, h, rg)
        for j in range(rg.count):
            best = (0, -1, -1)
            for dd in (1, 2, 3, 4, 5):
                lf, l = orc.lb_dff(dd, inst[j], caps[j])
                if lf >= 0 and (best[1] < 0 or lf > best[0]):
                    best = (lf, dd, l)
            assert (b[j], d[j], lam[j]) == best, j
    finally:
        cudalib.bp_lb_destroy(h)
