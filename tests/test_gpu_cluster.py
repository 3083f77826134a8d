"""The cluster kernel: prefix-count tables of 48-512 KB spread over the shared
memory of a cluster of 8 CTAs (c from 12287 to 131070; MT and CCM1 alone up
to 262142).  Bound, argmax and verdict against the oracle where the tables
move between one CTA, a cluster and the global scratch; for every kind of
unit (the merged u group, MT, RAD2 and CCM1 alone, BJ1 with FS1, FS1 and BJ1
alone, tables of mixed homes in one instance); for ragged batches, search
nodes with the reduction variants, the plain path, invalid instances and the
verdict mode; and unchanged with cluster tables off (the default)."""
import concurrent.futures as cf

import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

from test_gpu_parity import assert_same, oracle_batch, oracle_node, run_batch, run_nodes, to_dev
from test_gpu_reduction import large_item_nodes, nodes_with_caps, oracle_nodes

pytestmark = pytest.mark.gpu


def cluster_handle(cudalib, c=150, max_items=1 << 16):
    h = cudalib.bp_lb_create(c, max_items)
    cudalib.bp_lb_set_cluster_tables(h, True)
    return h

# the last capacities of each table home (bp_lb.h, the algorithm section)
BOUNDARY_CAPS = (12286, 12287, 24574, 24575, 40000, 65535, 65536, 99991, 131070, 131071,
                 262142, 262143)


def boundary_batch(seed):
    """Per capacity: uniform sizes with zero, full and half items mixed in;
    small items only; and equal sizes (many parameters tie at the maximum)."""
    rng = np.random.default_rng(seed)
    inst, caps = [], []
    for c in BOUNDARY_CAPS:
        n = 150 if c <= 70000 else 40
        w = rng.integers(0, c + 1, size=n)
        m = rng.random(n)
        w[m < 0.05] = 0
        w[(m >= 0.05) & (m < 0.1)] = c
        if c % 2 == 0:
            w[(m >= 0.1) & (m < 0.15)] = c // 2
        inst += [w, rng.integers(1, c // 2 + 1, size=n), np.full(n // 3, c // 3 + 1)]
        caps += [c, c, c]
    rg = I.ragged_from_list(inst, caps)
    rg.bins = rng.integers(0, 80, size=rg.count).astype(np.int64)
    return rg


def test_cluster_capacity_boundaries(cudalib, orc):
    rg = boundary_batch(71)
    want = oracle_batch(orc, rg)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        assert cudalib.bp_lb_get_cluster_tables(h) == 0
        assert_same(run_batch(cudalib, h, rg), want, "cluster tables off (default)")
        cudalib.bp_lb_set_cluster_tables(h, True)
        assert cudalib.bp_lb_get_cluster_tables(h) == 1
        assert_same(run_batch(cudalib, h, rg), want, "cluster tables on")
        assert_same(run_batch(cudalib, h, rg, i64=True), want, "cluster tables on, int64")
        cudalib.bp_lb_set_cluster_tables(h, False)
        assert cudalib.bp_lb_get_cluster_tables(h) == 0
        assert_same(run_batch(cudalib, h, rg), want, "cluster tables off")
        assert cudalib.lib().bp_lb_set_cluster_tables(h, 2) == cudalib.BP_ERANGE
    finally:
        cudalib.bp_lb_destroy(h)


def test_cluster_long_streams_mixed_homes(cudalib, orc):
    """Streams of 2^15 items or more (no merged u group): at c = 13000 MT and
    CCM1 keep one CTA's tables while RAD2 and BJ1 with FS1 take clusters; at
    c = 30000 every unit is a cluster's."""
    rng = np.random.default_rng(72)
    inst = [rng.integers(1, 13001, size=33000), rng.integers(1, 30001, size=33000),
            rng.integers(1, 15001, size=34000)]
    caps = [13000, 30000, 30000]
    rg = I.ragged_from_list(inst, caps)
    rg.bins = np.array([17000, 16600, 8600], np.int64)
    with cf.ThreadPoolExecutor(3) as ex:
        want = list(ex.map(lambda i: orc.lb(inst[i], caps[i], int(rg.bins[i])), range(3)))
    want = tuple(np.array(x) for x in zip(*want))
    h = cluster_handle(cudalib)
    try:
        assert_same(run_batch(cudalib, h, rg), want, "long streams")
    finally:
        cudalib.bp_lb_destroy(h)


@pytest.mark.parametrize("mask", [(2,), (5,), (2, 5), (0, 3), (1,), (0,), (3,), (0, 1, 3),
                                  (0, 1, 2, 3, 4, 5)])
def test_cluster_units_under_masks(cudalib, orc, mask):
    """Each kind of unit: FS1 alone, BJ1 alone, BJ1 with FS1, the u group of
    two or three members, MT, RAD2 or CCM1 alone."""
    rng = np.random.default_rng(73 + sum(1 << d for d in mask))
    caps = [20000, 50000, 50001, 100000, 131070, 262142]
    inst = [rng.integers(0, c + 1, size=120) for c in caps]
    rg = I.ragged_from_list(inst, caps)
    rg.bins = np.full(rg.count, 30, np.int64)
    want = []
    for w, c in zip(inst, caps):
        best = (0, -1, -1)
        for d in mask:
            lf, lam = orc.lb_dff(d, w, c)
            if lf >= 0 and (best[1] < 0 or lf > best[0]):
                best = (lf, d, lam)
        want.append(best)
    h = cluster_handle(cudalib)
    try:
        cudalib.bp_lb_set_dff_mask(h, sum(1 << d for d in mask))
        b, d, lam, _ = run_batch(cudalib, h, rg)
        for j, (wb, wd, wl) in enumerate(want):
            assert (b[j], d[j], lam[j]) == (wb, wd, wl), (mask, j)
    finally:
        cudalib.bp_lb_destroy(h)


def test_cluster_search_nodes(cudalib, orc):
    nd = I.ragged_nodes(seed=74, count=48, n_lo=20, n_hi=1500, caps=(20000, 50000, 100000))
    with cf.ThreadPoolExecutor(8) as ex:
        want = list(ex.map(lambda j: oracle_node(orc, nd, j), range(nd.count)))
    want = tuple(np.array(x) for x in zip(*want))
    h = cluster_handle(cudalib)
    try:
        assert_same(run_nodes(cudalib, h, nd), want, "nodes")
        cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_VERDICT)
        got = run_nodes(cudalib, h, nd)
        assert np.array_equal(got[3], want[3]), "verdicts"
        cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_FULL)
    finally:
        cudalib.bp_lb_destroy(h)


@pytest.mark.parametrize("mode", [0, 1])
def test_cluster_reduction_variants(cudalib, orc, mode):
    nd, offs, bin_max = nodes_with_caps(75 + mode, count=24, caps=(30000, 90000))
    want = oracle_nodes(orc, nd, mode, offs, bin_max)
    d_offs, d_bm = to_dev(offs), to_dev(bin_max)
    h = cluster_handle(cudalib)
    try:
        cudalib.bp_lb_set_reduction(h, mode)
        cudalib.bp_lb_set_bin_max(h, d_offs, d_bm)
        b = run_nodes(cudalib, h, nd)
        for x, y in zip(b, want):
            assert np.array_equal(np.asarray(x), np.asarray(y)), mode
        cudalib.bp_lb_set_bin_max(h)
        nd2 = large_item_nodes(77 + mode, count=24, caps=(30000, 90000))
        b2 = run_nodes(cudalib, h, nd2)
        for x, y in zip(b2, oracle_nodes(orc, nd2, mode)):
            assert np.array_equal(np.asarray(x), np.asarray(y)), mode
    finally:
        cudalib.bp_lb_destroy(h)


@pytest.mark.parametrize("c", [20000, 100000])
def test_cluster_plain_path(cudalib, orc, c):
    rng = np.random.default_rng(c)
    h = cluster_handle(cudalib, c, 4096)
    try:
        for _ in range(3):
            w = rng.integers(0, c + 1, size=int(rng.integers(1, 400)))
            k = int(rng.integers(0, 200))
            assert cudalib.bp_lb_eval(h, w, k) == orc.lb(w, c, k)[:3]
        nd = I.ragged_nodes(seed=c + 1, count=4, n_lo=50, n_hi=800, caps=(c,))
        for j in range(nd.count):
            w, a, cc, k = nd.node(j)
            assert cudalib.bp_lb_eval_node(h, w, a, k) == oracle_node(orc, nd, j)[:3]
    finally:
        cudalib.bp_lb_destroy(h)


def test_cluster_invalid_instances(cudalib, orc):
    """A size above c (ragged) and an overfull bin (search node) at cluster
    capacities: -BP_ERANGE for them, exact results for their neighbours."""
    rng = np.random.default_rng(78)
    caps = [50000, 50000, 100000, 20000]
    inst = [rng.integers(0, c + 1, size=200) for c in caps]
    inst[1][17] = caps[1] + 1
    rg = I.ragged_from_list(inst, caps)
    rg.bins = np.full(rg.count, 40, np.int64)
    h = cluster_handle(cudalib)
    try:
        b, d, lam, f = run_batch(cudalib, h, rg)
        assert (b[1], d[1], lam[1], f[1]) == (-cudalib.BP_ERANGE, -1, -1, False)
        for j in (0, 2, 3):
            assert (b[j], d[j], lam[j], f[j]) == orc.lb(inst[j], caps[j], 40), j
        nd = I.ragged_nodes(seed=79, count=6, n_lo=100, n_hi=600, caps=(50000,))
        j = next(j for j in range(nd.count) if np.any(nd.node(j)[1] >= 0))
        s, e = nd.assign_offsets[j], nd.assign_offsets[j + 1]
        asg = nd.assign[s:e]
        i0 = int(np.nonzero(asg >= 0)[0][0])
        # every item of node j into one bin: overfull
        nd.assign[s:e] = np.where(asg >= 0, asg[i0], asg)
        w, a, c, k = nd.node(j)
        if np.sum(w[a >= 0]) <= c:  # make sure it overflows
            nd.assign[s:e] = asg[i0]
        got = run_nodes(cudalib, h, nd)
        assert got[0][j] == -cudalib.BP_ERANGE
        for i in range(nd.count):
            if i != j:
                assert tuple(x[i] for x in got) == oracle_node(orc, nd, i), i
    finally:
        cudalib.bp_lb_destroy(h)


def _late_lmax(w, c, cut, budget=1 << 21):
    """The last VB2 parameter of a cluster u-group unit's second plan
    (late_vb2_plan with the cut of MT, RAD2 and CCM1), restated from the
    plan's linear test; None when the plan leaves VB2 to its kernel."""
    w = np.asarray(w, dtype=np.int64)
    w = w[w > 0]
    small, big = w[2 * w < c], w[(2 * w > c) & (w < c)]
    nh, nf = int(np.sum(2 * w == c)), int(np.sum(w == c))
    ns, nb = len(small), len(big)
    kk = min(cut, len(w))
    K = 2 * nb + nh + 2 * nf
    D = int(small.sum()) - int((c - big).sum())
    alpha = 2 * D - c * (2 * kk - K)
    beta = 2 * ns * (c - 1) + c * (2 * kk - K) - c * (2 * ns - 2 * nb + 1) + 2
    if alpha >= 0 or 2 * alpha + beta <= 0:
        return None
    lmax = min(c, (beta - 1) // (-alpha))
    U = (c - 1) // 2
    return lmax if U * lmax * lmax // (2 * c) + lmax <= budget else None


def test_cluster_vb2_long_parameters(cudalib, orc):
    """Sizes uniform over [1, c] at c = 10^5, n = 10^4: the cut of MT, RAD2
    and CCM1 leaves VB2 parameters up to 1 000-2 800 on the cluster's count
    table (cluster_vb2: a thread per parameter below 512, a warp per
    parameter above, each CTA summing the terms in its own slice) and up to
    4 800-6 000 (beyond the second plan's budget) to the generic kernel;
    bound and argmax equal the oracle's, and the same with cluster tables
    off."""
    c = 100_000
    full = I.large_instances("uniform_full", c, count=64, n=10_000, seed=2, dtype=np.int32)
    pick = [21, 25, 45, 55, 56, 0]
    inst = [np.asarray(full.instance(j)) for j in pick]
    rg = I.ragged_from_list(inst, [c] * len(pick))
    rg.bins = np.zeros(rg.count, np.int64)
    with cf.ThreadPoolExecutor(len(pick)) as ex:
        want = list(ex.map(lambda w: orc.lb(w, c, 0), inst))
        ucut = list(ex.map(lambda w: max(orc.lb_dff(d, w, c)[0] for d in (0, 1, 3)), inst))
    lm = [_late_lmax(w, c, u) for w, u in zip(inst, ucut)]
    assert sum(1 for x in lm if x is not None and x >= 1000) >= 3, lm
    want = tuple(np.array(x) for x in zip(*want))
    h = cluster_handle(cudalib)
    try:
        assert_same(run_batch(cudalib, h, rg), want, "cluster tables on")
        cudalib.bp_lb_set_cluster_tables(h, False)
        assert_same(run_batch(cudalib, h, rg), want, "cluster tables off")
    finally:
        cudalib.bp_lb_destroy(h)
