"""Verdict-only mode (Alg. 2's early exit): the verdict bound <= k is exact for
every instance; the reported bound and argmax are a genuine (DFF, lambda)
bound of the instance -- above k exactly when the instance is infeasible."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

from test_gpu_parity import oracle_batch, oracle_node, run_batch, run_nodes

pytestmark = pytest.mark.gpu


def check_verdicts(orc, rg_or_nodes, got, want, caps, witness_sizes, what):
    gb, gd, gl, gf = got
    wb, wd, wl, wf = want
    bad = np.nonzero(gf != wf)[0]
    assert len(bad) == 0, f"{what}: verdict mismatches at {bad[:5]}"
    for j in range(len(gb)):
        k = int(rg_or_nodes.bins[j])
        assert (gb[j] > k) == (not gf[j]), (what, j)
        assert gb[j] <= wb[j], (what, j)          # never above the maximum
        # the witness is a real bound of the instance
        assert orc.lb_param(int(gd[j]), int(gl[j]), witness_sizes(j), caps[j]) == gb[j], (what, j)


def mixed_ragged(orc, seed, count=160):
    """Reduced search-node instances with k around their bound: about half
    infeasible, half feasible."""
    rng = np.random.default_rng(seed)
    inst, caps = [], []
    for _ in range(count):
        c = int(rng.choice([150, 1000, 9999, 20000, 70000]))
        n = int(rng.integers(1, 900 if c < 50000 else 200))
        w = I.uniform_sizes(rng, n, 1, c)
        inst.append(w)
        caps.append(c)
    rg = I.ragged_from_list(inst, caps)
    full = oracle_batch(orc, rg)[0]
    rg.bins = np.maximum(0, full + rng.integers(-2, 2, size=count)).astype(np.int64)
    return rg


@pytest.mark.parametrize("algo", [0, 1])
def test_verdict_batch_mixed(cudalib, orc, algo):
    rg = mixed_ragged(orc, 41)
    want = oracle_batch(orc, rg)
    assert 0 < int(np.sum(~want[3])) < rg.count            # both verdicts occur
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_algorithm(h, algo)
        cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_VERDICT)
        assert cudalib.bp_lb_get_result_mode(h) == cudalib.RESULT_VERDICT
        for shape in (0, 5, 7):
            cudalib.bp_lb_set_launch_shape(h, cudalib.MODE_RAGGED_I32, shape)
            got = run_batch(cudalib, h, rg)
            check_verdicts(orc, rg, got, want, rg.capacity, rg.instance, f"algo {algo} shape {shape}")
        # back to the full maximum: exact bound and argmax again
        cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_FULL)
        got = run_batch(cudalib, h, rg)
        for x, y in zip(got, want):
            assert np.array_equal(np.asarray(x), np.asarray(y))
    finally:
        cudalib.bp_lb_destroy(h)


def test_verdict_nodes_search_batch(cudalib, orc):
    """The search-node workload in verdict mode (every node feasible there: the
    VB2 parameters whose upper bound is <= k are skipped)."""
    nd = I.search_nodes(seed=1, n=500, c=10_000, nodes=256)
    want = tuple(np.array(x) for x in zip(*[oracle_node(orc, nd, j) for j in range(nd.count)]))
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_VERDICT)
        got = run_nodes(cudalib, h, nd)

        def reduced(j):
            w, a, c, k = nd.node(j)
            return orc.reduce(w, a, k, c)
        check_verdicts(orc, nd, got, want, [10_000] * nd.count, reduced, "nodes")
    finally:
        cudalib.bp_lb_destroy(h)


def test_verdict_nodes_tight_bins(cudalib, orc):
    """Nodes whose k is the number of bins already used: many infeasible."""
    nd = I.ragged_nodes(seed=17, count=120, n_lo=20, n_hi=1500, caps=(150, 1000, 9999),
                        frac_hi=0.9)
    for j in range(nd.count):
        a = nd.assign[nd.assign_offsets[j]:nd.assign_offsets[j + 1]]
        nd.bins[j] = max(int(a.max()) + 1, 1)
    want = tuple(np.array(x) for x in zip(*[oracle_node(orc, nd, j) for j in range(nd.count)]))
    assert int(np.sum(~want[3])) > 0
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_VERDICT)
        got = run_nodes(cudalib, h, nd)

        def reduced(j):
            w, a, c, k = nd.node(j)
            return orc.reduce(w, a, k, c)
        caps = [int(nd.base.capacity[nd.node_base[j]]) for j in range(nd.count)]
        check_verdicts(orc, nd, got, want, caps, reduced, "tight nodes")
    finally:
        cudalib.bp_lb_destroy(h)


def test_verdict_plain_and_long_instance(cudalib, orc):
    """The plain path and an instance longer than one staging chunk."""
    rng = np.random.default_rng(5)
    c = 5000
    w = I.uniform_sizes(rng, 6000, 1, c // 2)
    full = orc.lb(w, c, 0)[0]
    h = cudalib.bp_lb_create(c, 1 << 14)
    try:
        cudalib.bp_lb_set_result_mode(h, cudalib.RESULT_VERDICT)
        for k in (full - 1, full, full + 1):
            got = cudalib.bp_lb_eval(h, w, k)       # (bound, dff, lambda)
            assert (got[0] > k) == (full > k)
            assert orc.lb_param(got[1], got[2], w, c) == got[0]
        rg = I.ragged_from_list([w, w, w], [c, c, c])
        rg.bins = np.array([full - 1, full, full + 1], dtype=np.int64)
        got = run_batch(cudalib, h, rg)
        assert list(got[3]) == [False, True, True]
        for j in range(3):
            assert orc.lb_param(int(got[1][j]), int(got[2][j]), w, c) == got[0][j]
    finally:
        cudalib.bp_lb_destroy(h)
