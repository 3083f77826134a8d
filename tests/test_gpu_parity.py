"""Bit-exact parity of the CUDA path with the CPU oracle (bound, argmax, verdict),
through the C ABI.  Sizes span several lambda-tiles, several item chunks and
ragged tails; full-size workloads are checked on sampled outputs."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

pytestmark = pytest.mark.gpu


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def to_dev(x, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def run_batch(cudalib, h, rg: I.Ragged, i64=False):
    import torch
    B = rg.count
    out_b = torch.empty(B, dtype=torch.int64, device="cuda")
    out_a = cudalib.argmax_tensor(B)
    out_f = torch.empty(B, dtype=torch.uint8, device="cuda")
    sizes = to_dev(rg.sizes.astype(np.int64 if i64 else np.int32))
    cudalib.bp_lb_eval_batch(h, to_dev(rg.offsets.astype(np.int64)), sizes,
                             to_dev(rg.capacity.astype(np.int64)), to_dev(rg.bins.astype(np.int64)),
                             out_b, out_a, out_f)
    torch.cuda.synchronize()
    d, lam = cudalib.decode_argmax(out_a)
    return out_b.cpu().numpy(), d, lam, out_f.cpu().numpy().astype(bool)


def node_tensors(nd: I.Nodes):
    return dict(base_offsets=to_dev(nd.base.offsets.astype(np.int64)),
                base_sizes=to_dev(nd.base.sizes.astype(np.int32)),
                base_capacity=to_dev(nd.base.capacity.astype(np.int64)),
                node_base=to_dev(nd.node_base.astype(np.int32)),
                assign_offsets=to_dev(nd.assign_offsets.astype(np.int64)),
                assign=to_dev(nd.assign.astype(np.int32)),
                bins=to_dev(nd.bins.astype(np.int64)))


def run_nodes(cudalib, h, nd: I.Nodes, max_bins=None):
    import torch
    B = nd.count
    out_b = torch.empty(B, dtype=torch.int64, device="cuda")
    out_a = cudalib.argmax_tensor(B)
    out_f = torch.empty(B, dtype=torch.uint8, device="cuda")
    mb = int(nd.bins.max()) if max_bins is None else max_bins
    cudalib.bp_lb_eval_nodes(h, max_bins=mb, out_bound=out_b, out_argmax=out_a, out_feasible=out_f,
                             **node_tensors(nd))
    torch.cuda.synchronize()
    d, lam = cudalib.decode_argmax(out_a)
    return out_b.cpu().numpy(), d, lam, out_f.cpu().numpy().astype(bool)


def debug_params(cudalib, h, sizes, c, dff, lam):
    import torch
    out = torch.empty(len(dff), dtype=torch.int64, device="cuda")
    cudalib.bp_lb_debug_params(h, to_dev(np.asarray(sizes, np.int32)), c,
                               to_dev(np.asarray(dff, np.int32)), to_dev(np.asarray(lam, np.int64)),
                               out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def assert_same(got, want, what=""):
    gb, gd, gl, gf = got
    wb, wd, wl, wf = want
    bad = np.nonzero((gb != wb) | (gd != wd) | (gl != wl) | (gf != wf))[0]
    assert len(bad) == 0, (f"{what}: {len(bad)} mismatches, first {bad[:5]}: got "
                           f"{[(gb[i], gd[i], gl[i], gf[i]) for i in bad[:3]]} want "
                           f"{[(wb[i], wd[i], wl[i], wf[i]) for i in bad[:3]]}")


def oracle_batch(orc, rg: I.Ragged):
    b, d, l, f = orc.lb_batch(rg.offsets, rg.sizes.astype(np.int64), rg.capacity, rg.bins)
    return b, d.astype(np.int32), l, f


def oracle_node(orc, nd: I.Nodes, j):
    w, a, c, k = nd.node(j)
    wr = orc.reduce(w, a, k, c)
    b, d, l, f = orc.lb(wr, c, k)
    return b, d, l, f


def random_ragged(rng, B, c_lo, c_hi, n_hi, zero_full=True):
    inst, caps = [], []
    for _ in range(B):
        c = int(rng.integers(c_lo, c_hi + 1))
        n = int(rng.integers(0, n_hi + 1))
        w = rng.integers(0, c + 1, size=n)
        if zero_full and n:
            m = rng.random(n)
            w[m < 0.05] = 0
            w[(m >= 0.05) & (m < 0.1)] = c
            if c % 2 == 0:
                w[(m >= 0.1) & (m < 0.15)] = c // 2
        inst.append(w)
        caps.append(c)
    rg = I.ragged_from_list(inst, caps)
    rg.bins = rng.integers(0, 60, size=B).astype(np.int64)
    return rg


# ---------------------------------------------------------------------------
# plain path
# ---------------------------------------------------------------------------
def test_plain_single_check(cudalib, orc):
    rg = I.plain_single()
    c, k, w = int(rg.capacity[0]), int(rg.bins[0]), rg.instance(0)
    h = cudalib.bp_lb_create(c, 1024)
    try:
        got = cudalib.bp_lb_eval(h, w, k)
        b, d, l, f = orc.lb(w, c, k)
        assert got == (b, d, l)
        # repeated calls give the same answer (scratch is self-cleaning)
        for _ in range(3):
            assert cudalib.bp_lb_eval(h, w, k) == got
        # empty instance
        assert cudalib.bp_lb_eval(h, [], 0) == (0, 0, 0)
        with pytest.raises(cudalib.BpLbError):
            cudalib.bp_lb_eval(h, [c + 1], 1)
    finally:
        cudalib.bp_lb_destroy(h)


@pytest.mark.parametrize("c", [1, 2, 3, 5, 6, 8, 13, 150, 1000, 9999, 65535, 65536, 70001])
def test_plain_random(cudalib, orc, c):
    rng = np.random.default_rng(c)
    h = cudalib.bp_lb_create(c, 4096)
    try:
        for _ in range(4 if c < 60000 else 2):
            n = int(rng.integers(0, 40 if c < 60000 else 12))
            w = rng.integers(0, c + 1, size=n)
            k = int(rng.integers(0, 20))
            got = cudalib.bp_lb_eval(h, w, k)
            b, d, l, f = orc.lb(w, c, k)
            assert got == (b, d, l), (c, list(w))
    finally:
        cudalib.bp_lb_destroy(h)


def test_plain_node(cudalib, orc):
    nd = I.search_nodes(nodes=24)
    h = cudalib.bp_lb_create(10_000, 4096)
    try:
        for j in range(nd.count):
            w, a, c, k = nd.node(j)
            got = cudalib.bp_lb_eval_node(h, w, a, k)
            b, d, l, _ = oracle_node(orc, nd, j)
            assert got == (b, d, l), j
        # an overfull bin is a domain error
        w, a, c, k = nd.node(0)
        a = np.zeros_like(a)
        with pytest.raises(cudalib.BpLbError) as e:
            cudalib.bp_lb_eval_node(h, w, a, k)
        assert e.value.status == cudalib.BP_ERANGE
    finally:
        cudalib.bp_lb_destroy(h)


# ---------------------------------------------------------------------------
# batched path
# ---------------------------------------------------------------------------
def test_batch_random_small(cudalib, handle, orc):
    rng = np.random.default_rng(1)
    rg = random_ragged(rng, 400, 1, 400, 60)
    assert_same(run_batch(cudalib, handle, rg), oracle_batch(orc, rg), "small")


def test_batch_int64_sizes(cudalib, handle, orc):
    rng = np.random.default_rng(2)
    rg = random_ragged(rng, 100, 1, 3000, 80)
    want = oracle_batch(orc, rg)
    assert_same(run_batch(cudalib, handle, rg, i64=True), want, "i64")
    assert_same(run_batch(cudalib, handle, rg, i64=False), want, "i32")


def test_batch_fast_path_boundaries(cudalib, handle, orc):
    """Capacities on both sides of every fast-path limit of the kernel."""
    rng = np.random.default_rng(3)
    caps = [65534, 65535, 65536, 65537, 131071, 131072, 131073]
    inst = [rng.integers(0, c + 1, size=int(rng.integers(1, 9))) for c in caps]
    rg = I.ragged_from_list(inst, caps)
    assert_same(run_batch(cudalib, handle, rg), oracle_batch(orc, rg), "boundaries")


def test_batch_multi_tile_multi_chunk(cudalib, handle, orc):
    """c = 10^4 (about 31 lambda tiles) and r up to 4500 items (three staging chunks)."""
    rng = np.random.default_rng(4)
    inst = [rng.integers(1, 5001, size=n) for n in (1, 2047, 2048, 2049, 4500)]
    inst.append(rng.integers(0, 10_001, size=3001))
    rg = I.ragged_from_list(inst, [10_000] * len(inst))
    assert_same(run_batch(cudalib, handle, rg), oracle_batch(orc, rg), "multi")


def test_batch_degenerate(cudalib, handle, orc):
    inst = [[], [0, 0, 0], [5, 5, 5], [1], [3, 3, 3], [2, 2], [4] * 9, [0], [7, 0, 7]]
    caps = [5, 5, 5, 1, 5, 4, 8, 9, 7]
    rg = I.ragged_from_list(inst, caps)
    assert_same(run_batch(cudalib, handle, rg), oracle_batch(orc, rg), "degenerate")
    # every capacity from 1 to 40 with a few items each
    rng = np.random.default_rng(5)
    inst = [rng.integers(0, c + 1, size=int(rng.integers(0, 7))) for c in range(1, 41)]
    rg = I.ragged_from_list(inst, list(range(1, 41)))
    assert_same(run_batch(cudalib, handle, rg), oracle_batch(orc, rg), "tiny capacities")


def test_batch_domain_errors(cudalib, handle, orc):
    inst = [[1, 2], [1, 9], [1, 2], [-1, 2], [3], [1, 2]]
    rg = I.ragged_from_list(inst, [8, 8, 0, 8, 8, 8], bins=[1, 1, 1, 1, -1, 2])
    b, d, l, f = run_batch(cudalib, handle, rg)
    assert list(b) [:5] == [orc.lb([1, 2], 8, 1)[0], -2, -2, -2, -2]
    assert list(d[1:5]) == [-1] * 4 and not f[1:5].any()
    assert b[5] == orc.lb([1, 2], 8, 2)[0]


def test_batch_alone_equals_in_batch(cudalib, handle, orc):
    rng = np.random.default_rng(6)
    rg = random_ragged(rng, 50, 1, 2000, 200)
    whole = run_batch(cudalib, handle, rg)
    for b in range(0, 50, 7):
        one = I.ragged_from_list([rg.instance(b)], [rg.capacity[b]], [rg.bins[b]])
        got = run_batch(cudalib, handle, one)
        assert tuple(x[0] for x in got) == tuple(x[b] for x in whole)


def test_large_capacity_sampled(cudalib, handle, orc):
    """Capacities past the fp32 and 32-bit fast paths (up to 2^30): lambda-sampled
    per-parameter bounds against the oracle's per-parameter bound."""
    rng = np.random.default_rng(7)
    for c in (4194303, 4194304, 4194305, 21262214, 21262215, 2 ** 28, 2 ** 28 + 1, 2 ** 30):
        w = rng.integers(0, c + 1, size=int(rng.integers(1, 40)))
        dff, lam = [], []
        for d in range(6):
            lo, hi, n = orc.param_range(d, c)
            if n == 0:
                continue
            ls = set(rng.integers(lo, hi + 1, size=40).tolist()) | {lo, hi, min(hi, lo + 1)}
            for l in sorted(ls):
                dff.append(d)
                lam.append(l)
        got = debug_params(cudalib, handle, w, c, dff, lam)
        want = [orc.lb_param(d, l, w, c) for d, l in zip(dff, lam)]
        assert list(got) == want, c


def test_debug_params_rejects_bad_lambda(cudalib, handle):
    got = debug_params(cudalib, handle, [3, 4], 10, [0, 1, 6, 3], [6, 2, 1, 5])
    assert got[0] == -2 and got[1] == -2 and got[2] == -2 and got[3] >= 0


# ---------------------------------------------------------------------------
# search nodes (device reduction fused into the evaluation)
# ---------------------------------------------------------------------------
def test_nodes_search_batch_full_size_sampled(cudalib, handle, orc):
    """The 4096-node search batch (n = 500, c = 10^4) in the benchmark's launch
    configuration; 48 sampled nodes against the oracle (reduction + bound)."""
    nd = I.search_nodes()
    got = run_nodes(cudalib, handle, nd)
    rng = np.random.default_rng(8)
    for j in sorted(rng.choice(nd.count, size=48, replace=False)):
        want = oracle_node(orc, nd, j)
        assert (got[0][j], got[1][j], got[2][j], got[3][j]) == want, j


def test_nodes_small_exhaustive(cudalib, handle, orc):
    nd = I.ragged_nodes(seed=9, count=300, n_lo=1, n_hi=300, caps=(6, 7, 150, 1000, 4999))
    got = run_nodes(cudalib, handle, nd)
    want = [oracle_node(orc, nd, j) for j in range(nd.count)]
    want = tuple(np.array(x) for x in zip(*want))
    assert_same(got, want, "nodes")


def test_nodes_errors(cudalib, handle, orc):
    nd = I.search_nodes(nodes=4)
    nd.assign = nd.assign.copy()
    k = int(nd.bins[0])
    nd.assign[nd.assign_offsets[1]:nd.assign_offsets[2]] = 0          # node 1: overfull bin 0
    nd.assign[nd.assign_offsets[2]] = k                                # node 2: bin out of range
    got = run_nodes(cudalib, handle, nd)
    assert got[0][1] == -2 and got[0][2] == -2
    for j in (0, 3):
        assert (got[0][j], got[1][j], got[2][j], got[3][j]) == oracle_node(orc, nd, j)


def test_reduce_nodes_exact(cudalib, handle, orc):
    import torch
    nd = I.ragged_nodes(seed=10, count=200, n_lo=0, n_hi=400, caps=(150, 1000))
    B = nd.count
    n = np.diff(nd.assign_offsets)
    cap_r = n + nd.bins
    out_off = np.zeros(B, np.int64)
    out_off[1:] = np.cumsum(cap_r)[:-1]
    out_sizes = torch.full((int(cap_r.sum()) + 1,), -7, dtype=torch.int32, device="cuda")
    out_count = torch.empty(B, dtype=torch.int64, device="cuda")
    t = node_tensors(nd)
    cudalib.bp_lb_reduce_nodes(handle, t["base_offsets"], t["base_sizes"], t["base_capacity"],
                               t["node_base"], t["assign_offsets"], t["assign"], t["bins"],
                               int(nd.bins.max()), to_dev(out_off), out_sizes, out_count)
    torch.cuda.synchronize()
    cnt = out_count.cpu().numpy()
    sz = out_sizes.cpu().numpy()
    for j in range(B):
        w, a, c, k = nd.node(j)
        want = orc.reduce(w, a, k, c)
        assert cnt[j] == len(want), j
        assert np.array_equal(sz[out_off[j]:out_off[j] + cnt[j]], want), j


# ---------------------------------------------------------------------------
# every compiled launch shape, and the autotuner
# ---------------------------------------------------------------------------
def test_every_launch_shape_is_exact(cudalib, orc):
    rng = np.random.default_rng(11)
    rg = random_ragged(rng, 120, 1, 5000, 300)
    rg.sizes = rg.sizes.astype(np.int64)
    want = oracle_batch(orc, rg)
    nd = I.ragged_nodes(seed=12, count=60, n_lo=1, n_hi=2600, caps=(150, 1000, 9000))
    want_nodes = tuple(np.array(x) for x in zip(*[oracle_node(orc, nd, j) for j in range(nd.count)]))
    h = cudalib.bp_lb_create(150, 4096)
    try:
        for shape in range(cudalib.bp_lb_num_launch_shapes()):
            for mode in (cudalib.MODE_RAGGED_I32, cudalib.MODE_RAGGED_I64, cudalib.MODE_NODES,
                         cudalib.MODE_PLAIN_RAGGED, cudalib.MODE_PLAIN_NODES):
                cudalib.bp_lb_set_launch_shape(h, mode, shape)
            assert_same(run_batch(cudalib, h, rg), want, f"shape {shape} i32")
            assert_same(run_batch(cudalib, h, rg, i64=True), want, f"shape {shape} i64")
            assert_same(run_nodes(cudalib, h, nd), want_nodes, f"shape {shape} nodes")
            w = rg.instance(3)
            assert cudalib.bp_lb_eval(h, w[w <= 150], 7)[0] == orc.lb(w[w <= 150], 150, 7)[0]
            wn, an, cn, kn = nd.node(5)
            if cn == 150:
                assert cudalib.bp_lb_eval_node(h, wn, an, kn)[:3] == oracle_node(orc, nd, 5)[:3]
    finally:
        cudalib.bp_lb_destroy(h)


def test_autotune_plain_node(cudalib, orc):
    nd = I.search_nodes(nodes=4)
    h = cudalib.bp_lb_create(10_000, 4096)
    try:
        w, a, c, k = nd.node(1)
        best, us = cudalib.bp_lb_autotune_plain_node(h, w, a, k, reps=3)
        nshapes = cudalib.bp_lb_num_launch_shapes()
        assert len(us) == 2 * nshapes and us[best] == min(us)
        assert cudalib.bp_lb_get_launch_shape(h, cudalib.MODE_PLAIN_NODES) == best % nshapes
        assert cudalib.bp_lb_eval_node(h, w, a, k) == oracle_node(orc, nd, 1)[:3]
    finally:
        cudalib.bp_lb_destroy(h)


def test_autotune_nodes(cudalib, handle, orc):
    import torch
    nd = I.search_nodes(nodes=256)
    t = node_tensors(nd)
    out_b = torch.empty(nd.count, dtype=torch.int64, device="cuda")
    out_a = cudalib.argmax_tensor(nd.count)
    best, ms = cudalib.bp_lb_autotune_nodes(handle, max_bins=int(nd.bins.max()), out_bound=out_b,
                                            out_argmax=out_a, reps=2, **t)
    assert 0 <= best < cudalib.bp_lb_num_launch_shapes()
    assert all(x > 0 for x in ms) and ms[best] == min(ms)
    assert cudalib.bp_lb_get_launch_shape(handle, cudalib.MODE_NODES) == best
    for j in (0, 100, 255):
        assert (int(out_b[j]),) == (oracle_node(orc, nd, j)[0],)


# ---------------------------------------------------------------------------
# prefix-count variant (default) and direct evaluation give identical results
# ---------------------------------------------------------------------------
def test_prefix_and_direct_match_oracle(cudalib, orc):
    rng = np.random.default_rng(13)
    caps = [1, 2, 3, 7, 150, 999, 4096, 12286, 12287, 24000, 24574, 24575, 70000]
    inst = [rng.integers(0, c + 1, size=int(rng.integers(0, 60 if c < 20000 else 20)))
            for c in caps]
    # zeros, full and half items
    inst[5][:3] = [0, 999, 499] if len(inst[5]) >= 3 else inst[5][:3]
    # equal sizes: many parameters tie at the maximum (first index must win)
    for c in (96, 1000, 5040, 12285):
        for w in (1, c // 3 + 1, c // 2, c // 4, c - 1, c):
            caps.append(c)
            inst.append(np.full(int(rng.integers(1, 40)), w))
    rg = I.ragged_from_list(inst, caps)
    want = oracle_batch(orc, rg)
    nd = I.ragged_nodes(seed=14, count=80, n_lo=1, n_hi=3000, caps=(150, 1000, 9999, 12286))
    want_nodes = tuple(np.array(x) for x in zip(*[oracle_node(orc, nd, j) for j in range(nd.count)]))
    h = cudalib.bp_lb_create(4096, 4096)
    try:
        for algo in (cudalib.ALGO_DIRECT, cudalib.ALGO_PREFIX):
            cudalib.bp_lb_set_algorithm(h, algo)
            assert cudalib.bp_lb_get_algorithm(h) == algo
            assert_same(run_batch(cudalib, h, rg), want, f"algo {algo} ragged")
            assert_same(run_nodes(cudalib, h, nd), want_nodes, f"algo {algo} nodes")
            w = inst[6]
            assert cudalib.bp_lb_eval(h, w, 3)[:3] == orc.lb(w, 4096, 3)[:3]
    finally:
        cudalib.bp_lb_destroy(h)


# ---------------------------------------------------------------------------
# the prefix-count kernel beside the VB2 kernel (default) or after it
# ---------------------------------------------------------------------------
def test_overlap_and_serial_identical(cudalib, orc):
    nd = I.ragged_nodes(seed=19, count=300, n_lo=1, n_hi=2500, caps=(150, 1000, 9999, 30000))
    rng = np.random.default_rng(19)
    rg = random_ragged(rng, 120, 1, 20000, 400)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        got = {}
        for pc in (0, 1, 2, 4):
            cudalib.bp_lb_set_overlap(h, pc)
            got[pc] = (run_nodes(cudalib, h, nd), run_batch(cudalib, h, rg))
        for pc in (1, 2, 4):
            for a, b in zip(got[pc], got[0]):
                for x, y in zip(a, b):
                    assert np.array_equal(x, y), pc
        for j in range(0, nd.count, 23):
            assert (int(got[2][0][0][j]),) == (oracle_node(orc, nd, j)[0],)
        assert_same(got[2][1], oracle_batch(orc, rg), "overlap batch")
        with pytest.raises(cudalib.BpLbError):
            cudalib.bp_lb_set_overlap(h, 9)
    finally:
        cudalib.bp_lb_destroy(h)


def test_prefix_long_stream_unmerged(cudalib, handle, orc):
    """A stream of 2^15 items or more: the prefix kernel's per-DFF tiles (the
    merged u-group tile needs 16-bit counts)."""
    rng = np.random.default_rng(29)
    inst = [rng.integers(1, 1001, size=40000), rng.integers(1, 501, size=33000),
            rng.integers(1, 1001, size=300)]
    rg = I.ragged_from_list(inst, [1000, 1000, 1000])
    assert_same(run_batch(cudalib, handle, rg), oracle_batch(orc, rg), "long streams")


@pytest.mark.parametrize("count", [4095, 4096, 4097, 8193])
def test_plan_pass_boundaries(cudalib, orc, count):
    """Batches just below, at and above one planner pass (1024 threads x 4
    instances; one pass also makes VB2's tile table, more take a second):
    every instance's bound, argmax and verdict against the oracle."""
    rng = np.random.default_rng(count)
    caps = [int(c) for c in rng.choice([150, 151, 1000, 4999], size=count)]
    inst = [rng.integers(1, c // 2 + 1, size=int(rng.integers(1, 30))) for c in caps]
    rg = I.ragged_from_list(inst, caps)
    rg.bins = rng.integers(0, 20, size=count).astype(np.int64)
    want = oracle_batch(orc, rg)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        assert_same(run_batch(cudalib, h, rg), want, "pass boundary %d" % count)
    finally:
        cudalib.bp_lb_destroy(h)
