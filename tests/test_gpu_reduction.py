"""Reduction variants of the search-node mode (bp_lb_set_reduction,
bp_lb_set_bin_max; not defined in the paper): the device results -- bound,
argmax, verdict, and the reduced instances of bp_lb_reduce_nodes -- equal the
oracle's restatement (orc_reduce_ex, whose validity tests/test_oracle_reduction.py
pins by brute force) on every node."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

from test_gpu_parity import node_tensors, run_nodes, to_dev

pytestmark = pytest.mark.gpu


def large_item_nodes(seed, count=160, caps=(150, 1000, 9999)):
    """Search nodes whose items are all large (U[c/5, c/2]) and mostly packed,
    so that many bins have less free space than the smallest unpacked item."""
    rng = np.random.default_rng(seed)
    sizes, cs, ks = [], [], []
    for _ in range(count):
        c = int(rng.choice(caps))
        n = int(rng.integers(5, 400))
        w = rng.integers(c // 5, c // 2 + 1, size=n)
        sizes.append(w)
        cs.append(c)
        ks.append(I.bins_for(w, c) + int(rng.integers(0, 3)))
    base = I.ragged_from_list(sizes, cs, bins=ks)
    assigns = I.prepack(rng, sizes, cs, ks, 0.95)
    return I._nodes_from(base, np.arange(count), assigns, ks)


def nodes_with_caps(seed, count=160, caps=(150, 1000, 9999)):
    """Nodes and per-bin maximum loads: each bin's cap lies between its
    packed load and c, mostly near c; some bins get exactly their load."""
    rng = np.random.default_rng(seed)
    nd = large_item_nodes(seed, count, caps)
    offs = np.zeros(nd.count + 1, np.int64)
    offs[1:] = np.cumsum(nd.bins)
    bin_max = np.zeros(int(offs[-1]), np.int32)
    for j in range(nd.count):
        w, a, c, k = nd.node(j)
        load = np.bincount(a[a >= 0], weights=w[a >= 0], minlength=k).astype(np.int64)
        cap = c - ((c - load) * rng.random(k) * 0.3).astype(np.int64)
        tight = rng.random(k) < 0.05
        cap[tight] = load[tight]
        bin_max[offs[j]:offs[j + 1]] = np.clip(cap, load, c)
    return nd, offs, bin_max


def oracle_nodes(orc, nd, mode, offs=None, bin_max=None):
    out = []
    for j in range(nd.count):
        w, a, c, k = nd.node(j)
        bm = None if bin_max is None else bin_max[offs[j]:offs[j + 1]]
        red = orc.reduce_ex(w, a, k, c, mode, bm)
        out.append(orc.lb(red, c, k))
    return tuple(np.array(x) for x in zip(*out))


def same(got, want, what):
    for x, y in zip(got, want):
        assert np.array_equal(np.asarray(x), np.asarray(y)), what


@pytest.mark.parametrize("algo", [1, 0])
def test_close_mode_batched_and_plain(cudalib, orc, algo):
    nd = large_item_nodes(31)
    want = oracle_nodes(orc, nd, 1)
    assert int(np.sum(want[0] != oracle_nodes(orc, nd, 0)[0])) >= 5   # closing matters here
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_algorithm(h, algo)
        cudalib.bp_lb_set_reduction(h, cudalib.REDUCE_CLOSE)
        assert cudalib.bp_lb_get_reduction(h) == cudalib.REDUCE_CLOSE
        same(run_nodes(cudalib, h, nd), want, f"close, algo {algo}")
        for j in range(0, nd.count, 16):             # the plain node path
            w, a, c, k = nd.node(j)
            hp = cudalib.bp_lb_create(c, 4096)
            cudalib.bp_lb_set_reduction(hp, cudalib.REDUCE_CLOSE)
            assert cudalib.bp_lb_eval_node(hp, w, a, k) == (want[0][j], want[1][j], want[2][j])
            cudalib.bp_lb_destroy(hp)
        cudalib.bp_lb_set_reduction(h, cudalib.REDUCE_LOADS)
        same(run_nodes(cudalib, h, nd), oracle_nodes(orc, nd, 0), "loads")
    finally:
        cudalib.bp_lb_destroy(h)


@pytest.mark.parametrize("mode", [0, 1])
def test_bin_max_batched(cudalib, orc, mode):
    nd, offs, bin_max = nodes_with_caps(32 + mode)
    want = oracle_nodes(orc, nd, mode, offs, bin_max)
    d_offs, d_bm = to_dev(offs), to_dev(bin_max)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_reduction(h, mode)
        cudalib.bp_lb_set_bin_max(h, d_offs, d_bm)
        for algo in (1, 0):
            cudalib.bp_lb_set_algorithm(h, algo)
            same(run_nodes(cudalib, h, nd), want, f"caps, mode {mode}, algo {algo}")
        cudalib.bp_lb_set_bin_max(h)                   # cleared: the plain loads again
        same(run_nodes(cudalib, h, nd), oracle_nodes(orc, nd, mode), "cleared")
    finally:
        cudalib.bp_lb_destroy(h)


def test_bin_max_below_load_is_an_error(cudalib, orc):
    nd, offs, bin_max = nodes_with_caps(35, count=40)
    bad = None
    for j in range(nd.count):
        w, a, c, k = nd.node(j)
        load = np.bincount(a[a >= 0], weights=w[a >= 0], minlength=k)
        nz = np.nonzero(load > 0)[0]
        if len(nz):
            bin_max[offs[j] + nz[0]] = int(load[nz[0]]) - 1
            bad = j
            break
    assert bad is not None
    d_offs, d_bm = to_dev(offs), to_dev(bin_max)   # alive while set on the handle
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_bin_max(h, d_offs, d_bm)
        got = run_nodes(cudalib, h, nd)
        assert got[0][bad] == -cudalib.BP_ERANGE
        for j in range(nd.count):
            if j != bad:
                w, a, c, k = nd.node(j)
                red = orc.reduce_ex(w, a, k, c, 0, bin_max[offs[j]:offs[j + 1]])
                assert got[0][j] == orc.lb(red, c, k)[0]
    finally:
        cudalib.bp_lb_destroy(h)


@pytest.mark.parametrize("mode", [0, 1])
def test_reduce_nodes_variants(cudalib, orc, mode):
    import torch
    nd, offs, bin_max = nodes_with_caps(36 + mode, count=120, caps=(150, 1000))
    B = nd.count
    cap_r = np.diff(nd.assign_offsets) + nd.bins
    out_off = np.zeros(B, np.int64)
    out_off[1:] = np.cumsum(cap_r)[:-1]
    out_sizes = torch.full((int(cap_r.sum()) + 1,), -7, dtype=torch.int32, device="cuda")
    out_count = torch.empty(B, dtype=torch.int64, device="cuda")
    t = node_tensors(nd)
    d_offs, d_bm = to_dev(offs), to_dev(bin_max)   # alive while set on the handle
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_reduction(h, mode)
        for caps in (False, True):
            if caps:
                cudalib.bp_lb_set_bin_max(h, d_offs, d_bm)
            cudalib.bp_lb_reduce_nodes(h, t["base_offsets"], t["base_sizes"], t["base_capacity"],
                                       t["node_base"], t["assign_offsets"], t["assign"], t["bins"],
                                       int(nd.bins.max()), to_dev(out_off), out_sizes, out_count)
            torch.cuda.synchronize()
            cnt, sz = out_count.cpu().numpy(), out_sizes.cpu().numpy()
            for j in range(B):
                w, a, c, k = nd.node(j)
                want = orc.reduce_ex(w, a, k, c, mode, bin_max[offs[j]:offs[j + 1]] if caps else None)
                assert cnt[j] == len(want), (j, caps)
                assert np.array_equal(sz[out_off[j]:out_off[j] + cnt[j]], want), (j, caps)
    finally:
        cudalib.bp_lb_destroy(h)
