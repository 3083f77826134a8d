"""Full-size workloads against the oracle: the large-instance sweep (n = 10^4,
c in {10^5, 10^6}, three size families, batches of 64, int32 and int64 sizes)
and the ragged batch of 10^4 search nodes replayed from a CUDA graph.  The
oracle recomputes sampled instances whole where it can do so in seconds, and
otherwise sampled parameters one by one; the GPU's argmax must attain its
bound and no sampled parameter may exceed it."""
import concurrent.futures as cf

import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _dev(x, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


def _run_batch(B, h, rg, autotune=False):
    import torch
    tdt = torch.int64 if rg.sizes.dtype == np.int64 else torch.int32
    t = (_dev(rg.offsets, torch.int64), _dev(rg.sizes, tdt), _dev(rg.capacity, torch.int64),
         _dev(rg.bins, torch.int64))
    ob = torch.empty(rg.count, dtype=torch.int64, device="cuda")
    oa = B.argmax_tensor(rg.count)
    of = torch.empty(rg.count, dtype=torch.uint8, device="cuda")
    if autotune:
        B.bp_lb_autotune_batch(h, *t, ob, oa, of, reps=1)
    B.bp_lb_eval_batch(h, *t, ob, oa, of)
    torch.cuda.synchronize()
    d, l = B.decode_argmax(oa)
    return ob.cpu().numpy(), d, l, of.cpu().numpy().astype(bool)


def _debug(B, h, sizes, c, dff, lam):
    import torch
    out = torch.empty(len(dff), dtype=torch.int64, device="cuda")
    B.bp_lb_debug_params(h, _dev(np.asarray(sizes), torch.int32), c,
                         _dev(np.asarray(dff), torch.int32), _dev(np.asarray(lam), torch.int64), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _sample_params(orc, rng, c, m):
    dff, lam = [], []
    for _ in range(m):
        d = int(rng.integers(0, 6))
        lo, hi, n = orc.param_range(d, c)
        if n:
            dff.append(d)
            lam.append(int(rng.integers(lo, hi + 1)))
    return dff, lam


def _check_sampled(B, h, orc, w, c, bound, d_star, l_star, rng, m=120):
    """The argmax attains the bound; sampled parameters agree with the oracle
    and do not exceed the bound."""
    dff, lam = _sample_params(orc, rng, c, m)
    dff.append(int(d_star))
    lam.append(int(l_star))
    got = _debug(B, h, w, c, dff, lam)
    assert got[-1] == bound, (c, d_star, l_star)
    assert np.all(got <= bound)
    want = [orc.lb_param(d, l, w, c) for d, l in zip(dff, lam)]
    assert list(got) == want


@pytest.mark.parametrize("c", [10 ** 5, 10 ** 6])
def test_large_sweep_full_size(cudalib, orc, c):
    B = cudalib
    h = B.bp_lb_create(150, 1024)
    rng = np.random.default_rng(c)
    try:
        for fam in I.FAMILIES:
            for dt in ((np.int32, np.int64) if fam == "uniform_wide" else (np.int32,)):
                rg = I.large_instances(fam, c, count=64, n=10_000, seed=2, dtype=dt)
                b, d, l, f = _run_batch(B, h, rg, autotune=(dt == np.int32))
                assert np.all(b > 0) and np.all(f == (b <= rg.bins))
                for i in rng.choice(64, size=3, replace=False):
                    w = rg.instance(i).astype(np.int64)
                    _check_sampled(B, h, orc, w, c, b[i], d[i], l[i], rng)
                if c == 10 ** 5 and dt == np.int32:
                    # whole instances through the oracle (a few seconds each, in parallel)
                    picks = [0, 31]
                    with cf.ThreadPoolExecutor(len(picks)) as ex:
                        res = list(ex.map(lambda i: orc.lb(rg.instance(i), c, int(rg.bins[i])),
                                          picks))
                    for i, want in zip(picks, res):
                        assert (b[i], d[i], l[i], f[i]) == want, (fam, i)
    finally:
        B.bp_lb_destroy(h)


def test_wide_capacity_whole_instances(cudalib, orc):
    """c = 10^6 (CCM1, BJ1 and VB2 on their wide-capacity paths) with n = 120:
    whole instances through the oracle."""
    B = cudalib
    h = B.bp_lb_create(150, 1024)
    try:
        inst = [I.large_instances(fam, 10 ** 6, count=1, n=120, seed=5).instance(0)
                for fam in I.FAMILIES]
        rg = I.ragged_from_list(inst, [10 ** 6] * len(inst))
        got = _run_batch(B, h, rg)
        with cf.ThreadPoolExecutor(len(inst)) as ex:
            want = list(ex.map(lambda i: orc.lb(inst[i], 10 ** 6, int(rg.bins[i])),
                               range(len(inst))))
        for i, wv in enumerate(want):
            assert tuple(x[i] for x in got) == wv, i
    finally:
        B.bp_lb_destroy(h)


def test_ragged_nodes_graph_full_size(cudalib, orc):
    """The 10^4-node ragged batch (n in [50, 5000], c in {150, 10^3, 10^4, 10^5})
    captured in a CUDA graph and replayed; sampled nodes against the oracle."""
    import torch
    B = cudalib
    nd = I.ragged_nodes(seed=3)
    t_in = dict(base_offsets=_dev(nd.base.offsets, torch.int64),
                base_sizes=_dev(nd.base.sizes, torch.int32),
                base_capacity=_dev(nd.base.capacity, torch.int64),
                node_base=_dev(nd.node_base, torch.int32),
                assign_offsets=_dev(nd.assign_offsets, torch.int64),
                assign=_dev(nd.assign, torch.int32), bins=_dev(nd.bins, torch.int64))
    mb = int(nd.bins.max())
    ob = torch.empty(nd.count, dtype=torch.int64, device="cuda")
    oa = B.argmax_tensor(nd.count)
    of = torch.empty(nd.count, dtype=torch.uint8, device="cuda")
    h = B.bp_lb_create(150, 1024)
    try:
        B.bp_lb_reserve(h, nd.count)
        cs = torch.cuda.Stream()
        with torch.cuda.stream(cs):  # warm-up outside capture
            B.bp_lb_eval_nodes(h, max_bins=mb, out_bound=ob, out_argmax=oa, out_feasible=of,
                               stream=cs, **t_in)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cs):
            B.bp_lb_eval_nodes(h, max_bins=mb, out_bound=ob, out_argmax=oa, out_feasible=of,
                               stream=cs, **t_in)
        ob.fill_(-99)
        g.replay()
        g.replay()
        torch.cuda.synchronize()
        b = ob.cpu().numpy()
        d, l = B.decode_argmax(oa)
        f = of.cpu().numpy().astype(bool)
        assert np.all(b >= 0)
        rng = np.random.default_rng(4)
        caps = nd.base.capacity
        small = [j for j in rng.permutation(nd.count) if caps[j] <= 10_000][:24]

        def whole(j):
            w, a, c, k = nd.node(j)
            return orc.lb(orc.reduce(w, a, k, c), c, k)

        with cf.ThreadPoolExecutor(8) as ex:
            res = list(ex.map(whole, small))
        for j, want in zip(small, res):
            assert (b[j], d[j], l[j], f[j]) == want, j
        big = [j for j in rng.permutation(nd.count) if caps[j] == 100_000][:6]
        for j in big:
            w, a, c, k = nd.node(j)
            wr = orc.reduce(w, a, k, c)
            _check_sampled(B, h, orc, wr, c, b[j], d[j], l[j], rng, m=60)
    finally:
        B.bp_lb_destroy(h)


def test_hard_nodes_full_size(cudalib, orc):
    """The hard search-node batch (4096 partial packings of a triplet instance
    with k = n/3 bins, most nodes with a bound above L1, so that pruning
    against L1 skips little): sampled nodes against the oracle, with pruning
    on and off (identical results), and most bounds above L1."""
    import torch
    B = cudalib
    nd = I.hard_nodes()
    t_in = dict(base_offsets=_dev(nd.base.offsets, torch.int64),
                base_sizes=_dev(nd.base.sizes, torch.int32),
                base_capacity=_dev(nd.base.capacity, torch.int64),
                node_base=_dev(nd.node_base, torch.int32),
                assign_offsets=_dev(nd.assign_offsets, torch.int64),
                assign=_dev(nd.assign, torch.int32), bins=_dev(nd.bins, torch.int64))
    mb = int(nd.bins.max())
    h = B.bp_lb_create(150, 1024)
    try:
        res = []
        for prune in (True, False):
            B.bp_lb_set_pruning(h, prune)
            ob = torch.empty(nd.count, dtype=torch.int64, device="cuda")
            oa = B.argmax_tensor(nd.count)
            of = torch.empty(nd.count, dtype=torch.uint8, device="cuda")
            B.bp_lb_eval_nodes(h, max_bins=mb, out_bound=ob, out_argmax=oa, out_feasible=of,
                               **t_in)
            torch.cuda.synchronize()
            d, l = B.decode_argmax(oa)
            res.append((ob.cpu().numpy(), d, l, of.cpu().numpy().astype(bool)))
        for x, y in zip(*res):
            assert np.array_equal(x, y)
        b, d, l, f = res[0]
        w0, _, c, _ = nd.node(0)
        L1 = -(-int(np.asarray(w0, np.int64).sum()) // c)   # the reduction keeps the total
        assert np.mean(b > L1) > 0.5
        rng = np.random.default_rng(8)
        sample = rng.choice(nd.count, 40, replace=False)

        def whole(j):
            w, a, c, k = nd.node(j)
            return orc.lb(orc.reduce(w, a, k, c), c, k)

        with cf.ThreadPoolExecutor(8) as ex:
            want = list(ex.map(whole, sample))
        for j, wv in zip(sample, want):
            assert (b[j], d[j], l[j], f[j]) == wv, j
    finally:
        B.bp_lb_destroy(h)
