"""Sharding over ranks, on CPU with the gloo backend (world size 2): the
checks of a batch split by estimated work with no exchange, and one
instance's parameter range split with a single MAX all-reduce of the packed
key.  The per-rank evaluation here is the oracle (no GPU in these tests);
the host logic is the library's (paper_2402_14821_gb300/shard.py)."""
import os
import socket

import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I
from paper_2402_14821_gb300 import shard


def test_partition_by_work_covers_and_balances():
    rng = np.random.default_rng(0)
    work = rng.integers(1, 10_000, size=257)
    for world in (1, 2, 3, 8):
        parts = shard.partition_by_work(work, world)
        assert len(parts) == world
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(len(work)))      # each check once
        loads = [int(work[p].sum()) for p in parts]
        assert max(loads) - min(loads) <= int(work.max())         # LPT bound


def test_param_ranges_and_keys():
    for total, world in ((0, 2), (1, 2), (10, 3), (30_933, 8)):
        r = shard.param_ranges(total, world)
        assert r[0][0] == 0 and r[-1][1] == total
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
    k = shard.make_key(129, 7)
    assert shard.split_key(k) == (129, 7)
    assert shard.make_key(5, 3) > shard.make_key(5, 4) > shard.make_key(4, 0)


def check_work_of_nodes(orc, nd):
    r = [len(orc.reduce(*nd.node(j)[:2], nd.node(j)[3], nd.node(j)[2])) for j in range(nd.count)]
    c = [int(nd.base.capacity[nd.node_base[j]]) for j in range(nd.count)]
    return shard.check_work(r, c)


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        orc = oracle.load()
        # (i) independent checks: each rank evaluates its own shard, no exchange
        nd = I.ragged_nodes(seed=23, count=24, n_lo=5, n_hi=300, caps=(150, 1000))
        parts = shard.partition_by_work(check_work_of_nodes(orc, nd), world)
        mine = {}
        for j in parts[rank]:
            w, a, c, k = nd.node(int(j))
            mine[int(j)] = orc.lb(orc.reduce(w, a, k, c), c, k)
        t = shard.max_over_ranks(float(len(parts[rank])))
        # (ii) one instance over parameter ranges: one MAX all-reduce of the key
        rng = np.random.default_rng(9)
        c = 157
        w = [int(x) for x in rng.integers(1, c + 1, 40)]
        counts = shard.param_counts(c)
        offs = np.concatenate([[0], np.cumsum(counts)])
        g0, g1 = shard.param_ranges(int(offs[-1]), world)[rank]
        best = 0
        for g in range(g0, g1):
            d = int(np.searchsorted(offs, g, side="right") - 1)
            lo = orc.param_range(d, c)[0]
            lam = lo + (g - int(offs[d]))
            best = max(best, shard.make_key(orc.lb_param(d, lam, w, c), g))
        key = shard.allreduce_max_key(best)
        q.put((rank, mine, t, key))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_ranks_gloo(orc):
    pytest.importorskip("torch.distributed")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # (i): the shards together are the whole batch, each check once, and equal
    # the checks evaluated alone
    nd = I.ragged_nodes(seed=23, count=24, n_lo=5, n_hi=300, caps=(150, 1000))
    merged = {}
    for _, mine, _, _ in out:
        assert not set(mine) & set(merged)
        merged.update(mine)
    assert sorted(merged) == list(range(nd.count))
    for j in range(nd.count):
        w, a, c, k = nd.node(j)
        assert merged[j] == orc.lb(orc.reduce(w, a, k, c), c, k)
    # max over ranks of the per-rank times
    assert out[0][2] == out[1][2] == max(float(len(p)) for p in shard.partition_by_work(
        check_work_of_nodes(orc, nd), 2))
    # (ii): the all-reduced key is the full bound and its first argmax
    rng = np.random.default_rng(9)
    c = 157
    w = [int(x) for x in rng.integers(1, c + 1, 40)]
    lb, d, lam, _ = orc.lb(w, c, 0)
    counts = shard.param_counts(c)
    g = sum(counts[:d]) + (lam - orc.param_range(d, c)[0])
    assert out[0][3] == out[1][3] == shard.make_key(lb, g)
