"""One instance evaluated over ranges of its flattened parameter index
(bp_lb_eval_range; the split of one check over GPUs): for random partitions
of [0, P(c)) into 1 to 8 ranges -- empty ranges, ranges inside one DFF and
ranges ending exactly at a DFF's boundary included -- the maximum of the
ranges' packed keys is the full bound and its first argmax, equal to the
oracle's and to bp_lb_eval_batch's; a one-parameter range gives that
parameter's own bound.  Run on one GPU, rank after rank."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I
from paper_2402_14821_gb300 import shard
from test_gpu_parity import run_batch

pytestmark = pytest.mark.gpu


def _dev32(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(x, np.int32))).cuda()


def _key(cudalib, h, sizes, c, g0, g1):
    import torch
    out = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    cudalib.bp_lb_eval_range(h, sizes, c, g0, g1, out)
    torch.cuda.synchronize()
    return int(out.item())


def _full_key(orc, w, c):
    lb, d, lam, _ = orc.lb(w, c, 0)
    g = sum(shard.param_counts(c)[:d]) + lam - orc.param_range(d, c)[0]
    return shard.make_key(lb, g)


def _partitions(rng, P, counts):
    offs = list(np.cumsum([0] + list(counts)))
    yield [0, P]                                            # one range
    yield [0] + offs[1:-1] + [P]                            # one range per DFF
    for world in (2, 3, 5, 8):
        cuts = sorted(int(x) for x in rng.integers(0, P + 1, size=world - 1))
        yield [0] + cuts + [P]                              # random, maybe empty
    yield [0] + [r[0] for r in shard.param_ranges(P, 4)[1:]] + [P]  # even split


@pytest.mark.parametrize("c", [150, 1000, 10_000, 70_000])
def test_range_partitions_give_the_full_key(cudalib, orc, handle, c):
    rng = np.random.default_rng(c)
    counts = shard.param_counts(c)
    P = sum(counts)
    for n in (0, 7, 300):
        w = rng.integers(0, c + 1, size=n)
        d_w = _dev32(w)
        want = _full_key(orc, w, c) if n else shard.make_key(0, 0)
        for cuts in _partitions(rng, P, counts):
            keys = [_key(cudalib, handle, d_w, c, g0, g1) for g0, g1 in zip(cuts[:-1], cuts[1:])]
            assert max(keys) == want, (c, n, cuts)
        # against the batched path too
        if n:
            rg = I.ragged_from_list([w], [c], bins=[0])
            b, d, lam, _ = run_batch(cudalib, handle, rg)
            g = sum(counts[:d[0]]) + lam[0] - orc.param_range(int(d[0]), c)[0]
            assert shard.make_key(b[0], g) == want


def test_one_parameter_ranges(cudalib, orc, handle):
    rng = np.random.default_rng(3)
    c = 1000
    counts = shard.param_counts(c)
    offs = np.concatenate([[0], np.cumsum(counts)])
    w = rng.integers(1, c + 1, size=50)
    d_w = _dev32(w)
    for g in list(offs[:-1]) + list(offs[1:] - 1) + [int(x) for x in rng.integers(0, offs[-1], 30)]:
        g = int(g)
        d = int(np.searchsorted(offs, g, side="right") - 1)
        lam = orc.param_range(d, c)[0] + g - int(offs[d])
        assert _key(cudalib, handle, d_w, c, g, g + 1) == shard.make_key(orc.lb_param(d, lam, w, c), g)


def test_range_large_capacity_split(cudalib, orc, handle):
    """c = 3 * 10^5 (VB2's fp32 path): the ranks' maximum equals the batched
    path's key, and each rank's key is attained inside its own range."""
    rng = np.random.default_rng(11)
    c = 300_000
    w = rng.integers(1, c + 1, size=400)
    d_w = _dev32(w)
    P = sum(shard.param_counts(c))
    rg = I.ragged_from_list([w], [c], bins=[0])
    b, d, lam, _ = run_batch(cudalib, handle, rg)
    g = sum(shard.param_counts(c)[:d[0]]) + lam[0] - orc.param_range(int(d[0]), c)[0]
    keys = []
    for rank, (g0, g1) in enumerate(shard.param_ranges(P, 6)):
        k = _key(cudalib, handle, d_w, c, g0, g1)
        assert g0 <= shard.split_key(k)[1] < g1
        keys.append(k)
        assert shard.rank_key(handle, d_w, c, rank, 6) == k
    assert max(keys) == shard.make_key(b[0], g)


def test_range_errors(cudalib, handle):
    import torch
    c = 100
    P = sum(shard.param_counts(c))
    d_w = _dev32([5, 101, 7])                                  # a size above c
    assert _key(cudalib, handle, d_w, c, 0, P) == -2           # -BP_ERANGE
    assert _key(cudalib, handle, _dev32([5, 6]), c, 10, 10) == 0   # empty range
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    for g0, g1 in ((0, P + 1), (5, 4), (-1, 3)):
        with pytest.raises(cudalib.BpLbError) as e:
            cudalib.bp_lb_eval_range(handle, _dev32([1]), c, g0, g1, out)
        assert e.value.status == cudalib.BP_ERANGE
