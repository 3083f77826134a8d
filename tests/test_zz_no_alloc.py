"""bp_lb_eval_batch_noalloc: the batched check for callers that cannot allocate
device memory where they check (their device memory belongs to another
allocator, or cudaFree's device-wide synchronisation is not acceptable in
their loop).  It must give exactly what the oracle and the allocating
bp_lb_eval_batch give, call after call, although every call reuses the same
fixed scratch array -- up to the largest batch it takes, at capacities on
every evaluation path, with invalid instances reported per instance.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

pytestmark = pytest.mark.gpu

ERANGE = 2


def _batch(seed, B, c_hi, n_hi):
    rng = np.random.default_rng(seed)
    inst, caps = [], []
    for _ in range(B):
        c = int(rng.integers(1, c_hi))
        inst.append(rng.integers(0, c + 1, size=int(rng.integers(0, n_hi))))
        caps.append(c)
    rg = I.ragged_from_list(inst, caps)
    rg.bins = rng.integers(0, 200, size=B).astype(np.int64)
    return rg


def _dev(rg):
    import torch
    d = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    return (d(rg.offsets, torch.int64), d(rg.sizes, torch.int32), d(rg.capacity, torch.int64),
            d(rg.bins, torch.int64))


def _outs(B):
    import torch
    return (torch.full((B,), -99, dtype=torch.int64, device="cuda"),
            torch.full((B, 2), -99, dtype=torch.int64, device="cuda"),
            torch.full((B,), 7, dtype=torch.uint8, device="cuda"))


def _decode(cudalib, outs):
    d, lam = cudalib.decode_argmax(outs[1])
    return outs[0].cpu().numpy(), d, lam, outs[2].cpu().numpy().astype(bool)


def _check_oracle(cudalib, orc, rg, outs, idx):
    b, d, lam, f = _decode(cudalib, outs)
    for j in idx:
        want = orc.lb(rg.instance(j), int(rg.capacity[j]), int(rg.bins[j]))
        assert (b[j], d[j], lam[j], f[j]) == want, j


def test_noalloc_matches_oracle_and_allocating_batch_twice_in_a_row(cudalib, orc):
    import torch
    # the first call on the device does the set-up; B = 0 is a warm-up
    cudalib.lib().bp_lb_eval_batch_noalloc(0, None, None, None, None, None, None, None, None)
    h = cudalib.bp_lb_create(150, 1024)
    try:
        for seed, B, c_hi, n_hi, sample in ((21, 300, 2000, 200, None),
                                            (22, 1000, 12_000, 700, 40)):
            rg = _batch(seed, B, c_hi, n_hi)
            args = _dev(rg)
            ref = _outs(B)
            cudalib.bp_lb_eval_batch(h, *args, *ref)
            idx = range(B) if sample is None else \
                np.random.default_rng(seed).choice(B, sample, replace=False)
            for call in range(2):                 # the same batch twice in a row
                got = _outs(B)
                cudalib.bp_lb_eval_batch_noalloc(*args, *got)
                torch.cuda.synchronize()
                # integer results: the tolerance is exact equality
                for g, r in zip(got, ref):
                    assert torch.equal(g, r), (seed, call)
                _check_oracle(cudalib, orc, rg, got, idx)
    finally:
        cudalib.bp_lb_destroy(h)


def test_noalloc_full_batch_wide_capacities_and_errors(cudalib, orc):
    """B = BP_NOALLOC_MAX_BATCH fills the scratch array (tile table, slots and
    counters all at their largest); capacities on the generic kernel's fp32
    and 64-bit VB2 paths; invalid instances get -BP_ERANGE, argmax (-1, -1)
    and verdict 0 while their neighbours are unaffected."""
    import torch
    B = cudalib.NOALLOC_MAX_BATCH
    rng = np.random.default_rng(23)
    inst, caps = [], []
    for _ in range(B):
        c = int(rng.integers(1, 3000))
        inst.append(rng.integers(0, c + 1, size=int(rng.integers(0, 100))))
        caps.append(c)
    wide = list(range(0, B, 512))                 # 8 instances at 65535 < c <= 10^6
    for j in wide:
        caps[j] = int(rng.integers(65536, 10 ** 6 + 1))
        inst[j] = rng.integers(1, caps[j] + 1, size=6)
    wider = [100, 1100, 2100]                      # c > 2^22: the 64-bit paths
    for j in wider:
        caps[j] = int(rng.integers((1 << 22) + 1, 1 << 24))
        inst[j] = rng.integers(1, caps[j] + 1, size=2)
    bad = [7, 777, 3000, 4095]
    caps[7] = 0                                    # capacity below 1
    caps[3000] = (1 << 30) + 1                     # capacity above 2^30
    inst[777] = np.array([5, caps[777] + 1])       # a size above c
    bins = rng.integers(0, 200, size=B).astype(np.int64)
    bins[4095] = -1                                # a negative bin count
    rg = I.ragged_from_list(inst, caps, bins=bins)
    args = _dev(rg)
    h = cudalib.bp_lb_create(150, 1024)
    try:
        ref = _outs(B)
        cudalib.bp_lb_eval_batch(h, *args, *ref)
        for call in range(2):
            got = _outs(B)
            cudalib.bp_lb_eval_batch_noalloc(*args, *got)
            torch.cuda.synchronize()
            for g, r in zip(got, ref):
                assert torch.equal(g, r), call
            b, d, lam, f = _decode(cudalib, got)
            for j in bad:
                assert (b[j], d[j], lam[j], f[j]) == (-ERANGE, -1, -1, False), j
            _check_oracle(cudalib, orc, rg, got, wide + list(range(1, 400, 13)))
    finally:
        cudalib.bp_lb_destroy(h)


def test_noalloc_rejects_oversize_batch(cudalib):
    import torch
    B = cudalib.NOALLOC_MAX_BATCH + 1
    z = torch.zeros(B + 1, dtype=torch.int64, device="cuda")
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(B, dtype=torch.int64, device="cuda")
    with pytest.raises(cudalib.BpLbError) as e:
        cudalib.bp_lb_eval_batch_noalloc(z, s, z[:B], z[:B], out)
    assert e.value.status == cudalib.BP_ERANGE
