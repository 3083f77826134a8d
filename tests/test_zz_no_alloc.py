"""bp_lb_eval_batch_noalloc: the batched check for callers that cannot allocate
device memory where they check (their device memory belongs to another
allocator, or cudaFree's device-wide synchronisation is not acceptable in
their loop).  It must give exactly what the allocating bp_lb_eval_batch gives,
call after call, although every call reuses the same fixed scratch array.

This file is named to be collected last, so that a run stopping at the first
failure has already run every other test; it also passes on its own."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

pytestmark = pytest.mark.gpu


def _batch(seed, B):
    rng = np.random.default_rng(seed)
    inst, caps = [], []
    for _ in range(B):
        c = int(rng.integers(1, 12_000))
        w = rng.integers(0, c + 1, size=int(rng.integers(0, 700)))
        inst.append(w)
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


def test_noalloc_matches_allocating_batch_twice_in_a_row(cudalib):
    import torch
    h = cudalib.bp_lb_create(150, 1024)
    try:
        for seed, B in ((21, 300), (22, 1000)):   # two different batches back to back
            rg = _batch(seed, B)
            args = _dev(rg)
            ref = _outs(B)
            cudalib.bp_lb_eval_batch(h, *args, *ref)
            for call in range(2):                 # and the same batch twice
                got = _outs(B)
                cudalib.bp_lb_eval_batch_noalloc(*args, *got)
                torch.cuda.synchronize()
                # integer results: the tolerance is exact equality
                for g, r in zip(got, ref):
                    assert torch.equal(g, r), (seed, call)
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
