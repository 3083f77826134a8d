"""FS1 on the prefix-count kernel -- its sum read from the twice-scanned
w-domain table that BJ1 uses (Sec. 3.1, FS1) -- equals the oracle's FS1
bound and argmax: on a tile of its own (FS1 alone), on BJ1's first tile (FS1
with BJ1), inside the full bound, with the tables in shared memory and in the
global scratch, batched and on the plain path."""
import math

import numpy as np
import pytest

from paper_2402_14821_gb300 import binding as B
from paper_2402_14821_gb300 import instances as I

from test_gpu_parity import oracle_batch, run_batch

pytestmark = pytest.mark.gpu

# highly composite capacities (many l' = l + 1 share factors with c), small
# ones, and both sides of the shared-memory limit of the w-domain table
CAPS = (1, 2, 3, 6, 12, 60, 101, 720, 2520, 5040, 10100, 12286, 12287, 55440, 100_000)
FS1, BJ1 = 2, 5


def fs1_instances(seed, per_cap=4, n_hi=160):
    """Sizes on FS1's breakpoints: multiples of c / gcd(c, l') (where c
    divides w l'), ceil(j c / l') and one below, c, 0, and uniform ones."""
    rng = np.random.default_rng(seed)
    inst, caps = [], []
    for c in CAPS:
        for _ in range(per_cap):
            ws = []
            for lp in rng.integers(2, 102, size=4):
                g = c // math.gcd(c, int(lp))
                ws += [m * g for m in range(1, c // g + 1)][:12]
                j = rng.integers(1, int(lp) + 1, size=6)
                x = -(-(j * c) // int(lp))
                ws += list(x) + list(np.maximum(x - 1, 0))
            ws += [c, c, 0]
            n = int(rng.integers(0, n_hi))
            w = np.concatenate([np.asarray(ws, dtype=np.int64), rng.integers(0, c + 1, size=n)])
            w = w[rng.permutation(len(w))][: int(rng.integers(1, len(w) + 1))]
            inst.append(w)
            caps.append(c)
    return I.ragged_from_list(inst, caps)


def want_masked(orc, rg, dffs):
    """Bound and first argmax (paper order) over the DFFs in dffs."""
    out = []
    for j in range(rg.count):
        w, c = rg.instance(j), int(rg.capacity[j])
        best = (0, -1, -1)
        for d in dffs:
            lf, lam = orc.lb_dff(d, w, c)
            if lf >= 0 and (best[1] < 0 or lf > best[0]):
                best = (lf, d, lam)
        out.append(best)
    return out


def test_fs1_routes_to_prefix():
    for c in CAPS:
        want = B.ALGO_PREFIX if c <= 1_048_574 else B.ALGO_DIRECT
        assert B.bp_lb_dff_route(FS1, c, 400, B.ALGO_PREFIX) == want
        assert B.bp_lb_dff_route(FS1, c, 400, B.ALGO_DIRECT) == B.ALGO_DIRECT


@pytest.mark.parametrize("mask", [(FS1,), (FS1, BJ1)])
@pytest.mark.parametrize("algo", [0, 1])
def test_fs1_masked_batch(cudalib, orc, algo, mask):
    rg = fs1_instances(90 + algo)
    rg.bins = np.zeros(rg.count, dtype=np.int64) + 2
    want = want_masked(orc, rg, mask)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_algorithm(h, algo)
        cudalib.bp_lb_set_dff_mask(h, sum(1 << d for d in mask))
        b, dd, ll, _ = run_batch(cudalib, h, rg)
        for j in range(rg.count):
            assert (b[j], dd[j], ll[j]) == want[j], (j, int(rg.capacity[j]), mask, algo)
    finally:
        cudalib.bp_lb_destroy(h)


def test_fs1_full_bound_batch(cudalib, orc):
    rg = fs1_instances(93, per_cap=2, n_hi=60)
    want = oracle_batch(orc, rg)
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        for algo in (1, 0):
            cudalib.bp_lb_set_algorithm(h, algo)
            got = run_batch(cudalib, h, rg)
            for x, y in zip(got, want):
                assert np.array_equal(np.asarray(x), np.asarray(y)), algo
    finally:
        cudalib.bp_lb_destroy(h)


@pytest.mark.parametrize("c", [720, 5040, 12286, 55440])
def test_fs1_plain_path(cudalib, orc, c):
    """The plain check splits BJ1 into short tiles; FS1 rides on the first."""
    rg = fs1_instances(94)
    idx = [j for j in range(rg.count) if int(rg.capacity[j]) == c]
    h = cudalib.bp_lb_create(c, 4096)
    try:
        for mask in ((FS1,), (FS1, BJ1)):
            cudalib.bp_lb_set_dff_mask(h, sum(1 << d for d in mask))
            for j in idx:
                w = rg.instance(j)
                want = want_masked(orc, I.ragged_from_list([w], [c]), mask)[0]
                assert cudalib.bp_lb_eval(h, w, 2) == want, (c, j, mask)
        cudalib.bp_lb_set_dff_mask(h, 63)
        for j in idx[:2]:
            w = rg.instance(j)
            assert cudalib.bp_lb_eval(h, w, 2)[:3] == tuple(orc.lb(w, c, 0)[:3])
    finally:
        cudalib.bp_lb_destroy(h)
