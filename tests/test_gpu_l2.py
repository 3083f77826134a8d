"""L2 on the device (the comparator) equals the oracle's L2 from its
definition; per-DFF bounds through the DFF mask equal the oracle's L_f."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I

from test_gpu_parity import oracle_batch, run_batch, to_dev

pytestmark = pytest.mark.gpu


def run_l2(cudalib, h, rg):
    import torch
    out = torch.empty(rg.count, dtype=torch.int64, device="cuda")
    cudalib.bp_lb_l2_batch(h, to_dev(rg.offsets.astype(np.int64)), to_dev(rg.sizes.astype(np.int32)),
                           to_dev(rg.capacity.astype(np.int64)), out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_l2_matches_oracle(cudalib, handle, orc):
    rng = np.random.default_rng(71)
    inst, caps = [], []
    for _ in range(300):
        c = int(rng.integers(1, 400))
        n = int(rng.integers(0, 80))
        w = rng.integers(0, c + 1, size=n)
        m = rng.random(n)
        w[m < 0.1] = c // 2                      # exactly half (c even: 2w = c)
        w[(m >= 0.1) & (m < 0.15)] = c // 2 + 1
        w[(m >= 0.15) & (m < 0.2)] = c
        w[(m >= 0.2) & (m < 0.25)] = 0
        inst.append(w)
        caps.append(c)
    # larger ones: several sort passes, prefix sums over many segments
    for n, c in ((8192, 1000), (5000, 77777), (2049, 10_000), (8191, 150)):
        inst.append(rng.integers(1, c + 1, size=n))
        caps.append(c)
    rg = I.ragged_from_list(inst, caps)
    got = run_l2(cudalib, handle, rg)
    for j in range(rg.count):
        want = orc.l2(rg.instance(j), int(rg.capacity[j])) if len(rg.instance(j)) < 3000 else None
        if want is not None:
            assert got[j] == want, (j, int(rg.capacity[j]))
        else:  # the oracle's definition is O(n c): check the pin L2 = max(L_MT, #{w > c/2}) instead
            w, c = rg.instance(j), int(rg.capacity[j])
            lmt = orc.lb_dff(0, w, c)[0]
            assert got[j] == max(lmt, int(np.sum(2 * np.asarray(w) > c)))


def test_l2_errors(cudalib, handle):
    rg = I.ragged_from_list([np.array([1, 2, 3]), np.array([5, 11]), np.ones(8193, np.int64)],
                            [10, 10, 100])
    got = run_l2(cudalib, handle, rg)
    assert got[0] >= 1 and got[1] == -cudalib.BP_ERANGE and got[2] == -cudalib.BP_ERANGE


@pytest.mark.parametrize("algo", [0, 1])
def test_dff_mask_gives_each_dff_bound(cudalib, orc, algo):
    rng = np.random.default_rng(72)
    inst, caps = [], []
    for c in (1, 2, 4, 5, 8, 9, 150, 1000, 9999, 30000):
        for _ in range(4):
            inst.append(rng.integers(0, c + 1, size=int(rng.integers(0, 120))))
            caps.append(c)
    rg = I.ragged_from_list(inst, caps)
    rg.bins = np.zeros(rg.count, dtype=np.int64) + 3
    h = cudalib.bp_lb_create(150, 1 << 16)
    try:
        cudalib.bp_lb_set_algorithm(h, algo)
        for d in range(6):
            cudalib.bp_lb_set_dff_mask(h, 1 << d)
            assert cudalib.bp_lb_get_dff_mask(h) == 1 << d
            b, dd, ll, f = run_batch(cudalib, h, rg)
            for j in range(rg.count):
                w, c = rg.instance(j), int(rg.capacity[j])
                lf, lam = orc.lb_dff(d, w, c)
                if lf < 0:                       # empty range at this capacity
                    assert (b[j], dd[j], ll[j]) == (0, -1, -1), (d, j)
                else:
                    assert (b[j], dd[j], ll[j]) == (lf, d, lam), (d, j, c)
                assert f[j] == (b[j] <= 3)
        # two DFFs: the maximum of the two, first argmax in paper order
        cudalib.bp_lb_set_dff_mask(h, (1 << 3) | (1 << 5))
        b, dd, ll, f = run_batch(cudalib, h, rg)
        for j in range(rg.count):
            w, c = rg.instance(j), int(rg.capacity[j])
            c3, c5 = orc.lb_dff(3, w, c), orc.lb_dff(5, w, c)
            want = (c3[0], 3, c3[1]) if c3[0] >= c5[0] else (c5[0], 5, c5[1])
            if c3[0] < 0:
                want = (c5[0], 5, c5[1])
            assert (b[j], dd[j], ll[j]) == want, j
        cudalib.bp_lb_set_dff_mask(h, 63)
        assert all(x == y for x, y in zip(run_batch(cudalib, h, rg)[0], oracle_batch(orc, rg)[0]))
        with pytest.raises(cudalib.BpLbError):
            cudalib.bp_lb_set_dff_mask(h, 0)
        # the plain path with one DFF
        cudalib.bp_lb_set_dff_mask(h, 1 << 3)
        w = rg.instance(30)
        hp = cudalib.bp_lb_create(int(rg.capacity[30]), 4096)
        cudalib.bp_lb_set_dff_mask(hp, 1 << 3)
        lf, lam = orc.lb_dff(3, w, int(rg.capacity[30]))
        assert cudalib.bp_lb_eval(hp, w, 3) == (lf, 3, lam)
        cudalib.bp_lb_destroy(hp)
    finally:
        cudalib.bp_lb_destroy(h)
