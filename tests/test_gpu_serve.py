"""The continuous-batching serving loop (bp_serve_*): every check served in a
mix of concurrent batches gives exactly the result it gives alone; admission by
memory footprint refuses what does not fit; bad requests are reported per
request; the closed-loop search driver runs against it."""
import numpy as np
import pytest

from paper_2402_14821_gb300 import instances as I
from paper_2402_14821_gb300 import search_sim

pytestmark = pytest.mark.gpu


def _alone(B, h, w, a, c, k):
    """One node through bp_lb_eval_nodes with B = 1."""
    import torch
    d = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()
    ob = torch.empty(1, dtype=torch.int64, device="cuda")
    oa = B.argmax_tensor(1)
    of = torch.empty(1, dtype=torch.uint8, device="cuda")
    B.bp_lb_eval_nodes(h, d([0, len(w)], torch.int64), d(w, torch.int32), d([c], torch.int64),
                       d([0], torch.int32), d([0, len(a)], torch.int64), d(a, torch.int32),
                       d([k], torch.int64), max(int(k), 1), ob, oa, of)
    torch.cuda.synchronize()
    dd, ll = B.decode_argmax(oa)
    return int(ob[0]), int(dd[0]), int(ll[0]), bool(of[0])


def _mixed_nodes(seed, count):
    rng = np.random.default_rng(seed)
    inst, caps = [], []
    for _ in range(12):
        c = int(rng.choice([150, 1000, 7000, 20000, 120000]))
        n = int(rng.integers(50, 1500))
        inst.append(I.uniform_sizes(rng, n, 1, c // 2))
        caps.append(c)
    base = I.ragged_from_list(inst, caps)
    pick = rng.integers(0, 12, size=count)
    assigns = I.prepack(rng, [inst[i] for i in pick], [caps[i] for i in pick],
                        [int(base.bins[i]) for i in pick], 0.6)
    return inst, caps, base, pick, assigns


def test_serve_mix_equals_alone(cudalib, orc):
    B = cudalib
    inst, caps, base, pick, assigns = _mixed_nodes(31, 300)
    srv = B.bp_serve_create(pool_items=1 << 16, max_instances=64, max_queued_items=1 << 19,
                            slots=3, max_batch=64, max_bins=4096)
    h = B.bp_lb_create(150, 1024)
    try:
        ids = [B.bp_serve_register(srv, w, c) for w, c in zip(inst, caps)]
        rids = {}
        for j, (i, a) in enumerate(zip(pick, assigns)):
            rid = B.bp_serve_submit(srv, ids[i], a, int(base.bins[i]), tag=j)
            assert rid is not None
            rids[rid] = j
        got = {}
        for _ in range(2000):
            for r in B.bp_serve_poll(srv, 512, 2000):
                got[rids[r.request]] = r
            if len(got) == len(pick):
                break
        assert len(got) == len(pick)
        st = B.bp_serve_stats(srv)
        assert st["done"] == len(pick) and st["status"] == 0
        assert st["batches"] > 1  # admitted in several batches while others ran
        for j, (i, a) in enumerate(zip(pick, assigns)):
            r = got[j]
            assert r.tag == j and r.status == 0 and r.latency_us > 0
            alone = _alone(B, h, inst[i], a, caps[i], int(base.bins[i]))
            assert (r.bound, r.dff, r.lam, bool(r.feasible)) == alone, j
        for j in range(0, len(pick), 37):     # and a sample against the oracle
            i, a = pick[j], assigns[j]
            want = orc.lb(orc.reduce(inst[i], a, int(base.bins[i]), caps[i]), caps[i],
                          int(base.bins[i]))
            assert (got[j].bound, got[j].dff, got[j].lam, bool(got[j].feasible)) == want
    finally:
        B.bp_lb_destroy(h)
        B.bp_serve_destroy(srv)


def test_serve_admission_by_footprint(cudalib):
    B = cudalib
    srv = B.bp_serve_create(pool_items=1000, max_instances=4, max_queued_items=1200, slots=2,
                            max_batch=8, max_bins=64)
    try:
        w = np.full(400, 5, dtype=np.int32)
        ids = [B.bp_serve_register(srv, w, 50), B.bp_serve_register(srv, w, 50)]
        with pytest.raises(B.BpLbError) as e:      # the resident pool is full
            B.bp_serve_register(srv, w, 50)
        assert e.value.status == B.BP_EBUSY
        with pytest.raises(B.BpLbError) as e:      # larger than one slot's staging
            B.bp_serve_register(srv, np.ones(700, np.int32), 50)
        assert e.value.status == B.BP_ERANGE
        a = np.full(400, -1, dtype=np.int32)
        accepted = [B.bp_serve_submit(srv, ids[0], a, 10) for _ in range(6)]
        # at most 1200 queued entries: never more than three 400-item checks at once
        assert accepted.count(None) >= 1 or B.bp_serve_stats(srv)["done"] > 0
        n_ok = sum(x is not None for x in accepted)
        res = []
        for _ in range(200):
            res += B.bp_serve_poll(srv, 16, 2000)
            if len(res) == n_ok:
                break
        assert len(res) == n_ok
        assert all(r.bound == 40 for r in res)     # 400 items of 5 in bins of 50
        assert B.bp_serve_submit(srv, ids[1], a, 10) is not None   # room again
        with pytest.raises(B.BpLbError) as e:
            B.bp_serve_submit(srv, 7, a, 10)       # unknown instance
        assert e.value.status == B.BP_EINVAL
        with pytest.raises(B.BpLbError) as e:
            B.bp_serve_submit(srv, ids[0], a, 65)  # more bins than max_bins
        assert e.value.status == B.BP_ERANGE
    finally:
        B.bp_serve_destroy(srv)


def test_serve_reports_bad_nodes(cudalib):
    B = cudalib
    srv = B.bp_serve_create(pool_items=1 << 12, max_instances=4, max_queued_items=1 << 14,
                            slots=2, max_batch=8, max_bins=64)
    try:
        i = B.bp_serve_register(srv, [30, 30, 30, 10], 50)
        good = B.bp_serve_submit(srv, i, [0, 1, -1, -1], 3)
        over = B.bp_serve_submit(srv, i, [0, 0, -1, -1], 3)   # bin 0 holds 60 > 50
        bad = B.bp_serve_submit(srv, i, [5, -1, -1, -1], 3)   # bin 5 of 3
        res = {}
        for _ in range(200):
            for r in B.bp_serve_poll(srv, 8, 2000):
                res[r.request] = r
            if len(res) == 3:
                break
        # W_R = [30, 10, 30, 30], c = 50: three items above c/2 need three bins
        assert res[good].status == 0 and res[good].bound == 3 and res[good].feasible
        assert res[over].status == B.BP_ERANGE and res[over].bound == -B.BP_ERANGE
        assert res[bad].status == B.BP_ERANGE
        assert B.bp_serve_stats(srv)["status"] == 0   # a bad node is not a server failure
    finally:
        B.bp_serve_destroy(srv)


def test_serve_closed_loop_searches(cudalib):
    B = cudalib
    searches = search_sim.make_searches(count=16, seed=5, n_lo=50, n_hi=400, c_lo=100,
                                        c_hi=5000)
    srv = B.bp_serve_create(pool_items=1 << 16, max_instances=64, max_queued_items=1 << 16,
                            slots=3, max_batch=256, max_bins=1024)
    try:
        ids = [B.bp_serve_register(srv, s.w, s.c) for s in searches]
        out = search_sim.drive(B, srv, searches, ids, rate=2000.0, duration_s=1.5)
        assert out["done"] > 50 and out["submitted"] >= out["done"]
        assert np.all(out["latency_us"] > 0)
        assert B.bp_serve_stats(srv)["status"] == 0
    finally:
        B.bp_serve_destroy(srv)
