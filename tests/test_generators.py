"""The seeded workload generators: determinism and the stated recipes."""
import numpy as np

from paper_2402_14821_gb300 import instances as I


def test_plain_single_recipe():
    a, b = I.plain_single(), I.plain_single()
    assert np.array_equal(a.sizes, b.sizes)
    w = a.instance(0)
    assert len(w) == 50 and w.min() >= 20 and w.max() <= 100
    assert a.capacity[0] == 150 and a.bins[0] == -(-int(w.sum()) // 150) + 1


def test_search_nodes_recipe():
    nd = I.search_nodes(nodes=256)
    w, a, c, k = nd.node(0)
    assert len(w) == 500 and c == 10_000 and w.min() >= 1 and w.max() <= 5000
    fr = []
    for j in range(nd.count):
        w, a, c, k = nd.node(j)
        assert a.min() >= -1 and a.max() < k
        load = np.bincount(a[a >= 0], weights=w[a >= 0], minlength=k)
        assert load.max() <= c
        fr.append(np.mean(a >= 0))
    assert 0.0 <= min(fr) and max(fr) <= 0.6 and np.mean(fr) > 0.05
    nd2 = I.search_nodes(nodes=256)
    assert np.array_equal(nd.assign, nd2.assign)


def test_triplets_fill_bins_exactly():
    c = 100_000
    w = I.triplet_sizes(np.random.default_rng(0), 3000, c)
    assert len(w) == 3000
    assert int(w.sum()) == 1000 * c
    assert np.all(4 * w > c) and np.all(2 * w < c)


def test_large_families():
    for fam in I.FAMILIES:
        r = I.large_instances(fam, 10 ** 5, count=2, n=999)
        assert r.count == 2 and r.sizes.min() >= 1 and r.sizes.max() <= 10 ** 5


def test_ragged_nodes_recipe():
    nd = I.ragged_nodes(count=200)
    assert nd.count == 200
    caps = set(int(x) for x in nd.base.capacity)
    assert caps <= set(I.RAGGED_CAPS)
    for j in range(0, 200, 17):
        w, a, c, k = nd.node(j)
        assert 50 <= len(w) <= 5000 and w.max() <= c // 2
        load = np.bincount(a[a >= 0], weights=w[a >= 0], minlength=k)
        assert load.max() <= c
