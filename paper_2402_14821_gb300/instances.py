"""Seeded synthetic bin-packing workloads.

This module only draws inputs: item sizes, capacities, bin counts and partial
packings (item -> bin assignments).  It computes no lower bound, no reduction
and nothing else the feasibility check itself computes, so both the CUDA path's
tests and the CPU oracle's tests can draw from it.

The paper evaluates on Falkenauer U/T, Scholl 1-3 and Weibull instances
(Sec. 5).  None of those files are used here: the families below only take
their shapes (uniform sizes with c = 150 like Falkenauer U, triplets that fill
a bin exactly like Falkenauer T, wide capacities like Scholl 3 / Weibull).
Every generator takes an explicit seed and uses numpy's PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def bins_for(sizes: np.ndarray, c: int) -> int:
    """The bin count the workloads use: ceil(sum / c) + 1 (one spare bin)."""
    s = int(np.asarray(sizes, dtype=np.int64).sum())
    return (s + c - 1) // c + 1


@dataclass
class Ragged:
    """B instances as ragged arrays (offsets[B+1] into sizes)."""
    offsets: np.ndarray     # int64 [B+1]
    sizes: np.ndarray       # int32 or int64 [offsets[-1]]
    capacity: np.ndarray    # int64 [B]
    bins: np.ndarray        # int64 [B]

    @property
    def count(self) -> int:
        return len(self.offsets) - 1

    def instance(self, b: int) -> np.ndarray:
        return self.sizes[self.offsets[b]:self.offsets[b + 1]]


@dataclass
class Nodes:
    """Search nodes: partial packings of base instances.

    Node j packs a subset of the items of base instance ``node_base[j]``:
    ``assign[assign_offsets[j] + i]`` is -1 when item i is unpacked, else the
    bin (0..bins[j]-1) it sits in.  No bin is filled above capacity.
    """
    base: Ragged            # the base instances (their ``bins`` are the search's k)
    node_base: np.ndarray   # int32 [B]
    assign_offsets: np.ndarray  # int64 [B+1]
    assign: np.ndarray      # int32 [assign_offsets[-1]]
    bins: np.ndarray        # int64 [B]

    @property
    def count(self) -> int:
        return len(self.node_base)

    def node(self, j: int):
        b = int(self.node_base[j])
        return (self.base.instance(b), self.assign[self.assign_offsets[j]:self.assign_offsets[j + 1]],
                int(self.base.capacity[b]), int(self.bins[j]))


def ragged_from_list(instances, capacities, bins=None, dtype=np.int32) -> Ragged:
    lens = np.array([len(x) for x in instances], dtype=np.int64)
    offsets = np.zeros(len(instances) + 1, dtype=np.int64)
    np.cumsum(lens, out=offsets[1:])
    sizes = (np.concatenate([np.asarray(x, dtype=dtype) for x in instances])
             if len(instances) and offsets[-1] > 0 else np.zeros(0, dtype=dtype))
    cap = np.asarray(capacities, dtype=np.int64)
    if bins is None:
        bins = [bins_for(x, int(c)) for x, c in zip(instances, cap)]
    return Ragged(offsets, sizes, cap, np.asarray(bins, dtype=np.int64))


# ---------------------------------------------------------------------------
# size families
# ---------------------------------------------------------------------------
def uniform_sizes(rng: np.random.Generator, n: int, lo: int, hi: int) -> np.ndarray:
    """n sizes uniform in the closed range [lo, hi]."""
    return rng.integers(lo, hi + 1, size=n, dtype=np.int64)


def triplet_sizes(rng: np.random.Generator, n: int, c: int) -> np.ndarray:
    """floor(n/3) triplets a + b + t = c with every size strictly inside (c/4, c/2).

    a and b are drawn uniformly in the open interval (c/4, c/2); the triplet is
    redrawn unless t = c - a - b also lies strictly inside it.  The items are
    shuffled.  (The shape of Falkenauer's T class; no file of that class is
    reproduced.)
    """
    lo = c // 4 + 1                     # smallest integer > c/4
    hi = (c - 1) // 2                   # largest integer < c/2
    m = n // 3
    out = np.empty((m, 3), dtype=np.int64)
    filled = 0
    while filled < m:
        need = m - filled
        a = rng.integers(lo, hi + 1, size=2 * need + 16)
        b = rng.integers(lo, hi + 1, size=2 * need + 16)
        t = c - a - b
        ok = (4 * t > c) & (2 * t < c)
        a, b, t = a[ok][:need], b[ok][:need], t[ok][:need]
        k = len(a)
        out[filled:filled + k, 0] = a
        out[filled:filled + k, 1] = b
        out[filled:filled + k, 2] = t
        filled += k
    flat = out.reshape(-1)
    rng.shuffle(flat)
    return flat


# ---------------------------------------------------------------------------
# partial packings
# ---------------------------------------------------------------------------
def prepack(rng: np.random.Generator, sizes_list, caps, ks, frac_hi: float):
    """Random partial packings, one per instance, vectorised over instances.

    For each instance: draw p ~ U[0, frac_hi], take the first floor(p*n) items
    of a random permutation, and for each of them in that order draw one bin
    uniformly in [0, k); the item is packed there if it still fits (load + w <=
    c), else it stays unpacked.  Returns a list of int32 assignment arrays.
    """
    B = len(sizes_list)
    out = []
    GROUP = 1024
    for g0 in range(0, B, GROUP):
        g1 = min(B, g0 + GROUP)
        G = g1 - g0
        ns = np.array([len(sizes_list[j]) for j in range(g0, g1)], dtype=np.int64)
        nmax = int(ns.max()) if G else 0
        W = np.zeros((G, max(nmax, 1)), dtype=np.int64)
        for j in range(G):
            W[j, :ns[j]] = sizes_list[g0 + j]
        kk = np.asarray(ks[g0:g1], dtype=np.int64)
        cc = np.asarray(caps[g0:g1], dtype=np.int64)
        p = rng.uniform(0.0, frac_hi, size=G)
        m = np.floor(p * ns).astype(np.int64)
        keys = rng.random((G, max(nmax, 1)))
        keys[np.arange(max(nmax, 1))[None, :] >= ns[:, None]] = 2.0  # padding sorts last
        perm = np.argsort(keys, axis=1, kind="stable")
        binsel = (rng.random((G, max(nmax, 1))) * kk[:, None]).astype(np.int64)
        kmax = int(kk.max()) if G else 1
        load = np.zeros((G, max(kmax, 1)), dtype=np.int64)
        asg = np.full((G, max(nmax, 1)), -1, dtype=np.int32)
        rows = np.arange(G)
        for t in range(int(m.max()) if G else 0):
            act = t < m
            r = rows[act]
            it = perm[r, t]
            bn = binsel[r, t]
            w = W[r, it]
            fits = load[r, bn] + w <= cc[r]
            r, it, bn, w = r[fits], it[fits], bn[fits], w[fits]
            load[r, bn] += w
            asg[r, it] = bn
        for j in range(G):
            out.append(asg[j, :ns[j]].copy())
    return out


def _nodes_from(base: Ragged, node_base, assigns, bins) -> Nodes:
    lens = np.array([len(a) for a in assigns], dtype=np.int64)
    aoff = np.zeros(len(assigns) + 1, dtype=np.int64)
    np.cumsum(lens, out=aoff[1:])
    asg = np.concatenate(assigns).astype(np.int32) if len(assigns) else np.zeros(0, np.int32)
    return Nodes(base, np.asarray(node_base, dtype=np.int32), aoff, asg,
                 np.asarray(bins, dtype=np.int64))


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------
def plain_single(seed: int = 0, n: int = 50, c: int = 150) -> Ragged:
    """One instance: n sizes uniform in [20, 100], c = 150, k = ceil(sum/c) + 1."""
    rng = _rng(seed)
    w = uniform_sizes(rng, n, 20, 100)
    return ragged_from_list([w], [c])


def search_nodes(seed: int = 1, n: int = 500, c: int = 10_000, nodes: int = 4096,
                 frac_hi: float = 0.6) -> Nodes:
    """One base instance (n sizes uniform in [1, c/2]) and `nodes` partial packings
    committing a uniform 0..60% of its items to random bins without overflow."""
    rng = _rng(seed)
    w = uniform_sizes(rng, n, 1, c // 2)
    base = ragged_from_list([w], [c])
    k = int(base.bins[0])
    assigns = prepack(rng, [w] * nodes, [c] * nodes, [k] * nodes, frac_hi)
    return _nodes_from(base, np.zeros(nodes, np.int32), assigns, [k] * nodes)


def hard_nodes(seed: int = 5, n: int = 501, c: int = 10_000, nodes: int = 4096,
               frac_hi: float = 0.6) -> Nodes:
    """Search nodes whose bounds mostly exceed L1: one triplet instance (n items
    in (c/4, c/2) filling n/3 bins exactly, Falkenauer-T-like), k = n/3 bins --
    the optimum, the bin count a search that has found it tries to beat -- and
    `nodes` partial packings committing a uniform 0..60% of the items to random
    bins without overflow.  A random partial packing rarely completes to the
    perfect packing, so most nodes are infeasible with a bound above L1."""
    rng = _rng(seed)
    w = triplet_sizes(rng, n, c)
    k = len(w) // 3
    base = ragged_from_list([w], [c], bins=[k])
    assigns = prepack(rng, [w] * nodes, [c] * nodes, [k] * nodes, frac_hi)
    return _nodes_from(base, np.zeros(nodes, np.int32), assigns, [k] * nodes)


FAMILIES = ("uniform_wide", "triplets", "uniform_full")


def large_instances(family: str, c: int, count: int = 64, n: int = 10_000, seed: int = 2,
                    dtype=np.int32) -> Ragged:
    """`count` instances of n items: 'uniform_wide' sizes in [c/10, c/2],
    'triplets' (3*floor(n/3) items filling bins exactly), 'uniform_full' sizes in [1, c]."""
    rng = _rng(seed * 1_000_003 + FAMILIES.index(family) * 101 + c % 997)
    inst = []
    for _ in range(count):
        if family == "uniform_wide":
            w = uniform_sizes(rng, n, c // 10, c // 2)
        elif family == "triplets":
            w = triplet_sizes(rng, n, c)
        elif family == "uniform_full":
            w = uniform_sizes(rng, n, 1, c)
        else:
            raise ValueError(family)
        inst.append(w)
    return ragged_from_list(inst, [c] * count, dtype=dtype)


RAGGED_CAPS = (150, 1_000, 10_000, 100_000)


def ragged_nodes(seed: int = 3, count: int = 10_000, n_lo: int = 50, n_hi: int = 5000,
                 caps=RAGGED_CAPS, frac_hi: float = 0.5) -> Nodes:
    """`count` independent instances, n uniform in [n_lo, n_hi], c drawn from `caps`,
    sizes uniform in [1, c/2], each with one partial packing of a uniform 0..50% of
    its items (one search node per instance)."""
    rng = _rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    cs = np.asarray(caps, dtype=np.int64)[rng.integers(0, len(caps), size=count)]
    inst = [uniform_sizes(rng, int(n), 1, int(c) // 2) for n, c in zip(ns, cs)]
    base = ragged_from_list(inst, cs)
    assigns = prepack(rng, inst, cs, base.bins, frac_hi)
    return _nodes_from(base, np.arange(count, dtype=np.int32), assigns, base.bins)


def random_small(rng: np.random.Generator, n_max: int, c_max: int):
    """A small random instance for exhaustive-style tests: (sizes, c)."""
    c = int(rng.integers(1, c_max + 1))
    n = int(rng.integers(0, n_max + 1))
    return rng.integers(0, c + 1, size=n, dtype=np.int64), c


def strength_families(seed: int = 6):
    """Seeded stand-ins shaped like the paper's benchmark classes (Sec. 5; no
    instance of those sets is reproduced), for comparing bound strength
    (Table 1's statistics) at the root of the search:
      U   c = 150, sizes U[20, 100], n in {120, 250, 500, 1000}
      T   c = 1000, triplets filling bins exactly, n in {60, 120, 249, 501}
          (optimum n / 3 by construction)
      S1  n in {50, 100, 200, 500}, c in {100, 120, 150}, sizes U[1, 100],
          U[20, 100] or U[30, 100] (at most about three items per bin)
      S2  c = 1000, n as S1, sizes U[a (1 - d), a (1 + d)] with mean
          a in {c/3, c/5, c/7, c/9}, d in {0.2, 0.5, 0.9} (three to nine per bin)
      S3  c = 100000, n = 200, sizes U[20000, 35000]
      W   n in {100, 200}, sizes 1 + floor(1000 X), X ~ Weibull(k),
          k in {0.5, 1.0, ..., 5.0}, c = round(s max w), s in {1.0, 1.4, 2.0}
    Returns a list of (family, Ragged, optimum or None per instance)."""
    rng = _rng(seed)
    fams = []

    def add(name, inst, caps, opt=None):
        fams.append((name, ragged_from_list(inst, caps), opt))

    inst, caps = [], []
    for n in (120, 250, 500, 1000):
        for _ in range(20):
            inst.append(uniform_sizes(rng, n, 20, 100))
            caps.append(150)
    add("U", inst, caps)
    inst, caps, opt = [], [], []
    for n in (60, 120, 249, 501):
        for _ in range(20):
            inst.append(triplet_sizes(rng, n, 1000))
            caps.append(1000)
            opt.append(n // 3)
    add("T", inst, caps, opt)
    inst, caps = [], []
    for n in (50, 100, 200, 500):
        for c in (100, 120, 150):
            for lo in (1, 20, 30):
                for _ in range(5):
                    inst.append(uniform_sizes(rng, n, lo, 100))
                    caps.append(c)
    add("S1", inst, caps)
    inst, caps = [], []
    for n in (50, 100, 200, 500):
        for a in (1000 // 3, 1000 // 5, 1000 // 7, 1000 // 9):
            for d in (0.2, 0.5, 0.9):
                for _ in range(2):
                    inst.append(uniform_sizes(rng, n, max(1, int(a * (1 - d))), int(a * (1 + d))))
                    caps.append(1000)
    add("S2", inst, caps)
    inst, caps = [], []
    for _ in range(10):
        inst.append(uniform_sizes(rng, 200, 20000, 35000))
        caps.append(100000)
    add("S3", inst, caps)
    inst, caps = [], []
    for n in (100, 200):
        for k in np.arange(0.5, 5.01, 0.5):
            w = 1 + np.floor(1000.0 * rng.weibull(float(k), size=n)).astype(np.int64)
            for s in (1.0, 1.4, 2.0):
                inst.append(w.copy())
                caps.append(int(round(s * int(w.max()))))
    add("W", inst, caps)
    return fams

