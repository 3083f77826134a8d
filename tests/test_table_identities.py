"""CPU pins of the identities and upper bounds the device kernels rely on
(csrc/bp_lb_prefix.cuh, csrc/bp_lb_kernels.cuh), restated here in plain
Python over value tables and checked against the oracle's per-(DFF, lambda)
bounds on small random instances:

- FS1 from the twice-scanned table NN (Sec. 3.1, FS1): S = c sum_j
  N(ceil(j c / l')) - sum over the multiples of their sizes;
- BJ1 from D(x) = NN(c + 1 - x) - NN(1 + x): S = sum_{i=1}^{floor(c/l)} D(i l),
  with D built from NN in place pair by pair;
- VB2 from the signed counts N'(x) = #small[u >= x] - #big[u >= x]:
  acc = sum_j N'(floor(j c / l) + 1);
- the pruning upper bounds: BJ1 and CCM1 against L1, VB2 against any cut kk
  (per parameter and through the linear function G over a range).
A mistake in one of them would make the GPU path diverge from the oracle
only on instances that exercise it; here each is checked on its own."""
import numpy as np
import pytest


def cdiv(a, b):
    return -(-a // b)


def tables(w, c):
    H = np.zeros(c + 3, np.int64)
    for x in w:
        H[x] += 1
    N = np.cumsum(H[::-1])[::-1]            # N[x] = #[w >= x], x in [0, c + 2]
    NN = np.cumsum(N[::-1])[::-1]           # NN[x] = sum_{y >= x} N[y]
    return N, NN


def classes(w, c):
    w = [int(x) for x in w if x > 0]
    small = [x for x in w if 2 * x < c]
    big = [c - x for x in w if 2 * x > c and x < c]
    nh = sum(1 for x in w if 2 * x == c)
    nf = sum(1 for x in w if x == c)
    return small, big, nh, nf


def instances(seed, count, c_hi=120, n_hi=25):
    rng = np.random.default_rng(seed)
    for it in range(count):
        c = int(rng.integers(1, c_hi))
        n = int(rng.integers(0, n_hi))
        w = rng.integers(0, c + 1, n)
        if it % 3 == 0 and n:
            w[: n // 3] = c // 2
        if it % 4 == 0 and n:
            w[: n // 4] = c
        yield [int(x) for x in w], c


def test_fs1_from_the_w_table(orc):
    for w, c in instances(1, 150):
        N, NN = tables(w, c)
        for l in range(1, 101):
            lp = l + 1
            cnt = sum(int(N[cdiv(j * c, lp)]) for j in range(1, lp + 1))
            div = sum((j * c // lp) * int(N[j * c // lp] - N[j * c // lp + 1])
                      for j in range(1, lp + 1) if (j * c) % lp == 0)
            assert cdiv(c * cnt - div, c * l) == orc.lb_param(2, l, w, c), (w, c, l)


def test_bj1_from_the_d_table(orc):
    for w, c in instances(2, 150):
        _, NN = tables(w, c)
        T = NN[: c + 2].copy()
        for x in range(0, c // 2 + 1):      # in place, pair by pair
            a, b = T[1 + x], T[c + 1 - x]
            T[1 + x], T[c + 1 - x] = b - a, a - b
        for l in range(1, c + 1):
            q, cm = c // l, c % l
            S = sum(int(T[1 + i * l]) for i in range(1, q + 1))
            assert cdiv(S, q * (l - cm)) == orc.lb_param(5, l, w, c), (w, c, l)


def test_vb2_from_the_signed_counts(orc):
    for w, c in instances(3, 120):
        small, big, nh, nf = classes(w, c)
        U = (c - 1) // 2
        Np = np.zeros(U + 2, np.int64)
        for u in small:
            Np[1:u + 1] += 1
        for u in big:
            Np[1:u + 1] -= 1
        K = 2 * len(big) + nh + 2 * nf
        for l in range(2, c + 1):
            acc, j = 0, 0
            while (j * c) // l + 1 <= U:
                acc += int(Np[(j * c) // l + 1])
                j += 1
            S = 2 * (acc - len(small) + len(big)) + (l - 1) * K
            assert cdiv(S, 2 * (l - 1)) == orc.lb_param(4, l, w, c), (w, c, l)


def test_pruning_upper_bounds(orc):
    """A parameter the kernels skip never has a bound above the cut."""
    rng = np.random.default_rng(4)
    skipped = {"bj1": 0, "ccm1": 0, "vb2": 0}
    for w, c in instances(5, 150):
        small, big, nh, nf = classes(w, c)
        ns, nb = len(small), len(big)
        sumw = sum(w)
        L1 = cdiv(sumw, c)
        sws, sub = sum(small), sum(big)
        kS = 2 * nb + nh + 2 * nf
        for l in range(1, c + 1):               # BJ1 against L1
            if L1 * (c - c % l) >= sumw:
                skipped["bj1"] += 1
                assert orc.lb_param(5, l, w, c) <= L1
        for l in range(1, c // 2 + 1):          # CCM1 against L1
            q = c // l
            if 2 * sws - 2 * sub + 2 * nb * (l - 1) + q * l * kS <= 2 * q * l * L1:
                skipped["ccm1"] += 1
                assert orc.lb_param(3, l, w, c) <= L1
        L = len(w)
        D = sws - sub
        for _ in range(3):                      # VB2 against a cut kk in [0, L]
            kk = int(rng.integers(0, L + 1))
            alpha = 2 * D - c * (2 * kk - kS)
            beta = 2 * ns * (c - 1) + c * (2 * kk - kS) - c * (2 * ns - 2 * nb + 1) + 2
            for l in range(2, c + 1):
                M = ((l - 1) * (2 * kk - kS) + 2 * ns - 2 * nb) >> 1
                may = l * D + ns * (c - 1) > (M + 1) * c - 1
                if alpha * l + beta <= 0:
                    assert not may, (w, c, l, kk)   # the range test is a relaxation
                if not may:
                    skipped["vb2"] += 1
                    assert orc.lb_param(4, l, w, c) <= kk, (w, c, l, kk)
    assert min(skipped.values()) > 100
