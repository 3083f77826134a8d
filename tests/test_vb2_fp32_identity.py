"""CPU pin of the exactness argument behind VB2's fp32-corrected quotient
(csrc/bp_lb_eval.cuh, vb2_list_float), used for 65535 < c <= 2^22.

For each list entry u (1 <= u < c/2: u = w for a small item, c - w for a
big one) the kernel stages a = fl32(u / c), the correctly rounded float32
quotient, and for a parameter l forms, with one fused multiply-add,
fl32(l a + 1.5 2^23).  Because l a <= 2^21, that sum lies in [2^23, 2^24),
where float32's spacing is 1: the fma rounds l a to the nearest integer
q~ (ties to even) and its bit pattern is 0x4B400000 + q~.  The kernel then
takes ceil(u l / c) = q~ + [rho > 0], rho = u l - c q~, with 2 rho formed in
wrapping 32-bit arithmetic.  That is right iff |q~ - u l / c| < 1 and
|2 rho| < 2^31.

Here the same steps are emulated exactly: numpy's float32 division is the
IEEE correctly rounded one, the product l a of a float32 by an integer
below 2^23 is exact in float64 (24 + 23 bits < 53), and np.rint rounds it to
the nearest integer with ties to even -- which is the fma's single rounding
on the unit grid of [2^23, 2^24) (1.5 2^23 is even, so parities agree).
Checked exhaustively over u at the range's ends c in {65536, 65537,
2^22 - 1, 2^22} for a sample of l that includes the smallest, the largest
(l = c) and powers of two, and on random (c, u, l) in between."""
import numpy as np
import pytest

F32_ROUND_BITS = 0x4B400000


def emulate(u, lam, c):
    """(the kernel's ceil(u l / c), 2 rho) for int64 arrays u, one l and c."""
    a = u.astype(np.float32) / np.float32(c)      # fl32(u / c), correctly rounded
    prod = np.float64(lam) * a.astype(np.float64)  # exact: 24-bit mantissa x l < 2^23
    q = np.rint(prod).astype(np.int64)             # the fma's rounding on the unit grid
    # the fma's result lies in [2^23, 2^24): its bit pattern is 0x4B400000 + q
    bits = (np.float32(1.5 * 2 ** 23) + q.astype(np.float32)).view(np.uint32).astype(np.int64)
    assert np.all(bits - F32_ROUND_BITS == q)
    two_rho = 2 * u * lam - 2 * c * q
    return q + (two_rho > 0), two_rho


def check(c, u, lams):
    for lam in lams:
        got, two_rho = emulate(u, int(lam), c)
        want = -((-u * int(lam)) // c)             # ceil(u l / c)
        assert np.all(np.abs(two_rho) < 2 ** 31), (c, lam)
        bad = np.nonzero(got != want)[0]
        assert len(bad) == 0, (c, lam, u[bad[:5]])


def lambda_sample(c, rng, k=40):
    lams = {2, 3, 4, 5, 7, 8, 1000, c // 2, c // 2 + 1, c - 2, c - 1, c}
    p = 16
    while p <= c:
        lams.update((p - 1, p, p + 1))
        p *= 2
    lams.update(int(x) for x in rng.integers(2, c + 1, size=k))
    return sorted(x for x in lams if 2 <= x <= c)


@pytest.mark.parametrize("c", [65536, 65537, (1 << 22) - 1, 1 << 22])
def test_exhaustive_in_u(c):
    rng = np.random.default_rng(c)
    u = np.arange(1, (c + 1) // 2, dtype=np.int64)  # every u with 2u < c
    check(c, u, lambda_sample(c, rng))


def test_random_capacities():
    rng = np.random.default_rng(7)
    for _ in range(200):
        c = int(rng.integers(65536, (1 << 22) + 1))
        u = rng.integers(1, (c + 1) // 2, size=4000, dtype=np.int64)
        check(c, u, [int(x) for x in rng.integers(2, c + 1, size=4)] + [c])


def test_emulation_has_teeth():
    """The check fails where the argument's premises fail: far past 2^22 the
    product l a leaves [0, 2^21] and the rounded quotient can be off by more
    than one; and without the correction term [rho > 0] the rounded quotient
    is not the ceiling."""
    c = (1 << 24) + 3
    u = np.arange(1, 20001, dtype=np.int64) * 411
    with pytest.raises(AssertionError):
        check(c, u, [c])
    c = 1 << 22
    u = np.arange(1, (c + 1) // 2, 7, dtype=np.int64)
    got = np.rint(np.float64(3) * (u.astype(np.float32) / np.float32(c)).astype(np.float64))
    want = -((-u * 3) // c)
    assert np.any(got.astype(np.int64) != want)   # q~ alone is not the ceiling
