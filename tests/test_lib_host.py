"""CPU-only checks of the CUDA library: it builds, loads, exports every entry
point include/bp_lb.h declares, and its host-side helpers (parameter ranges,
exact division by invariant integers) are right.  No kernel runs here."""
import ctypes
import os
import re

import pytest

from paper_2402_14821_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.lib()


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "bp_lb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bp_(?:lb|serve)_\w+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 12
    cdll = ctypes.CDLL(binding.LIB_PATH)
    for n in names:
        assert hasattr(cdll, n), n
    assert set(names) == set(binding.EXPORTED)


def test_strerror(lib):
    assert binding.strerror(0) == "ok"
    assert "range" in binding.strerror(2)


def test_param_count_matches_oracle(lib, orc):
    for c in list(range(1, 64)) + [150, 1000, 65535, 65536, 10 ** 6, 2 ** 30]:
        for d in range(6):
            n, lo, hi = binding.bp_lb_param_count(d, c)
            olo, ohi, on = orc.param_range(d, c)
            assert n == on, (d, c)
            if n:
                assert (lo, hi) == (olo, ohi)
    assert binding.bp_lb_param_count(6, 10)[0] == -1
    assert binding.bp_lb_param_count(0, 0)[0] == -1
    assert binding.bp_lb_param_count(0, 2 ** 30 + 1)[0] == -1


def test_exact_division_small_exhaustive(lib):
    # every divisor up to 2^11 on every numerator up to 2^12
    assert binding.bp_lb_selfcheck_division(1, 2048, 4096, 64) == 0


def test_exact_division_wide(lib):
    # divisors near powers of two and at the top of the range, random numerators < 2^31
    for lo in (2 ** 15 - 8, 2 ** 16 - 8, 2 ** 20 - 8, 2 ** 24 - 8, 2 ** 30 - 8, 2 ** 31 - 64):
        assert binding.bp_lb_selfcheck_division(lo, lo + 63, 64, 4000) == 0
    assert binding.bp_lb_selfcheck_division(0, 5, 5, 0) == -1


def test_create_rejects_bad_arguments(lib):
    for cap, items in ((0, 10), (2 ** 30 + 1, 10), (10, 0), (10, 2 ** 20 + 1)):
        with pytest.raises(binding.BpLbError) as e:
            binding.bp_lb_create(cap, items)
        assert e.value.status == binding.BP_ERANGE


def test_serve_rejects_bad_arguments_before_any_device_work(lib):
    for args in ((0, 4, 100, 2, 8, 16), (100, 0, 100, 2, 8, 16), (100, 4, 0, 2, 8, 16),
                 (100, 4, 100, 0, 8, 16), (100, 4, 100, 17, 8, 16), (100, 4, 100, 2, 0, 16),
                 (100, 4, 100, 2, 8, 16385)):
        with pytest.raises(binding.BpLbError) as e:
            binding.bp_serve_create(*args)
        assert e.value.status == binding.BP_ERANGE
    assert binding.lib().bp_serve_destroy(None) == binding.BP_OK
    assert binding.lib().bp_serve_stats(None, None, None, None, None, None) == binding.BP_EINVAL


def test_dff_route(lib):
    P, D = binding.ALGO_PREFIX, binding.ALGO_DIRECT
    # VB2 is always direct; MT/RAD2/FS1/CCM1/BJ1 go to the prefix tables
    # (shared memory up to 48 KiB, else a 4 MiB global slice per CTA:
    # FS1, BJ1 4 (c + 2) bytes; RAD2 8 ((c-1)/2 + 2); MT, CCM1 4 ((c-1)/2 + 2))
    assert binding.bp_lb_dff_route(4, 1000, 500, P) == D
    for d in (0, 1, 2, 3, 5):
        assert binding.bp_lb_dff_route(d, 10_000, 630, P) == P
        assert binding.bp_lb_dff_route(d, 10_000, 630, D) == D
        assert binding.bp_lb_dff_route(d, 100_000, 500, P) == P      # global tables
    for d in (2, 5):
        assert binding.bp_lb_dff_route(d, 1_048_574, 10, P) == P
        assert binding.bp_lb_dff_route(d, 1_048_575, 10, P) == D
    assert binding.bp_lb_dff_route(1, 1_048_574, 10, P) == P
    assert binding.bp_lb_dff_route(1, 1_048_575, 10, P) == D
    for d in (0, 3):
        assert binding.bp_lb_dff_route(d, 2_097_150, 10, P) == P
        assert binding.bp_lb_dff_route(d, 2_097_151, 10, P) == D
    # reduced sizes that could sum past 2^31 stay direct
    assert binding.bp_lb_dff_route(3, 10_000, 300_000, P) == D
    # FS1's count sum (at most 101 sum w / c) must fit 32 bits: streams below 2^25
    assert binding.bp_lb_dff_route(2, 10, (1 << 25) - 1, P) == P
    assert binding.bp_lb_dff_route(2, 10, 1 << 25, P) == D
    assert binding.bp_lb_dff_route(6, 10, 1, P) == -1
