"""CPU oracle for the DFF-based feasibility check (arXiv 2402.14821).

TEST INFRASTRUCTURE ONLY.  The arithmetic lives in ``bp_oracle.c`` (plain C,
int64, the literal definitions of Sec. 3.1 and Alg. 2); this module compiles it
with gcc and marshals numpy arrays through ctypes.  Only the tests, the smoke
check and the benchmark's CPU-baseline leg may import this package; the CUDA
library never does, and this package imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MT, RAD2, FS1, CCM1, VB2, BJ1 = range(6)
NAMES = ("MT", "RAD2", "FS1", "CCM1", "VB2", "BJ1")

_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_u8p = ctypes.POINTER(ctypes.c_uint8)


def build(src: str = _SRC, out: str = _LIB, extra_flags=()) -> str:
    """Compile the oracle into a shared library (gcc, -O2, no tuning)."""
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra_flags, src, "-o", out]
    subprocess.run(cmd, check=True)
    return out


def _bind(lib):
    lib.orc_param_range.argtypes = [ctypes.c_int, ctypes.c_int64, _i64p, _i64p]
    lib.orc_param_range.restype = ctypes.c_int64
    lib.orc_dff.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64]
    lib.orc_dff.restype = ctypes.c_int64
    lib.orc_lb_param.argtypes = [ctypes.c_int, ctypes.c_int64, _i64p, ctypes.c_int64, ctypes.c_int64]
    lib.orc_lb_param.restype = ctypes.c_int64
    lib.orc_lb_dff.argtypes = [ctypes.c_int, _i64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                               _i64p]
    lib.orc_lb_dff.restype = ctypes.c_int64
    lib.orc_lb.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                           _i64p, _i32p, _i64p]
    lib.orc_lb.restype = ctypes.c_int
    lib.orc_reduce.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _i64p]
    lib.orc_reduce.restype = ctypes.c_int64
    lib.orc_reduce_ex.argtypes = [_i64p, _i32p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                  ctypes.c_int, _i64p, _i64p]
    lib.orc_reduce_ex.restype = ctypes.c_int64
    lib.orc_l1.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int64]
    lib.orc_l1.restype = ctypes.c_int64
    lib.orc_l2.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int64]
    lib.orc_l2.restype = ctypes.c_int64
    lib.orc_opt_bins.argtypes = [_i64p, ctypes.c_int64, ctypes.c_int64]
    lib.orc_opt_bins.restype = ctypes.c_int64
    lib.orc_dff_knapsack_max.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64]
    lib.orc_dff_knapsack_max.restype = ctypes.c_int64
    lib.orc_lb_batch.argtypes = [ctypes.c_int64, _i64p, _i64p, _i64p, _i64p, ctypes.c_int,
                                 _i64p, _i32p, _i64p, _u8p]
    lib.orc_lb_batch.restype = ctypes.c_int
    return lib


class Oracle:
    """ctypes view of one compiled oracle library."""

    def __init__(self, path: str):
        self.path = path
        self.lib = _bind(ctypes.CDLL(path))

    # -- helpers -----------------------------------------------------------
    @staticmethod
    def _arr64(x):
        a = np.ascontiguousarray(np.asarray(x, dtype=np.int64))
        return a, a.ctypes.data_as(_i64p)

    # -- API ---------------------------------------------------------------
    def param_range(self, d: int, c: int):
        lo, hi = ctypes.c_int64(), ctypes.c_int64()
        n = self.lib.orc_param_range(d, c, ctypes.byref(lo), ctypes.byref(hi))
        return lo.value, hi.value, n

    def dff(self, d: int, w: int, lam: int, c: int) -> int:
        return self.lib.orc_dff(d, w, lam, c)

    def lb_param(self, d: int, lam: int, wr, c: int) -> int:
        a, p = self._arr64(wr)
        return self.lib.orc_lb_param(d, lam, p, len(a), c)

    def lb_dff(self, d: int, wr, c: int, vb2_cap: bool = False):
        """L_f of one DFF: (bound, first attaining lambda); bound -1 for an empty range."""
        a, p = self._arr64(wr)
        l = ctypes.c_int64()
        v = self.lib.orc_lb_dff(d, p, len(a), c, int(vb2_cap), ctypes.byref(l))
        return v, l.value

    def lb(self, wr, c: int, k: int, vb2_cap: bool = False):
        """Returns (bound, dff, lambda, feasible)."""
        a, p = self._arr64(wr)
        b, d, l = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
        ok = self.lib.orc_lb(p, len(a), c, k, int(vb2_cap), ctypes.byref(b), ctypes.byref(d),
                             ctypes.byref(l))
        if ok < 0:
            raise ValueError("oracle: invalid instance")
        return b.value, d.value, l.value, bool(ok)

    def reduce(self, w, assign, k: int, c: int) -> np.ndarray:
        a, p = self._arr64(w)
        asg = np.ascontiguousarray(np.asarray(assign, dtype=np.int32))
        out = np.zeros(len(a) + max(k, 0), dtype=np.int64)
        r = self.lib.orc_reduce(p, asg.ctypes.data_as(_i32p), len(a), k, c, out.ctypes.data_as(_i64p))
        if r < 0:
            raise ValueError("oracle: invalid partial packing")
        return out[:r].copy()

    def reduce_ex(self, w, assign, k: int, c: int, mode: int = 0, bin_max=None) -> np.ndarray:
        """A reduction variant (orc_reduce_ex): mode 1 closes bins that no
        unpacked item fits; bin_max caps each bin's load."""
        a, p = self._arr64(w)
        asg = np.ascontiguousarray(np.asarray(assign, dtype=np.int32))
        out = np.zeros(len(a) + max(k, 0), dtype=np.int64)
        bm = None
        if bin_max is not None:
            bm = np.ascontiguousarray(np.asarray(bin_max, dtype=np.int64))
            if len(bm) != k:
                raise ValueError("bin_max needs one entry per bin")
        r = self.lib.orc_reduce_ex(p, asg.ctypes.data_as(_i32p), len(a), k, c, int(mode),
                                   bm.ctypes.data_as(_i64p) if bm is not None else None,
                                   out.ctypes.data_as(_i64p))
        if r < 0:
            raise ValueError("oracle: invalid partial packing")
        return out[:r].copy()

    def l1(self, w, c: int) -> int:
        a, p = self._arr64(w)
        return self.lib.orc_l1(p, len(a), c)

    def l2(self, w, c: int) -> int:
        a, p = self._arr64(w)
        return self.lib.orc_l2(p, len(a), c)

    def opt_bins(self, w, c: int) -> int:
        a, p = self._arr64(w)
        return self.lib.orc_opt_bins(p, len(a), c)

    def dff_knapsack_max(self, d: int, lam: int, c: int) -> int:
        return self.lib.orc_dff_knapsack_max(d, lam, c)

    def lb_batch(self, offsets, sizes, cap, bins, vb2_cap: bool = False):
        """Ragged batch; returns (bound, dff, lambda, feasible) arrays."""
        o, po = self._arr64(offsets)
        s, ps = self._arr64(sizes)
        cp_, pc = self._arr64(cap)
        bn, pb = self._arr64(bins)
        B = len(o) - 1
        ob = np.zeros(B, np.int64)
        od = np.zeros(B, np.int32)
        ol = np.zeros(B, np.int64)
        of = np.zeros(B, np.uint8)
        rc = self.lib.orc_lb_batch(B, po, ps, pc, pb, int(vb2_cap), ob.ctypes.data_as(_i64p),
                                   od.ctypes.data_as(_i32p), ol.ctypes.data_as(_i64p),
                                   of.ctypes.data_as(_u8p))
        if rc != 0:
            raise ValueError("oracle: invalid instance in batch")
        return ob, od, ol, of.astype(bool)


_default: Oracle | None = None


def load() -> Oracle:
    """The oracle compiled from bp_oracle.c (built on first use if missing or stale)."""
    global _default
    if _default is None:
        if not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            build()
        _default = Oracle(_LIB)
    return _default
