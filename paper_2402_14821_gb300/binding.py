"""Thin Python binding of the C ABI in include/bp_lb.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device
buffers are torch CUDA tensors (only their data pointers are passed); the
stream defaults to torch's current stream.  The CUDA library must have been
built (``paper_2402_14821_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbp_lb.so")

BP_OK, BP_EINVAL, BP_ERANGE, BP_ENOMEM, BP_ECUDA, BP_ETIMEOUT, BP_EBUSY = range(7)
DFF_NAMES = ("MT", "RAD2", "FS1", "CCM1", "VB2", "BJ1")

_c_i64 = ctypes.c_int64
_c_i32 = ctypes.c_int32
_vp = ctypes.c_void_p
_i64p = ctypes.POINTER(ctypes.c_int64)


class BpArgmax(ctypes.Structure):
    _fields_ = [("dff", ctypes.c_int32), ("pad", ctypes.c_int32), ("lam", ctypes.c_int64)]


class BpServeResult(ctypes.Structure):
    _fields_ = [("request", ctypes.c_int64), ("tag", ctypes.c_int64), ("bound", ctypes.c_int64),
                ("dff", ctypes.c_int32), ("argpad", ctypes.c_int32), ("lam", ctypes.c_int64),
                ("latency_us", ctypes.c_double), ("status", ctypes.c_int32),
                ("feasible", ctypes.c_uint8), ("pad", ctypes.c_uint8 * 3)]


class BpLbError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status})")


_lib = None


def _bind(lib):
    P = ctypes.POINTER
    sig = {
        "bp_lb_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "bp_lb_create": (ctypes.c_int, [_c_i64, _c_i64, P(_vp)]),
        "bp_lb_destroy": (ctypes.c_int, [_vp]),
        "bp_lb_reserve": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_eval": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, _i64p, P(BpArgmax)]),
        "bp_lb_eval_node": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i64, _i64p, P(BpArgmax)]),
        "bp_lb_eval_batch": (ctypes.c_int, [_vp, _c_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "bp_lb_eval_batch_i64": (ctypes.c_int, [_vp, _c_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "bp_lb_eval_nodes": (ctypes.c_int, [_vp, _c_i32, _c_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                            _c_i64, _vp, _vp, _vp, _vp]),
        "bp_lb_reduce_nodes": (ctypes.c_int, [_vp, _c_i32, _c_i32, _vp, _vp, _vp, _vp, _vp, _vp,
                                              _vp, _c_i64, _vp, _vp, _vp, _vp]),
        "bp_lb_debug_params": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, _vp, _vp, _c_i64, _vp, _vp]),
        "bp_lb_param_count": (_c_i64, [_c_i32, _c_i64, _i64p, _i64p]),
        "bp_lb_num_launch_shapes": (ctypes.c_int, []),
        "bp_lb_launch_shape_info": (ctypes.c_int, [_c_i32, P(_c_i32), P(_c_i32), P(_c_i32),
                                                   P(_c_i32)]),
        "bp_lb_set_launch_shape": (ctypes.c_int, [_vp, _c_i32, _c_i32]),
        "bp_lb_get_launch_shape": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_autotune_batch": (ctypes.c_int, [_vp, _c_i32, _vp, _vp, _c_i32, _vp, _vp, _vp, _vp,
                                                _vp, _c_i32, _vp, P(_c_i32), _vp]),
        "bp_lb_autotune_nodes": (ctypes.c_int, [_vp, _c_i32, _c_i32, _vp, _vp, _vp, _vp, _vp, _vp,
                                                _vp, _c_i64, _vp, _vp, _vp, _c_i32, _vp, P(_c_i32),
                                                _vp]),
        "bp_lb_selfcheck_division": (_c_i64, [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                              _c_i64]),
        "bp_lb_eval_batch_noalloc": (ctypes.c_int, [_c_i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
        "bp_lb_autotune_plain_node": (ctypes.c_int, [_vp, _vp, _vp, _c_i64, _c_i64, _c_i32, _vp,
                                                     P(_c_i32)]),
        "bp_lb_set_algorithm": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_set_result_mode": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_set_pruning": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_kernel_work": (ctypes.c_int, [_vp, _vp]),
        "bp_lb_set_reduction": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_get_reduction": (ctypes.c_int, [_vp]),
        "bp_lb_set_bin_max": (ctypes.c_int, [_vp, _vp, _vp]),
        "bp_lb_get_pruning": (ctypes.c_int, [_vp]),
        "bp_lb_set_vb2_cap": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_probe_int_issue": (ctypes.c_int, [_c_i32, _c_i32, _vp, _vp, _i64p]),
        "bp_lb_eval_range": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, _c_i64, _c_i64, _vp, _vp]),
        "bp_lb_get_vb2_cap": (ctypes.c_int, [_vp]),
        "bp_lb_set_dff_mask": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_set_overlap": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_set_cluster_tables": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_get_cluster_tables": (ctypes.c_int, [_vp]),
        "bp_lb_kernel_times4": (ctypes.c_int, [_vp, P(ctypes.c_double), P(_c_i64)]),
        "bp_lb_l2_batch": (ctypes.c_int, [_vp, _c_i32, _vp, _vp, _vp, _vp, _vp]),
        "bp_lb_get_dff_mask": (ctypes.c_int, [_vp]),
        "bp_lb_get_result_mode": (ctypes.c_int, [_vp]),
        "bp_lb_get_algorithm": (ctypes.c_int, [_vp]),
        "bp_lb_set_kernel_timing": (ctypes.c_int, [_vp, _c_i32]),
        "bp_lb_dff_route": (ctypes.c_int, [_c_i32, _c_i64, _c_i64, _c_i32]),
        "bp_lb_kernel_times": (ctypes.c_int, [_vp, P(ctypes.c_double), P(ctypes.c_double),
                                              P(ctypes.c_double), P(_c_i64)]),
        "bp_serve_create": (ctypes.c_int, [_c_i64, _c_i32, _c_i64, _c_i32, _c_i32, _c_i64, P(_vp)]),
        "bp_serve_destroy": (ctypes.c_int, [_vp]),
        "bp_serve_register": (ctypes.c_int, [_vp, _vp, _c_i64, _c_i64, P(_c_i32)]),
        "bp_serve_submit": (ctypes.c_int, [_vp, _c_i32, _vp, _c_i64, _c_i64, P(_c_i64)]),
        "bp_serve_poll": (ctypes.c_int, [_vp, P(BpServeResult), _c_i32, P(_c_i32), _c_i32]),
        "bp_serve_stats": (ctypes.c_int, [_vp, P(_c_i64), P(_c_i64), P(_c_i64), P(_c_i64),
                                          P(_c_i64)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2402_14821_gb300.build.build()")
        _lib = _bind(ctypes.CDLL(LIB_PATH))
    return _lib


EXPORTED = ("bp_lb_strerror", "bp_lb_create", "bp_lb_destroy", "bp_lb_reserve", "bp_lb_eval",
            "bp_lb_eval_node", "bp_lb_eval_batch", "bp_lb_eval_batch_i64", "bp_lb_eval_nodes",
            "bp_lb_reduce_nodes", "bp_lb_debug_params", "bp_lb_param_count",
            "bp_lb_selfcheck_division", "bp_lb_num_launch_shapes", "bp_lb_launch_shape_info",
            "bp_lb_set_launch_shape", "bp_lb_get_launch_shape", "bp_lb_autotune_batch",
            "bp_lb_autotune_nodes", "bp_lb_eval_batch_noalloc", "bp_lb_autotune_plain_node",
            "bp_serve_create", "bp_serve_destroy", "bp_serve_register", "bp_serve_submit",
            "bp_serve_poll", "bp_serve_stats", "bp_lb_set_algorithm", "bp_lb_get_algorithm",
            "bp_lb_set_kernel_timing", "bp_lb_kernel_times", "bp_lb_dff_route",
            "bp_lb_set_result_mode", "bp_lb_get_result_mode", "bp_lb_set_dff_mask",
            "bp_lb_get_dff_mask", "bp_lb_l2_batch", "bp_lb_set_overlap", "bp_lb_set_pruning",
            "bp_lb_get_pruning", "bp_lb_kernel_work", "bp_lb_set_reduction",
            "bp_lb_get_reduction", "bp_lb_set_bin_max", "bp_lb_set_vb2_cap",
            "bp_lb_get_vb2_cap", "bp_lb_eval_range", "bp_lb_probe_int_issue",
            "bp_lb_set_cluster_tables", "bp_lb_get_cluster_tables", "bp_lb_kernel_times4")

ALGO_DIRECT, ALGO_PREFIX = 0, 1
RESULT_FULL, RESULT_VERDICT = 0, 1
REDUCE_LOADS, REDUCE_CLOSE = 0, 1

NOALLOC_MAX_BATCH = 4096

MODE_RAGGED_I32, MODE_RAGGED_I64, MODE_NODES, MODE_PLAIN_RAGGED, MODE_PLAIN_NODES = range(5)


def strerror(status: int) -> str:
    return lib().bp_lb_strerror(status).decode()


def _check(status: int, where: str):
    if status != BP_OK:
        raise BpLbError(status, where)


# -- tensor marshalling --------------------------------------------------------
def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def argmax_tensor(B: int, device="cuda"):
    """A [B, 2] int64 tensor laid out as B bp_argmax_t records."""
    import torch
    return torch.empty((B, 2), dtype=torch.int64, device=device)


def decode_argmax(t):
    """(dff int32 array, lambda int64 array) from an argmax tensor / array."""
    a = t.cpu().numpy() if hasattr(t, "cpu") else np.asarray(t)
    a = np.ascontiguousarray(a, dtype=np.int64)
    return (a[:, 0] & 0xFFFFFFFF).astype(np.int64).astype(np.int32), a[:, 1].copy()


# -- handle ----------------------------------------------------------------------
def bp_lb_create(capacity: int, max_items: int):
    h = _vp()
    _check(lib().bp_lb_create(int(capacity), int(max_items), ctypes.byref(h)), "bp_lb_create")
    return h


def bp_lb_destroy(h):
    _check(lib().bp_lb_destroy(h), "bp_lb_destroy")


def bp_lb_reserve(h, max_batch: int):
    _check(lib().bp_lb_reserve(h, int(max_batch)), "bp_lb_reserve")


# -- plain path ------------------------------------------------------------------
def bp_lb_eval(h, sizes, bins: int):
    """Host sizes (int32) -> (bound, dff, lambda)."""
    a = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32))
    b = ctypes.c_int64()
    am = BpArgmax()
    _check(lib().bp_lb_eval(h, a.ctypes.data, len(a), int(bins), ctypes.byref(b), ctypes.byref(am)),
           "bp_lb_eval")
    return b.value, am.dff, am.lam


def bp_lb_eval_node(h, w, assign, bins: int):
    """Host base sizes + assignment -> (bound, dff, lambda)."""
    wa = np.ascontiguousarray(np.asarray(w, dtype=np.int32))
    aa = np.ascontiguousarray(np.asarray(assign, dtype=np.int32))
    if len(wa) != len(aa):
        raise ValueError("w and assign differ in length")
    b = ctypes.c_int64()
    am = BpArgmax()
    _check(lib().bp_lb_eval_node(h, wa.ctypes.data, aa.ctypes.data, len(wa), int(bins),
                                 ctypes.byref(b), ctypes.byref(am)), "bp_lb_eval_node")
    return b.value, am.dff, am.lam


# -- batched path ------------------------------------------------------------------
def bp_lb_eval_batch(h, offsets, sizes, capacity, bins, out_bound, out_argmax=None,
                     out_feasible=None, stream=None):
    import torch
    B = offsets.numel() - 1
    fn = lib().bp_lb_eval_batch if sizes.dtype == torch.int32 else lib().bp_lb_eval_batch_i64
    if sizes.dtype not in (torch.int32, torch.int64):
        raise TypeError("sizes must be int32 or int64")
    _check(fn(h, B, _ptr(offsets, torch.int64, "offsets"), _ptr(sizes, None, "sizes"),
              _ptr(capacity, torch.int64, "capacity"), _ptr(bins, torch.int64, "bins"),
              _ptr(out_bound, torch.int64, "out_bound"), _ptr(out_argmax, torch.int64, "out_argmax"),
              _ptr(out_feasible, torch.uint8, "out_feasible"), _stream(stream)), "bp_lb_eval_batch")


def bp_lb_l2_batch(h, offsets, sizes, capacity, out_l2, stream=None):
    """Martello-Toth L2 of each ragged instance (int32 sizes) into out_l2 (int64)."""
    import torch
    _check(lib().bp_lb_l2_batch(h, offsets.numel() - 1, _ptr(offsets, torch.int64, "offsets"),
                                _ptr(sizes, torch.int32, "sizes"),
                                _ptr(capacity, torch.int64, "capacity"),
                                _ptr(out_l2, torch.int64, "out_l2"), _stream(stream)),
           "bp_lb_l2_batch")


def bp_lb_eval_batch_noalloc(offsets, sizes, capacity, bins, out_bound, out_argmax=None,
                             out_feasible=None, stream=None):
    """bp_lb_eval_batch without a handle and without any device allocation (for
    callers that cannot allocate where they check); at most NOALLOC_MAX_BATCH
    instances; calls that overlap on the GPU race (they share fixed scratch)."""
    import torch
    _check(lib().bp_lb_eval_batch_noalloc(
        offsets.numel() - 1, _ptr(offsets, torch.int64, "offsets"), _ptr(sizes, torch.int32, "sizes"),
        _ptr(capacity, torch.int64, "capacity"), _ptr(bins, torch.int64, "bins"),
        _ptr(out_bound, torch.int64, "out_bound"), _ptr(out_argmax, torch.int64, "out_argmax"),
        _ptr(out_feasible, torch.uint8, "out_feasible"), _stream(stream)),
        "bp_lb_eval_batch_noalloc")


def bp_lb_eval_batch_i64(h, offsets, sizes, capacity, bins, out_bound, out_argmax=None,
                         out_feasible=None, stream=None):
    import torch
    if sizes.dtype != torch.int64:
        raise TypeError("sizes must be int64")
    bp_lb_eval_batch(h, offsets, sizes, capacity, bins, out_bound, out_argmax, out_feasible, stream)


def bp_lb_eval_nodes(h, base_offsets, base_sizes, base_capacity, node_base, assign_offsets,
                     assign, bins, max_bins: int, out_bound, out_argmax=None, out_feasible=None,
                     stream=None):
    import torch
    B = node_base.numel()
    I = base_offsets.numel() - 1
    _check(lib().bp_lb_eval_nodes(
        h, B, I, _ptr(base_offsets, torch.int64, "base_offsets"),
        _ptr(base_sizes, torch.int32, "base_sizes"), _ptr(base_capacity, torch.int64, "base_capacity"),
        _ptr(node_base, torch.int32, "node_base"), _ptr(assign_offsets, torch.int64, "assign_offsets"),
        _ptr(assign, torch.int32, "assign"), _ptr(bins, torch.int64, "bins"), int(max_bins),
        _ptr(out_bound, torch.int64, "out_bound"), _ptr(out_argmax, torch.int64, "out_argmax"),
        _ptr(out_feasible, torch.uint8, "out_feasible"), _stream(stream)), "bp_lb_eval_nodes")


def bp_lb_reduce_nodes(h, base_offsets, base_sizes, base_capacity, node_base, assign_offsets,
                       assign, bins, max_bins: int, out_offsets, out_sizes, out_count, stream=None):
    import torch
    B = node_base.numel()
    I = base_offsets.numel() - 1
    _check(lib().bp_lb_reduce_nodes(
        h, B, I, _ptr(base_offsets, torch.int64, "base_offsets"),
        _ptr(base_sizes, torch.int32, "base_sizes"), _ptr(base_capacity, torch.int64, "base_capacity"),
        _ptr(node_base, torch.int32, "node_base"), _ptr(assign_offsets, torch.int64, "assign_offsets"),
        _ptr(assign, torch.int32, "assign"), _ptr(bins, torch.int64, "bins"), int(max_bins),
        _ptr(out_offsets, torch.int64, "out_offsets"), _ptr(out_sizes, torch.int32, "out_sizes"),
        _ptr(out_count, torch.int64, "out_count"), _stream(stream)), "bp_lb_reduce_nodes")


def bp_lb_debug_params(h, sizes, c: int, dff, lam, out_lb, stream=None):
    import torch
    _check(lib().bp_lb_debug_params(h, _ptr(sizes, torch.int32, "sizes"), sizes.numel(), int(c),
                                    _ptr(dff, torch.int32, "dff"), _ptr(lam, torch.int64, "lam"),
                                    dff.numel(), _ptr(out_lb, torch.int64, "out_lb"),
                                    _stream(stream)), "bp_lb_debug_params")


def bp_lb_param_count(d: int, c: int):
    lo, hi = ctypes.c_int64(), ctypes.c_int64()
    n = lib().bp_lb_param_count(int(d), int(c), ctypes.byref(lo), ctypes.byref(hi))
    return n, lo.value, hi.value


def bp_lb_set_algorithm(h, algo: int):
    _check(lib().bp_lb_set_algorithm(h, int(algo)), "bp_lb_set_algorithm")


def bp_lb_get_algorithm(h) -> int:
    return lib().bp_lb_get_algorithm(h)


def bp_lb_set_result_mode(h, mode: int):
    """RESULT_FULL (exact maximum and argmax) or RESULT_VERDICT (exact verdict,
    early exit; the bound is a genuine witness, not the maximum)."""
    _check(lib().bp_lb_set_result_mode(h, int(mode)), "bp_lb_set_result_mode")


def bp_lb_get_result_mode(h) -> int:
    return lib().bp_lb_get_result_mode(h)


def bp_lb_kernel_work(h):
    """(VB2 pairs by the VB2 kernel, VB2 pairs by the generic kernel, VB2
    parameters evaluated, VB2 parameters pruned) since the last query; counted
    while kernel timing is on."""
    out = np.zeros(4, dtype=np.int64)
    _check(lib().bp_lb_kernel_work(h, out.ctypes.data), "bp_lb_kernel_work")
    return tuple(int(x) for x in out)


def bp_lb_set_reduction(h, mode: int):
    """REDUCE_LOADS (the paper's reduction) or REDUCE_CLOSE (bins that no
    unpacked item fits count as full)."""
    _check(lib().bp_lb_set_reduction(h, int(mode)), "bp_lb_set_reduction")


def bp_lb_get_reduction(h) -> int:
    return lib().bp_lb_get_reduction(h)


def bp_lb_set_bin_max(h, offsets=None, bin_max=None):
    """Per-bin maximum loads (device int64 offsets [B+1], int32 caps) for the
    batched search-node calls; no arguments clears them.  The tensors must
    stay alive while they are set."""
    import torch
    _check(lib().bp_lb_set_bin_max(h, _ptr(offsets, torch.int64, "offsets"),
                                   _ptr(bin_max, torch.int32, "bin_max")),
           "bp_lb_set_bin_max")


def bp_lb_set_pruning(h, on: bool):
    """VB2 pruning on (default) or off; results are identical either way."""
    _check(lib().bp_lb_set_pruning(h, int(bool(on))), "bp_lb_set_pruning")


def bp_lb_get_pruning(h) -> int:
    return lib().bp_lb_get_pruning(h)


def bp_lb_eval_range(h, sizes, c: int, g0: int, g1: int, out_key, stream=None):
    """Packed key (bound << 32 | 2^32 - 1 - g) of one reduced instance (int32
    CUDA tensor) over the flattened parameter indices [g0, g1), written to the
    int64 CUDA tensor out_key[0]."""
    import torch
    n = int(sizes.numel())
    _check(lib().bp_lb_eval_range(h, _ptr(sizes, torch.int32, "sizes") if n else None, n, int(c),
                                  int(g0), int(g1), _ptr(out_key, torch.int64, "out_key"),
                                  _stream(stream)), "bp_lb_eval_range")


def bp_lb_probe_int_issue(blocks_per_sm: int, trips: int, sink, stream=None) -> int:
    """Launches the integer-issue probe; returns the lane operations it performs
    (time the launch with CUDA events on `stream`)."""
    import torch
    ops = ctypes.c_int64()
    _check(lib().bp_lb_probe_int_issue(int(blocks_per_sm), int(trips),
                                       _ptr(sink, torch.int32, "sink"), _stream(stream),
                                       ctypes.byref(ops)), "bp_lb_probe_int_issue")
    return ops.value


def bp_lb_set_vb2_cap(h, on: bool):
    """The paper's VB2 parameter cap (Sec. 4) on or off (default off)."""
    _check(lib().bp_lb_set_vb2_cap(h, int(bool(on))), "bp_lb_set_vb2_cap")


def bp_lb_get_vb2_cap(h) -> int:
    return lib().bp_lb_get_vb2_cap(h)


def bp_lb_set_overlap(h, prefix_ctas_per_sm: int):
    """Prefix-count kernel CTAs per SM beside the VB2 kernel (0: one kernel after another)."""
    _check(lib().bp_lb_set_overlap(h, int(prefix_ctas_per_sm)), "bp_lb_set_overlap")


def bp_lb_set_cluster_tables(h, on: bool):
    """Prefix-count tables of 48-512 KB in a cluster's shared memory (default) or not."""
    _check(lib().bp_lb_set_cluster_tables(h, int(bool(on))), "bp_lb_set_cluster_tables")


def bp_lb_get_cluster_tables(h) -> int:
    return lib().bp_lb_get_cluster_tables(h)


def bp_lb_set_dff_mask(h, mask: int):
    """Bit d keeps DFF d (MT, RAD2, FS1, CCM1, VB2, BJ1) in the bound; 63 = all."""
    _check(lib().bp_lb_set_dff_mask(h, int(mask)), "bp_lb_set_dff_mask")


def bp_lb_get_dff_mask(h) -> int:
    return lib().bp_lb_get_dff_mask(h)


def bp_lb_set_kernel_timing(h, on: bool):
    _check(lib().bp_lb_set_kernel_timing(h, int(bool(on))), "bp_lb_set_kernel_timing")


def bp_lb_kernel_times(h):
    """(ms in the prefix-count kernel, ms in the VB2 kernel, ms in the generic
    direct kernel, calls) since the last query."""
    p, v, d, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(lib().bp_lb_kernel_times(h, ctypes.byref(p), ctypes.byref(v), ctypes.byref(d),
                                    ctypes.byref(n)),
           "bp_lb_kernel_times")
    return p.value, v.value, d.value, n.value


def bp_lb_kernel_times4(h):
    """(ms in the cluster kernel, the prefix-count kernel, the VB2 kernel, the
    generic direct kernel, calls) since the last query."""
    ms = (ctypes.c_double * 4)()
    n = ctypes.c_int64()
    _check(lib().bp_lb_kernel_times4(h, ms, ctypes.byref(n)), "bp_lb_kernel_times4")
    return ms[0], ms[1], ms[2], ms[3], n.value


def bp_lb_dff_route(d: int, c: int, stream_len: int, algo: int = 1) -> int:
    """ALGO_PREFIX or ALGO_DIRECT: the path that evaluates DFF d of such an instance."""
    return lib().bp_lb_dff_route(int(d), int(c), int(stream_len), int(algo))


def bp_lb_num_launch_shapes() -> int:
    return lib().bp_lb_num_launch_shapes()


def bp_lb_launch_shape_info(shape: int):
    """(nt, t, g, min_blocks) of one compiled launch shape."""
    v = [ctypes.c_int32() for _ in range(4)]
    _check(lib().bp_lb_launch_shape_info(int(shape), *[ctypes.byref(x) for x in v]),
           "bp_lb_launch_shape_info")
    return tuple(x.value for x in v)


def bp_lb_set_launch_shape(h, mode: int, shape: int):
    _check(lib().bp_lb_set_launch_shape(h, int(mode), int(shape)), "bp_lb_set_launch_shape")


def bp_lb_get_launch_shape(h, mode: int) -> int:
    return lib().bp_lb_get_launch_shape(h, int(mode))


def bp_lb_autotune_batch(h, offsets, sizes, capacity, bins, out_bound, out_argmax=None,
                         out_feasible=None, reps: int = 3, stream=None):
    """Times every launch shape on this batch; keeps the fastest.  Returns
    (best shape, [ms per shape])."""
    import torch
    n = bp_lb_num_launch_shapes()
    ms = (ctypes.c_float * n)()
    best = ctypes.c_int32()
    _check(lib().bp_lb_autotune_batch(
        h, offsets.numel() - 1, _ptr(offsets, torch.int64, "offsets"), _ptr(sizes, None, "sizes"),
        int(sizes.dtype == torch.int64), _ptr(capacity, torch.int64, "capacity"),
        _ptr(bins, torch.int64, "bins"), _ptr(out_bound, torch.int64, "out_bound"),
        _ptr(out_argmax, torch.int64, "out_argmax"), _ptr(out_feasible, torch.uint8, "out_feasible"),
        int(reps), ms, ctypes.byref(best), _stream(stream)), "bp_lb_autotune_batch")
    return best.value, list(ms)


def bp_lb_autotune_nodes(h, base_offsets, base_sizes, base_capacity, node_base, assign_offsets,
                         assign, bins, max_bins: int, out_bound, out_argmax=None, out_feasible=None,
                         reps: int = 3, stream=None):
    """Times every launch shape on this node batch; keeps the fastest.  Returns
    (best shape, [ms per shape])."""
    import torch
    n = bp_lb_num_launch_shapes()
    ms = (ctypes.c_float * n)()
    best = ctypes.c_int32()
    _check(lib().bp_lb_autotune_nodes(
        h, node_base.numel(), base_offsets.numel() - 1, _ptr(base_offsets, torch.int64, "base_offsets"),
        _ptr(base_sizes, torch.int32, "base_sizes"), _ptr(base_capacity, torch.int64, "base_capacity"),
        _ptr(node_base, torch.int32, "node_base"), _ptr(assign_offsets, torch.int64, "assign_offsets"),
        _ptr(assign, torch.int32, "assign"), _ptr(bins, torch.int64, "bins"), int(max_bins),
        _ptr(out_bound, torch.int64, "out_bound"), _ptr(out_argmax, torch.int64, "out_argmax"),
        _ptr(out_feasible, torch.uint8, "out_feasible"), int(reps), ms, ctypes.byref(best),
        _stream(stream)), "bp_lb_autotune_nodes")
    return best.value, list(ms)


def bp_lb_autotune_plain_node(h, w, assign, bins: int, reps: int = 20):
    """Times the plain node path with every algorithm and launch shape; keeps the
    fastest.  Returns (best index, [microseconds per call]): index a * shapes + s
    for algorithm a (0 direct, 1 prefix) and shape s."""
    wa = np.ascontiguousarray(np.asarray(w, dtype=np.int32))
    aa = np.ascontiguousarray(np.asarray(assign, dtype=np.int32))
    n = 2 * bp_lb_num_launch_shapes()
    us = (ctypes.c_float * n)()
    best = ctypes.c_int32()
    _check(lib().bp_lb_autotune_plain_node(h, wa.ctypes.data, aa.ctypes.data, len(wa), int(bins),
                                           int(reps), us, ctypes.byref(best)),
           "bp_lb_autotune_plain_node")
    return best.value, list(us)


def bp_lb_selfcheck_division(d_lo: int, d_hi: int, n_hi: int, samples: int) -> int:
    return lib().bp_lb_selfcheck_division(d_lo, d_hi, n_hi, samples)


# -- serving -------------------------------------------------------------------------
def bp_serve_create(pool_items: int, max_instances: int, max_queued_items: int, slots: int = 3,
                    max_batch: int = 4096, max_bins: int = 16384):
    s = _vp()
    _check(lib().bp_serve_create(int(pool_items), int(max_instances), int(max_queued_items),
                                 int(slots), int(max_batch), int(max_bins), ctypes.byref(s)),
           "bp_serve_create")
    return s


def bp_serve_destroy(s):
    _check(lib().bp_serve_destroy(s), "bp_serve_destroy")


def bp_serve_register(s, sizes, capacity: int) -> int:
    a = np.ascontiguousarray(np.asarray(sizes, dtype=np.int32))
    i = ctypes.c_int32()
    _check(lib().bp_serve_register(s, a.ctypes.data, len(a), int(capacity), ctypes.byref(i)),
           "bp_serve_register")
    return i.value


def bp_serve_submit(s, instance: int, assign, bins: int, tag: int = 0):
    """Returns the request id, or None when admission refused it (BP_EBUSY)."""
    a = np.ascontiguousarray(np.asarray(assign, dtype=np.int32))
    rid = ctypes.c_int64()
    st = lib().bp_serve_submit(s, int(instance), a.ctypes.data, int(bins), int(tag),
                               ctypes.byref(rid))
    if st == BP_EBUSY:
        return None
    _check(st, "bp_serve_submit")
    return rid.value


def bp_serve_poll(s, max_results: int = 1024, wait_us: int = 0):
    """List of finished results (BpServeResult records)."""
    buf = (BpServeResult * max_results)()
    cnt = ctypes.c_int32()
    st = lib().bp_serve_poll(s, buf, int(max_results), ctypes.byref(cnt), int(wait_us))
    if st not in (BP_OK, BP_ETIMEOUT):
        _check(st, "bp_serve_poll")
    return [buf[i] for i in range(cnt.value)]


def bp_serve_stats(s):
    v = [ctypes.c_int64() for _ in range(5)]
    st = lib().bp_serve_stats(s, *[ctypes.byref(x) for x in v])
    return dict(zip(("pending", "queued_items", "batches", "done", "refused"),
                    (x.value for x in v)), status=st)
