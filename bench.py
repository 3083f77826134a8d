#!/usr/bin/env python3
"""Benchmark of the DFF lower-bound feasibility check on GB300.

Workload (one step): the search-node batch -- one base instance of n = 500
items with sizes uniform in [1, c/2], c = 10^4, k = ceil(sum/c) + 1 bins, and
4096 partial packings of it (a uniform 0..60% of the items committed to random
bins without overflow).  A step reduces every node on the device (Sec. 3,
Fig. 3) and evaluates the full collection of DFF bounds (Alg. 2, all six DFFs
and all their integer parameters) for each of them: one bp_lb_eval_nodes call.

Reported: batched feasibility checks/s (value), item-parameter evals/s, the
plain one-check-per-launch path (bp_lb_eval_node: H2D, one launch, D2H, sync)
with its p50/p99 latency, the end-to-end rate with host buffers, the roofline
of the evaluation kernel against the integer issue rate, and the CPU oracle on
a bounded sample of the same workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
(N > 1 under torch.distributed.run: every rank runs its own batch; weak scaling.)
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "feasibility checks/s and item-param evals/s, batched vs plain; p50/p99 ms"
UNIT = "checks/s"
WORKLOAD = "search-node batch: {} partial packings of n=500 items, sizes U[1,c/2], c=10000"
NODES, N_ITEMS, CAP = 4096, 500, 10_000

# Thread instructions per (item, parameter) pair of each DFF's item-by-item
# evaluation: measured with ncu where the workloads use the path
# (smsp__inst_executed.sum x 32 / pairs of one launch, pruning off, one
# instance of n = 10^4; profiles/item_kernels_instructions_per_eval.md):
#   generic kernel at c = 10^6: MT 2.39, RAD2 4.59, CCM1 2.87 (its wide path,
#   c > 131071), VB2 5.71 (fp32-corrected path, 65535 < c <= 2^22), BJ1 5.45
#   (wide path, c > 65535); VB2 kernel (fixed point, c <= 65535): 2.68.
# The paths no workload puts on the item-by-item kernels keep the integer
# operations counted from the source expressions of csrc/bp_lb_eval.cuh:
# FS1 7 (mul, mul-high, shift, add, mul, compare, conditional add), CCM1 1 at
# c <= 131071 (one multiply-high-add), BJ1 5 at c <= 65535, VB2 5 above 2^22.
def ops_per_eval(d, c):
    return {0: 2.39, 1: 4.59, 2: 7,
            3: 1 if c <= 131071 else 2.87,
            4: 2.68 if c <= 65535 else (5.71 if c <= 1 << 22 else 5),
            5: 5 if c <= 65535 else 5.45}[d]
SM_COUNT_NOMINAL = 152
# DRAM bytes (read + write) per search node of one launch of each kernel, from
# one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum of a 512-node
# launch, divided by 512: traffic grows with the nodes, each node's inputs
# being read from DRAM once; profiles/prefix_kernel_search_nodes.md), or None
# while the kernel has changed since the last capture.
TRAFFIC_BYTES_PER_NODE = {"prefix": 2352, "vb2": None, "direct": None}

# Prefix-count kernel: its algorithmic work is shared-memory table traffic, in
# 32-bit words -- zeroing, histogram updates, three accesses per entry and
# scan, and the lookups of every parameter it does not prune (csrc/
# bp_lb_prefix.cuh) -- against one 32-lane word access per SM per clock.
PREFIX_CTA_BLOCKS, PREFIX_WARP_BLOCKS, PREFIX_MAX_HEAVY, PREFIX_PRUNE_MIN = 1024, 32, 256, 4


def param_counts(c):
    from paper_2402_14821_gb300 import binding as B
    return [B.bp_lb_param_count(d, c)[0] for d in range(6)]


def reduced_sizes(nd):
    """r of each node: unpacked items + non-empty bins (all sizes are >= 1)."""
    r = np.empty(nd.count, dtype=np.int64)
    for j in range(nd.count):
        a = nd.assign[nd.assign_offsets[j]:nd.assign_offsets[j + 1]]
        r[j] = int(np.sum(a == -1)) + len(np.unique(a[a >= 0]))
    return r


def _warp_end(X):
    """First parameter of the prefix kernel's thread phase (CCM1: X = U, BJ1: X = c)."""
    return max(min(X // PREFIX_CTA_BLOCKS + 1, 1 + PREFIX_MAX_HEAVY), X // PREFIX_WARP_BLOCKS + 1)


def prefix_smem_words(nd, prune=True):
    """Shared-memory words of one prefix-kernel launch on a search-node batch
    with every node at capacity c <= 12286 (tables in shared memory, u group
    merged, FS1 on BJ1's tile, one tile each), pruning as in the kernel
    (against L1: prune_bj1, prune_ccm1)."""
    total = 0
    cache = {}
    for j in range(nd.count):
        w, a, c, k = nd.node(j)
        w = np.asarray(w, dtype=np.int64)
        a = np.asarray(a)
        loads = np.bincount(a[a >= 0], weights=w[a >= 0], minlength=k).astype(np.int64)
        red = np.concatenate([w[a < 0], loads])
        n_as = int(np.sum(a >= 0))
        U = (c - 1) // 2
        nU, nW = U + 2, c + 2
        small = red[(red > 0) & (2 * red < c)]
        big = red[(2 * red > c) & (red < c)]
        nh, nf, nb = int(np.sum(2 * red == c)), int(np.sum(red == c)), len(big)
        sumw = int(red.sum())
        L1 = -(-sumw // c)
        sws, sub = int(small.sum()), int((c - big).sum())
        kS = 2 * nb + nh + 2 * nf
        key = (c, sumw)
        if key not in cache:
            # BJ1: one lookup per multiple of l (the D table), none when c mod l
            # = 0; pruned in the CTA and warp phases, and in the thread phase
            # when it has at least PREFIX_PRUNE_MIN terms
            lam = np.arange(1, c + 1, dtype=np.int64)
            q, cm = c // lam, c % lam
            heavy = lam < _warp_end(c)
            cut = prune & (L1 * (c - cm) >= sumw) & (heavy | (q >= PREFIX_PRUNE_MIN))
            keep = (cm > 0) & ~cut
            lp = np.arange(2, 102)
            fs1 = 2 * int(lp.sum()) + 2 * int(sum(np.gcd(c, lp)))
            cache[key] = int(q[keep].sum()) + fs1 + 4 * (c // 2 + 1)   # + NN -> D
        # node loads, once per tile: zero k, one atomic per packed item, read k
        loads_words = 2 * (k + n_as + k)
        # u group: E and packed counts (zero, 2 updates per small or big item,
        # 2 scans), MT 1 lookup per parameter, RAD2 3, CCM1 floor(U / l)
        lam = np.arange(1, c // 2 + 1, dtype=np.int64)
        q = c // lam
        ccm1_keep = ~(prune & (2 * sws - 2 * sub + 2 * nb * (lam - 1) + q * lam * kS
                               <= 2 * q * lam * L1)
                      & ((lam < _warp_end(U)) | (q >= PREFIX_PRUNE_MIN)))
        ccm1 = int((U // lam)[ccm1_keep].sum())
        pc = param_counts(c)
        u_words = 2 * nU + 2 * (len(small) + nb) + 6 * nU + pc[0] + 3 * pc[1] + ccm1
        # VB2 on the u-group tile (vb2_table_plan): floor((U l - 1) / c) + 1
        # lookups for each l in [2, lmax] when pruning leaves only those
        if prune and c <= VB2_FIXED_CAP:
            L = len(w) + k
            kk = min(L1, L)
            D = sws - sub
            alpha = 2 * D - c * (2 * kk - kS)
            beta = 2 * len(small) * (c - 1) + c * (2 * kk - kS) - c * (2 * len(small) - 2 * nb + 1) + 2
            if alpha < 0 and 2 * alpha + beta > 0:
                lmax = min(c, (beta - 1) // (-alpha))
                if U * lmax * lmax // (2 * c) + lmax <= 1 << 16:
                    lv = np.arange(2, lmax + 1, dtype=np.int64)
                    u_words += int(((U * lv - 1) // c + 1).sum())
        # w group: NN (zero, one update per reduced item, scanned twice), FS1, BJ1
        w_words = nW + len(red) + 3 * nW + cache[key]
        total += loads_words + u_words + w_words
    return total


VB2_FIXED_CAP = 65535


def kernel_of(d, c, stream_len, algo=1):
    """Which batched kernel evaluates DFF d: "prefix" (the prefix-count kernel,
    where bp_lb_dff_route says so), "vb2" (VB2 at c <= 65535, its own kernel)
    or "direct" (the generic direct kernel)."""
    from paper_2402_14821_gb300 import binding as B
    if B.bp_lb_dff_route(d, c, stream_len, algo) == B.ALGO_PREFIX:
        return "prefix"
    return "vb2" if d == 4 and c <= VB2_FIXED_CAP else "direct"


def algorithmic_work(nd, algo=1):
    """(item-parameter pairs of the whole check, {kernel: integer ops}) of one
    batch: the generic direct kernel evaluates every (item, parameter) pair of
    the DFFs other than VB2 routed to it; MT, RAD2, FS1, CCM1 and BJ1 go to the
    prefix-count kernel where their tables fit.  VB2's pairs are pruned on the
    device, which counts the ones it evaluates (bp_lb_kernel_work)."""
    r = reduced_sizes(nd)
    evals = 0
    ops = {"vb2": 0, "direct": 0, "prefix": 0}
    for j in range(nd.count):
        b = int(nd.node_base[j])
        c = int(nd.base.capacity[b])
        L = int(nd.base.offsets[b + 1] - nd.base.offsets[b]) + int(nd.bins[j])
        cnt = param_counts(c)
        for d in range(6):
            evals += int(r[j]) * cnt[d]
            k = kernel_of(d, c, L, algo)
            if k != "prefix" and d != 4:
                ops[k] += r[j] * cnt[d] * ops_per_eval(d, c)
    return evals, ops


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self._t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------------------
# CPU oracle leg
# ---------------------------------------------------------------------------
def _oracle_node_fn(nd):
    import oracle
    orc = oracle.load()

    def one(j):
        w, a, c, k = nd.node(j % nd.count)
        orc.lb(orc.reduce(w, a, k, c), c, k)
    return one


def oracle_sample_size(nd, budget_s: float, threads: int) -> int:
    """Nodes the oracle checks in about budget_s seconds of wall time on
    `threads` host threads (from the time of one node)."""
    one = _oracle_node_fn(nd)
    t0 = time.perf_counter()
    one(0)
    t_one = max(time.perf_counter() - t0, 1e-4)
    return int(min(nd.count, max(threads, budget_s * threads / t_one)))


def oracle_run(nd, first: int, m: int, threads: int) -> float:
    """Wall seconds of the oracle (reduction + full bound) over nodes first ..
    first + m - 1 (mod the batch), on `threads` host threads (ctypes releases
    the GIL)."""
    one = _oracle_node_fn(nd)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        list(ex.map(one, range(first, first + m)))
    return time.perf_counter() - t0


def oracle_rate(nd, budget_s: float, threads: int):
    """Checks/s of the oracle over a bounded sample of the nodes (about
    budget_s seconds of wall time): (rate, nodes, wall seconds)."""
    m = oracle_sample_size(nd, budget_s, threads)
    wall = oracle_run(nd, 0, m, threads)
    return m / wall, m, wall


# ---------------------------------------------------------------------------
def main():
    global NODES
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=150)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--nodes", type=int, default=NODES,
                    help="search nodes per batch (4096 is the benchmark workload)")
    ap.add_argument("--plain-sample", type=int, default=1024)
    ap.add_argument("--shape", type=int, default=-1,
                    help="fix the batched launch shape (default: autotune on the batch)")
    ap.add_argument("--cpu-budget", type=float, default=15.0,
                    help="CPU-seconds of oracle work for the cpu_baseline sample")
    ap.add_argument("--workload", choices=("search", "plain", "large", "ragged", "serve", "table1",
                                           "issue", "hard"),
                    default="search",
                    help="search: the benchmark line (4096 search nodes); plain: one check of "
                         "n=50, c=150 per call (bp_lb_eval), 10^4 calls; large: n=10^4, "
                         "c in {1e5, 1e6}, three size families, batches of 64; ragged: 10^4 "
                         "ragged search nodes in one CUDA-graph launch; serve: 256 simulated "
                         "searches against the continuous-batching server, offered rates swept; "
                         "issue: the integer-issue probe alone; hard: the hard search-node "
                         "batch alone (the benchmark line's hard_nodes record)")
    ap.add_argument("--large-cases", default="",
                    help="large: comma-separated c:family cases (default: both c, all families)")
    ap.add_argument("--large-count", type=int, default=64, help="large: instances per batch")
    ap.add_argument("--dff-mask", type=int, default=63, help="large: DFFs in the bound (bits)")
    ap.add_argument("--no-prune", action="store_true", help="large: pruning off (all the work)")
    ap.add_argument("--large-dtypes", default="int32,int64", help="large: size types")
    ap.add_argument("--cluster", choices=("auto", "on", "off"), default="auto",
                    help="cluster tables (bp_lb_set_cluster_tables) of every handle: auto = the "
                         "handle's default, switched by the autotuner where one runs; on / off "
                         "forced, also after autotuning")
    ap.add_argument("--records", default="hard,large",
                    help="secondary records of the benchmark line (comma-separated: hard, large; "
                         "'none' for the search-node step alone, e.g. under a profiler)")
    args = ap.parse_args()
    global CLUSTER_TABLES
    CLUSTER_TABLES = args.cluster
    if args.workload != "search":
        return run_sweep(args)

    NODES = args.nodes
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    from paper_2402_14821_gb300 import instances as I

    if args.impl == "reference":
        if rank != 0:
            return
        nd = I.search_nodes(seed=1, n=N_ITEMS, c=CAP, nodes=NODES)
        threads = os.cpu_count() or 1
        # one step = the oracle over a fixed bounded sample of m nodes (about
        # `budget` seconds), consecutive steps taking consecutive nodes;
        # ms_per_step is the wall time of the step that ran
        budget = max(1.0, 45.0 / max(1, args.steps + args.warmup))
        m = oracle_sample_size(nd, budget, threads)
        walls = []
        for i in range(args.warmup + args.steps):
            wall = oracle_run(nd, i * m, m, threads)
            if i >= args.warmup:
                walls.append(wall)
        t_step = float(np.mean(walls))
        value = m / t_step
        line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": t_step * 1e3, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
                "config": {"workload": WORKLOAD.format(NODES), "nodes": NODES, "n": N_ITEMS, "c": CAP,
                           "nodes_per_step": m,
                           "step": f"the oracle over {m} of the {NODES} nodes (a bounded sample; "
                                   "consecutive steps take consecutive nodes)"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": f"{m} of the {NODES} nodes per step, reduction + "
                                           f"full bound, {threads} host threads"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    from paper_2402_14821_gb300 import binding as B
    from paper_2402_14821_gb300 import build

    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    build.build()
    dev = torch.device("cuda")
    stream = torch.cuda.current_stream()

    # the integer issue peak this device sustains (the ALU-bound kernels'
    # roofline denominator), measured before anything else runs
    ipeak = issue_peak(B, stream)

    nd = I.search_nodes(seed=1 + rank, n=N_ITEMS, c=CAP, nodes=NODES)
    evals, ops = algorithmic_work(nd)

    def d(x, dt):
        return torch.from_numpy(np.ascontiguousarray(x)).to(dt).to(dev)

    t_in = dict(base_offsets=d(nd.base.offsets, torch.int64), base_sizes=d(nd.base.sizes, torch.int32),
                base_capacity=d(nd.base.capacity, torch.int64), node_base=d(nd.node_base, torch.int32),
                assign_offsets=d(nd.assign_offsets, torch.int64), assign=d(nd.assign, torch.int32),
                bins=d(nd.bins, torch.int64))
    max_bins = int(nd.bins.max())
    out_b = torch.empty(NODES, dtype=torch.int64, device=dev)
    out_a = B.argmax_tensor(NODES)
    out_f = torch.empty(NODES, dtype=torch.uint8, device=dev)
    h = new_handle(B, CAP, 1 << 16)
    B.bp_lb_reserve(h, NODES)
    # autotuner: pick the launch shape on this batch (not timed)
    if args.shape >= 0:
        shape, shape_ms = args.shape, []
        B.bp_lb_set_launch_shape(h, B.MODE_NODES, shape)
    else:
        shape, shape_ms = B.bp_lb_autotune_nodes(h, max_bins=max_bins, out_bound=out_b,
                                                 out_argmax=out_a, out_feasible=out_f, reps=2,
                                                 stream=stream, **t_in)
        cluster_setting(B, h)

    def step():
        B.bp_lb_eval_nodes(h, max_bins=max_bins, out_bound=out_b, out_argmax=out_a,
                           out_feasible=out_f, stream=stream, **t_in)

    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident batched path ---------------------------------------
    for _ in range(max(3, args.warmup)):
        step()
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # the steps as a user runs them (no per-kernel events between the kernels)
    with ClockSampler(torch.cuda.current_device()) as clk:
        barrier()
        for e0, e1 in ev:
            flush.zero_()
            e0.record(stream)
            step()
            e1.record(stream)
        barrier()
    step_ms = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
    # the same steps again with events around each kernel, on its stream, for
    # the per-kernel times of the roofline (they separate the kernels, so this
    # pass's steps are a little longer)
    B.bp_lb_set_kernel_timing(h, True)
    B.bp_lb_kernel_times(h)
    ev_k = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in range(max(3, args.steps // 3))]
    barrier()
    for e0, e1 in ev_k:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    barrier()
    step_ms_timed = np.array([e0.elapsed_time(e1) for e0, e1 in ev_k])
    ms_cluster, ms_prefix, ms_vb2, ms_direct, n_calls = B.bp_lb_kernel_times4(h)
    cluster_used = B.bp_lb_get_cluster_tables(h) == 1
    kwork = B.bp_lb_kernel_work(h)        # VB2 pairs and parameters actually evaluated
    B.bp_lb_set_kernel_timing(h, False)
    t_direct = ms_direct / max(1, n_calls)
    t_vb2 = ms_vb2 / max(1, n_calls)
    t_prefix = ms_prefix / max(1, n_calls)
    t_cluster = ms_cluster / max(1, n_calls)
    t_step = float(step_ms.mean())
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_step = float(t.item())
    value = NODES * world / (t_step / 1e3)

    # ---- end to end through the C ABI with host buffers ---------------------
    pin = {k: v.cpu().pin_memory() for k, v in t_in.items()}
    h_b = torch.empty(NODES, dtype=torch.int64).pin_memory()
    h_a = torch.empty((NODES, 2), dtype=torch.int64).pin_memory()
    h_f = torch.empty(NODES, dtype=torch.uint8).pin_memory()
    h2d = sum(v.numel() * v.element_size() for v in pin.values())
    d2h = h_b.numel() * 8 + h_a.numel() * 8 + h_f.numel()

    def e2e_step():
        for k2, v in pin.items():
            t_in[k2].copy_(v, non_blocking=True)
        step()
        h_b.copy_(out_b, non_blocking=True)
        h_a.copy_(out_a, non_blocking=True)
        h_f.copy_(out_f, non_blocking=True)

    for _ in range(3):
        e2e_step()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    barrier()
    t_e2e = e0.elapsed_time(e1) / args.steps
    e2e_value = NODES * world / (t_e2e / 1e3)

    # ---- plain path: one check per launch ------------------------------------
    w0, a0, c0, k0 = nd.node(0)
    plain_best, plain_us = B.bp_lb_autotune_plain_node(h, w0, a0, k0, reps=20)
    nshapes = B.bp_lb_num_launch_shapes()
    plain_shape = {"algorithm": ("direct", "prefix")[plain_best // nshapes],
                   "shape": plain_best % nshapes}
    lat = []
    for j in range(min(args.plain_sample, NODES)):
        w, a, c, k = nd.node(j)
        t0 = time.perf_counter()
        B.bp_lb_eval_node(h, w, a, k)
        lat.append(time.perf_counter() - t0)
    lat = np.array(lat[8:]) * 1e3  # drop the first calls (warm-up)
    plain_rate = 1e3 / float(lat.mean())

    # correctness spot check of the timed batch against the plain path
    torch.cuda.synchronize()
    for j in (0, NODES // 2, NODES - 1):
        w, a, c, k = nd.node(j)
        assert B.bp_lb_eval_node(h, w, a, k)[0] == int(out_b[j].item())
    full_feasible = out_f.clone()

    # ---- verdict-only mode (early exit): same batch, same launch shape --------
    B.bp_lb_set_result_mode(h, B.RESULT_VERDICT)
    for _ in range(3):
        step()
    barrier()
    vev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for e0, e1 in vev:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    barrier()
    v_ms = np.array([e0.elapsed_time(e1) for e0, e1 in vev])
    assert torch.equal(out_f, full_feasible)   # the same verdicts as the full maximum
    B.bp_lb_set_result_mode(h, B.RESULT_FULL)
    t_verdict = float(v_ms.mean())

    # ---- the same batch with pruning off (identical results, all the work) ----
    B.bp_lb_set_pruning(h, False)
    for _ in range(3):
        step()
    barrier()
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(min(args.steps, 30))]
    B.bp_lb_set_kernel_timing(h, True)
    B.bp_lb_kernel_times(h)
    for e0, e1 in pev:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    barrier()
    t_noprune = float(np.mean([e0.elapsed_time(e1) for e0, e1 in pev]))
    np_k = B.bp_lb_kernel_times(h)
    B.bp_lb_kernel_work(h)
    B.bp_lb_set_kernel_timing(h, False)
    assert torch.equal(out_f, full_feasible)
    B.bp_lb_set_pruning(h, True)
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([t_verdict], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_verdict = float(t.item())

    B.bp_lb_destroy(h)
    if rank != 0:
        return

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak_ops = ipeak["lane_ops_per_s"]                # measured integer issue rate
    sm_mhz = ipeak["sm_mhz"]                          # SM clock sampled during the probe
    peak_words = sms * 32 * sm_mhz * 1e6              # one 32-lane shared access / clk / SM

    # ---- secondary records on this GPU: hard nodes, the large sweep ------------
    recs = set(args.records.split(","))
    hard = hard_nodes_record(B, stream, flush, min(args.steps, 30), peak_ops) if "hard" in recs else None
    large = large_record(B, stream, flush, peak_ops) if "large" in recs else None

    # ---- CPU oracle baseline ---------------------------------------------------
    threads = os.cpu_count() or 1
    cpu_rate, cpu_m, cpu_wall = oracle_rate(nd, args.cpu_budget, threads)
    calls = max(1, n_calls)
    # work per step actually done by each kernel: the VB2 pairs the kernels
    # counted (pruning skips the rest), the generic kernel's other DFFs, the
    # prefix kernel's shared-memory words (host model of the same pruning)
    vb2_pairs = kwork[0] / calls
    work = {"vb2": vb2_pairs * ops_per_eval(4, CAP),
            "direct": ops["direct"] + kwork[1] / calls * ops_per_eval(4, CAP),
            "prefix": float(prefix_smem_words(nd))}
    tms = {"vb2": t_vb2, "direct": t_direct, "prefix": t_prefix}
    peak = {"vb2": peak_ops, "direct": peak_ops, "prefix": peak_words}
    frac = {kk: (work[kk] / (tms[kk] / 1e3) / peak[kk] if tms[kk] > 0 and work[kk] > 0 else None)
            for kk in tms}
    dom = max(tms, key=lambda kk: tms[kk])           # the kernel that takes longest
    achieved = work[dom] / (tms[dom] / 1e3)
    kernel_name = {"vb2": "vb2_kernel (VB2 item by item, fixed-point quotients, pruned)",
                   "direct": "eval_kernel (generic direct evaluation)",
                   "prefix": "prefix_kernel (MT, RAD2, FS1, CCM1, BJ1 from shared-memory "
                             "prefix tables, pruned against L1; VB2 from the count table when "
                             "pruning leaves only small lambda)"}[dom]
    basis = ({"prefix": f"{sms} SMs x 32 lanes x {sm_mhz:.0f} MHz, the SM clock measured under "
                        "the issue probe (one 32-bit shared-memory word per lane per clock: "
                        "128 B/clk/SM); work = shared-memory words of table building and lookups"}
             .get(dom, f"measured integer issue rate {peak_ops / 1e12:.2f} T lane-ops/s "
                       "(bp_lb_probe_int_issue, see issue_peak); work = integer ops of the "
                       "(item, parameter) pairs evaluated"))
    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": WORKLOAD.format(NODES), "nodes": NODES, "n": N_ITEMS, "c": CAP,
                   "evals_per_step": evals, "l2": "flushed (256 MB write) before every timed step",
                   "parallelism": f"independent batches per rank x{world}"},
        "evals_per_s": evals * world / (t_step / 1e3),
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "plain": {"value": plain_rate, "unit": UNIT, "p50_ms": float(np.percentile(lat, 50)),
                  "p99_ms": float(np.percentile(lat, 99)), "sample": len(lat),
                  "launch_shape": plain_shape, "autotune_us": [round(x, 2) for x in plain_us],
                  "call": "bp_lb_eval_node (H2D, 1 launch, D2H, sync)"},
        "batched_over_plain": value / world / plain_rate,
        "verdict": {"value": NODES * world / (t_verdict / 1e3), "unit": UNIT,
                    "ms_per_step": t_verdict, "p50_ms": float(np.percentile(v_ms, 50)),
                    "p99_ms": float(np.percentile(v_ms, 99)),
                    "mode": "verdict only (Alg. 2 early exit; VB2 parameters whose upper "
                            "bound is <= k skipped); same verdicts as the full maximum"},
        "pruning": {"vb2_params_evaluated": kwork[2] / calls, "vb2_params_pruned": kwork[3] / calls,
                    "vb2_pairs_evaluated": vb2_pairs,
                    "off": {"value": NODES * world / (t_noprune / 1e3), "unit": UNIT,
                            "ms_per_step": t_noprune,
                            "kernel_ms": {"prefix": np_k[0] / max(1, np_k[3]),
                                          "vb2": np_k[1] / max(1, np_k[3]),
                                          "direct": np_k[2] / max(1, np_k[3])}},
                    "note": "exact: results identical with pruning off (bp_lb_set_pruning)"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak[dom] / 1e9,
                     "unit": "Gword/s" if dom == "prefix" else "Gop/s", "frac": frac[dom],
                     "traffic": (TRAFFIC_BYTES_PER_NODE[dom] * NODES
                                 if TRAFFIC_BYTES_PER_NODE[dom] is not None else None),
                     "peak_basis": basis,
                     "kernel": kernel_name + ", its own CUDA-event time per launch",
                     "prefix_kernel_ms": t_prefix, "vb2_kernel_ms": t_vb2,
                     "direct_kernel_ms": t_direct, "cluster_kernel_ms": t_cluster,
                     "kernel_events_pass_ms_per_step": float(step_ms_timed.mean()),
                     "prefix_kernel_frac": frac["prefix"], "vb2_kernel_frac": frac["vb2"],
                     "direct_kernel_frac": frac["direct"]},
        "launch_shape": {"chosen": shape, "nt_t_g_minb": list(B.bp_lb_launch_shape_info(shape)),
                         "autotune_ms": [round(x, 4) for x in shape_ms]},
        # plan, prefix, VB2 and generic kernels per step, and the cluster
        # kernel when the autotuner left cluster tables on
        "gpu_launches": (4 + (1 if cluster_used else 0)) * args.steps,
        "clocks": clocks,
        "issue_peak": ipeak,
        "hard_nodes": hard,
        "large": large,
        "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{cpu_m} of the {NODES} nodes (reduction + full bound), "
                                   f"{cpu_wall:.1f} s wall on {threads} threads"},
    }
    print(json.dumps(line))


# ---------------------------------------------------------------------------
# secondary workloads (not the benchmark line): large instances, ragged batch
# ---------------------------------------------------------------------------
CLUSTER_TABLES = "auto"


def cluster_setting(B, h):
    """Applies the run's forced cluster-table setting (none under auto)."""
    if CLUSTER_TABLES != "auto":
        B.bp_lb_set_cluster_tables(h, CLUSTER_TABLES == "on")


def new_handle(B, c, max_items):
    """A handle with the run's cluster-table setting."""
    h = B.bp_lb_create(c, max_items)
    cluster_setting(B, h)
    return h


def _dev(x, dt):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).to(dt).cuda()


def _time_steps(step, steps, flush, stream):
    """Per-step CUDA-event times (ms) with an L2 flush before every step."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    torch.cuda.synchronize()
    for e0, e1 in ev:
        flush.zero_()
        e0.record(stream)
        step()
        e1.record(stream)
    torch.cuda.synchronize()
    return np.array([e0.elapsed_time(e1) for e0, e1 in ev])


def issue_peak(B, stream, launches=25, target_ms=30.0):
    """The integer issue rate the device sustains, measured by the library's
    probe (bp_lb_probe_int_issue: integer multiply-adds and xors only, both
    half-rate pipes busy): lane operations per second of its launches timed
    with CUDA events, and the SM clock sampled meanwhile."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    bps = 4
    sink = torch.empty(sms * bps * 256, dtype=torch.int32, device="cuda")
    ops1 = B.bp_lb_probe_int_issue(bps, 1, sink, stream)
    trips = max(1, int(target_ms * 1e-3 * sms * 4 * 32 * 2.07e9 / ops1))
    for _ in range(3):
        B.bp_lb_probe_int_issue(bps, trips, sink, stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(launches)]
    with ClockSampler(torch.cuda.current_device()) as clk:
        for e0, e1 in ev:
            e0.record(stream)
            ops = B.bp_lb_probe_int_issue(bps, trips, sink, stream)
            e1.record(stream)
        torch.cuda.synchronize()
    ms = np.array([e0.elapsed_time(e1) for e0, e1 in ev])
    clocks = clk.summary()
    rate = ops / (float(np.median(ms)) / 1e3)
    mhz = clocks.get("sm_mhz") or float(measured_peaks().get("sm_max_mhz", 2070.0))
    nominal = sms * 4 * 32 * mhz * 1e6
    return {"lane_ops_per_s": rate, "ms_per_launch": float(np.median(ms)), "launches": launches,
            "lane_ops_per_launch": ops, "sm_mhz": mhz, "clocks": clocks,
            "nominal_at_that_clock": nominal, "frac_of_nominal": rate / nominal,
            "probe": "bp_lb_probe_int_issue: 4 CTAs x 256 threads per SM, 8 independent "
                     "chains per thread of one integer multiply-add (FMA pipe) and one xor "
                     "(ALU pipe) per step"}


def node_tensors(nd):
    import torch
    return dict(base_offsets=_dev(nd.base.offsets, torch.int64),
                base_sizes=_dev(nd.base.sizes, torch.int32),
                base_capacity=_dev(nd.base.capacity, torch.int64),
                node_base=_dev(nd.node_base, torch.int32),
                assign_offsets=_dev(nd.assign_offsets, torch.int64),
                assign=_dev(nd.assign, torch.int32), bins=_dev(nd.bins, torch.int64))


def hard_nodes_record(B, stream, flush, steps, peak_ops, shape=-1):
    """The search-node step on nodes whose bounds mostly exceed L1 (triplet
    instance, k = n/3; instances.hard_nodes), pruning on and off, per kernel."""
    import torch
    from paper_2402_14821_gb300 import instances as I
    nd = I.hard_nodes()
    t_in = node_tensors(nd)
    mb = int(nd.bins.max())
    ob = torch.empty(nd.count, dtype=torch.int64, device="cuda")
    oa = B.argmax_tensor(nd.count)
    of = torch.empty(nd.count, dtype=torch.uint8, device="cuda")
    h = new_handle(B, 150, 1024)
    out = {"workload": f"{nd.count} partial packings (uniform 0..60% committed) of one triplet "
                       "instance, n=501 sizes in (c/4, c/2) filling 167 bins exactly, c=10000, "
                       "k=167 bins (the optimum)"}
    try:
        B.bp_lb_reserve(h, nd.count)
        if shape >= 0:
            B.bp_lb_set_launch_shape(h, B.MODE_NODES, shape)
        else:
            shape, _ = B.bp_lb_autotune_nodes(h, max_bins=mb, out_bound=ob, out_argmax=oa,
                                              out_feasible=of, reps=2, stream=stream, **t_in)
            cluster_setting(B, h)
        step = lambda: B.bp_lb_eval_nodes(h, max_bins=mb, out_bound=ob, out_argmax=oa,
                                          out_feasible=of, stream=stream, **t_in)
        res = {}
        for prune in (True, False):
            B.bp_lb_set_pruning(h, prune)
            for _ in range(3):
                step()
            B.bp_lb_set_kernel_timing(h, True)
            B.bp_lb_kernel_times(h)
            ms = _time_steps(step, steps if prune else max(3, steps // 3), flush, stream)
            kc, kp, kv, kd, kn = B.bp_lb_kernel_times4(h)
            kw = B.bp_lb_kernel_work(h)
            B.bp_lb_set_kernel_timing(h, False)
            n = max(1, kn)
            res[prune] = (ob.cpu().numpy().copy(), of.cpu().numpy().copy())
            t = float(ms.mean())
            vb2_frac = (kw[0] / n * ops_per_eval(4, CAP) / (kv / n / 1e3) / peak_ops
                        if kv > 0 and kw[0] > 0 else None)
            out["pruning_on" if prune else "pruning_off"] = {
                "value": nd.count / (t / 1e3), "unit": UNIT, "ms_per_step": t,
                "p50_ms": float(np.percentile(ms, 50)), "p99_ms": float(np.percentile(ms, 99)),
                "kernel_ms": {"cluster": kc / n, "prefix": kp / n, "vb2": kv / n,
                              "direct": kd / n},
                "vb2_pairs_evaluated": kw[0] / n, "vb2_params_pruned": kw[3] / n,
                "vb2_kernel_frac_of_issue_peak": vb2_frac}
        B.bp_lb_set_pruning(h, True)
        assert np.array_equal(res[True][0], res[False][0])   # pruning is exact
        b = res[True][0]
        w0, _, c, _ = nd.node(0)
        L1 = -(-int(np.asarray(w0, np.int64).sum()) // c)  # the reduction keeps the total
        out.update({"launch_shape": shape, "frac_nodes_bound_above_L1": float(np.mean(b > L1)),
                    "frac_nodes_infeasible": float(np.mean(res[True][1] == 0)),
                    "pruning_speedup": out["pruning_off"]["ms_per_step"] /
                                       out["pruning_on"]["ms_per_step"]})
    finally:
        B.bp_lb_destroy(h)
    return out


LARGE_CASES = ((10 ** 5, "uniform_wide"), (10 ** 5, "triplets"), (10 ** 5, "uniform_full"),
               (10 ** 6, "triplets"))


def large_record(B, stream, flush, peak_ops, cases=LARGE_CASES, steps=3):
    """The large-instance sweep (n = 10^4, 64 instances per batch, int32 sizes):
    per case the batch time, checks/s and the item-by-item kernels' fraction of
    the integer issue peak (integer ops of the (item, parameter) pairs they
    evaluate, VB2's counted by the kernels, over their own CUDA-event time)."""
    import torch
    from paper_2402_14821_gb300 import instances as I
    h = new_handle(B, 150, 1024)
    res = []
    try:
        for c, fam in cases:
            rg = I.large_instances(fam, c, count=64, n=10_000, seed=2, dtype=np.int32)
            evals, ops = ragged_work(rg)
            t = (_dev(rg.offsets, torch.int64), _dev(rg.sizes, torch.int32),
                 _dev(rg.capacity, torch.int64), _dev(rg.bins, torch.int64))
            ob = torch.empty(rg.count, dtype=torch.int64, device="cuda")
            oa = B.argmax_tensor(rg.count)
            shape, _ = B.bp_lb_autotune_batch(h, *t, ob, oa, reps=1, stream=stream)
            cluster_setting(B, h)
            step = lambda: B.bp_lb_eval_batch(h, *t, ob, oa, stream=stream)
            step()
            B.bp_lb_set_kernel_timing(h, True)
            B.bp_lb_kernel_times(h)
            ms = _time_steps(step, steps, flush, stream)
            kc, kp, kv, kd, kn = B.bp_lb_kernel_times4(h)
            kw = B.bp_lb_kernel_work(h)
            B.bp_lb_set_kernel_timing(h, False)
            n = max(1, kn)
            td = (kv + kd) / n
            ops += (kw[0] + kw[1]) / n * ops_per_eval(4, c)
            tm = float(ms.mean())
            off = None
            if c <= 10 ** 5:
                # the same batch with pruning off: all the item-by-item work
                B.bp_lb_set_pruning(h, False)
                step()
                B.bp_lb_set_kernel_timing(h, True)
                B.bp_lb_kernel_times(h)
                ms_off = _time_steps(step, steps, flush, stream)
                kc2, kp2, kv2, kd2, kn2 = B.bp_lb_kernel_times4(h)
                kw2 = B.bp_lb_kernel_work(h)
                B.bp_lb_set_kernel_timing(h, False)
                B.bp_lb_set_pruning(h, True)
                n2 = max(1, kn2)
                td2 = (kv2 + kd2) / n2
                ops2 = ragged_work(rg)[1] + (kw2[0] + kw2[1]) / n2 * ops_per_eval(4, c)
                off = {"ms_per_batch": float(ms_off.mean()), "item_kernels_ms": td2,
                       "prefix_kernel_ms": kp2 / n2, "cluster_kernel_ms": kc2 / n2,
                       "item_kernel_ops": ops2,
                       "item_kernels_frac_of_issue_peak": ops2 / (td2 / 1e3) / peak_ops
                       if td2 > 0 else None}
            res.append({"c": c, "family": fam, "instances": 64, "n": 10_000, "dtype": "int32",
                        "ms_per_batch": tm, "checks_per_s": 64 / (tm / 1e3),
                        "evals_per_s_equivalent": evals / (tm / 1e3), "launch_shape": shape,
                        "prefix_kernel_ms": kp / n, "cluster_kernel_ms": kc / n,
                        "item_kernels_ms": td, "item_kernel_ops": ops,
                        "item_kernels_frac_of_issue_peak": ops / (td / 1e3) / peak_ops
                        if td > 0 else None, "pruning_off": off})
            del t, ob, oa
    finally:
        B.bp_lb_destroy(h)
    return res


def ragged_work(rg, algo=1):
    """(evals, item-by-item integer ops of the direct kernel but VB2's, which
    the device counts) of a ragged batch of reduced instances."""
    evals = ops = 0
    for b in range(rg.count):
        c = int(rg.capacity[b])
        r = int(rg.offsets[b + 1] - rg.offsets[b])
        cnt = param_counts(c)
        evals += r * sum(cnt)
        ops += r * sum(cnt[d] * ops_per_eval(d, c) for d in range(6)
                       if d != 4 and kernel_of(d, c, r, algo) != "prefix")
    return evals, ops


def bound_strength(B, I, h, stream, flush):
    """Table 1's statistics on the synthetic families (root of the search, no
    packing): per DFF the instances where it is the only one / one of those
    reaching the optimum (known for the triplet family) and the best bound
    among the six, and the sum of its bounds; every bound against L2; and the
    time of the collection and of L2 on the device."""
    import torch
    names = ["MT", "RAD2", "FS1", "CCM1", "VB2", "BJ1"]
    res = []
    tot = {nm: dict(only_opt=0, total_opt=0, only_best=0, total_best=0, sum=0, above_l2=0,
                    equal_l2=0, below_l2=0) for nm in names}
    coll_tot = dict(instances=0, above_l2=0, equal_l2=0, below_l2=0, opt=0, l2_opt=0, with_opt=0)
    for fam, rg, opt in I.strength_families():
        t = (_dev(rg.offsets, torch.int64), _dev(rg.sizes, torch.int32),
             _dev(rg.capacity, torch.int64), _dev(rg.bins, torch.int64))
        ob = torch.empty(rg.count, dtype=torch.int64, device="cuda")
        oa = B.argmax_tensor(rg.count)
        per = np.zeros((6, rg.count), dtype=np.int64)
        for d in range(6):
            B.bp_lb_set_dff_mask(h, 1 << d)
            B.bp_lb_eval_batch(h, *t, ob, oa, stream=stream)
            torch.cuda.synchronize()
            per[d] = ob.cpu().numpy()
        B.bp_lb_set_dff_mask(h, 63)
        B.bp_lb_eval_batch(h, *t, ob, oa, stream=stream)
        ms_coll = float(_time_steps(lambda: B.bp_lb_eval_batch(h, *t, ob, oa, stream=stream), 5,
                                    flush, stream).mean())
        lb = ob.cpu().numpy()
        l2t = torch.empty(rg.count, dtype=torch.int64, device="cuda")
        B.bp_lb_l2_batch(h, t[0], t[1], t[2], l2t, stream=stream)
        ms_l2 = float(_time_steps(lambda: B.bp_lb_l2_batch(h, t[0], t[1], t[2], l2t, stream=stream),
                                  5, flush, stream).mean())
        l2 = l2t.cpu().numpy()
        l1 = np.array([-(-int(rg.instance(j).sum()) // int(rg.capacity[j])) for j in range(rg.count)])
        assert np.array_equal(lb, per.max(axis=0))        # the collection is the max of its DFFs
        best = per.max(axis=0)
        nbest = (per == best[None, :]).sum(axis=0)
        row = {"family": fam, "instances": rg.count, "ms_collection": ms_coll, "ms_l2": ms_l2,
               "sum_l1": int(l1.sum()), "sum_l2": int(l2.sum()), "sum_collection": int(lb.sum()),
               "collection_vs_l2": {"above": int((lb > l2).sum()), "equal": int((lb == l2).sum()),
                                    "below": int((lb < l2).sum())}, "dff": {}}
        if opt is not None:
            opt = np.asarray(opt)
            nopt = (per == opt[None, :]).sum(axis=0)
            row["optimum_reached"] = {"collection": int((lb == opt).sum()), "L2": int((l2 == opt).sum())}
            coll_tot["opt"] += int((lb == opt).sum())
            coll_tot["l2_opt"] += int((l2 == opt).sum())
            coll_tot["with_opt"] += rg.count
        for d, nm in enumerate(names):
            x = per[d]
            e = {"total_best": int((x == best).sum()), "only_best": int(((x == best) & (nbest == 1)).sum()),
                 "sum": int(x.sum()), "above_l2": int((x > l2).sum()), "equal_l2": int((x == l2).sum()),
                 "below_l2": int((x < l2).sum())}
            if opt is not None:
                e["total_opt"] = int((x == opt).sum())
                e["only_opt"] = int(((x == opt) & (nopt == 1)).sum())
            row["dff"][nm] = e
            for k2, v in e.items():
                tot[nm][k2] += v
        for k2 in ("above", "equal", "below"):
            coll_tot[k2 + "_l2"] += row["collection_vs_l2"][k2]
        coll_tot["instances"] += rg.count
        print(json.dumps(row), flush=True)
        res.append(row)
    res.append({"family": "all", "dff": tot, "collection": coll_tot})
    print(json.dumps(res[-1]), flush=True)
    # throughput of L2 against the collection on one larger batch
    rng = np.random.default_rng(61)
    rg = I.ragged_from_list([I.uniform_sizes(rng, 1000, 20, 100) for _ in range(4096)], [150] * 4096)
    t = (_dev(rg.offsets, torch.int64), _dev(rg.sizes, torch.int32),
         _dev(rg.capacity, torch.int64), _dev(rg.bins, torch.int64))
    ob = torch.empty(rg.count, dtype=torch.int64, device="cuda")
    l2t = torch.empty(rg.count, dtype=torch.int64, device="cuda")
    B.bp_lb_l2_batch(h, t[0], t[1], t[2], l2t, stream=stream)
    B.bp_lb_eval_batch(h, *t, ob, stream=stream)
    ms_l2 = float(_time_steps(lambda: B.bp_lb_l2_batch(h, t[0], t[1], t[2], l2t, stream=stream),
                              10, flush, stream).mean())
    ms_c = float(_time_steps(lambda: B.bp_lb_eval_batch(h, *t, ob, stream=stream), 10, flush,
                             stream).mean())
    res.append({"throughput": "4096 instances, n = 1000, sizes U[20, 100], c = 150",
                "l2_instances_per_s": 4096 / (ms_l2 / 1e3), "l2_ms": ms_l2,
                "collection_instances_per_s": 4096 / (ms_c / 1e3), "collection_ms": ms_c,
                "l2_below_collection": int((l2t < ob).sum().item())})
    print(json.dumps(res[-1]), flush=True)
    return res


def run_sweep(args):
    import torch
    from paper_2402_14821_gb300 import binding as B
    from paper_2402_14821_gb300 import build
    from paper_2402_14821_gb300 import instances as I

    torch.cuda.set_device(0)
    build.build()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ipeak = issue_peak(B, stream)
    peak = ipeak["lane_ops_per_s"]
    h = new_handle(B, 150, 1 << 16)
    out = {"workload": args.workload, "results": [], "issue_peak": ipeak}
    with ClockSampler(torch.cuda.current_device()) as clk:
        if args.workload == "issue":
            out["results"].append({k: v for k, v in ipeak.items() if k != "clocks"})
        elif args.workload == "hard":
            out["results"].append(hard_nodes_record(B, stream, flush, max(3, min(args.steps, 30)),
                                                    peak, args.shape))
        elif args.workload == "large":
            steps = max(1, min(args.steps, 5))
            cases = ([(int(float(x.split(":")[0])), x.split(":")[1]) for x in args.large_cases.split(",")]
                     if args.large_cases else [(c, f) for c in (10 ** 5, 10 ** 6) for f in I.FAMILIES])
            B.bp_lb_set_dff_mask(h, args.dff_mask)
            B.bp_lb_set_pruning(h, not args.no_prune)
            count = args.large_count
            for c, fam in cases:
                for dt in [np.dtype(x).type for x in args.large_dtypes.split(",")]:
                    rg = I.large_instances(fam, c, count=count, n=10_000, seed=2, dtype=dt)
                    evals, ops = ragged_work(rg)
                    tdt = torch.int32 if dt == np.int32 else torch.int64
                    t = (_dev(rg.offsets, torch.int64), _dev(rg.sizes, tdt),
                         _dev(rg.capacity, torch.int64), _dev(rg.bins, torch.int64))
                    ob = torch.empty(rg.count, dtype=torch.int64, device="cuda")
                    oa = B.argmax_tensor(rg.count)
                    if args.shape >= 0:
                        shape = args.shape
                        B.bp_lb_set_launch_shape(h, B.MODE_RAGGED_I32 if dt == np.int32
                                                 else B.MODE_RAGGED_I64, shape)
                    else:
                        shape, _ = B.bp_lb_autotune_batch(h, *t, ob, oa, reps=1)
                        cluster_setting(B, h)
                    step = lambda: B.bp_lb_eval_batch(h, *t, ob, oa, stream=stream)
                    step()
                    B.bp_lb_set_kernel_timing(h, True)
                    B.bp_lb_kernel_times(h)
                    ms = _time_steps(step, steps, flush, stream)
                    kc, kp, kv, kd, kn = B.bp_lb_kernel_times4(h)
                    kw = B.bp_lb_kernel_work(h)
                    B.bp_lb_set_kernel_timing(h, False)
                    tm = float(ms.mean())
                    td = (kv + kd) / max(1, kn)
                    ops += (kw[0] + kw[1]) / max(1, kn) * ops_per_eval(4, c)
                    out["results"].append({
                        "c": c, "family": fam, "dtype": np.dtype(dt).name, "instances": count,
                        "dff_mask": args.dff_mask, "pruning": not args.no_prune, "evals": evals,
                        "n": 10_000, "ms_per_batch": tm, "checks_per_s": count / (tm / 1e3),
                        "evals_per_s": evals / (tm / 1e3), "launch_shape": shape,
                        "item_kernels_ms": td, "vb2_kernel_ms": kv / max(1, kn),
                        "prefix_kernel_ms": kp / max(1, kn),
                        "cluster_kernel_ms": kc / max(1, kn),
                        "roofline_frac": ops / (td / 1e3) / peak})
                    print(json.dumps(out["results"][-1]), flush=True)
        elif args.workload == "plain":
            import oracle
            rg = I.plain_single(seed=0)
            w, c, k = rg.instance(0), int(rg.capacity[0]), int(rg.bins[0])
            hp = new_handle(B, c, 1024)
            for _ in range(100):
                B.bp_lb_eval(hp, w, k)
            lat = []
            for _ in range(10_000):
                t0 = time.perf_counter()
                B.bp_lb_eval(hp, w, k)
                lat.append(time.perf_counter() - t0)
            lat = np.array(lat) * 1e3
            got = B.bp_lb_eval(hp, w, k)
            B.bp_lb_destroy(hp)
            orc = oracle.load()
            t0 = time.perf_counter()
            reps = 200
            for _ in range(reps):
                want = orc.lb(w, c, k)
            t_orc = (time.perf_counter() - t0) / reps
            evals = len(w) * sum(param_counts(c))
            out["results"].append({
                "n": len(w), "c": c, "bins": k, "bound": got[0], "matches_oracle": got == want[:3],
                "checks_per_s": 1e3 / float(lat.mean()), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "evals_per_check": evals,
                "oracle_1thread_checks_per_s": 1.0 / t_orc,
                "oracle_1thread_evals_per_s": evals / t_orc})
            print(json.dumps(out["results"][-1]), flush=True)
        elif args.workload == "serve":
            from paper_2402_14821_gb300 import search_sim
            searches = search_sim.make_searches(count=256, seed=4)
            tot = lambda c: sum(param_counts(c))
            srv = B.bp_serve_create(pool_items=1 << 23, max_instances=256,
                                    max_queued_items=3 << 20, slots=3, max_batch=256,
                                    max_bins=16384)
            ids = [B.bp_serve_register(srv, s.w, s.c) for s in searches]
            for rate in (10.0, 100.0, 1e3, 1e4, 1e5, 1e6):
                res = search_sim.drive(B, srv, searches, ids, rate=rate, duration_s=4.0,
                                       param_total=tot)
                lat = res["latency_us"] / 1e3
                el = res["elapsed_s"]
                out["results"].append({
                    "offered_checks_per_s": rate, "achieved_checks_per_s": res["done"] / el,
                    "evals_per_s": res["evals"] / el, "done": res["done"],
                    "submitted": res["submitted"], "refused": res["refused"],
                    "infeasible": res["infeasible"],
                    "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                    "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None})
                print(json.dumps(out["results"][-1]), flush=True)
            out["server"] = B.bp_serve_stats(srv)
            B.bp_serve_destroy(srv)
        elif args.workload == "table1":
            out["results"] = bound_strength(B, I, h, stream, flush)
        else:  # ragged
            nd = I.ragged_nodes(seed=3)
            evals, kops = algorithmic_work(nd)
            ops = kops["direct"]
            t_in = dict(base_offsets=_dev(nd.base.offsets, torch.int64),
                        base_sizes=_dev(nd.base.sizes, torch.int32),
                        base_capacity=_dev(nd.base.capacity, torch.int64),
                        node_base=_dev(nd.node_base, torch.int32),
                        assign_offsets=_dev(nd.assign_offsets, torch.int64),
                        assign=_dev(nd.assign, torch.int32), bins=_dev(nd.bins, torch.int64))
            mb = int(nd.bins.max())
            ob = torch.empty(nd.count, dtype=torch.int64, device="cuda")
            oa = B.argmax_tensor(nd.count)
            of = torch.empty(nd.count, dtype=torch.uint8, device="cuda")
            B.bp_lb_reserve(h, nd.count)
            shape, shape_ms = B.bp_lb_autotune_nodes(h, max_bins=mb, out_bound=ob, out_argmax=oa,
                                                     out_feasible=of, reps=1, **t_in)
            cluster_setting(B, h)
            direct = lambda: B.bp_lb_eval_nodes(h, max_bins=mb, out_bound=ob, out_argmax=oa,
                                                out_feasible=of, stream=stream, **t_in)
            # capture the whole batch (planning + persistent evaluation) in a CUDA graph
            g = torch.cuda.CUDAGraph()
            cs = torch.cuda.Stream()
            cs.wait_stream(stream)
            with torch.cuda.stream(cs):
                direct()
            stream.wait_stream(cs)
            torch.cuda.synchronize()
            with torch.cuda.graph(g, stream=cs):
                B.bp_lb_eval_nodes(h, max_bins=mb, out_bound=ob, out_argmax=oa, out_feasible=of,
                                   stream=cs, **t_in)
            g.replay()
            torch.cuda.synchronize()
            steps = max(3, min(args.steps, 20))
            ms_graph = _time_steps(g.replay, steps, flush, stream)
            B.bp_lb_set_kernel_timing(h, True)
            B.bp_lb_kernel_times(h)
            ms_direct = _time_steps(direct, steps, flush, stream)
            kc, kp, kv, kd, kn = B.bp_lb_kernel_times4(h)
            kw = B.bp_lb_kernel_work(h)
            B.bp_lb_set_kernel_timing(h, False)
            # VB2 on its kernel up to c = 65535, on the generic one above
            ops += (kw[0] * ops_per_eval(4, 9999) + kw[1] * ops_per_eval(4, 100_000)) / max(1, kn)
            td = (kv + kd) / max(1, kn)
            tm = float(ms_graph.mean())
            out["results"].append({
                "instances": nd.count, "ms_per_batch_graph": tm,
                "ms_per_batch_direct": float(ms_direct.mean()),
                "checks_per_s": nd.count / (tm / 1e3), "evals_per_s": evals / (tm / 1e3),
                "evals_per_batch": evals, "launch_shape": shape,
                "autotune_ms": [round(x, 3) for x in shape_ms],
                "item_kernels_ms": td, "vb2_kernel_ms": kv / max(1, kn),
                "prefix_kernel_ms": kp / max(1, kn), "cluster_kernel_ms": kc / max(1, kn),
                "roofline_frac": ops / (td / 1e3) / peak})
            print(json.dumps(out["results"][-1]), flush=True)
    out["clocks"] = clk.summary()
    B.bp_lb_destroy(h)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
