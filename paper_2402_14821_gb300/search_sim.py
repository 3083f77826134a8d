"""Simulated depth-first searches that generate feasibility checks.

Load generator for the serving loop: each search walks one instance with the
decreasing-best-fit strategy of Sec. 5 ("resolution procedure"): items in
decreasing size, each committed to the bin with the smallest residual that
still fits it; after every commitment it issues a feasibility check of the
partial packing and, when the check fails (bound > k), backtracks by removing
that bin from the item's choices.  A search that packs every item, or runs out
of choices, starts over.  It is a workload driver, not a solver: no other
propagation, symmetry breaking or dominance rule is applied.

The decision to backtrack uses the server's answer (the verdict), so the
sequence of checks is closed-loop.  Offered load is set by exponentially
distributed think times between a search's result and its next check.
"""
from __future__ import annotations

import heapq
import time

import numpy as np

from . import instances as I


class DFSearch:
    def __init__(self, sizes: np.ndarray, c: int, k: int):
        self.w = np.asarray(sizes, dtype=np.int64)
        self.c = int(c)
        self.k = int(k)
        self.order = np.argsort(-self.w, kind="stable")
        self.restart()

    def restart(self):
        n = len(self.w)
        self.assign = np.full(n, -1, dtype=np.int32)
        self.load = np.zeros(self.k, dtype=np.int64)
        self.depth = 0                 # items of `order` committed so far
        self.tried = [set()]           # bins already refused for the item at each depth
        self.restarts = getattr(self, "restarts", -1) + 1

    def _best_fit(self, item: int, banned) -> int:
        room = self.c - self.load
        ok = room >= self.w[item]
        if banned:
            ok[list(banned)] = False
        if not ok.any():
            return -1
        cand = np.nonzero(ok)[0]
        return int(cand[np.argmin(room[cand])])

    def next_check(self):
        """Commits the next item and returns the assignment to check, or None
        when the search has to restart (solution found or exhausted)."""
        while True:
            if self.depth == len(self.w):
                self.restart()
            item = int(self.order[self.depth])
            b = self._best_fit(item, self.tried[self.depth])
            if b >= 0:
                self.assign[item] = b
                self.load[b] += self.w[item]
                self.depth += 1
                self.tried.append(set())
                self._last = (item, b)
                return self.assign.copy()
            # no bin left for this item: undo the previous commitment
            if self.depth == 0:
                self.restart()
                continue
            self._undo()

    def _undo(self):
        self.tried.pop()
        self.depth -= 1
        item = int(self.order[self.depth])
        b = int(self.assign[item])
        self.assign[item] = -1
        self.load[b] -= self.w[item]
        self.tried[self.depth].add(b)

    def on_result(self, feasible: bool):
        if not feasible:
            self._undo()


def make_searches(count: int = 256, seed: int = 4, n_lo: int = 100, n_hi: int = 20_000,
                  c_lo: int = 1_000, c_hi: int = 1_000_000):
    """`count` searches over instances with n ~ U[n_lo, n_hi], c ~ U[c_lo, c_hi],
    sizes U[1, c/2] and k = ceil(sum/c) + 1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        n = int(rng.integers(n_lo, n_hi + 1))
        c = int(rng.integers(c_lo, c_hi + 1))
        w = I.uniform_sizes(rng, n, 1, c // 2)
        out.append(DFSearch(w, c, I.bins_for(w, c)))
    return out


def reduced_size(assign: np.ndarray) -> int:
    """r of a partial packing: unpacked items plus non-empty bins (sizes >= 1)."""
    return int(np.sum(assign == -1)) + len(np.unique(assign[assign >= 0]))


def drive(server_api, srv, searches, ids, rate: float, duration_s: float, seed: int = 0,
          param_total=None):
    """Runs the closed loop for `duration_s` seconds at an offered rate of
    `rate` checks/s (think times ~ Exp(len(searches) / rate) per search).
    `server_api` is the binding module; `ids[i]` is search i's instance id.
    Returns a dict of counts and the latencies (microseconds) of completed checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    S = len(searches)
    mean_think = S / rate
    ready = [(float(rng.exponential(mean_think)), i) for i in range(S)]
    heapq.heapify(ready)
    waiting = {}
    lat, submitted, refused, done, infeasible, evals = [], 0, 0, 0, 0, 0
    work = {}
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        if now >= duration_s:
            break
        while ready and ready[0][0] <= now:
            _, i = heapq.heappop(ready)
            a = searches[i].next_check()
            rid = server_api.bp_serve_submit(srv, ids[i], a, searches[i].k, tag=i)
            if rid is None:                       # admission refused: retry shortly
                refused += 1
                searches[i]._undo()
                heapq.heappush(ready, (now + 0.001, i))
                continue
            waiting[rid] = i
            if param_total is not None:
                work[rid] = reduced_size(a) * param_total(searches[i].c)
            submitted += 1
        wait_us = 200 if waiting else 0
        if ready:
            wait_us = int(max(0, min(wait_us, (ready[0][0] - now) * 1e6)))
        for r in server_api.bp_serve_poll(srv, 4096, wait_us):
            i = waiting.pop(r.request)
            evals += work.pop(r.request, 0)
            done += 1
            lat.append(r.latency_us)
            feas = bool(r.feasible)
            infeasible += not feas
            searches[i].on_result(feas)
            heapq.heappush(ready, (time.perf_counter() - t0 + float(rng.exponential(mean_think)), i))
        if not waiting and not ready:
            break
    elapsed = time.perf_counter() - t0
    # drain what is still in flight (not counted)
    deadline = time.perf_counter() + 30
    while waiting and time.perf_counter() < deadline:
        for r in server_api.bp_serve_poll(srv, 4096, 1000):
            i = waiting.pop(r.request)
            searches[i].on_result(bool(r.feasible))
    return {"offered_rate": rate, "elapsed_s": elapsed, "submitted": submitted, "done": done,
            "refused": refused, "infeasible": infeasible, "evals": evals,
            "latency_us": np.array(lat)}
