"""Continuous batching of hull requests over a device-resident pool of point
sets, admitted by a device-memory budget.

A request names a set (a range of rows of the pool).  The server keeps a
FIFO of requests that have arrived.  Whenever one of its streams is idle it
forms the next batch from the head of the FIFO -- within a point cap, a set
cap, and the device memory free in its arena -- and launches it as one
hull_batch_ranges call on that stream.  No points are copied: only the
requests' start rows and sizes (16 bytes each) go to the device.

Memory.  The server owns one device buffer of `budget_bytes` (the arena),
allocated once.  Each batch takes one region of it, first fit, holding its
workspace (hull_batch_workspace_bytes), its outputs and its metadata; the
region is returned when the batch's completion event has fired.  A batch is
formed only if its region fits in the arena's largest free block now, so the
bytes in flight never exceed the budget.  If the head of the FIFO does not
fit yet it waits (nothing behind it may overtake it: arrival order is kept);
if it could not fit even in an empty arena it is refused with
HULL_ERR_BUDGET.

Completion is detected by polling each batch's CUDA event; a request's
latency is the GPU time of that event minus the request's arrival time,
both measured from one start event.

The method itself (section 2, Steps 1-3, and the hull of the survivors)
runs entirely in the library's kernels; this module only schedules and
accounts memory.
"""
from __future__ import annotations

import bisect
import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np

HULL_ERR_BUDGET = 6
ALIGN = 256


def align_up(v: int, a: int = ALIGN) -> int:
    return (int(v) + a - 1) // a * a


class Arena:
    """First-fit allocator of byte ranges in [0, capacity), every range
    ALIGN-aligned; free blocks are coalesced.  Host bookkeeping only."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity) // ALIGN * ALIGN
        self.free_blocks: list[tuple[int, int]] = [(0, self.capacity)] if self.capacity > 0 else []
        self.used: dict[int, int] = {}
        self.in_use = 0
        self.peak = 0

    def largest_free(self) -> int:
        return max((s for _, s in self.free_blocks), default=0)

    def alloc(self, nbytes: int):
        """Offset of a new range of nbytes (rounded up to ALIGN), or None."""
        n = align_up(max(int(nbytes), 1))
        for k, (off, size) in enumerate(self.free_blocks):
            if size >= n:
                if size == n:
                    del self.free_blocks[k]
                else:
                    self.free_blocks[k] = (off + n, size - n)
                self.used[off] = n
                self.in_use += n
                self.peak = max(self.peak, self.in_use)
                return off
        return None

    def free(self, off: int):
        n = self.used.pop(off)
        self.in_use -= n
        k = bisect.bisect_left(self.free_blocks, (off, 0))
        self.free_blocks.insert(k, (off, n))
        # merge with the next block, then with the previous one
        if k + 1 < len(self.free_blocks) and off + n == self.free_blocks[k + 1][0]:
            self.free_blocks[k] = (off, n + self.free_blocks[k + 1][1])
            del self.free_blocks[k + 1]
        if k > 0 and self.free_blocks[k - 1][0] + self.free_blocks[k - 1][1] == off:
            po, ps = self.free_blocks[k - 1]
            self.free_blocks[k - 1] = (po, ps + self.free_blocks[k][1])
            del self.free_blocks[k]


class Batcher:
    """FIFO of waiting requests.  take(room) forms the next batch in arrival
    order: the longest prefix of the FIFO with at most max_sets requests and
    max_points points (a single request above max_points goes alone) whose
    memory, need(points, sets), fits in `room` bytes.  If even the head
    alone does not fit in `room` it waits and take returns [] -- unless it
    could never fit (need above `budget`): then it is moved to `refused`
    and the next request is considered."""

    def __init__(self, max_points: int, max_sets: int, need=None, budget: int | None = None):
        if max_points < 1 or max_sets < 1:
            raise ValueError("batch caps must be positive")
        self.max_points = int(max_points)
        self.max_sets = int(max_sets)
        self.need = need or (lambda points, sets: 0)
        self.budget = budget
        self.q: collections.deque = collections.deque()
        self.refused: list[int] = []

    def push(self, rid: int, size: int):
        self.q.append((int(rid), int(size)))

    def __len__(self):
        return len(self.q)

    def take(self, room: int | None = None) -> list[tuple[int, int]]:
        while self.q and self.budget is not None and self.need(self.q[0][1], 1) > self.budget:
            self.refused.append(self.q.popleft()[0])
        # the longest prefix within the point and set caps, then (memory
        # grows with the prefix) the longest part of it that fits `room`,
        # found by bisection: a few memory evaluations per batch
        k, pts, prefix = 0, 0, [0]
        for rid, size in self.q:
            if k >= self.max_sets or (k and pts + size > self.max_points):
                break
            k += 1
            pts += size
            prefix.append(pts)
        if room is not None and k and self.need(prefix[k], k) > room:
            lo, hi = 0, k  # need(prefix[lo], lo) fits (lo = 0: nothing), need(prefix[hi], hi) does not
            while hi - lo > 1:
                mid = (lo + hi) // 2
                if self.need(prefix[mid], mid) <= room:
                    lo = mid
                else:
                    hi = mid
            k = lo
        return [self.q.popleft() for _ in range(k)]


@dataclass
class ServeResult:
    latency_s: np.ndarray      # per request, in request order (NaN: refused)
    completion_s: np.ndarray   # per request, from the start event (NaN: refused)
    batches: int
    points: int
    makespan_s: float          # first arrival to last completion
    refused: list = field(default_factory=list)
    peak_bytes: int = 0        # largest device memory held by batches in flight
    budget_bytes: int = 0
    deferred: int = 0          # times the head of the FIFO waited for memory

    def summary(self) -> dict:
        ok = ~np.isnan(self.latency_s)
        lat = self.latency_s[ok] * 1e3
        return {"requests": int(len(self.latency_s)), "served": int(ok.sum()), "refused": len(self.refused),
                "batches": self.batches,
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_ms": float(lat.mean()) if len(lat) else None, "max_ms": float(lat.max()) if len(lat) else None,
                "gpoints_per_s": self.points / self.makespan_s / 1e9 if self.makespan_s > 0 else None,
                "peak_bytes_in_flight": int(self.peak_bytes), "budget_bytes": int(self.budget_bytes),
                "deferred_for_memory": int(self.deferred)}


def batch_bytes(cp, n_total: int, S: int, opt) -> int:
    """Device bytes of one batch: its workspace, hull indices (int64 per
    point), hull offsets (S+1) and metadata (starts and offsets, 2S+1)."""
    return (align_up(cp.hull_batch_workspace_bytes(n_total, S, opt)) + align_up(8 * max(n_total, 1))
            + align_up(8 * (S + 1)) + align_up(8 * (2 * S + 1)))


def batch_bytes_fn(cp, opt):
    """batch_bytes with the options converted once (a call per batch size)."""
    lib = cp.load()
    copt = opt.c()
    ref = ctypes.byref(copt)

    def need(n_total: int, S: int) -> int:
        return (align_up(lib.hull_batch_workspace_bytes(int(n_total), int(S), ref)) + align_up(8 * max(n_total, 1))
                + align_up(8 * (S + 1)) + align_up(8 * (2 * S + 1)))
    return need


class Server:
    """Batches in flight on up to `streams` streams, their memory carved out
    of one arena of budget_bytes device bytes."""

    def __init__(self, pool, budget_bytes: int = 64 << 30, max_points: int = 256 << 20, max_sets: int = 2048,
                 streams: int = 2, opt=None):
        import torch
        import paper_1405_3454_gb300 as cp
        self.cp = cp
        self.torch = torch
        self.pool = pool
        self.n_xy = cp._check_points(pool)
        self.opt = opt or cp.Options()
        self.max_points, self.max_sets = int(max_points), int(max_sets)
        self.budget = int(budget_bytes)
        self._need = batch_bytes_fn(cp, self.opt)
        self._copt = self.opt.c()
        dev = pool.device
        self.arena = Arena(self.budget)
        self.mem = torch.empty(self.arena.capacity, dtype=torch.uint8, device=dev)
        self.base = int(self.mem.data_ptr())
        self.slots = []
        for _ in range(streams):
            self.slots.append({
                "stream": torch.cuda.Stream(device=dev),
                "meta_h": torch.empty(2 * self.max_sets + 1, dtype=torch.int64).pin_memory(),
                "event": torch.cuda.Event(enable_timing=True),
                "busy": None, "region": None, "out": None, "hoff": None,
            })

    def need(self, n_total: int, S: int) -> int:
        return self._need(n_total, S)

    def batcher(self, max_points: int | None = None, max_sets: int | None = None) -> Batcher:
        return Batcher(max_points or self.max_points, min(max_sets or self.max_sets, self.max_sets), self.need,
                       self.arena.capacity)

    def free_slot(self):
        for s in self.slots:
            if s["busy"] is None:
                return s
        return None

    def room(self) -> int:
        return self.arena.largest_free()

    def launch(self, slot, starts: np.ndarray, sizes: np.ndarray, tag) -> bool:
        """Enqueue one batch on an idle slot's stream: set k = pool rows
        starts[k] .. starts[k] + sizes[k].  Returns False (nothing enqueued)
        when its memory does not fit in the arena now; raises HullError
        (HULL_ERR_BUDGET) when it would not fit in an empty arena."""
        cp, torch = self.cp, self.torch
        S = len(starts)
        n_total = int(np.sum(sizes))
        if S > self.max_sets:
            raise ValueError("batch exceeds the set cap")
        need = self.need(n_total, S)
        if need > self.arena.capacity:
            raise cp.HullError(HULL_ERR_BUDGET, "Server.launch")
        off = self.arena.alloc(need)
        if off is None:
            return False
        ws_bytes = int(cp.load().hull_batch_workspace_bytes(n_total, S, ctypes.byref(self._copt)))
        p_ws = self.base + off
        p_out = p_ws + align_up(ws_bytes)
        p_hoff = p_out + align_up(8 * max(n_total, 1))
        p_meta = p_hoff + align_up(8 * (S + 1))
        # host metadata: starts [S], then offsets [S+1] (pinned, one copy)
        m = slot["meta_h"].numpy()
        m[:S] = starts
        m[S] = 0
        np.cumsum(sizes, out=m[S + 1:2 * S + 1])
        st = slot["stream"]
        mo = off + (p_meta - p_ws)  # byte offsets of the parts within the arena
        ob = off + (p_out - p_ws)
        hb = off + (p_hoff - p_ws)
        meta_d = self.mem[mo:mo + 8 * (2 * S + 1)].view(torch.int64)
        with torch.cuda.stream(st):
            meta_d.copy_(slot["meta_h"][:2 * S + 1], non_blocking=True)
            code = cp.hull_batch_ranges(self.pool.data_ptr(), self.n_xy, p_meta, p_meta + 8 * S, S, n_total, p_ws,
                                        ws_bytes, p_out, p_hoff, self.opt, int(st.cuda_stream))
            if code:
                self.arena.free(off)
                raise cp.HullError(code, "hull_batch_ranges")
            slot["event"].record(st)
        slot["busy"] = tag
        slot["region"] = off
        # views of the outputs (valid until the region is reused by a later launch)
        slot["out"] = self.mem[ob:ob + 8 * max(n_total, 1)].view(torch.int64)
        slot["hoff"] = self.mem[hb:hb + 8 * (S + 1)].view(torch.int64)
        return True

    def poll(self):
        """Batches that have completed: [(slot, tag)]; their slots become
        idle and their memory returns to the arena (their outputs stay
        readable until the next launch)."""
        done = []
        for s in self.slots:
            if s["busy"] is not None and s["event"].query():
                done.append((s, s["busy"]))
                s["busy"] = None
                self.arena.free(s["region"])
                s["region"] = None
        return done


def simulate(server: Server, set_starts: np.ndarray, set_sizes: np.ndarray, req_set: np.ndarray,
             arrivals_s: np.ndarray, max_points: int | None = None, max_sets: int | None = None) -> ServeResult:
    """Open-loop run: request r asks for the hull of pool set req_set[r] and
    arrives at arrivals_s[r] seconds (non-decreasing) after the start."""
    torch = server.torch
    n = len(req_set)
    batcher = server.batcher(max_points, max_sets)
    completion = np.full(n, np.nan)
    server.arena.peak = server.arena.in_use
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    start.record(torch.cuda.current_stream())
    start.synchronize()
    t0 = time.perf_counter()
    nxt, finished, batches, points, deferred = 0, 0, 0, 0, 0
    waiting_for_memory = False
    while finished + len(batcher.refused) < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals_s[nxt] <= now:
            batcher.push(nxt, set_sizes[req_set[nxt]])
            nxt += 1
        for slot, rids in server.poll():
            completion[rids] = start.elapsed_time(slot["event"]) * 1e-3
            finished += len(rids)
        slot = server.free_slot() if len(batcher) else None
        if slot is not None:
            batch = batcher.take(server.room())
            if batch:
                rids = np.fromiter((r for r, _ in batch), dtype=np.int64, count=len(batch))
                sets = req_set[rids]
                if not server.launch(slot, set_starts[sets], set_sizes[sets], rids):
                    raise RuntimeError("a batch formed within the arena's largest free block did not fit")
                batches += 1
                points += int(set_sizes[sets].sum())
                waiting_for_memory = False
            elif len(batcher):
                deferred += 0 if waiting_for_memory else 1
                waiting_for_memory = True
    latency = completion - arrivals_s[:n]
    return ServeResult(latency_s=latency, completion_s=completion, batches=batches, points=points,
                       makespan_s=float(np.nanmax(completion) - arrivals_s[0]) if finished else 0.0,
                       refused=list(batcher.refused), peak_bytes=server.arena.peak, budget_bytes=server.budget,
                       deferred=deferred)
