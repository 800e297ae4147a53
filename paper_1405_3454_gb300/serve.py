"""Continuous batching of hull requests over a device-resident pool of point
sets.

A request names a set (a range of rows of the pool).  The server keeps a
FIFO of requests that have arrived and, whenever one of its slots is free,
launches every waiting request that fits the slot (point and set caps) as one
hull_batch_ranges call on the slot's own stream: no points are copied, only
the requests' start rows and sizes (16 bytes each) go to the device.  A slot
owns its workspace and output buffers, sized once for its caps, so serving
allocates nothing per batch.  Completion is detected by polling the slot's
CUDA event; a request's latency is the GPU time of that event minus the
request's arrival time, both measured from one start event.

The method itself (section 2, Steps 1-3, and the hull of the survivors)
runs entirely in the library's kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass

import numpy as np


class Batcher:
    """FIFO of waiting requests; take() forms the next batch in arrival order
    without exceeding max_points points or max_sets requests (a single
    request larger than max_points is taken alone)."""

    def __init__(self, max_points: int, max_sets: int):
        if max_points < 1 or max_sets < 1:
            raise ValueError("batch caps must be positive")
        self.max_points = int(max_points)
        self.max_sets = int(max_sets)
        self.q: collections.deque = collections.deque()

    def push(self, rid: int, size: int):
        self.q.append((int(rid), int(size)))

    def __len__(self):
        return len(self.q)

    def take(self) -> list[tuple[int, int]]:
        out, pts = [], 0
        while self.q and len(out) < self.max_sets:
            rid, size = self.q[0]
            if out and pts + size > self.max_points:
                break
            self.q.popleft()
            out.append((rid, size))
            pts += size
        return out


@dataclass
class ServeResult:
    latency_s: np.ndarray      # per request, in request order
    completion_s: np.ndarray   # per request, from the start event
    batches: int
    points: int
    makespan_s: float          # first arrival to last completion

    def summary(self) -> dict:
        lat = self.latency_s * 1e3
        return {"requests": int(len(lat)), "batches": self.batches,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "max_ms": float(lat.max()),
                "gpoints_per_s": self.points / self.makespan_s / 1e9}


class Server:
    """Up to `slots` batches in flight, each on its own stream."""

    def __init__(self, pool, max_points: int, max_sets: int, slots: int = 2, opt=None):
        import torch
        import paper_1405_3454_gb300 as cp
        self.cp = cp
        self.torch = torch
        self.pool = pool
        self.n_xy = cp._check_points(pool)
        self.opt = opt or cp.Options()
        self.max_points, self.max_sets = int(max_points), int(max_sets)
        dev = pool.device
        self.ws_bytes = cp.hull_batch_workspace_bytes(self.max_points, self.max_sets, self.opt)
        self.slots = []
        for _ in range(slots):
            self.slots.append({
                "stream": torch.cuda.Stream(device=dev),
                "ws": cp.workspace(self.ws_bytes, dev),
                "out": torch.empty(self.max_points, dtype=torch.int64, device=dev),
                "hoff": torch.empty(self.max_sets + 1, dtype=torch.int64, device=dev),
                "meta_h": torch.empty(2 * self.max_sets + 1, dtype=torch.int64).pin_memory(),
                "meta_d": torch.empty(2 * self.max_sets + 1, dtype=torch.int64, device=dev),
                "event": torch.cuda.Event(enable_timing=True),
                "busy": None,
            })

    def free_slot(self):
        for s in self.slots:
            if s["busy"] is None:
                return s
        return None

    def launch(self, slot, starts: np.ndarray, sizes: np.ndarray, tag):
        """Enqueue one batch: set k = pool rows starts[k] .. starts[k] + sizes[k]."""
        cp = self.cp
        S = len(starts)
        n_total = int(sizes.sum())
        if S > self.max_sets or n_total > self.max_points:
            raise ValueError("batch exceeds the slot's caps")
        # host metadata: starts [S], then offsets [S+1] (pinned, one copy)
        m = slot["meta_h"].numpy()
        m[:S] = starts
        m[S] = 0
        np.cumsum(sizes, out=m[S + 1:2 * S + 1])
        st = slot["stream"]
        d = slot["meta_d"]
        with self.torch.cuda.stream(st):
            d[:2 * S + 1].copy_(slot["meta_h"][:2 * S + 1], non_blocking=True)
            code = cp.hull_batch_ranges(self.pool.data_ptr(), self.n_xy, d.data_ptr(), d.data_ptr() + 8 * S, S,
                                        n_total, slot["ws"].data_ptr(), self.ws_bytes, slot["out"].data_ptr(),
                                        slot["hoff"].data_ptr(), self.opt, int(st.cuda_stream))
            if code:
                raise cp.HullError(code, "hull_batch_ranges")
            slot["event"].record(st)
        slot["busy"] = tag

    def poll(self):
        """Slots whose batch has completed: [(slot, tag)]; the slots become free."""
        done = []
        for s in self.slots:
            if s["busy"] is not None and s["event"].query():
                done.append((s, s["busy"]))
                s["busy"] = None
        return done


def simulate(server: Server, set_starts: np.ndarray, set_sizes: np.ndarray, req_set: np.ndarray,
             arrivals_s: np.ndarray, max_points: int | None = None, max_sets: int | None = None) -> ServeResult:
    """Open-loop run: request r asks for the hull of pool set req_set[r] and
    arrives at arrivals_s[r] seconds (non-decreasing) after the start."""
    torch = server.torch
    n = len(req_set)
    batcher = Batcher(max_points or server.max_points, max_sets or server.max_sets)
    completion = np.full(n, np.nan)
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    start.record(torch.cuda.current_stream())
    start.synchronize()
    t0 = time.perf_counter()
    nxt, finished, batches, points = 0, 0, 0, 0
    while finished < n:
        now = time.perf_counter() - t0
        while nxt < n and arrivals_s[nxt] <= now:
            batcher.push(nxt, set_sizes[req_set[nxt]])
            nxt += 1
        for slot, rids in server.poll():
            t_done = start.elapsed_time(slot["event"]) * 1e-3
            completion[rids] = t_done
            finished += len(rids)
        slot = server.free_slot() if len(batcher) else None
        if slot is not None:
            batch = batcher.take()
            rids = np.fromiter((r for r, _ in batch), dtype=np.int64, count=len(batch))
            sets = req_set[rids]
            server.launch(slot, set_starts[sets], set_sizes[sets], rids)
            batches += 1
            points += int(set_sizes[sets].sum())
    latency = completion - arrivals_s[:n]
    return ServeResult(latency_s=latency, completion_s=completion, batches=batches, points=points,
                       makespan_s=float(np.nanmax(completion) - arrivals_s[0]))
