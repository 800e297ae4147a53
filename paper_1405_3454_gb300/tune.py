"""Launch-shape tuner for batched calls.

The shapes a batch call can vary without changing any result (hull_options
`waves`, `unit_chunks`, `grid`) are timed on the caller's own workload and
the fastest is kept in a JSON cache keyed by (GPU name, size class): the
power of two of the batch's points and of its set count.  Host code only:
`run(shape)` does the timing (CUDA events around the library call in real
use; a table in the tests).
"""
from __future__ import annotations

import json
import math
import os

# (waves of the streaming search's static shares, chunks per unit of the
# inside test); grid 0 = resident blocks
CANDIDATES = [{"waves": w, "unit_chunks": u, "grid": 0} for w in (1, 2, 4, 8) for u in (16, 32, 64, 128)]


def default_cache_path() -> str:
    return os.environ.get("CUDAPRE_TUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "cudapre", "batch_shapes.json"))


def size_class(n_total: int, sets: int) -> str:
    return "n2^%d_s2^%d" % (int(math.log2(max(int(n_total), 1))), int(math.log2(max(int(sets), 1))))


class Tuner:
    def __init__(self, device: str, path: str | None = None):
        self.device = device
        self.path = path or default_cache_path()
        self.cache: dict = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.cache = json.load(f)
            except (OSError, ValueError):
                self.cache = {}

    def key(self, n_total: int, sets: int) -> str:
        return "%s|%s" % (self.device, size_class(n_total, sets))

    def lookup(self, n_total: int, sets: int):
        e = self.cache.get(self.key(n_total, sets))
        return dict(e["shape"]) if e else None

    def tune(self, n_total: int, sets: int, run, candidates=None, reps: int = 2) -> dict:
        """The cached shape for this size class, else the candidate with the
        least time (the least of `reps` runs each; ties keep the earlier
        candidate), which is cached and saved."""
        hit = self.lookup(n_total, sets)
        if hit is not None:
            return hit
        table = []
        best, best_t = None, math.inf
        for c in (candidates or CANDIDATES):
            t = min(float(run(dict(c))) for _ in range(max(1, reps)))
            table.append({"shape": dict(c), "ms": t})
            if t < best_t:
                best, best_t = dict(c), t
        self.cache[self.key(n_total, sets)] = {"shape": best, "ms": best_t, "table": table}
        self.save()
        return dict(best)

    def save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(self.cache, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def options(self, n_total: int, sets: int, base):
        """`base` (an Options) with the cached shape of this size class, if any."""
        import dataclasses
        shape = self.lookup(n_total, sets)
        return dataclasses.replace(base, **shape) if shape else base
