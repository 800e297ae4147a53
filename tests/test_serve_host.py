"""Host logic of the serving loop (no GPU): batch formation and the
serving workload's request stream."""
import numpy as np

import synth
from paper_1405_3454_gb300.serve import ALIGN, Arena, Batcher


def test_batcher_fifo_and_caps():
    b = Batcher(max_points=100, max_sets=3)
    for rid, size in enumerate([40, 30, 20, 10, 5, 200, 1]):
        b.push(rid, size)
    assert b.take() == [(0, 40), (1, 30), (2, 20)]      # set cap
    assert b.take() == [(3, 10), (4, 5)]                # next would exceed the point cap
    assert b.take() == [(5, 200)]                       # oversize request goes alone
    assert b.take() == [(6, 1)]
    assert b.take() == [] and len(b) == 0


def test_batcher_never_splits_or_reorders():
    rng = np.random.default_rng(3)
    sizes = rng.integers(1, 60, 500)
    b = Batcher(max_points=150, max_sets=7)
    for r, s in enumerate(sizes):
        b.push(r, int(s))
    seen = []
    while len(b):
        batch = b.take()
        assert 1 <= len(batch) <= 7
        assert len(batch) == 1 or sum(s for _, s in batch) <= 150
        seen.extend(r for r, _ in batch)
    assert seen == list(range(500))


def test_serving_requests_are_log_uniform_and_poisson():
    sets, arr = synth.serving_requests(20000, 160, 5)
    assert sets.min() >= 0 and sets.max() < 160
    counts = np.bincount(sets, minlength=160)
    assert counts.min() > 60  # uniform over the pool
    gaps = np.diff(arr)
    assert np.all(gaps > 0) and abs(gaps.mean() - 1.0) < 0.03  # unit-rate exponential
    assert abs(np.median(gaps) - np.log(2)) < 0.03


def test_serving_pool_deciles():
    xy, starts, sizes, shapes = synth.serving_pool(2, 11, 1e4, 1e5)
    edges = np.exp(np.linspace(np.log(1e4), np.log(1e5), 11))
    for j, s in enumerate(sizes):
        d = j // 2
        assert edges[d] - 1 <= s <= edges[d + 1]
    assert starts[0] == 0 and np.all(np.diff(starts) == sizes[:-1])
    assert len(xy) == sizes.sum() and set(shapes.tolist()) <= {0, 1, 2}


def test_arena_first_fit_coalesces_and_tracks_peak():
    a = Arena(10 * ALIGN)
    x = a.alloc(3 * ALIGN)
    y = a.alloc(ALIGN + 1)          # rounded up to 2 ALIGN
    z = a.alloc(5 * ALIGN)
    assert (x, y, z) == (0, 3 * ALIGN, 5 * ALIGN) and a.in_use == 10 * ALIGN
    assert a.alloc(1) is None and a.largest_free() == 0
    a.free(y)
    assert a.largest_free() == 2 * ALIGN and a.alloc(3 * ALIGN) is None
    a.free(x)                        # merges with y's block
    assert a.largest_free() == 5 * ALIGN
    a.free(z)                        # everything merges back
    assert a.free_blocks == [(0, 10 * ALIGN)] and a.in_use == 0 and a.peak == 10 * ALIGN


def test_batcher_defers_on_memory_keeps_fifo_and_refuses_the_impossible():
    need = lambda pts, sets: 10 * pts + 100 * sets    # fake sizes
    b = Batcher(max_points=1000, max_sets=4, need=need, budget=5000)
    for rid, size in enumerate([100, 300, 600, 20, 50]):
        b.push(rid, size)
    assert b.take(room=0) == []                       # head waits: nothing fits
    assert b.take(room=4300) == [(0, 100), (1, 300)]   # 10*400+200 = 4200; adding 600 would not fit
    # 600 alone needs 6100 > budget: refused, not deferred forever; the
    # requests behind it go on
    assert b.take(room=1000) == [(3, 20), (4, 50)]
    assert b.refused == [2] and len(b) == 0


def test_admission_simulation_never_exceeds_the_budget():
    # Requests of random sizes arrive; batches are formed within the arena's
    # largest free block and complete in random order.  The bytes in flight
    # stay within the budget, no request overtakes an earlier one, and only
    # requests that could never fit are refused.
    rng = np.random.default_rng(12)
    need = lambda pts, sets: 8 * pts + 256 * sets
    budget = 64 * 1024
    arena = Arena(budget)
    b = Batcher(max_points=4000, max_sets=5, need=need, budget=arena.capacity)
    sizes = rng.integers(1, 9000, 400)
    for r, s in enumerate(sizes):
        b.push(r, int(s))
    inflight, order = [], []
    while len(b) or inflight:
        batch = b.take(arena.largest_free()) if len(b) else []
        if batch:
            off = arena.alloc(need(sum(s for _, s in batch), len(batch)))
            assert off is not None and arena.in_use <= budget
            inflight.append(off)
            order.extend(r for r, _ in batch)
        elif inflight:
            arena.free(inflight.pop(int(rng.integers(len(inflight)))))
    assert order == sorted(order)
    assert sorted(order + b.refused) == list(range(400))
    assert b.refused == [r for r, s in enumerate(sizes) if need(int(s), 1) > arena.capacity]
    assert arena.peak <= budget and arena.in_use == 0
