"""Host logic of the serving loop (no GPU): batch formation and the
serving workload's request stream."""
import numpy as np

import synth
from paper_1405_3454_gb300.serve import Batcher


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
