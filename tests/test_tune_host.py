"""The batch launch-shape tuner (host logic, no GPU): it keeps the fastest
candidate of a timing table, caches it by (GPU name, size class) in a JSON
file, and reuses the cache without timing again."""
import json

import paper_1405_3454_gb300 as cp
from paper_1405_3454_gb300 import tune


def fake_table():
    # a made-up timing surface with one minimum
    return {(w, u): 5.0 + abs(w - 4) * 0.7 + abs(u - 64) / 32.0 for w in (1, 2, 4, 8) for u in (16, 32, 64, 128)}


def test_tuner_picks_the_fastest_and_caches(tmp_path):
    path = str(tmp_path / "shapes.json")
    table = fake_table()
    calls = []

    def run(shape):
        calls.append(shape)
        return table[(shape["waves"], shape["unit_chunks"])]

    t = tune.Tuner("GB300-test", path)
    best = t.tune(1_939_658_877, 4096, run)
    assert best == {"waves": 4, "unit_chunks": 64, "grid": 0}
    assert len(calls) == 2 * len(tune.CANDIDATES)
    # same size class: from the cache, no timing
    assert t.tune(1_800_000_000, 5000, run) == best and len(calls) == 2 * len(tune.CANDIDATES)
    # a new object reads the file
    t2 = tune.Tuner("GB300-test", path)
    assert t2.lookup(1_939_658_877, 4096) == best
    saved = json.load(open(path))
    (key,) = saved.keys()
    assert key == "GB300-test|n2^30_s2^12" and len(saved[key]["table"]) == len(tune.CANDIDATES)
    # another GPU or size class is tuned on its own
    assert tune.Tuner("other-gpu", path).lookup(1_939_658_877, 4096) is None
    assert t2.lookup(1 << 20, 4096) is None


def test_tuner_ties_keep_the_first_and_options_apply(tmp_path):
    t = tune.Tuner("dev", str(tmp_path / "s.json"))
    cands = [{"waves": 2, "unit_chunks": 16, "grid": 0}, {"waves": 8, "unit_chunks": 128, "grid": 0}]
    assert t.tune(1000, 10, lambda s: 1.0, cands) == cands[0]
    o = t.options(1000, 10, cp.Options(refine=False))
    assert (o.waves, o.unit_chunks, o.grid, o.refine) == (2, 16, 0, False)
    assert t.options(1 << 30, 10, cp.Options()) == cp.Options()
