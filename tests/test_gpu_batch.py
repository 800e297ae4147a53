"""Parity of hull_batch (through the C ABI) with the CPU oracle, set by set.

Every set's hull (global indices, CCW from the lexicographic minimum) must
equal the oracle's hull of that set alone, shifted by the set's offset.  The
batches mix the three input shapes, empty and tiny sets, sets starting at
odd rows (8-byte but not 16-byte aligned), sizes that span several blocks
of the streaming passes, and a set whose survivors exceed the one-block
hull's capacity (the cooperative large path).
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def convex_ring(k, r=float(1 << 23)):
    a = np.arange(k) * (2 * np.pi / k)
    return np.stack([np.round(r * np.cos(a)), np.round(r * np.sin(a))], 1).astype(np.float32)


def make_batch(sizes, seed, extra=None):
    sets = []
    for k, n in enumerate(sizes):
        sets.append(synth.shape(k % 3, n, seed + k, 0))
    if extra is not None:
        sets.extend(extra)
    offsets = np.zeros(len(sets) + 1, np.int64)
    offsets[1:] = np.cumsum([len(s) for s in sets])
    xy = np.concatenate(sets).astype(np.float32) if offsets[-1] else np.zeros((0, 2), np.float32)
    return sets, offsets, xy


def run_batch(cp, xy, offsets, opt):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda() if len(xy) else torch.zeros((0, 2), device="cuda")
    o = torch.from_numpy(offsets).cuda()
    out, hoff, ws = cp.batch(d, o, opt)
    torch.cuda.synchronize()
    hoff = hoff.cpu().numpy()
    out = out.cpu().numpy()
    return out, hoff, ws


def check(cp, sets, offsets, xy, opt):
    out, hoff, ws = run_batch(cp, xy, offsets, opt)
    assert cp.device_status(ws) == (0, 0)
    assert hoff[0] == 0
    for s, pts in enumerate(sets):
        got = out[hoff[s]:hoff[s + 1]]
        want = oracle.cudapre(pts)["hull"].astype(np.int64) + offsets[s] if len(pts) else np.zeros(0, np.int64)
        assert got.tolist() == want.tolist(), f"set {s} (n={len(pts)})"


SIZES = [0, 1, 2, 3, 5, 17, 100, 1000, 4097, 50_001, 0, 300_000, 2, 123_457, 7]


@pytest.mark.parametrize("angles,filt,refine", [(0, 1, 1), (0, 0, 1), (1, 1, 1), (0, 1, 0), (1, 0, 0)])
def test_batch_mixed_sets(gpu_lib, angles, filt, refine):
    sets, offsets, xy = make_batch(SIZES, 9100)
    check(gpu_lib, sets, offsets, xy, gpu_lib.Options(angles=angles, filter=filt, refine=bool(refine)))


def test_batch_large_path_set(gpu_lib):
    # a set of 20,000 points in convex position plus a disk: more survivors
    # than the one-block hull takes, between ordinary sets
    ring = np.concatenate([synth.disk(3000, 5, 1 << 20), convex_ring(20_000)]).astype(np.float32)
    sets, offsets, xy = make_batch([1000, 33, 70_000], 9200, extra=[ring, synth.square(999, 9201)])
    check(gpu_lib, sets, offsets, xy, gpu_lib.Options())
    check(gpu_lib, sets, offsets, xy, gpu_lib.Options(refine=False))


def test_batch_many_small_sets(gpu_lib):
    rng = np.random.default_rng(9300)
    sizes = [int(v) for v in np.floor(np.exp(rng.uniform(np.log(1), np.log(3e4), 600)))]
    sets, offsets, xy = make_batch(sizes, 9300)
    check(gpu_lib, sets, offsets, xy, gpu_lib.Options())


def degenerate_sets():
    """Sets whose survivors reach the one-block hull of a batch with
    duplicates, collinear runs, equal coordinates across its chunks, and
    convex position up to and past its capacity (1024 points)."""
    rng = np.random.default_rng(9350)
    t = np.arange(-300, 300, dtype=np.float32)
    line = np.stack([t, 2 * t], 1)[rng.permutation(600)]
    vline = np.stack([np.full(500, -9.0), np.repeat(np.arange(100), 5)], 1)[rng.permutation(500)]
    g = np.arange(-3, 4, dtype=np.float32)
    lattice = np.tile(np.stack(np.meshgrid(g, g), -1).reshape(-1, 2), (5, 1))[rng.permutation(245)]
    pair = np.tile(np.array([[0, 0], [5, 5]], np.float32), (20, 1))
    same = np.full((50, 2), 7, np.float32)
    negz = np.array([[-0.0, 3], [0.0, 3], [0.0, -3], [-0.0, -3], [4, 0], [-4, 0], [0, 0]], np.float32)
    rings = [convex_ring(k)[rng.permutation(k)] for k in (31, 32, 33, 1000, 1024, 1025)]
    # convex ring with every point repeated: equal coordinates in adjacent chunks
    rep = np.repeat(convex_ring(400), 2, axis=0)
    sq = synth.square(900, 9351, 1 << 10)  # dense lattice: many equal points
    return [line, vline, lattice, pair, same, negz, rep, sq] + rings


@pytest.mark.parametrize("refine", [True, False])
def test_batch_degenerate_sets(gpu_lib, refine):
    extra = [np.ascontiguousarray(a, dtype=np.float32) for a in degenerate_sets()]
    sets, offsets, xy = make_batch([], 0, extra=extra)
    check(gpu_lib, sets, offsets, xy, gpu_lib.Options(refine=refine))
    check(gpu_lib, sets, offsets, xy, gpu_lib.Options(refine=refine, filter=gpu_lib.HULL_FILTER_EXACT))


@pytest.mark.parametrize("refine", [True, False])
def test_single_degenerate_sets(gpu_lib, refine):
    # the same sets one at a time: the whole-GPU hull of a single set
    import torch
    cp = gpu_lib
    for k, pts in enumerate(degenerate_sets()):
        pts = np.ascontiguousarray(pts, dtype=np.float32)
        h, c, _ = cp.compute(torch.from_numpy(pts).cuda(), cp.Options(refine=refine))
        torch.cuda.synchronize()
        want = oracle.cudapre(pts)["hull"]
        assert cp.as_index(h, int(c.item())).tolist() == want.tolist(), f"set {k}"


def test_batch_plan_sample(gpu_lib):
    # the batch workload's own generator (log-uniform sizes, shape per set),
    # on 48 sets with sizes from 1e3 to 2e5
    S = 48
    xy, offsets, _ = synth.batch(S, 9400, 1e3, 2e5)
    sets = [xy[offsets[s]:offsets[s + 1]] for s in range(S)]
    check(gpu_lib, sets, np.asarray(offsets, np.int64), xy, gpu_lib.Options())


def test_batch_single_set_equals_hull_compute(gpu_lib):
    import torch
    cp = gpu_lib
    pts = synth.disk(1 << 20, 9500)
    out, hoff, _ = run_batch(cp, pts, np.array([0, len(pts)], np.int64), cp.Options())
    d = torch.from_numpy(pts).cuda()
    h, c, _ = cp.compute(d)
    torch.cuda.synchronize()
    assert out[hoff[0]:hoff[1]].tolist() == cp.as_index(h, int(c.item())).tolist()


def test_batch_empty_and_zero_sets(gpu_lib):
    cp = gpu_lib
    sets, offsets, xy = make_batch([0, 0, 0], 9600)
    out, hoff, ws = run_batch(cp, xy, offsets, cp.Options())
    assert hoff.tolist() == [0, 0, 0, 0]
    out, hoff, ws = run_batch(cp, np.zeros((0, 2), np.float32), np.array([0], np.int64), cp.Options())
    assert hoff.tolist() == [0]


def test_batch_bad_offsets_flagged(gpu_lib):
    cp = gpu_lib
    sets, offsets, xy = make_batch([100, 200, 300], 9700)
    bad = offsets.copy()
    bad[1], bad[2] = bad[2], bad[1]  # decreasing
    out, hoff, ws = run_batch(cp, xy, bad, cp.Options())
    assert cp.device_status(ws)[1] & cp.HULL_DEVICE_OFFSETS
    assert hoff.tolist() == [0, 0, 0, 0]


def test_batch_ranges_in_a_pool(gpu_lib):
    # sets taken anywhere in a resident pool: overlapping, repeated, empty,
    # out of order, starting at odd rows
    import torch
    cp = gpu_lib
    pool = np.concatenate([synth.disk(300_000, 9800), synth.square(200_001, 9801),
                           synth.gaussian(150_000, 9802)]).astype(np.float32)
    rng = np.random.default_rng(9803)
    ranges = [(0, 300_000), (300_000, 200_001), (500_001, 150_000), (12_345, 0), (7, 99_999), (7, 99_999),
              (640_000, 10_001), (123_457, 3), (1, 1)]
    for _ in range(40):
        a = int(rng.integers(0, len(pool)))
        b = int(rng.integers(0, min(60_000, len(pool) - a) + 1))
        ranges.append((a, b))
    d = torch.from_numpy(pool).cuda()
    starts = torch.tensor([r[0] for r in ranges], dtype=torch.int64, device="cuda")
    sizes = torch.tensor([r[1] for r in ranges], dtype=torch.int64, device="cuda")
    out, hoff, ws = cp.batch_ranges(d, starts, sizes)
    torch.cuda.synchronize()
    assert cp.device_status(ws) == (0, 0)
    out, hoff = out.cpu().numpy(), hoff.cpu().numpy()
    for s, (a, b) in enumerate(ranges):
        got = out[hoff[s]:hoff[s + 1]]
        want = (oracle.cudapre(pool[a:a + b])["hull"].astype(np.int64) + a) if b else np.zeros(0, np.int64)
        assert got.tolist() == want.tolist(), (s, a, b)


def test_batch_range_beyond_the_pool_flagged(gpu_lib):
    import torch
    cp = gpu_lib
    pool = torch.from_numpy(synth.disk(1000, 9804)).cuda()
    starts = torch.tensor([0, 900], dtype=torch.int64, device="cuda")
    sizes = torch.tensor([500, 200], dtype=torch.int64, device="cuda")
    out, hoff, ws = cp.batch_ranges(pool, starts, sizes)
    torch.cuda.synchronize()
    assert cp.device_status(ws)[1] & cp.HULL_DEVICE_OFFSETS
    assert hoff.cpu().tolist() == [0, 0, 0]


def test_server_slots_match_oracle_and_simulation_completes(gpu_lib):
    import torch
    from paper_1405_3454_gb300 import serve
    cp = gpu_lib
    pxy, starts, sizes, _ = synth.serving_pool(1, 9900, 1e3, 2e5)
    pool = torch.from_numpy(pxy).cuda()
    server = serve.Server(pool, budget_bytes=1 << 30, max_points=1 << 20, max_sets=64, streams=2)
    picks = [[0, 3, 5, 9, 9], [1, 2, 4, 6, 7, 8]]
    slots = []
    for k, p in enumerate(picks):
        slot = server.free_slot()
        assert server.launch(slot, starts[p], sizes[p], k)
        slots.append(slot)
    torch.cuda.synchronize()
    done = server.poll()
    assert sorted(t for _, t in done) == [0, 1] and server.free_slot() is not None
    for slot, p in zip(slots, picks):
        out, hoff = slot["out"].cpu().numpy(), slot["hoff"][:len(p) + 1].cpu().numpy()
        for s, j in enumerate(p):
            want = oracle.cudapre(pxy[starts[j]:starts[j] + sizes[j]])["hull"].astype(np.int64) + starts[j]
            assert out[hoff[s]:hoff[s + 1]].tolist() == want.tolist()
    req_set, unit = synth.serving_requests(500, len(sizes), 9901)
    res = serve.simulate(server, starts, sizes, req_set, unit / 20000.0)
    assert np.all(np.isfinite(res.completion_s)) and np.all(res.latency_s > 0)
    assert res.points == int(sizes[req_set].sum())


def test_set_alone_equals_in_batch_equals_in_serving_mix(gpu_lib):
    # One set's hull computed alone (hull_compute on its rows), inside a
    # batch of other sets (hull_batch_ranges) and inside a serving slot's
    # mix (Server.launch) is the same list of global indices.
    import torch
    from paper_1405_3454_gb300 import serve
    cp = gpu_lib
    pxy, starts, sizes, _ = synth.serving_pool(1, 9950, 1e3, 3e5)
    pool = torch.from_numpy(pxy).cuda()
    server = serve.Server(pool, budget_bytes=1 << 30, max_points=1 << 22, max_sets=32, streams=1)
    rng = np.random.default_rng(9951)
    for j in range(len(sizes)):
        a, b = int(starts[j]), int(sizes[j])
        h, c, _ = cp.compute(pool[a:a + b])
        torch.cuda.synchronize()
        alone = (cp.as_index(h, int(c.item())) + a).tolist()
        others = rng.choice(len(sizes), 6, replace=True).tolist()
        mix = others[:3] + [j] + others[3:]
        out, hoff, ws = cp.batch_ranges(pool, torch.tensor(starts[mix], device="cuda"),
                                        torch.tensor(sizes[mix], device="cuda"))
        torch.cuda.synchronize()
        assert cp.device_status(ws) == (0, 0)
        hoff = hoff.cpu().numpy()
        in_batch = out[hoff[3]:hoff[4]].cpu().tolist()
        slot = server.free_slot()
        assert server.launch(slot, starts[mix[::-1]], sizes[mix[::-1]], j)
        torch.cuda.synchronize()
        assert [t for _, t in server.poll()] == [j]
        so = slot["hoff"][:len(mix) + 1].cpu().numpy()
        k = len(mix) - 1 - 3
        in_serving = slot["out"][so[k]:so[k + 1]].cpu().tolist()
        assert alone == in_batch == in_serving, j
    want = oracle.cudapre(pxy[starts[0]:starts[0] + sizes[0]])["hull"].astype(np.int64) + starts[0]
    h, c, _ = cp.compute(pool[int(starts[0]):int(starts[0] + sizes[0])])
    assert (cp.as_index(h, int(c.item())) + starts[0]).tolist() == want.tolist()


def test_server_admits_by_memory_budget(gpu_lib):
    # A budget that holds one large batch at a time: requests wait for
    # memory (in arrival order), one that could never fit is refused, the
    # bytes in flight never exceed the budget, and every served hull is the
    # oracle's.
    import torch
    from paper_1405_3454_gb300 import serve
    cp = gpu_lib
    pxy, starts, sizes, _ = synth.serving_pool(1, 9960, 1e4, 4e5)
    pool = torch.from_numpy(pxy).cuda()
    big = int(np.argmax(sizes))
    budget = serve.batch_bytes(cp, int(sizes[big]) + 2000, 2, cp.Options()) + 4096
    server = serve.Server(pool, budget_bytes=budget, max_points=1 << 22, max_sets=8, streams=3)
    # a request above the budget is refused before any CUDA call
    huge = np.array([0], np.int64), np.array([len(pxy)], np.int64)
    if serve.batch_bytes(cp, len(pxy), 1, cp.Options()) > budget:
        with pytest.raises(cp.HullError):
            server.launch(server.free_slot(), huge[0], huge[1], -1)
    req_set = np.array([big, big, 0, big, 1, 2, big, 3], np.int64)
    res = serve.simulate(server, starts, sizes, req_set, np.zeros(len(req_set)))
    assert not res.refused and np.all(np.isfinite(res.completion_s))
    assert res.peak_bytes <= budget and res.deferred >= 1
    # a pool row range as one request larger than the whole budget
    starts2 = np.concatenate([starts, [0]]).astype(np.int64)
    sizes2 = np.concatenate([sizes, [len(pxy)]]).astype(np.int64)
    res2 = serve.simulate(server, starts2, sizes2, np.array([0, len(sizes), 1], np.int64), np.zeros(3))
    if serve.batch_bytes(cp, len(pxy), 1, cp.Options()) > budget:
        assert res2.refused == [1] and np.isnan(res2.latency_s[1])
    assert np.isfinite(res2.latency_s[0]) and np.isfinite(res2.latency_s[2])
    # served results are the oracle's hulls
    for j in (big, 0, 1):
        slot = server.free_slot()
        assert server.launch(slot, starts[[j]], sizes[[j]], j)
        torch.cuda.synchronize()
        server.poll()
        want = oracle.cudapre(pxy[starts[j]:starts[j] + sizes[j]])["hull"].astype(np.int64) + starts[j]
        h = slot["hoff"].cpu().numpy()
        assert slot["out"][h[0]:h[1]].cpu().tolist() == want.tolist()
