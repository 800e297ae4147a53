"""hull_batch run as a CUDA graph (hull_graph_*): capture, replay, replay on
new contents of the same buffers, update for other arguments -- every
result equal to the eager call and to the oracle's hull of each set alone."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _batch(seed, sizes, ring=0):
    sets = [synth.shape(k % 3, n, seed + k, 0) for k, n in enumerate(sizes)]
    if ring:
        a = np.arange(ring) * (2 * np.pi / ring)
        r = float(1 << 23)
        sets.append(np.stack([np.round(r * np.cos(a)), np.round(r * np.sin(a))], 1).astype(np.float32))
    offsets = np.zeros(len(sets) + 1, np.int64)
    offsets[1:] = np.cumsum([len(s) for s in sets])
    return sets, offsets, np.concatenate(sets).astype(np.float32)


def _hulls(out, hoff):
    out, hoff = out.cpu().numpy(), hoff.cpu().numpy()
    return [out[hoff[s]:hoff[s + 1]].tolist() for s in range(len(hoff) - 1)]


def _want(sets, offsets):
    return [(oracle.cudapre(p)["hull"] + offsets[s]).tolist() for s, p in enumerate(sets)]


def test_graph_replay_equals_eager_and_oracle(gpu_lib):
    import torch
    cp = gpu_lib
    sizes = [0, 1, 3, 1000, 70_001, 5, 300_000, 2, 12_345]
    sets, offsets, xy = _batch(7100, sizes, ring=20_000)  # the ring takes the large path
    n_total, S = int(offsets[-1]), len(sets)
    d = torch.from_numpy(xy).cuda()
    o = torch.from_numpy(offsets).cuda()
    want = _want(sets, offsets)
    eout, ehoff, _ = cp.batch(d, o)
    torch.cuda.synchronize()
    assert _hulls(eout, ehoff) == want
    wsb = cp.hull_batch_workspace_bytes(n_total, S)
    ws = cp.workspace(wsb)
    out = torch.empty(n_total, dtype=torch.int64, device="cuda")
    hoff = torch.empty(S + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    g = cp.Graph()
    with torch.cuda.stream(stream):
        for k in range(3):
            out.fill_(-1)
            g.batch_ranges(d, None, o, n_total, ws, out, hoff, stream=stream)
            stream.synchronize()
            assert cp.device_status(ws, stream) == (0, 0)
            assert _hulls(out, hoff) == want, k
    c = g.counts()
    assert c["captures"] == 1 and c["replays"] == 2 and c["instantiations"] == 1 and c["kernels"] > 5
    # new point data in the same buffers: a replay computes the new hulls
    sets2, offsets2, xy2 = _batch(7200, sizes, ring=20_000)
    assert np.array_equal(offsets2, offsets)
    d.copy_(torch.from_numpy(xy2))
    with torch.cuda.stream(stream):
        g.batch_ranges(d, None, o, n_total, ws, out, hoff, stream=stream)
        stream.synchronize()
    assert _hulls(out, hoff) == _want(sets2, offsets)
    assert g.counts()["replays"] == 3
    # other arguments: a capture that updates or replaces the graph
    sets3, offsets3, xy3 = _batch(7300, [50_000, 7, 120_000])
    d3 = torch.from_numpy(xy3).cuda()
    o3 = torch.from_numpy(offsets3).cuda()
    with torch.cuda.stream(stream):
        g.batch_ranges(d3, None, o3, int(offsets3[-1]), ws, out, hoff[:4], stream=stream)
        stream.synchronize()
        assert _hulls(out, hoff[:4]) == _want(sets3, offsets3)
        g.batch_ranges(d, None, o, n_total, ws, out, hoff, cp.Options(filter=cp.HULL_FILTER_EXACT), stream=stream)
        stream.synchronize()
        assert _hulls(out, hoff) == _want(sets2, offsets)
    c = g.counts()
    assert c["captures"] == 3 and c["updates"] + c["instantiations"] == 3
    g.close()


def test_graph_of_pool_ranges(gpu_lib):
    # ranges of a resident pool (the server's call) through a graph
    import torch
    cp = gpu_lib
    pool = np.concatenate([synth.disk(200_000, 7400), synth.gaussian(100_001, 7401)]).astype(np.float32)
    ranges = [(0, 200_000), (200_000, 100_001), (5, 99_999), (123_457, 3), (7, 0)]
    d = torch.from_numpy(pool).cuda()
    starts = torch.tensor([a for a, _ in ranges], dtype=torch.int64, device="cuda")
    offsets = torch.tensor(np.concatenate([[0], np.cumsum([b for _, b in ranges])]), dtype=torch.int64, device="cuda")
    n_total, S = int(offsets[-1].item()), len(ranges)
    ws = cp.workspace(cp.hull_batch_workspace_bytes(n_total, S))
    out = torch.empty(n_total, dtype=torch.int64, device="cuda")
    hoff = torch.empty(S + 1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    g = cp.Graph()
    with torch.cuda.stream(stream):
        for _ in range(2):
            g.batch_ranges(d, starts, offsets, n_total, ws, out, hoff, stream=stream)
            stream.synchronize()
            got = _hulls(out, hoff)
            for s, (a, b) in enumerate(ranges):
                want = (oracle.cudapre(pool[a:a + b])["hull"] + a).tolist() if b else []
                assert got[s] == want, s
    assert g.counts()["replays"] == 1
    g.close()
