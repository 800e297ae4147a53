"""Full-size parity at the benchmark's workload and launch configuration.

268,435,456 lattice points uniform in the disk of radius 2^24 (2 GiB), the
same generator stream and library defaults that bench.py times.  The CPU
oracle computes the extremes, the polygon, the survivor set and the hull of
the survivors over all points (about a minute of single-thread CPU), and
every output of the GPU must match it bit for bit, in both filter modes.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = 1 << 28
SEED = 1405345  # bench.py's seed for rank 0


@pytest.fixture(scope="module")
def disk_and_oracle():
    xy = synth.disk(N, SEED)
    ref = oracle.cudapre(xy)
    return xy, ref


@pytest.mark.parametrize("filt", [1, 0])
def test_disk_2p28_bit_exact(gpu_lib, disk_and_oracle, filt):
    import torch
    cp = gpu_lib
    xy, ref = disk_and_oracle
    d = torch.from_numpy(xy).cuda()
    opt = cp.Options(filter=filt)
    surv, cnt, ext, ws = cp.prefilter(d, opt)
    torch.cuda.synchronize()
    assert cp.as_index(ext).tolist() == ref["extremes"].tolist()
    m, pxy, _ = cp.read_polygon(ws)
    assert pxy == ref["poly_xy"].tolist()
    ns = int(cnt.item())
    assert ns == len(ref["survivors"])
    got = np.sort(cp.as_index(surv, ns))
    assert np.array_equal(got, ref["survivors"])
    del surv, ws
    for refine in (True, False):
        out, hcnt, ws2 = cp.compute(d, cp.Options(filter=filt, refine=refine))
        torch.cuda.synchronize()
        assert cp.as_index(out, int(hcnt.item())).tolist() == ref["hull"].tolist()
        del out, ws2
    # cumulative angles on a disk leave ~6.7 % outside the 12-gon
    assert 0.060 < ns / N < 0.072


def test_batch_4096_sets_sampled(gpu_lib):
    """The batched workload at full size (4096 sets, log-uniform sizes from
    1e3 to 4e6, about 1.9e9 points) through hull_batch with the bench's
    defaults; 16 sets, the largest among them, checked against the oracle
    one by one, and every hull offset checked for consistency."""
    import torch
    cp = gpu_lib
    S = 4096
    xy, off, _ = synth.batch(S, SEED + 17)
    n = int(off[-1])
    d = torch.from_numpy(xy).cuda()
    o = torch.from_numpy(off).cuda()
    out, hoff, ws = cp.batch(d, o)
    torch.cuda.synchronize()
    assert cp.device_status(ws) == (0, 0)
    hoff = hoff.cpu().numpy()
    assert hoff[0] == 0 and np.all(np.diff(hoff) >= 3)
    sizes = np.diff(off)
    pick = sorted(set([int(np.argmax(sizes)), int(np.argmin(sizes))] +
                      np.random.default_rng(17).choice(S, 14, replace=False).tolist()))
    for s in pick:
        got = out[hoff[s]:hoff[s + 1]].cpu().numpy()
        want = oracle.cudapre(xy[off[s]:off[s + 1]])["hull"].astype(np.int64) + off[s]
        assert got.tolist() == want.tolist(), s
    del d, out, ws
    assert n > 1_000_000_000


def test_near_edge_2p28_fp32_decisions_match_exact(gpu_lib):
    """The FP32 filter's error bound at scale: 2^28 points, half of them
    (1.3e8) on or within one unit inside the polygon's edges, where float32
    cannot decide and the bound must send the test to int64.  The survivor
    set, the polygon and the hull must equal the oracle's (exact integer
    arithmetic); a wrong bound would keep or drop some near-edge point."""
    import torch
    cp = gpu_lib
    xy, poly = synth.near_edge_mix(N, SEED + 41, lambda g: oracle.hull16(g, oracle.extremes(g))[1])
    _, opoly = oracle.hull16(xy, oracle.extremes(xy))
    assert opoly.tolist() == poly.tolist()
    osurv = oracle.prefilter(xy, opoly)
    d = torch.from_numpy(xy).cuda()
    surv, cnt, ext, ws = cp.prefilter(d)
    torch.cuda.synchronize()
    assert cp.read_polygon(ws)[1] == opoly.tolist()
    ns, nesc = cp.read_counters(ws)
    assert nesc > N // 8, nesc
    assert np.array_equal(np.sort(cp.as_index(surv, int(cnt.item()))), osurv)
    del surv, ws
    out, hcnt, _ = cp.compute(d)
    torch.cuda.synchronize()
    assert cp.as_index(out, int(hcnt.item())).tolist() == oracle.hull(xy, osurv).tolist()


def test_time_grows_linearly_with_n(gpu_lib):
    """Linear time: on the disk workload, 4x the points costs between 2x and
    4.4x the device time of hull_compute (at most linear growth, within
    noise; below 4x while the costs that do not grow with n, about 0.2 ms
    of the survivors' hull, still weigh), median of 7 timed calls after 3
    warm-up calls each."""
    import torch
    cp = gpu_lib
    ms = {}
    for n in (1 << 26, 1 << 28):
        d = torch.from_numpy(synth.disk(n, SEED)).cuda()
        ws = cp.workspace(cp.hull_workspace_bytes(n))
        t = []
        for k in range(10):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            cp.compute(d, ws=ws)
            b.record()
            torch.cuda.synchronize()
            if k >= 3:
                t.append(a.elapsed_time(b))
        ms[n] = float(np.median(t))
        del d, ws
    r = ms[1 << 28] / ms[1 << 26]
    assert 2.0 < r < 4.4, ms


@pytest.mark.parametrize("name", ["all_equal", "collinear", "ring"])
def test_reserved_slots_when_everything_survives(gpu_lib, name):
    """hull_compute on one set of 2^24 points or more reserves survivor slots
    ahead and fills a warp's last block with copies of one of its survivors.
    Sets where every point survives (a degenerate polygon, or points in
    convex position) use the most slots: the hull must still equal the
    oracle's, and the reported survivors exclude the copies."""
    import torch
    cp = gpu_lib
    n = 1 << 24
    rng = np.random.default_rng(24)
    if name == "all_equal":
        xy = np.tile(np.array([[3.0, -4.0]], np.float32), (n, 1))
    elif name == "collinear":
        k = rng.integers(-(1 << 20), 1 << 20, n)
        xy = np.stack([k * 7, k * -3], 1).astype(np.float32)
    else:
        a = rng.uniform(0, 2 * np.pi, n)
        xy = np.stack([np.round(8e6 * np.cos(a)), np.round(8e6 * np.sin(a))], 1).astype(np.float32)
    want = oracle.cudapre(xy)
    d = torch.from_numpy(xy).cuda()
    for refine in (True, False):
        out, cnt, ws = cp.compute(d, cp.Options(refine=refine))
        torch.cuda.synchronize()
        assert cp.device_status(ws) == (0, 0)
        assert cp.as_index(out[:int(cnt.item())], int(cnt.item())).tolist() == want["hull"].tolist()
        assert cp.read_stats(ws)["n_survivors"] == len(want["survivors"])
