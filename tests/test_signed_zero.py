"""Ties between -0.0 and +0.0 in the extreme search (section 2, Step 1).

-0.0 and +0.0 are equal values, so a tie between them goes to the lowest
index like any other tie.  The sets below put the extreme of several
directions at exactly 0: the bulk lies strictly inside one quadrant, and
copies of the origin with every sign pattern (plus points on the two axes)
sit at a low index and at higher ones -- in the same warp, in other warps,
in other blocks, and at the loose head and tail points.  Both orders occur:
the lowest index holding the -0.0 score, or the +0.0 one.

The CPU check confirms the data does what it is for: for some direction
the maximum score is 0, reached by a -0.0 at a lower index and a +0.0 at a
higher one, so ordering scores by their raw bit patterns (which puts -0.0
below +0.0) would pick the wrong index.  The GPU tests compare the 16
extremes, the polygon, the survivors and the hull with the oracle, for one
set and inside a batch.
"""
import numpy as np
import pytest

import oracle
import synth

QUADRANTS = [(1, 1), (1, -1), (-1, 1), (-1, -1)]


def tables():
    k = oracle.constants()  # pinned against the closed forms elsewhere
    s3, c75, s75, h = k["s3"], k["c75"], k["s75"], k["h"]
    return {0: [(1.0, 0.0), (s3, 0.5), (c75, s75), (-0.5, s3)],
            1: [(1.0, 0.0), (s3, 0.5), (h, h), (0.5, s3)]}


def zero_positions(n):
    # same warp (pairs 1 and 20 of a chunk), other warps (pair 300), other
    # blocks (middle and far end), the head point and the odd tail point
    return sorted({0, 2, 40, 41, 601, 5000, n // 2 + 1, n - 3, n - 1})


def signed_zero_set(n, quadrant, neg_first, seed):
    rng = np.random.default_rng(seed)
    sx, sy = quadrant
    r = 1 << 20
    xy = np.stack([sx * rng.integers(1, r, n), sy * rng.integers(1, r, n)], 1).astype(np.float32)
    pos = zero_positions(n)
    for k, p in enumerate(pos):
        negx = (k % 2 == 0) == neg_first      # alternate the sign of x, starting as asked
        negy = (k // 2) % 2 == 0
        zx = np.float32(-0.0) if negx else np.float32(0.0)
        zy = np.float32(-0.0) if negy else np.float32(0.0)
        if k % 3 == 2:
            xy[p] = (zx, sy * rng.integers(1, r))   # on the y axis: x' = 0, not the origin
        elif k % 3 == 1 and k > 1:
            xy[p] = (sx * rng.integers(1, r), zy)   # on the x axis
        else:
            xy[p] = (zx, zy)                        # a copy of the origin
    return xy


def cases(n=300_001):
    for q in QUADRANTS:
        for neg_first in (True, False):
            yield q, neg_first, signed_zero_set(n, q, neg_first, 7 + 2 * QUADRANTS.index(q) + neg_first)


def scores(xy, angles):
    """Binary64 scores of the 16 directions, slot order (larger is better)."""
    x = xy[:, 0].astype(np.float64)
    y = xy[:, 1].astype(np.float64)
    out = []
    for c, s in tables()[angles]:
        px = x * c - y * s
        py = x * s + y * c
        out += [-px, px, -py, py]
    return out


def bits_key(v):
    b = v.view(np.uint64)
    neg = (b >> np.uint64(63)).astype(bool)
    return np.where(neg, ~b, b | np.uint64(1 << 63))


def test_data_separates_signed_zero_ties():
    # (not gpu) the sets contain ties at 0 that an ordering by raw bits gets
    # wrong: the lowest index of the tie holds -0.0, a higher one +0.0
    hits = {True: 0, False: 0}
    for q, neg_first, xy in cases(20_001):
        for angles in (0, 1):
            want = oracle.extremes(xy, angles)
            for slot, sc in enumerate(scores(xy, angles)):
                key = bits_key(sc)
                by_bits = int(np.flatnonzero(key == key.max())[0])
                assert sc[want[slot]] == sc.max()
                if by_bits != want[slot]:
                    assert sc.max() == 0.0 and np.signbit(sc[want[slot]])
                    hits[neg_first] += 1
    assert hits[True] > 0 and hits[False] > 0, hits


@pytest.mark.gpu
@pytest.mark.parametrize("offset", [False, True])
def test_signed_zero_ties_single_set(gpu_lib, offset):
    from test_gpu_parity import MODES, check_compute, check_prefilter
    for q, neg_first, xy in cases():
        for angles, filt in MODES:
            check_prefilter(gpu_lib, xy, angles, filt, offset=offset)
        check_compute(gpu_lib, xy, 0, 1, offset=offset)
        check_compute(gpu_lib, xy, 1, 0, offset=offset)


@pytest.mark.gpu
@pytest.mark.parametrize("angles,filt", [(0, 1), (0, 0), (1, 1), (1, 0)])
def test_signed_zero_ties_in_a_batch(gpu_lib, angles, filt):
    import torch
    cp = gpu_lib
    sets = []
    for k, (q, neg_first, xy) in enumerate(cases(100_001)):
        sets.append(xy)
        sets.append(synth.shape(k % 3, 1 + 999 * k, 400 + k, 0))  # odd sizes: later sets start unaligned
    offsets = np.zeros(len(sets) + 1, np.int64)
    offsets[1:] = np.cumsum([len(s) for s in sets])
    xy = np.concatenate(sets).astype(np.float32)
    d = torch.from_numpy(xy).cuda()
    o = torch.from_numpy(offsets).cuda()
    opt = cp.Options(angles=angles, filter=filt)
    out, hoff, ws = cp.batch(d, o, opt)
    torch.cuda.synchronize()
    assert cp.device_status(ws) == (0, 0)
    out, hoff = out.cpu().numpy(), hoff.cpu().numpy()
    n_total, S = int(offsets[-1]), len(sets)
    for s, pts in enumerate(sets):
        info = cp.batch_read_set(ws, n_total, S, s)
        want_ext = oracle.extremes(pts, angles)
        assert info["extremes"] == np.where(want_ext < 0, 0xFFFFFFFF, want_ext).tolist(), s
        pidx, pxy = oracle.hull16(pts, want_ext)
        assert info["poly_idx"] == pidx.tolist() and info["poly_xy"] == pxy.tolist(), s
        want = oracle.cudapre(pts, angles)
        assert info["n_survivors"] == len(want["survivors"]), s
        got = out[hoff[s]:hoff[s + 1]]
        assert got.tolist() == (want["hull"] + offsets[s]).tolist(), s
