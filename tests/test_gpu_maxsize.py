"""The largest single set the ABI takes: n = 2^32 - 1 points (32 GiB of
points, about 145 GiB on the device with the workspace and the output).

The points are built so that the hull is known without running the oracle
over 4.3e9 points: 48 integer vertices of a convex polygon (their own hull,
by the oracle, fixes the expected order) placed at high indices, some also
copied to low indices (the lowest index must stand for equal points), and
every other point strictly inside the polygon (uniform in a square whose
corners lie inside the polygon's inscribed circle), drawn on the device from
a seeded generator.  Indices near 2^32 exercise every 32-bit index and
64-bit offset on the path."""
import math

import numpy as np
import pytest

import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N = (1 << 32) - 1
K = 48
R = float(1 << 23)


def polygon():
    a = np.arange(K) * (2 * math.pi / K)
    v = np.stack([np.round(R * np.cos(a)), np.round(R * np.sin(a))], 1).astype(np.float32)
    h = oracle.hull(v)
    assert len(h) == K  # every vertex is a hull vertex
    return v, h


def test_max_points_hull(gpu_lib):
    import torch
    cp = gpu_lib
    free, _ = torch.cuda.mem_get_info()
    need = N * 8 + cp.hull_workspace_bytes(N) + N * 4 + (4 << 30)
    if free < need:
        pytest.skip(f"needs {need / 2**30:.0f} GiB on the device, {free / 2**30:.0f} GiB free")
    v, h = polygon()
    xy = torch.empty((N, 2), dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(20140513)
    a = 0.6 * R  # corner radius 0.85 R, inside the inscribed radius R cos(pi / K)
    step = 1 << 28
    for s in range(0, N, step):
        e = min(N, s + step)
        xy[s:e].uniform_(-a, a, generator=g).round_()
    # the vertices at high indices (vertex k at N - 1 - 7k), and copies of
    # every third vertex at low indices (vertex k also at 5 + 11k)
    hi = np.array([N - 1 - 7 * k for k in range(K)], dtype=np.int64)
    lo = np.array([5 + 11 * k for k in range(0, K, 3)], dtype=np.int64)
    vt = torch.from_numpy(v).cuda()
    xy[torch.from_numpy(hi).cuda()] = vt
    xy[torch.from_numpy(lo).cuda()] = vt[torch.arange(0, K, 3, device="cuda")]
    first = hi.copy()
    first[0::3] = lo
    want = first[h].tolist()
    out, cnt, ws = cp.compute(xy)
    torch.cuda.synchronize()
    assert cp.device_status(ws) == (0, 0)
    assert int(cnt.item()) == K
    assert cp.as_index(out[:K], K).tolist() == want
