"""Parity of the 3D extension (section 5) on the GPU with the CPU oracle:
the 24 extremes, the facet planes of their polyhedron and the survivor set,
bit for bit, over sizes with every tail, the three shapes, both angle
tables and both arithmetic forms, degenerate sets and points on the
facets (which the float32 filter must escalate)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

MODES = [(a, f) for a in (0, 1) for f in (0, 1)]


def run3(cp, xyz, angles, filt):
    import torch
    d = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float32).reshape(-1, 3)).cuda()
    surv, cnt, ext, ws = cp.prefilter3(d, cp.Options(angles=angles, filter=filt))
    torch.cuda.synchronize()
    info = cp.read_polyhedron(ws)
    s = np.sort(cp.as_index(surv, int(cnt.item())))
    return cp.as_index(ext), info, s, ws


def check3(cp, xyz, angles, filt):
    e, info, s, ws = run3(cp, xyz, angles, filt)
    want = oracle.cudapre3(xyz, angles)
    assert e.tolist() == np.where(want["extremes"] < 0, 0xFFFFFFFF, want["extremes"]).tolist(), "extremes"
    assert info["planes"] == want["planes"].tolist(), "planes"
    assert s.tolist() == want["survivors"].tolist(), "survivors"
    assert info["device_status"] == 0
    return info


SIZES = [0, 1, 2, 3, 4, 5, 7, 17, 1000, 4099, 65537, 300_001]


@pytest.mark.parametrize("angles,filt", MODES)
@pytest.mark.parametrize("n", SIZES)
def test_3d_sizes_and_shapes(gpu_lib, n, angles, filt):
    for kind in (0, 1, 2):
        check3(gpu_lib, synth.shape3(kind, n, 500 + n, kind), angles, filt)


def degenerate3():
    rng = np.random.default_rng(8)
    yield "all_equal", np.tile(np.array([[3, -4, 5]], np.float32), (3000, 1))
    k = rng.integers(-1000, 1000, 20_000)
    yield "collinear", np.stack([k * 7, k * -3, k], 1).astype(np.float32)
    xy = rng.integers(-500, 500, size=(20_000, 2))
    yield "coplanar", np.stack([xy[:, 0], xy[:, 1], 2 * xy[:, 0] - xy[:, 1] + 9], 1).astype(np.float32)
    yield "small_lattice", synth.cube3(40_000, 9, r=6)
    z = synth.cube3(40_000, 10, r=30)
    z[z == 0] = -0.0
    yield "negative_zero", z
    c = rng.choice(np.array([-(1 << 19), 1 << 19, 0, 1, -1], np.float32), size=(30_000, 3))
    yield "domain_corners", c.astype(np.float32)
    s = 1000
    corners = np.array([(x, y, zz) for x in (-s, s) for y in (-s, s) for zz in (-s, s)], np.float32)
    inner = rng.integers(-s + 1, s, size=(10_000, 3)).astype(np.float32)
    yield "cube_corners_late", np.concatenate([inner, corners, corners])


@pytest.mark.parametrize("name,xyz", list(degenerate3()), ids=lambda v: v if isinstance(v, str) else "")
def test_3d_degenerate(gpu_lib, name, xyz):
    for angles, filt in MODES:
        check3(gpu_lib, xyz, angles, filt)


def test_3d_points_on_facets_escalate(gpu_lib):
    # a Gaussian cloud plus points on or within a unit of its polyhedron's
    # facets (never outside it, so the polyhedron stays): the float32 plane
    # tests cannot decide them and must escalate; results stay exact
    rng = np.random.default_rng(21)
    g = synth.gauss3(100_000, 22)
    ext = oracle.extremes3(g)
    planes = oracle.facets3(g, ext)
    verts = g[sorted(set(int(i) for i in ext))].astype(np.int64)
    # exact in int64: |N| < 2^42, |p| <= 2^19, so N.p - d stays below 2^63
    N, d = planes[:, :3], planes[:, 3]
    extra = np.zeros((0, 3), np.int64)
    while len(extra) < 60_000:
        for f in range(len(planes)):
            on = verts[verts @ N[f] == d[f]].astype(np.float64)  # the facet's vertices
            w = rng.dirichlet(np.ones(len(on)), size=1000)
            cand = np.rint(w @ on).astype(np.int64)
            s = cand @ N.T - d
            extra = np.concatenate([extra, cand[np.all(s <= 0, axis=1)]])  # on the facet or just inside
    xyz = np.concatenate([g, extra[:60_000].astype(np.float32)]).astype(np.float32)
    assert oracle.facets3(xyz, oracle.extremes3(xyz)).tolist() == planes.tolist()
    info = check3(gpu_lib, xyz, 0, 1)
    assert info["n_escalated"] > 1000, info["n_escalated"]
    check3(gpu_lib, xyz, 0, 0)


def test_3d_validate_and_alignment(gpu_lib):
    import torch
    cp = gpu_lib
    for bad in (0.5, np.nan, np.inf, 2.0 ** 19 + 1, -(2.0 ** 19 + 1)):
        xyz = synth.cube3(5000, 1, r=100)
        xyz[777, 2] = bad
        d = torch.from_numpy(xyz).cuda()
        surv, cnt, ext, ws = cp.prefilter3(d, cp.Options(validate=True))
        torch.cuda.synchronize()
        assert cp.read_polyhedron(ws)["device_status"] & cp.HULL_DEVICE_DOMAIN
        assert int(cnt.item()) == 0
    # a 4-byte (not 16-byte) aligned input is refused before any launch
    buf = torch.zeros(3 * 1001, dtype=torch.float32, device="cuda")
    v = buf[1:3001].view(1000, 3)
    with pytest.raises(cp.HullError):
        cp.prefilter3(v)


def test_3d_large_ball(gpu_lib):
    n = 1 << 24
    for kind in (1, 0):
        check3(gpu_lib, synth.shape3(kind, n, 31 + kind), 0, 1)
