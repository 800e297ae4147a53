"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact comparisons: the 16 extreme indices, the Step-2 polygon, the
survivor set (sorted indices; compaction order is unspecified) and the hull
index list (order included).  Sizes span several tiles and ragged tails;
edge cases cover empty input, tiny inputs, duplicates, collinear sets,
-0.0 and coordinates at +-2^24, and an 8-byte (not 16-byte) aligned input.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

MODES = [(a, f) for a in (0, 1) for f in (0, 1)]  # (angles, filter)


def to_dev(xy, offset=False):
    import torch
    a = np.ascontiguousarray(xy, dtype=np.float32).reshape(-1, 2)
    if not offset:
        return torch.from_numpy(a).cuda()
    # 8-byte but not 16-byte aligned view: one leading dummy point
    buf = torch.empty(a.shape[0] + 1, 2, dtype=torch.float32, device="cuda")
    buf[1:] = torch.from_numpy(a).cuda()
    v = buf[1:]
    assert v.data_ptr() % 16 == 8
    return v


def run_prefilter(cp, xy, angles, filt, offset=False):
    d = to_dev(xy, offset)
    surv, cnt, ext, ws = cp.prefilter(d, cp.Options(angles=angles, filter=filt))
    import torch
    torch.cuda.synchronize()
    n_s = int(cnt.item())
    s = np.sort(cp.as_index(surv, n_s))
    e = cp.as_index(ext)
    m, pxy, _ = cp.read_polygon(ws)
    return e, np.array(pxy, dtype=np.int64).reshape(-1, 2), s, ws


def oracle_ext(xy, angles):
    e = oracle.extremes(xy, angles)
    return np.where(e < 0, 0xFFFFFFFF, e)


def check_prefilter(cp, xy, angles, filt, offset=False):
    e, poly, surv, ws = run_prefilter(cp, xy, angles, filt, offset)
    oe = oracle_ext(xy, angles)
    assert e.tolist() == oe.tolist(), "extremes"
    if xy.shape[0]:
        _, opoly = oracle.hull16(xy, oracle.extremes(xy, angles))
    else:
        opoly = np.zeros((0, 2), dtype=np.int32)
    assert poly.tolist() == opoly.tolist(), "polygon"
    osurv = oracle.prefilter(xy, opoly)
    assert surv.tolist() == osurv.tolist(), "survivors"
    return ws


def check_compute(cp, xy, angles, filt, offset=False, refine=True):
    import torch
    d = to_dev(xy, offset)
    out, cnt, ws = cp.compute(d, cp.Options(angles=angles, filter=filt, refine=refine))
    torch.cuda.synchronize()
    h = cp.as_index(out, int(cnt.item()))
    want = oracle.hull(xy)
    assert h.tolist() == want.tolist(), "hull"
    return ws


SIZES = [0, 1, 2, 3, 4, 5, 7, 17, 255, 1000, 2047, 2048, 4097, 65537, 300001]


@pytest.mark.parametrize("angles,filt", MODES)
@pytest.mark.parametrize("n", SIZES)
def test_prefilter_sizes(gpu_lib, n, angles, filt):
    for kind in (0, 1, 2):
        xy = synth.shape(kind, n, 7 + n, 50 + kind)
        check_prefilter(gpu_lib, xy, angles, filt)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 1001, 65537])
def test_prefilter_unaligned_input(gpu_lib, n):
    for kind in (0, 1, 2):
        xy = synth.shape(kind, n, 9 + n, 60 + kind)
        for filt in (0, 1):
            check_prefilter(gpu_lib, xy, 0, filt, offset=True)
            check_compute(gpu_lib, xy, 0, filt, offset=True)


@pytest.mark.parametrize("refine", [True, False])
@pytest.mark.parametrize("angles,filt", MODES)
@pytest.mark.parametrize("n", [0, 1, 2, 3, 5, 17, 1000, 4097, 65537, 300001])
def test_compute_sizes(gpu_lib, n, angles, filt, refine):
    for kind in (0, 1, 2):
        xy = synth.shape(kind, n, 11 + n, 70 + kind)
        check_compute(gpu_lib, xy, angles, filt, refine=refine)


@pytest.mark.parametrize("refine", [True, False])
@pytest.mark.parametrize("k", [8190, 8192, 8193, 8200, 20000])
def test_one_block_and_large_paths_at_the_boundary(gpu_lib, k, refine):
    # Points in convex position survive every discard round, so the hull
    # stage sees exactly k survivors: both sides of the one-block limit.
    a = np.arange(k) * (2 * np.pi / k)
    r = float(1 << 23)
    xy = np.stack([np.round(r * np.cos(a)), np.round(r * np.sin(a))], 1).astype(np.float32)
    inner = synth.disk(5000, 3, 1 << 20)
    xy = np.concatenate([inner, xy]).astype(np.float32)
    check_compute(gpu_lib, xy, 0, 1, refine=refine)


def degenerate_sets():
    r = np.random.default_rng(5)
    yield "all_equal", np.tile(np.array([[3.0, -4.0]], np.float32), (5000, 1))
    yield "two_points", np.array([[0, 0], [5, 5]] * 3000, np.float32)
    k = r.integers(-1000, 1000, 20000)
    yield "collinear", np.stack([k * 7, k * -3], 1).astype(np.float32)
    sq = synth.square(40000, 3, 50)  # heavy duplication, many ties
    yield "small_lattice", sq
    z = sq.copy()
    z[z == 0] = -0.0
    yield "negative_zero", z
    big = r.choice(np.array([-(1 << 24), 1 << 24, 0, 1, -1], np.float32), size=(30000, 2))
    yield "domain_corners", big.astype(np.float32)
    tri = np.array([[0, 0], [6, 0], [0, 6], [1, 1], [3, 3], [0, 3], [3, 0]] * 1000, np.float32)
    yield "triangle_repeated", tri
    circ = []
    for t in range(4096):  # points in convex position: nothing can be discarded twice
        a = 2 * np.pi * t / 4096
        circ.append((round(8e6 * np.cos(a)), round(8e6 * np.sin(a))))
    yield "convex_position", np.array(circ, np.float32)


@pytest.mark.parametrize("name,xy", list(degenerate_sets()), ids=lambda v: v if isinstance(v, str) else "")
def test_degenerate(gpu_lib, name, xy):
    for angles, filt in MODES:
        check_prefilter(gpu_lib, xy, angles, filt)
        check_compute(gpu_lib, xy, angles, filt)
        check_compute(gpu_lib, xy, angles, filt, refine=False)


def test_config1_square_1m(gpu_lib):
    # 1,000,000 points uniform in [-2^20, 2^20]^2, plain exact and FP32-filtered
    xy = synth.square(1_000_000, synth.BASE_SEED, 1 << 20)
    for filt in (0, 1):
        check_prefilter(gpu_lib, xy, 0, filt)
        check_compute(gpu_lib, xy, 0, filt)


def test_filter_modes_identical_near_edges(gpu_lib):
    # Half Gaussian, half on/within one unit inside the polygon's edges: the
    # FP32 filter must escalate, and both modes must agree with the oracle.
    import torch
    n = 1 << 20
    xy, poly = synth.near_edge_mix(n, 17, lambda g: oracle.hull16(g, oracle.extremes(g))[1])
    _, poly_all = oracle.hull16(xy, oracle.extremes(xy))
    assert poly_all.tolist() == poly.tolist()
    ws = check_prefilter(gpu_lib, xy, 0, 1)
    ns, nesc = gpu_lib.read_counters(ws)
    assert nesc > n // 8, nesc  # many near-boundary decisions escalated
    check_prefilter(gpu_lib, xy, 0, 0)
    check_compute(gpu_lib, xy, 0, 1)


def test_launch_shapes_do_not_change_results(gpu_lib):
    import torch
    xy = synth.disk(500_000, 23)
    ref = None
    for grid in (1, 3, 64, 1000):
        d = to_dev(xy)
        surv, cnt, ext, ws = gpu_lib.prefilter(d, gpu_lib.Options(grid=grid))
        out, hcnt, _ = gpu_lib.compute(d, gpu_lib.Options(grid=grid))
        torch.cuda.synchronize()
        got = (gpu_lib.as_index(ext).tolist(), np.sort(gpu_lib.as_index(surv, int(cnt.item()))).tolist(),
               gpu_lib.as_index(out, int(hcnt.item())).tolist())
        if ref is None:
            ref = got
        assert got == ref, grid


def test_validate_flags_out_of_domain(gpu_lib):
    import torch
    for bad in (np.float32(0.5), np.float32(np.nan), np.float32(np.inf), np.float32(-np.inf),
                np.float32(2 ** 24 + 2), np.float32(-(2 ** 24 + 2)), np.float32(-0.5)):
        xy = synth.square(10000, 1, 100)
        xy[1234, 1] = bad
        d = to_dev(xy)
        out, cnt, ws = gpu_lib.compute(d, gpu_lib.Options(validate=True))
        torch.cuda.synchronize()
        code, bits = gpu_lib.device_status(ws)
        assert bits & gpu_lib.HULL_DEVICE_DOMAIN and code == 2
        assert int(cnt.item()) == 0
    # in-domain input passes validation, boundary values and -0.0 included
    xy = synth.square(10000, 1, 100)
    xy[10] = (2.0 ** 24, -(2.0 ** 24))
    xy[20] = (-0.0, 0.0)
    out, cnt, ws = gpu_lib.compute(to_dev(xy), gpu_lib.Options(validate=True))
    assert gpu_lib.device_status(ws) == (0, 0)
    assert gpu_lib.as_index(out, int(cnt.item())).tolist() == oracle.hull(xy).tolist()


def test_workspace_reuse_back_to_back(gpu_lib):
    import torch
    a = synth.disk(200_000, 31)
    b = synth.gaussian(150_000, 32)
    ws = gpu_lib.workspace(gpu_lib.hull_workspace_bytes(200_000))
    for xy in (a, b, a):
        out, cnt, _ = gpu_lib.compute(to_dev(xy), ws=ws)
        torch.cuda.synchronize()
        assert gpu_lib.as_index(out, int(cnt.item())).tolist() == oracle.hull(xy).tolist()
        out, cnt, _ = gpu_lib.compute(to_dev(xy), gpu_lib.Options(refine=False), ws=ws)
        torch.cuda.synchronize()
        assert gpu_lib.as_index(out, int(cnt.item())).tolist() == oracle.hull(xy).tolist()


@pytest.mark.parametrize("name,n", [("empty", 0), ("one", 1), ("tiny_square", 700), ("small_disk", 5000),
                                    ("disk_100k", 100_000), ("square_1m", 1_000_000)])
def test_no_prefilter_hull_equals_the_method(gpu_lib, name, n):
    # the paper's case (1): the hull of all points with no preprocessing
    # (every point goes to the small-set or the large-set hull) gives the
    # same hull as the method
    import torch
    cp = gpu_lib
    xy = synth.square(n, 31, 1 << 20) if "square" in name else synth.disk(n, 32)
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda() if n else torch.zeros((0, 2), device="cuda")
    out, cnt, _ = cp.compute(d, cp.Options(no_prefilter=True))
    torch.cuda.synchronize()
    got = cp.as_index(out, int(cnt.item())).tolist()
    want = oracle.cudapre(xy)["hull"].tolist() if n else []
    assert got == want


@pytest.mark.parametrize("name,xy", list(degenerate_sets()) + [
    ("all_equal_large", np.tile(np.array([[-7.0, 9.0]], np.float32), (20000, 1)))],
    ids=lambda v: v if isinstance(v, str) else "")
def test_no_prefilter_degenerate(gpu_lib, name, xy):
    # case (1) on sets with duplicates, collinear points and equal keys; sets
    # beyond the one-block path make their sort keys from the points (equal
    # points: no sort pass moves anything and the keys are written apart)
    import torch
    cp = gpu_lib
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    out, cnt, ws = cp.compute(d, cp.Options(no_prefilter=True))
    torch.cuda.synchronize()
    assert cp.device_status(ws) == (0, 0)
    assert cp.as_index(out, int(cnt.item())).tolist() == oracle.hull(xy).tolist()


def test_bounded_wait_timeout_reports_and_context_survives(gpu_lib):
    # A bounded device wait that nothing releases gives up, records the
    # timeout in the workspace status and returns; the context stays usable
    # and the next call on the same workspace clears the status.
    import torch
    cp = gpu_lib
    xy = synth.disk(100_000, 41)
    ws = cp.workspace(cp.hull_workspace_bytes(len(xy)))
    for limit in (1, 1 << 12, 1 << 20):
        cp.selftest_wait(ws, limit)
        torch.cuda.synchronize()
        assert cp.device_status(ws) == (5, cp.HULL_DEVICE_TIMEOUT)
    out, cnt, _ = cp.compute(to_dev(xy), ws=ws)
    torch.cuda.synchronize()
    assert cp.device_status(ws) == (0, 0)
    assert cp.as_index(out, int(cnt.item())).tolist() == oracle.hull(xy).tolist()


@pytest.mark.parametrize("name,lo,hi", [("square", 5e-5, 2e-3), ("disk", 0.060, 0.072),
                                        ("gaussian", 2e-5, 2e-3)])
def test_survivor_fraction_bands(gpu_lib, name, lo, hi):
    # Fraction of points left after Step 3 with cumulative angles: in a
    # square the corners are among the 16 extremes and only thin slivers
    # along the sides remain, a disk keeps the circular segments outside the
    # inscribed polygon, a Gaussian cloud only its sparse outer tail.
    import torch
    n = 1 << 24
    xy = {"square": lambda: synth.square(n, 51, 1 << 24), "disk": lambda: synth.disk(n, 52),
          "gaussian": lambda: synth.gaussian(n, 53)}[name]()
    surv, cnt, _, ws = gpu_lib.prefilter(to_dev(xy))
    torch.cuda.synchronize()
    assert lo <= int(cnt.item()) / n <= hi


def _crescent(n, seed):
    # lattice points of the disk of radius 2^23 outside an offset disk of
    # radius 0.9 * 2^23: hull and Step-2 polygon are round, the survivors and
    # the refinement winners form a crescent whose mean lies off-centre
    rng = np.random.default_rng(seed)
    r = float(1 << 23)
    out = np.zeros((0, 2))
    while len(out) < n:
        p = rng.uniform(-r, r, size=(2 * n, 2)).round()
        keep = (np.hypot(p[:, 0], p[:, 1]) <= r) & (np.hypot(p[:, 0] - 0.15 * r, p[:, 1]) > 0.9 * r)
        out = np.concatenate([out, p[keep]])
    return out[:n].astype(np.float32)


def _two_blobs(n, seed):
    # two lattice disks of radius 2^22, centres 2^24 apart: a stadium-like
    # hull with two long straight edges
    rng = np.random.default_rng(seed)
    r = float(1 << 22)
    out = np.zeros((0, 2))
    while len(out) < n:
        p = rng.uniform(-r, r, size=(2 * n, 2)).round()
        out = np.concatenate([out, p[np.hypot(p[:, 0], p[:, 1]) <= r]])
    out = out[:n]
    out[::2] += [-(2.0 ** 23), 0.0]
    out[1::2] += [2.0 ** 23 - 2.0 ** 22, 2.0 ** 21]
    return out.astype(np.float32)


@pytest.mark.parametrize("name", ["crescent", "two_blobs"])
def test_refinement_on_uneven_shapes(gpu_lib, name):
    # shapes whose refinement winners are far from round: the disk inside the
    # winners' polygon must be rejected or small, never wrong
    import torch
    for n in (70_000, 1 << 20):
        xy = _crescent(n, 61) if name == "crescent" else _two_blobs(n, 62)
        out, cnt, ws = gpu_lib.compute(to_dev(xy))
        torch.cuda.synchronize()
        assert gpu_lib.device_status(ws) == (0, 0)
        assert gpu_lib.as_index(out, int(cnt.item())).tolist() == oracle.hull(xy).tolist(), n


def _columns(n, seed, w, h):
    # n lattice points in w columns of height h: many points per column and
    # many exact copies, so the large-set hull sees long x runs and ties
    rng = np.random.default_rng(seed)
    xy = np.stack([rng.integers(-w, w + 1, n), rng.integers(-h, h + 1, n)], 1).astype(np.float32)
    return xy


@pytest.mark.parametrize("name", ["columns", "one_column", "two_columns", "copies_late"])
def test_large_path_columns_and_copies(gpu_lib, name):
    # The large-set hull keeps only the lowest and highest point of each x
    # column for its chains; columns, copies of the extreme points at high
    # and low indices and single-column sets must still give the oracle's
    # hull, through the case (1) path (every point) and through the
    # survivors of Step 3 without refinement (compaction order).
    import torch
    cp = gpu_lib
    if name == "columns":
        xy = _columns(300_000, 71, 60, 3000)
    elif name == "one_column":
        xy = _columns(50_000, 72, 0, 1 << 20)
    elif name == "two_columns":
        xy = _columns(50_000, 73, 1, 1 << 20)
        xy[:, 0] *= 5
    else:
        xy = _columns(120_000, 74, 300, 300)
        # copies of the extremes of every column, late in the set
        xy[-2000:] = xy[:2000][np.argsort(xy[:2000, 1])]
    want = oracle.hull(xy)
    d = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    for opt in (cp.Options(no_prefilter=True), cp.Options(refine=False), cp.Options()):
        out, cnt, ws = cp.compute(d, opt)
        torch.cuda.synchronize()
        assert cp.device_status(ws) == (0, 0)
        assert cp.as_index(out, int(cnt.item())).tolist() == want.tolist(), opt
