"""Pins of the 3D oracle (section 5: extremes of the set and of copies rotated
about one axis, their convex polyhedron, the strict-inside discard) against
things other than itself: the 2D oracle's extremes of the projection, numpy
first-occurrence argmin/argmax, hand-worked solids, Qhull's facets with
exact integer plane arithmetic, and the hull of the survivors."""
import math

import numpy as np
import pytest

import oracle
import synth


def test_group0_is_numpy_first_occurrence_and_z_slots_repeat():
    xyz = synth.cube3(50_000, 11, r=40)  # many ties
    for angles in (0, 1):
        e = oracle.extremes3(xyz, angles)
        for a in range(3):
            col = xyz[:, a]
            assert e[2 * a] == int(np.argmin(col)) and e[2 * a + 1] == int(np.argmax(col))
        for g in range(4):  # z' = z: every group's z slots are group 0's
            assert e[6 * g + 4] == e[4] and e[6 * g + 5] == e[5]


@pytest.mark.parametrize("angles", [0, 1])
def test_rotated_slots_are_the_2d_extremes_of_the_projection(angles):
    # x' and y' are the 2D rotation of (x, y): the 3D slots 6g + 0..3 must be
    # the 2D oracle's slots 4g + 0..3 of the xy projection
    for kind in (0, 1, 2):
        xyz = synth.shape3(kind, 30_001, 12 + kind)
        e3 = oracle.extremes3(xyz, angles)
        e2 = oracle.extremes(np.ascontiguousarray(xyz[:, :2]), angles)
        for g in range(4):
            assert e3[6 * g:6 * g + 4].tolist() == e2[4 * g:4 * g + 4].tolist()


def test_empty_and_tiny_sets():
    assert oracle.extremes3(np.zeros((0, 3), np.float32)).tolist() == [-1] * 24
    one = np.array([[5, -3, 2]], np.float32)
    assert oracle.extremes3(one).tolist() == [0] * 24
    assert oracle.facets3(one, oracle.extremes3(one)).shape == (0, 4)
    r = oracle.cudapre3(one)
    assert r["survivors"].tolist() == [0]


def _with_interior(corners, k=200, seed=3):
    # corners first, then points strictly inside their hull (convex
    # combinations with all weights > 0, rounded toward the centroid)
    rng = np.random.default_rng(seed)
    c = np.asarray(corners, np.int64)
    w = rng.dirichlet(np.ones(len(c)) * 2, size=k)
    pts = np.rint(w @ c)
    return np.concatenate([c, pts]).astype(np.float32)


def test_cube_has_six_axis_facets():
    s = 1000
    corners = [(x, y, z) for x in (-s, s) for y in (-s, s) for z in (-s, s)]
    xyz = _with_interior(corners)
    planes = oracle.facets3(xyz, list(range(8)))
    want = sorted([[1, 0, 0, s], [-1, 0, 0, s], [0, 1, 0, s], [0, -1, 0, s], [0, 0, 1, s], [0, 0, -1, s]])
    assert planes.tolist() == want
    surv = oracle.prefilter3(xyz, planes)
    # the corners survive; interior points strictly inside are discarded
    assert set(range(8)) <= set(surv.tolist())
    inside = [i for i in range(8, len(xyz)) if np.all(np.abs(xyz[i]) < s)]
    assert not set(inside) & set(surv.tolist())


def test_tetrahedron_planes_by_hand():
    xyz = np.array([[0, 0, 0], [4, 0, 0], [0, 4, 0], [0, 0, 4], [1, 1, 1], [4, 0, 0], [2, 2, 0]], np.float32)
    planes = oracle.facets3(xyz, list(range(7)))
    assert planes.tolist() == sorted([[-1, 0, 0, 0], [0, -1, 0, 0], [0, 0, -1, 0], [1, 1, 1, 4]])
    # (1,1,1) strictly inside; (2,2,0) on a face and the duplicate vertex survive
    assert oracle.prefilter3(xyz, planes).tolist() == [0, 1, 2, 3, 5, 6]


def test_degenerate_polyhedra_discard_nothing():
    flat = np.array([[x, y, 7] for x in range(-3, 4) for y in range(-3, 4)], np.float32)
    assert oracle.facets3(flat, list(range(len(flat)))).shape == (0, 4)
    line = np.array([[t, 2 * t, -t] for t in range(-5, 6)], np.float32)
    assert oracle.facets3(line, list(range(len(line)))).shape == (0, 4)
    for xyz in (flat, line):
        r = oracle.cudapre3(xyz)
        assert r["planes"].shape == (0, 4) and r["survivors"].tolist() == list(range(len(xyz)))


def _exact_plane(a, b, c):
    a, b, c = (tuple(int(v) for v in p) for p in (a, b, c))
    u = [b[i] - a[i] for i in range(3)]
    v = [c[i] - a[i] for i in range(3)]
    n = [u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]]
    d = sum(n[i] * a[i] for i in range(3))
    return n, d


def _qhull_planes(pts):
    """Facet planes of the hull of integer points from Qhull's simplices,
    each plane computed exactly from its three vertices, oriented outward,
    reduced; coplanar simplices give one plane."""
    from scipy.spatial import ConvexHull
    h = ConvexHull(pts.astype(np.float64))
    out = set()
    allp = [tuple(int(v) for v in p) for p in pts]
    for s in h.simplices:
        n, d = _exact_plane(pts[s[0]], pts[s[1]], pts[s[2]])
        side = [sum(n[i] * p[i] for i in range(3)) - d for p in allp]
        if max(side) > 0:
            assert min(side) >= 0
            n, d = [-v for v in n], -d
        g = math.gcd(math.gcd(abs(n[0]), abs(n[1])), math.gcd(abs(n[2]), abs(d)))
        out.add((n[0] // g, n[1] // g, n[2] // g, d // g))
    return sorted(list(p) for p in out)


@pytest.mark.parametrize("seed", range(12))
def test_facets_equal_qhull_exact_planes(seed):
    rng = np.random.default_rng(100 + seed)
    k = int(rng.integers(4, 40))
    pts = rng.integers(-(1 << 19), (1 << 19) + 1, size=(k, 3)).astype(np.float32)
    if seed % 3 == 0:  # a small lattice: coplanar facets with many points
        pts = rng.integers(-3, 4, size=(k, 3)).astype(np.float32)
    try:
        want = _qhull_planes(pts)
    except Exception:
        pytest.skip("Qhull rejects this set (flat)")
    got = oracle.facets3(pts, list(range(k)))
    assert got.tolist() == want


@pytest.mark.parametrize("kind", [0, 1, 2])
def test_prefilter_against_qhull_planes_and_survivor_hull(kind):
    from scipy.spatial import ConvexHull
    xyz = synth.shape3(kind, 20_000, 40 + kind)
    for angles in (0, 1):
        ext = oracle.extremes3(xyz, angles)
        uniq = sorted(set(int(i) for i in ext))
        planes = _qhull_planes(xyz[uniq])
        assert oracle.facets3(xyz, ext).tolist() == planes
        # strict inside test by exact Python integers on the Qhull planes
        P = np.array(planes, dtype=object)
        X = xyz.astype(np.int64).astype(object)
        s = X @ P[:, :3].T - P[:, 3]
        want = [i for i in range(len(xyz)) if not all(v < 0 for v in s[i])]
        surv = oracle.prefilter3(xyz, planes)
        assert surv.tolist() == want
        # the discarded points change no hull: same hull vertices
        full = set(ConvexHull(xyz.astype(np.float64)).vertices.tolist())
        part = ConvexHull(xyz[surv].astype(np.float64)).vertices
        assert set(surv[part].tolist()) == full


def test_check_domain3():
    ok = np.array([[0, -0.0, 1], [2.0 ** 19, -(2.0 ** 19), 5]], np.float32)
    assert oracle.check_domain3(ok)
    for bad in (np.nan, np.inf, 0.5, 2.0 ** 19 + 1, -(2.0 ** 19 + 1)):
        x = ok.copy()
        x[1, 2] = bad
        assert not oracle.check_domain3(x)
