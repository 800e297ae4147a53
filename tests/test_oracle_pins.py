"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed
forms, constructions whose extremes are known, a textbook or library routine
(numpy argmin/argmax, scipy's Qhull -- the library the paper itself used),
an O(n^3) brute force, an independent area-decomposition inside test,
hand-worked cases, and the remaining-point percentages printed in the paper.
"""
import json
import math
import os
from decimal import Decimal, getcontext
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rng(seed):
    return np.random.default_rng(seed)


# ----------------------------------------------------------------------------
# constants: correctly rounded closed forms (section 2, Step 1 rotations)

def test_constants_are_correctly_rounded_closed_forms():
    getcontext().prec = 60
    s3 = Decimal(3).sqrt() / 2
    s6, s2 = Decimal(6).sqrt(), Decimal(2).sqrt()
    want = {"s3": s3, "c75": (s6 - s2) / 4, "s75": (s6 + s2) / 4, "h": s2 / 2}
    got = oracle.constants()
    for k, v in want.items():
        assert got[k] == float(v), k  # float(Decimal) rounds to nearest
    # the libm route differs by one ulp and must not be what the oracle uses
    assert math.cos(math.radians(30)) != got["s3"]


# ----------------------------------------------------------------------------
# O1, Step 1: extremes

def polygon24(radius=1 << 23):
    """Vertices of a regular 24-gon (angles k*15 degrees), rounded to integers."""
    pts = []
    for k in range(24):
        a = math.radians(15 * k)
        pts.append((round(radius * math.cos(a)), round(radius * math.sin(a))))
    return np.array(pts, dtype=np.float32)


def support_vertex(angle_deg):
    """Index k of the 24-gon vertex at angle_deg (a multiple of 15)."""
    assert angle_deg % 15 == 0
    return (angle_deg // 15) % 24


@pytest.mark.parametrize("angles,thetas", [(oracle.ANGLES_CUMULATIVE, [0, 30, 75, 120]),
                                           (oracle.ANGLES_ABSOLUTE, [0, 30, 45, 60])])
def test_extremes_known_by_construction(angles, thetas):
    # Rotating the set counter-clockwise by theta makes the argmax of x' the
    # support point in direction -theta, argmax y' the one at 90 - theta, and
    # so on; every such direction is a vertex of the 24-gon, whose neighbours
    # are ~2.8e5 units behind it, far beyond any rounding.
    poly = polygon24()
    r = rng(1)
    interior = r.integers(-(1 << 21), 1 << 21, size=(500, 2)).astype(np.float32)
    xy = np.concatenate([interior, poly])
    off = interior.shape[0]
    ext = oracle.extremes(xy, angles)
    for g, th in enumerate(thetas):
        want = [180 - th, -th, 270 - th, 90 - th]  # argmin x', argmax x', argmin y', argmax y'
        for k in range(4):
            assert ext[4 * g + k] == off + support_vertex(want[k] % 360), (g, k)


def test_extremes_ties_take_lowest_index():
    poly = polygon24()
    xy = np.concatenate([poly, poly, poly])  # three copies
    for angles in (0, 1):
        ext = oracle.extremes(xy, angles)
        assert np.all(ext < 24)


def test_group0_matches_numpy_first_occurrence():
    r = rng(2)
    xy = r.integers(-50, 50, size=(5000, 2)).astype(np.float32)  # many ties
    ext = oracle.extremes(xy)
    assert ext[0] == np.argmin(xy[:, 0]) and ext[1] == np.argmax(xy[:, 0])
    assert ext[2] == np.argmin(xy[:, 1]) and ext[3] == np.argmax(xy[:, 1])


def test_group120_equals_group30_mapping():
    # With c, s the correctly rounded closed forms, x'(120) = -y'(30) and
    # y'(120) = x'(30) exactly, so argmax x'120 = argmin y'30, etc.  The
    # oracle computes both groups independently.
    for seed in range(5):
        r = rng(10 + seed)
        xy = r.integers(-(1 << 24), (1 << 24) + 1, size=(20000, 2)).astype(np.float32)
        e = oracle.extremes(xy)
        g30, g120 = e[4:8], e[12:16]
        assert g120[1] == g30[2]  # argmax x'120 == argmin y'30
        assert g120[0] == g30[3]  # argmin x'120 == argmax y'30
        assert g120[2] == g30[0]  # argmin y'120 == argmin x'30
        assert g120[3] == g30[1]  # argmax y'120 == argmax x'30


def _rn(fr: Fraction) -> float:
    return float(fr)  # Fraction -> float rounds to nearest even


def test_rotation_is_two_rounded_products_and_one_rounded_sum():
    # Exact rational arithmetic with explicit rounding steps, against the
    # oracle's double evaluation; includes points where a fused multiply-add
    # would round differently.
    c = oracle.constants()
    table = {1: (c["s3"], 0.5), 2: (c["c75"], c["s75"]), 3: (-0.5, c["s3"])}
    r = rng(3)
    pts = r.integers(-(1 << 24), (1 << 24) + 1, size=(3000, 2))
    diffs_vs_fma = 0
    for x, y in pts:
        for g, (cc, ss) in table.items():
            fx, fy, fc, fs = Fraction(int(x)), Fraction(int(y)), Fraction(cc), Fraction(ss)
            want_x = _rn(Fraction(_rn(fx * fc)) - Fraction(_rn(fy * fs)))
            want_y = _rn(Fraction(_rn(fx * fs)) + Fraction(_rn(fy * fc)))
            got = oracle.rotate(float(x), float(y), g)
            assert got == (want_x, want_y)
            fused = _rn(fx * fc - Fraction(_rn(fy * fs)))
            diffs_vs_fma += fused != want_x
    assert diffs_vs_fma > 0  # the sample does exercise the difference


# ----------------------------------------------------------------------------
# O2 / O4 / O5: hulls

def load_cases():
    with open(os.path.join(GOLDEN, "hand_worked.json")) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", load_cases(), ids=lambda c: c["name"])
def test_hand_worked_cases(case):
    xy = np.array(case["xy"], dtype=np.float32)
    res = oracle.cudapre(xy)
    assert res["poly_xy"].tolist() == case["polygon_xy"]
    assert res["survivors"].tolist() == case["survivors"]
    assert res["hull"].tolist() == case["hull"]
    assert oracle.hull(xy).tolist() == case["hull"]
    assert oracle.brute_hull(xy).tolist() == case["hull"]


def random_tiny_sets():
    r = rng(4)
    for t in range(400):
        n = int(r.integers(0, 40))
        span = int(r.choice([2, 3, 5, 50, 1 << 24]))
        xy = r.integers(-span, span + 1, size=(n, 2)).astype(np.float32)
        if t % 7 == 0 and n > 3:  # collinear points on a lattice line
            k = r.integers(-5, 6, size=n)
            xy = np.stack([k * 3, k * -2], axis=1).astype(np.float32)
        if t % 11 == 0 and n > 2:  # duplicated points
            xy[n // 2:] = xy[: n - n // 2]
        yield xy


def test_andrew_hull_equals_brute_force_hull():
    for xy in random_tiny_sets():
        assert oracle.hull(xy).tolist() == oracle.brute_hull(xy).tolist()


def test_hull_matches_qhull_vertex_set():
    # scipy.spatial.ConvexHull is Qhull, the library the paper used
    # (section 3).  Random points in a large range are in general position.
    from scipy.spatial import ConvexHull
    r = rng(5)
    for n in (10, 100, 3000):
        for shape in ("square", "disk"):
            xy = r.integers(-(1 << 24), (1 << 24) + 1, size=(n, 2)).astype(np.float32)
            if shape == "disk":
                xy = xy[(xy.astype(np.float64) ** 2).sum(1) <= float(1 << 48)]
            qh = ConvexHull(xy.astype(np.float64))
            ours = oracle.hull(xy)
            assert set(ours.tolist()) == set(qh.vertices.tolist())
            # both counter-clockwise: same cyclic order
            q = qh.vertices.tolist()
            k = q.index(int(ours[0]))
            assert q[k:] + q[:k] == ours.tolist()


def _orient(a, b, p):
    return (int(b[0]) - int(a[0])) * (int(p[1]) - int(a[1])) - (int(b[1]) - int(a[1])) * (int(p[0]) - int(a[0]))


def test_hull_invariants_strictly_convex_ccw_and_contains_all():
    r = rng(6)
    for xy in [synth.disk(20000, 7), synth.square(20000, 7, 1000), synth.gaussian(20000, 7, 1e5, 1 << 24)]:
        h = oracle.hull(xy)
        P = xy[h].astype(np.int64)
        m = len(h)
        assert m >= 3
        for k in range(m):
            assert _orient(P[k], P[(k + 1) % m], P[(k + 2) % m]) > 0  # strictly convex, CCW
        assert tuple(P[0]) == min(map(tuple, P))  # starts at the lexicographic minimum
        sample = xy[r.integers(0, xy.shape[0], size=2000)]
        for p in sample:
            for k in range(m):
                assert _orient(P[k], P[(k + 1) % m], p) >= 0


# ----------------------------------------------------------------------------
# O3, Step 3: strict-inside discard

def on_segment(a, b, p):
    if _orient(a, b, p) != 0:
        return False
    return (min(a[0], b[0]) <= p[0] <= max(a[0], b[0])) and (min(a[1], b[1]) <= p[1] <= max(a[1], b[1]))


def inside_by_crossing_number(poly, p):
    """Independent test (ray casting): p is strictly inside a simple polygon iff
    it is on no edge and a ray from p to +x crosses the boundary an odd number
    of times (half-open rule on vertex heights, exact rational comparison)."""
    m = len(poly)
    if m < 3:
        return False
    px, py = Fraction(int(p[0])), Fraction(int(p[1]))
    crossings = 0
    for k in range(m):
        a = [int(v) for v in poly[k]]
        b = [int(v) for v in poly[(k + 1) % m]]
        if on_segment(a, b, p):
            return False
        if (a[1] > py) != (b[1] > py):
            x_at = Fraction(a[0]) + (py - a[1]) * Fraction(b[0] - a[0], b[1] - a[1])
            if x_at > px:
                crossings += 1
    return crossings % 2 == 1


def test_strict_inside_matches_ray_casting():
    for t in range(40):
        xy = synth.gaussian(1500, 100 + t, 50.0, 1 << 24) if t % 2 else synth.square(1500, 100 + t, 40)
        e = oracle.extremes(xy)
        _, poly = oracle.hull16(xy, e)
        surv = set(oracle.prefilter(xy, poly).tolist())
        for i in range(xy.shape[0]):
            assert (i not in surv) == inside_by_crossing_number(poly, xy[i]), (t, i)


def test_survivor_hull_equals_full_hull():
    # The method's correctness argument (section 2): points strictly inside a
    # polygon of input points are interior, so the hull is unchanged.
    for k, xy in enumerate([synth.square(200000, 11), synth.disk(200000, 11), synth.gaussian(200000, 11)]):
        res = oracle.cudapre(xy)
        assert res["hull"].tolist() == oracle.hull(xy).tolist(), k


def test_polygon_vertices_are_hull_vertices_or_on_hull():
    for xy in [synth.disk(50000, 12), synth.gaussian(50000, 12)]:
        e = oracle.extremes(xy)
        _, poly = oracle.hull16(xy, e)
        h = oracle.hull(xy)
        P = xy[h].astype(np.int64)
        m = len(h)
        for v in poly:
            assert all(_orient(P[k], P[(k + 1) % m], v) >= 0 for k in range(m))
            assert any(_orient(P[k], P[(k + 1) % m], v) == 0 for k in range(m))


def test_remaining_fraction_matches_paper_tables_absolute_angles():
    # Table 2 prints 3.39-3.46 % remaining for circles and Table 1 prints
    # 0.02-0.06 % for squares; Figure 1 and section 5 rotate by 30/45/60.
    with open(os.path.join(GOLDEN, "paper_tables.json")) as f:
        tab = json.load(f)
    n = 1_000_000
    circ = tab["circle_remaining_percent"]["remaining_percent"][0]
    sq = tab["square_remaining_percent"]["remaining_percent"][0]
    xy = synth.disk(n, 21)
    e = oracle.extremes(xy, oracle.ANGLES_ABSOLUTE)
    _, poly = oracle.hull16(xy, e)
    f_disk = 100.0 * len(oracle.prefilter(xy, poly)) / n
    assert abs(f_disk - circ) < 0.15, f_disk
    xy = synth.square(n, 21, 1 << 24)
    e = oracle.extremes(xy, oracle.ANGLES_ABSOLUTE)
    _, poly = oracle.hull16(xy, e)
    f_sq = 100.0 * len(oracle.prefilter(xy, poly)) / n
    assert f_sq <= 2 * sq, f_sq


def test_remaining_fraction_cumulative_angles_closed_form():
    # Cumulative angles 0/30/75/120 give support directions at
    # {0,15,60,90,105,150,...} degrees (12 distinct); the inscribed polygon of
    # a disk leaves 1 - sum(sin(gap))/(2 pi) of its area outside.
    dirs = sorted({(-t + 90 * k) % 360 for t in (0, 30, 75, 120) for k in range(4)})
    gaps = [(dirs[(i + 1) % len(dirs)] - dirs[i]) % 360 for i in range(len(dirs))]
    frac = 1 - sum(math.sin(math.radians(g)) for g in gaps) / (2 * math.pi)
    n = 1_000_000
    xy = synth.disk(n, 22)
    res = oracle.cudapre(xy)
    f = len(res["survivors"]) / n
    assert len(dirs) == 12
    assert abs(f - frac) < 0.003, (f, frac)
    assert len(res["poly_xy"]) == 12


def test_check_domain_accepts_exactly_the_stated_domain():
    # The domain (finite, integer-valued, |v| <= 2^24, -0.0 equal to 0) fixed
    # where the paper is silent on precision.  Each bad value, alone in an
    # otherwise valid set, in either coordinate, must be rejected; the
    # boundary values must pass.
    base = np.array([[1.0, 2.0], [-3.0, 4.0], [5.0, -6.0]], np.float32)
    good = [0.0, -0.0, 1.0, -1.0, 2.0 ** 24, -(2.0 ** 24), 2.0 ** 24 - 1, 12345678.0]
    bad = [np.nan, np.inf, -np.inf, 0.5, -0.5, 2.0 ** 24 + 2, -(2.0 ** 24 + 2), 2.0 ** 25, 1e30, 8388607.5,
           np.float32(1.5e-45)]
    assert oracle.check_domain(base)
    assert oracle.check_domain(np.zeros((0, 2), np.float32))
    for v in good:
        for c in (0, 1):
            xy = base.copy()
            xy[1, c] = v
            assert oracle.check_domain(xy), (v, c)
    for v in bad:
        for row in (0, 2):
            for c in (0, 1):
                xy = base.copy()
                xy[row, c] = v
                assert not oracle.check_domain(xy), (v, row, c)


@pytest.mark.parametrize("threads", [1, 2, 3, 8, 0])
def test_multithreaded_oracle_equals_single_thread(threads):
    # the all-cores CPU baseline runs oracle_cudapre_mt; it must give exactly
    # the single-thread oracle's extremes, polygon, survivors and hull,
    # including lowest-index ties that straddle the threads' ranges
    for kind, n, seed in ((1, 200_001, 3), (0, 65_536, 4), (2, 100_003, 5), (1, 5, 6), (0, 0, 7)):
        xy = synth.shape(kind, n, seed, 9)
        if n > 1000:
            xy[n // 2] = xy[n // 5]      # a duplicate of an early point late in the set
            xy[n - 1] = xy[0]
        for angles in (0, 1):
            want = oracle.cudapre(xy, angles)
            got, used = oracle.cudapre_mt(xy, angles, threads)
            assert used >= 1
            for k in ("extremes", "poly_xy", "survivors", "hull"):
                assert np.array_equal(got[k], want[k]), (kind, n, angles, k)
    sq = synth.square(40_000, 8, 50)   # heavy duplication: many ties across ranges
    for angles in (0, 1):
        got, _ = oracle.cudapre_mt(sq, angles, threads)
        want = oracle.cudapre(sq, angles)
        for k in ("extremes", "poly_xy", "survivors", "hull"):
            assert np.array_equal(got[k], want[k]), k
