"""The error bounds that make the FP32 filters exact (CPU, exact rational
arithmetic).

The extreme search orders points by float32 values: positive multiples k of
the rotated coordinates that one fused multiply-add computes from float32
constants.  For lattice points within +-2^24 each such value must lie within
3 (30, 45 and 60 degrees) or 6 (75 degrees) of k times the binary64
definition (the oracle's rotation); the bands that decide when binary64 is
consulted (16 and 32) are more than twice those bounds.

The inside test evaluates s = fma(A, px, fma(B, py, C)) with the float32
roundings A', B', C' of the exact edge coefficients and trusts the sign of
s when |s| > E, E the bound built with the polygon's edge records; its sign
must then equal that of the exact int64 orientation.

Every float32 operation is emulated exactly: the exact result rounded once
to nearest-even float32."""
import math
import random
from fractions import Fraction

import oracle


def rn32(q: Fraction) -> Fraction:
    """q rounded to the nearest float32 (ties to even); no overflow here."""
    if q == 0:
        return Fraction(0)
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    scale = Fraction(2) ** (e - 23)
    m = a / scale  # in [2^23, 2^24)
    mi = math.floor(m)
    rem = m - mi
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and mi % 2 == 1):
        mi += 1
    return sign * mi * scale


def f32(x: float) -> Fraction:
    return rn32(Fraction(x))


C = oracle.constants()
S3, C75, H = Fraction(C["s3"]), Fraction(C["c75"]), Fraction(C["h"])
F_2S3 = f32(2 * C["s3"])
# tan 75 = 2 + sqrt(3), rounded to float32 from a 60-digit value
T75 = rn32(Fraction(2) + Fraction(int(math.isqrt(3 * 10 ** 120)), 10 ** 60))


def fma32(a: Fraction, b: Fraction, c: Fraction) -> Fraction:
    return rn32(a * b + c)


def cases(count, seed):
    rng = random.Random(seed)
    lim = 1 << 24
    pts = [(lim, lim), (-lim, -lim), (lim, -lim), (-lim, lim), (lim - 1, 1 - lim), (0, lim), (lim, 0),
           (1 << 23, (1 << 23) + 1), (-(1 << 22) - 3, (1 << 24) - 5)]
    for _ in range(count):
        pts.append((rng.randint(-lim, lim), rng.randint(-lim, lim)))
    return pts


def test_projection_values_within_bound():
    worst = {}
    for x, y in cases(3000, 1):
        X, Y = Fraction(x), Fraction(y)
        v30 = [Fraction(v) for v in oracle.rotate(x, y, 1, 0)]
        v75 = [Fraction(v) for v in oracle.rotate(x, y, 2, 0)]
        v45 = [Fraction(v) for v in oracle.rotate(x, y, 2, 1)]
        v60 = [Fraction(v) for v in oracle.rotate(x, y, 3, 1)]
        checks = {
            "2x30": (fma32(X, F_2S3, -Y), 2 * v30[0], 3),
            "2y30": (fma32(Y, F_2S3, X), 2 * v30[1], 3),
            "x75": (fma32(Y, -T75, X), v75[0] / C75, 6),
            "y75": (fma32(X, T75, Y), v75[1] / C75, 6),
            "x45": (rn32(X - Y), v45[0] / H, 3),
            "y45": (rn32(X + Y), v45[1] / H, 3),
            "2x60": (fma32(-Y, F_2S3, X), 2 * v60[0], 3),
            "2y60": (fma32(X, F_2S3, Y), 2 * v60[1], 3),
        }
        for name, (v32, exact, bound) in checks.items():
            d = abs(v32 - exact)
            assert d <= bound, (name, x, y, float(d))
            worst[name] = max(worst.get(name, 0), d)
    # the bands (16, 32) are over twice the bounds
    assert 16 > 2 * 3 and 32 > 2 * 6
    assert all(float(w) > 0 for w in worst.values())  # the rounding is really exercised


def edge_bound(A, B, Cc):
    """The inside test's static bound for an edge, without its upward
    roundings (the library's is at least this large)."""
    u = Fraction(1, 1 << 24)
    k2 = 2 + Fraction(1, 1 << 22)
    A_, B_, C_ = rn32(Fraction(A)), rn32(Fraction(B)), rn32(Fraction(Cc))
    E = abs(A_) + k2 * abs(B_) + k2 * abs(C_) * u + abs(A) + abs(B) + abs(Cc) * u
    return 2 * E, A_, B_, C_


def test_edge_sign_decided_only_outside_the_bound():
    rng = random.Random(2)
    lim = 1 << 24
    decided = 0
    for _ in range(400):
        ax, ay = rng.randint(-lim, lim), rng.randint(-lim, lim)
        bx, by = rng.randint(-lim, lim), rng.randint(-lim, lim)
        if (ax, ay) == (bx, by):
            continue
        dx, dy = bx - ax, by - ay
        A, B, Cc = -dy, dx, dy * ax - dx * ay  # orient(a, b, p) = A px + B py + C
        E, A_, B_, C_ = edge_bound(A, B, Cc)
        norm = math.hypot(dx, dy)
        for _ in range(40):
            # points near the line (within about 40 units), some far away
            t = rng.random()
            off = rng.uniform(-40, 40) if rng.random() < 0.8 else rng.uniform(-1e6, 1e6)
            px = round(ax + t * dx - off * dy / norm)
            py = round(ay + t * dy + off * dx / norm)
            if abs(px) > lim or abs(py) > lim:
                continue
            s = fma32(A_, Fraction(px), fma32(B_, Fraction(py), C_))
            orient = A * px + B * py + Cc
            if s > E:
                assert orient > 0, (ax, ay, bx, by, px, py)
                decided += 1
            elif s < -E:
                assert orient < 0, (ax, ay, bx, by, px, py)
                decided += 1
    assert decided > 1000


def test_inner_box_compare_is_exact_for_lattice_points():
    # The inside test's quick discard by the inner box: dx = fl(x - c) in
    # float32 (x, c integers within +-2^24), then |dx| <= h with h an integer
    # at most 2^24 - 1.  Whenever the float32 compare passes, the exact
    # |x - c| <= h holds (a difference that rounds exceeds 2^24 > h), so no
    # point outside the box is discarded.  Random cases plus the edges of the
    # domain and of the rounding range.
    rnd = random.Random(1405)
    B = 1 << 24
    edge = [-B, -B + 1, -B + 2, -1, 0, 1, B - 2, B - 1, B]
    cases = [(x, c) for x in edge for c in edge]
    cases += [(rnd.randint(-B, B), rnd.randint(-B, B)) for _ in range(20000)]
    cases += [(c + d, c) for c in (-B, -B + 1, 0, B - 1) for d in range(-3, 4) if abs(c + d) <= B]
    hs = [0, 1, 2, 1000, (1 << 23) + 1, B - 3, B - 2, B - 1]
    for x, c in cases:
        dx = abs(rn32(Fraction(x) - Fraction(c)))  # one float32 subtraction
        for h in hs:
            if dx <= h:
                assert abs(x - c) <= h, (x, c, h)
