/* synth.c -- seeded synthetic point sets for tests and benchmarks.
 *
 * This module holds input generators only: it computes no extreme point, no
 * hull and no inside test.  Both the CPU oracle and the CUDA path consume the
 * arrays it writes.  Every value is a pure function of (seed, stream, index,
 * attempt) through the SplitMix64 finaliser (Steele, Lea and Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014), so the
 * output does not depend on the thread count.
 *
 * Output format: float32 xy interleaved, [n][2], integer-valued coordinates
 * with |v| <= 2^24 -- the domain in which orientation tests are exact in int64.
 * The 3D generators (cube3, ball3, gauss3) write float32 xyz interleaved,
 * [n][3], integer-valued with |v| <= 2^19, the domain of the 3D extension.
 *
 * Shapes follow the paper's data groups (section 3): uniform points in a
 * square and in a circle (the rbox data), plus Gaussian clusters standing in
 * for the projected mesh vertices of Table 3, which are not available.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

static uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Counter-based draw number k of point i in stream `stream`. */
static uint64_t draw(uint64_t seed, uint64_t stream, uint64_t i, uint64_t k) {
  uint64_t h = mix64(seed ^ mix64(stream + 0x5851F42D4C957F2Dull));
  h = mix64(h ^ i);
  return mix64(h ^ (k * 0xD6E8FEB86659FD93ull));
}

/* Uniform integer in [-r, r]. */
static int64_t uni_int(uint64_t u, int64_t r) {
  uint64_t span = (uint64_t)(2 * r + 1);
  return (int64_t)(u % span) - r;
}

/* Uniform double in (0, 1]. */
static double uni01(uint64_t u) { return ((double)(u >> 11) + 1.0) * 0x1p-53; }

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) {
  return v < lo ? lo : (v > hi ? hi : v);
}

uint64_t synth_mix64(uint64_t z) { return mix64(z); }
uint64_t synth_draw(uint64_t seed, uint64_t stream, uint64_t i, uint64_t k) {
  return draw(seed, stream, i, k);
}

/* Uniform integer points in the square [-r, r]^2. */
void synth_square(float* xy, int64_t n, uint64_t seed, uint64_t stream,
                  int64_t r) {
#pragma omp parallel for schedule(static) if (n > 65536)
  for (int64_t i = 0; i < n; ++i) {
    xy[2 * i] = (float)uni_int(draw(seed, stream, (uint64_t)i, 0), r);
    xy[2 * i + 1] = (float)uni_int(draw(seed, stream, (uint64_t)i, 1), r);
  }
}

/* Uniform integer points in the disk x^2 + y^2 <= r^2 (r <= 2^24): candidate
 * k of point i is uniform in the square; the first accepted one is kept. */
void synth_disk(float* xy, int64_t n, uint64_t seed, uint64_t stream,
                int64_t r) {
#pragma omp parallel for schedule(static) if (n > 65536)
  for (int64_t i = 0; i < n; ++i) {
    for (uint64_t k = 0;; ++k) {
      int64_t x = uni_int(draw(seed, stream, (uint64_t)i, 2 * k), r);
      int64_t y = uni_int(draw(seed, stream, (uint64_t)i, 2 * k + 1), r);
      if (x * x + y * y <= r * r) {
        xy[2 * i] = (float)x;
        xy[2 * i + 1] = (float)y;
        break;
      }
    }
  }
}

/* Integer-valued Gaussian points (Box-Muller), standard deviation sigma,
 * rounded to nearest and clipped to [-clip, clip] per coordinate. */
void synth_gaussian(float* xy, int64_t n, uint64_t seed, uint64_t stream,
                    double sigma, int64_t clip) {
  const double two_pi = 6.283185307179586;
#pragma omp parallel for schedule(static) if (n > 65536)
  for (int64_t i = 0; i < n; ++i) {
    double u1 = uni01(draw(seed, stream, (uint64_t)i, 0));
    double u2 = uni01(draw(seed, stream, (uint64_t)i, 1));
    double rad = sqrt(-2.0 * log(u1)) * sigma;
    double x = rad * cos(two_pi * u2);
    double y = rad * sin(two_pi * u2);
    xy[2 * i] = (float)clampi(llrint(x), -clip, clip);
    xy[2 * i + 1] = (float)clampi(llrint(y), -clip, clip);
  }
}

static int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b, r = a % b;
  if (r != 0 && ((r < 0) != (b < 0))) --q;
  return q;
}

static int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

static int64_t gcd64(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

/* Points on, or within one unit inside of, the edges of a given convex
 * counter-clockwise polygon poly[m][2] (integer vertices).  Point i picks an
 * edge a->b and a position t in [0.05, 0.95] along it.  Where the edge has
 * interior lattice points (gcd(|dx|, |dy|) > 1) every fourth point is put
 * exactly on the edge; otherwise the point sits on the major-axis lattice line
 * at parameter t and the other coordinate is rounded toward the polygon's
 * interior (the left of a->b), so its distance to the edge line is < 1 and it
 * is on the inner side or on the line.  Points of axis-parallel edges are put
 * one unit inside instead.  Used to force near-boundary inside tests.
 * m < 3 writes nothing and returns 0. */
int synth_near_edge(float* xy, int64_t n, uint64_t seed, uint64_t stream,
                    const int32_t* poly, int m) {
  if (m < 3) return 0;
#pragma omp parallel for schedule(static) if (n > 65536)
  for (int64_t i = 0; i < n; ++i) {
    uint64_t ue = draw(seed, stream, (uint64_t)i, 0);
    int e = (int)(ue % (uint64_t)m);
    int64_t ax = poly[2 * e], ay = poly[2 * e + 1];
    int64_t bx = poly[2 * ((e + 1) % m)], by = poly[2 * ((e + 1) % m) + 1];
    int64_t dx = bx - ax, dy = by - ay;
    double t = 0.05 + 0.9 * uni01(draw(seed, stream, (uint64_t)i, 1));
    int64_t g = gcd64(dx, dy);
    int64_t qx, qy;
    if (g > 1 && (draw(seed, stream, (uint64_t)i, 2) & 3) == 0) {
      int64_t k = 1 + (int64_t)(draw(seed, stream, (uint64_t)i, 3) %
                                (uint64_t)(g - 1));
      qx = ax + k * (dx / g);
      qy = ay + k * (dy / g);
    } else if ((dy < 0 ? -dy : dy) >= (dx < 0 ? -dx : dx)) {
      /* steep edge: integer y, x on the line rounded toward the interior;
       * the interior is +x when -dy > 0 */
      qy = ay + llrint(t * (double)dy);
      int64_t num = (qy - ay) * dx; /* x = ax + num / dy */
      qx = ax + (-dy > 0 ? ceil_div(num, dy) : floor_div(num, dy));
    } else {
      /* shallow edge: integer x, y on the line rounded toward the interior;
       * the interior is +y when dx > 0 */
      qx = ax + llrint(t * (double)dx);
      int64_t num = (qx - ax) * dy; /* y = ay + num / dx */
      qy = ay + (dx > 0 ? ceil_div(num, dx) : floor_div(num, dx));
    }
    /* an axis-parallel edge lies on a line of axis extremes; keep its points
     * one unit inside so that they never tie with those extremes */
    if (dx == 0) qx += (-dy > 0) ? 1 : -1;
    if (dy == 0) qy += (dx > 0) ? 1 : -1;
    xy[2 * i] = (float)qx;
    xy[2 * i + 1] = (float)qy;
  }
  return 1;
}

/* Scatter src[n][2] through the affine permutation i -> (a*i + b) mod n with
 * a odd-and-coprime-to-n chosen from the seed (an invertible shuffle that is
 * cheap for 2^28 points). */
void synth_permute(const float* src, float* dst, int64_t n, uint64_t seed) {
  if (n <= 0) return;
  uint64_t a = (mix64(seed ^ 0xA5A5A5A5ull) % (uint64_t)n) | 1u;
  while (gcd64((int64_t)a, n) != 1) a += 2;
  uint64_t b = mix64(seed ^ 0x3C3C3C3Cull) % (uint64_t)n;
#pragma omp parallel for schedule(static) if (n > 65536)
  for (int64_t i = 0; i < n; ++i) {
    uint64_t j = (uint64_t)(((__uint128_t)a * (uint64_t)i + b) % (uint64_t)n);
    dst[2 * j] = src[2 * i];
    dst[2 * j + 1] = src[2 * i + 1];
  }
}

/* Set sizes floor(exp(U(ln lo, ln hi))) and a shape id in {0 square,
 * 1 disk, 2 gaussian} for each of s sets. */
void synth_set_plan(int64_t s, uint64_t seed, double lo, double hi,
                    int64_t* sizes, int32_t* shapes) {
  for (int64_t k = 0; k < s; ++k) {
    double u = uni01(draw(seed, 0x5E75, (uint64_t)k, 0));
    double v = exp(log(lo) + u * (log(hi) - log(lo)));
    int64_t sz = (int64_t)floor(v);
    if (sz < (int64_t)lo) sz = (int64_t)lo;
    if (sz > (int64_t)hi) sz = (int64_t)hi;
    sizes[k] = sz;
    shapes[k] = (int32_t)(draw(seed, 0x5E75, (uint64_t)k, 1) % 3u);
  }
}

/* ---- 3D point sets (float32 xyz interleaved, [n][3]) ------------------- */

/* Uniform integer points in the cube [-r, r]^3. */
void synth_cube3(float* xyz, int64_t n, uint64_t seed, uint64_t stream, int64_t r) {
#pragma omp parallel for schedule(static) if (n > 65536)
  for (int64_t i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) xyz[3 * i + c] = (float)uni_int(draw(seed, stream, (uint64_t)i, (uint64_t)c), r);
}

/* Uniform integer points in the ball x^2 + y^2 + z^2 <= r^2 (indexed
 * rejection from the cube, as synth_disk). */
void synth_ball3(float* xyz, int64_t n, uint64_t seed, uint64_t stream, int64_t r) {
#pragma omp parallel for schedule(static) if (n > 65536)
  for (int64_t i = 0; i < n; ++i) {
    for (uint64_t k = 0;; ++k) {
      int64_t x = uni_int(draw(seed, stream, (uint64_t)i, 3 * k), r);
      int64_t y = uni_int(draw(seed, stream, (uint64_t)i, 3 * k + 1), r);
      int64_t z = uni_int(draw(seed, stream, (uint64_t)i, 3 * k + 2), r);
      if (x * x + y * y + z * z <= r * r) {
        xyz[3 * i] = (float)x;
        xyz[3 * i + 1] = (float)y;
        xyz[3 * i + 2] = (float)z;
        break;
      }
    }
  }
}

/* Integer-valued Gaussian points (Box-Muller per coordinate pair), standard
 * deviation sigma, rounded to nearest and clipped to [-clip, clip]. */
void synth_gauss3(float* xyz, int64_t n, uint64_t seed, uint64_t stream, double sigma, int64_t clip) {
  const double two_pi = 6.283185307179586;
#pragma omp parallel for schedule(static) if (n > 65536)
  for (int64_t i = 0; i < n; ++i) {
    double u1 = uni01(draw(seed, stream, (uint64_t)i, 0));
    double u2 = uni01(draw(seed, stream, (uint64_t)i, 1));
    double u3 = uni01(draw(seed, stream, (uint64_t)i, 2));
    double u4 = uni01(draw(seed, stream, (uint64_t)i, 3));
    double r1 = sqrt(-2.0 * log(u1)) * sigma, r2 = sqrt(-2.0 * log(u3)) * sigma;
    xyz[3 * i] = (float)clampi(llrint(r1 * cos(two_pi * u2)), -clip, clip);
    xyz[3 * i + 1] = (float)clampi(llrint(r1 * sin(two_pi * u2)), -clip, clip);
    xyz[3 * i + 2] = (float)clampi(llrint(r2 * cos(two_pi * u4)), -clip, clip);
  }
}
