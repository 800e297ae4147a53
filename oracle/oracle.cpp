// oracle.cpp -- plain, slow, obviously-correct CPU oracle for the CudaPre
// convex-hull preprocessing method (Mei, arXiv 1405.3454).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file: only the test suite, the smoke check and the CPU-baseline
// leg of the benchmark use it.  It shares no code, header, constant table or
// helper with the CUDA implementation.
//
// Build: g++ -std=c++17 -O2 -ffp-contract=off -shared -fPIC (no FMA
// contraction, so every double operation below is one IEEE round-to-nearest
// operation, exactly as written).
//
// What it computes (paper section 2, "The procedure of our algorithm"):
//   O1 oracle_extremes  -- Step 1: min/max of x and y of the original set and
//                          of three rotated copies (16 extreme points).
//   O2 oracle_hull16    -- Step 2: Andrew's monotone chain over those points
//                          (the correction note: reference [6] is Andrew's).
//   O3 oracle_prefilter -- Step 3: discard every point strictly inside the
//                          polygon; the others remain (section 3, case (2)).
//   O4 oracle_hull      -- the final hull of a point subset, again by Andrew's
//                          monotone chain; applied to all points it is the
//                          plain definition of the convex hull.
//   O5 oracle_brute_hull-- O(n^3) definition of the hull for tiny inputs.
//   oracle_cudapre_mt   -- the same steps split over host threads, for the
//                          all-cores CPU baseline (tested equal to the
//                          single-thread oracle).
//   oracle3_*           -- the 3D extension sketched in section 5: extremes
//                          of the set and of copies rotated about one axis,
//                          their convex polyhedron, the strict-inside discard.
//
// Conventions where the paper is silent (each is a stated reading):
//   * Rotation is counter-clockwise: x' = x c - y s, y' = x s + y c, each
//     rotated set derived from the ORIGINAL coordinates.
//   * Angle table "cumulative": 0, 30, 75 (=30+45), 120 (=30+45+45) degrees,
//     the reading of "rotate in 30, 45, and 45 degrees" (section 2, Step 1).
//     Angle table "absolute": 0, 30, 45, 60 degrees (Figure 1, section 5).
//   * c and s are the correctly rounded doubles of the closed forms
//     (sqrt(3)/2, (sqrt(6)-sqrt(2))/4, ...), never cos(radians(t)).
//   * Projections are evaluated in double as RN(RN(x*c) - RN(y*s)) and
//     RN(RN(x*s) + RN(y*c)), no fused multiply-add.
//   * Ties among equal projections go to the lowest point index.
//   * "Inside" means strictly inside: points on the polygon boundary remain.
//     A polygon with fewer than 3 vertices discards nothing.
//   * Hulls are strictly convex (collinear boundary points are not vertices),
//     counter-clockwise, starting at the lexicographically smallest (x, y)
//     vertex; among points with equal coordinates the lowest index is used.
//   * Coordinates are finite integer-valued floats with |v| <= 2^24, so every
//     orientation determinant is exact in int64.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// Correctly rounded closed forms (hex double literals).
//   S3  = sqrt(3)/2        C75 = (sqrt(6)-sqrt(2))/4
//   S75 = (sqrt(6)+sqrt(2))/4   H = sqrt(2)/2
const double S3 = 0x1.bb67ae8584caap-1;
const double C75 = 0x1.0907dc1930690p-2;
const double S75 = 0x1.ee8dd4748bf15p-1;
const double H = 0x1.6a09e667f3bcdp-1;

struct Rot {
  double c, s;
};

// Angle tables (section 2 / Step 1 and Figure 1): group 0 is the original set.
void angle_table(int angles, Rot out[4]) {
  out[0] = {1.0, 0.0};  // 0 degrees
  out[1] = {S3, 0.5};   // 30 degrees
  if (angles == 0) {
    out[2] = {C75, S75};  // 75 degrees = 30 + 45
    out[3] = {-0.5, S3};  // 120 degrees = 30 + 45 + 45
  } else {
    out[2] = {H, H};    // 45 degrees
    out[3] = {0.5, S3}; // 60 degrees
  }
}

// Rotated x coordinate: RN(RN(x*c) - RN(y*s)).
double rot_x(double x, double y, Rot r) {
  double a = x * r.c;
  double b = y * r.s;
  return a - b;
}

// Rotated y coordinate: RN(RN(x*s) + RN(y*c)).
double rot_y(double x, double y, Rot r) {
  double a = x * r.s;
  double b = y * r.c;
  return a + b;
}

int64_t to_i(float v) { return (int64_t)v; }

// Orientation determinant of (a, b, p): > 0 when p is to the left of a->b.
int64_t orient(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t px,
               int64_t py) {
  return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

struct Pt {
  int64_t x, y, idx;
};

bool lex_less(const Pt& a, const Pt& b) {
  if (a.x != b.x) return a.x < b.x;
  if (a.y != b.y) return a.y < b.y;
  return a.idx < b.idx;
}

// Andrew's monotone chain over points sorted by (x, y, idx) with equal
// coordinates already collapsed to their lowest index.  Pops while the turn is
// not strictly left, so the hull is strictly convex.  Returns the vertices
// counter-clockwise from the lexicographically smallest point.
std::vector<Pt> andrew(const std::vector<Pt>& p) {
  size_t k = p.size();
  if (k <= 1) return p;
  std::vector<Pt> lower, upper;
  for (size_t i = 0; i < k; ++i) {
    while (lower.size() >= 2 &&
           orient(lower[lower.size() - 2].x, lower[lower.size() - 2].y,
                  lower.back().x, lower.back().y, p[i].x, p[i].y) <= 0)
      lower.pop_back();
    lower.push_back(p[i]);
  }
  for (size_t j = k; j-- > 0;) {
    while (upper.size() >= 2 &&
           orient(upper[upper.size() - 2].x, upper[upper.size() - 2].y,
                  upper.back().x, upper.back().y, p[j].x, p[j].y) <= 0)
      upper.pop_back();
    upper.push_back(p[j]);
  }
  std::vector<Pt> hull(lower.begin(), lower.end() - 1);
  hull.insert(hull.end(), upper.begin(), upper.end() - 1);
  return hull;
}

// Sort by (x, y, idx) and keep the first (lowest index) of each run of equal
// coordinates.
std::vector<Pt> sorted_unique(std::vector<Pt> p) {
  std::sort(p.begin(), p.end(), lex_less);
  std::vector<Pt> u;
  for (const Pt& q : p)
    if (u.empty() || u.back().x != q.x || u.back().y != q.y) u.push_back(q);
  return u;
}

}  // namespace

extern "C" {

int oracle_abi_version(void) { return 1; }

// The projection constants, for the test that checks them against the closed
// forms: out = {S3, C75, S75, H}.
void oracle_constants(double* out) {
  out[0] = S3;
  out[1] = C75;
  out[2] = S75;
  out[3] = H;
}

// Rotated coordinates of one point, for tests: out = {x', y'} of group g.
void oracle_rotate(float x, float y, int angles, int g, double* out) {
  Rot t[4];
  angle_table(angles, t);
  out[0] = rot_x((double)x, (double)y, t[g]);
  out[1] = rot_y((double)x, (double)y, t[g]);
}

// Returns 1 when every coordinate is finite, integer-valued and |v| <= 2^24.
int oracle_check_domain(const float* xy, int64_t n) {
  for (int64_t i = 0; i < 2 * n; ++i) {
    float v = xy[i];
    if (!std::isfinite(v)) return 0;
    if (std::fabs(v) > 16777216.0f) return 0;
    if (std::floor(v) != v) return 0;
  }
  return 1;
}

// O1 -- Step 1 (section 2): the 16 extreme points.  For group g (angle table
// entry g) the output slots are [4g+0] argmin x', [4g+1] argmax x',
// [4g+2] argmin y', [4g+3] argmax y'.  Every group is computed independently
// from the original coordinates.  Lowest index wins ties (strict comparisons
// while scanning in increasing index).  n == 0 writes -1 everywhere.
void oracle_extremes(const float* xy, int64_t n, int angles, int64_t* out_idx) {
  Rot t[4];
  angle_table(angles, t);
  for (int g = 0; g < 4; ++g) {
    int64_t imin_x = -1, imax_x = -1, imin_y = -1, imax_y = -1;
    double min_x = 0, max_x = 0, min_y = 0, max_y = 0;
    for (int64_t i = 0; i < n; ++i) {
      double x = (double)xy[2 * i];
      double y = (double)xy[2 * i + 1];
      double px = rot_x(x, y, t[g]);
      double py = rot_y(x, y, t[g]);
      if (imin_x < 0 || px < min_x) { min_x = px; imin_x = i; }
      if (imax_x < 0 || px > max_x) { max_x = px; imax_x = i; }
      if (imin_y < 0 || py < min_y) { min_y = py; imin_y = i; }
      if (imax_y < 0 || py > max_y) { max_y = py; imax_y = i; }
    }
    out_idx[4 * g + 0] = imin_x;
    out_idx[4 * g + 1] = imax_x;
    out_idx[4 * g + 2] = imin_y;
    out_idx[4 * g + 3] = imax_y;
  }
}

// O2 -- Step 2 (section 2): the convex polygon of the (up to 16) extreme
// points by Andrew's monotone chain.  Duplicate indices and equal coordinates
// collapse to the lowest index.  Writes m <= 16 vertices counter-clockwise
// from the lexicographically smallest: poly_idx[m] point indices and
// poly_xy[2m] integer coordinates.  Returns m (0 when n == 0).
int oracle_hull16(const float* xy, const int64_t* ext_idx, int64_t* poly_idx,
                  int32_t* poly_xy) {
  std::vector<Pt> pts;
  for (int k = 0; k < 16; ++k) {
    int64_t i = ext_idx[k];
    if (i < 0) continue;
    pts.push_back({to_i(xy[2 * i]), to_i(xy[2 * i + 1]), i});
  }
  std::vector<Pt> hull = andrew(sorted_unique(pts));
  for (size_t k = 0; k < hull.size(); ++k) {
    poly_idx[k] = hull[k].idx;
    poly_xy[2 * k] = (int32_t)hull[k].x;
    poly_xy[2 * k + 1] = (int32_t)hull[k].y;
  }
  return (int)hull.size();
}

// Strict inside test of one integer point against the CCW polygon: every edge
// must see the point strictly to its left.  Fewer than 3 vertices: never.
int oracle_strictly_inside(const int32_t* poly_xy, int m, int64_t px,
                           int64_t py) {
  if (m < 3) return 0;
  for (int k = 0; k < m; ++k) {
    int j = (k + 1) % m;
    if (orient(poly_xy[2 * k], poly_xy[2 * k + 1], poly_xy[2 * j],
               poly_xy[2 * j + 1], px, py) <= 0)
      return 0;
  }
  return 1;
}

// O3 -- Step 3 (section 2): discard the points strictly inside the polygon.
// Writes the indices of the remaining points in ascending order and returns
// their count.
int64_t oracle_prefilter(const float* xy, int64_t n, const int32_t* poly_xy,
                         int m, int64_t* surv_idx) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!oracle_strictly_inside(poly_xy, m, to_i(xy[2 * i]),
                                to_i(xy[2 * i + 1])))
      surv_idx[c++] = i;
  }
  return c;
}

// O4 -- convex hull of the points idx[0..k) (k == n and idx == NULL means
// all points) by Andrew's monotone chain.  Writes hull point indices
// counter-clockwise from the lexicographically smallest vertex, lowest index
// among equal coordinates; returns the vertex count.
int64_t oracle_hull(const float* xy, const int64_t* idx, int64_t k,
                    int64_t* hull_idx) {
  std::vector<Pt> pts;
  pts.reserve((size_t)k);
  for (int64_t j = 0; j < k; ++j) {
    int64_t i = idx ? idx[j] : j;
    pts.push_back({to_i(xy[2 * i]), to_i(xy[2 * i + 1]), i});
  }
  std::vector<Pt> hull = andrew(sorted_unique(std::move(pts)));
  for (size_t j = 0; j < hull.size(); ++j) hull_idx[j] = hull[j].idx;
  return (int64_t)hull.size();
}

// O5 -- brute-force hull for tiny inputs (n <= 256), straight from the
// definition: after collapsing equal coordinates to the lowest index, the
// directed pair (i, j) is a hull edge when every other point k has
// orient(i, j, k) >= 0 and every point with orient 0 lies on the closed
// segment [i, j].  The vertices are the tails of those edges, walked from the
// lexicographically smallest vertex.  Returns -1 if n is too large.
int64_t oracle_brute_hull(const float* xy, int64_t n, int64_t* hull_idx) {
  if (n > 256) return -1;
  std::vector<Pt> raw;
  for (int64_t i = 0; i < n; ++i)
    raw.push_back({to_i(xy[2 * i]), to_i(xy[2 * i + 1]), i});
  std::vector<Pt> p = sorted_unique(raw);
  size_t u = p.size();
  if (u <= 2) {
    for (size_t j = 0; j < u; ++j) hull_idx[j] = p[j].idx;
    return (int64_t)u;
  }
  std::vector<int> next(u, -1);
  for (size_t i = 0; i < u; ++i) {
    for (size_t j = 0; j < u; ++j) {
      if (i == j) continue;
      bool edge = true;
      for (size_t k = 0; k < u && edge; ++k) {
        if (k == i || k == j) continue;
        int64_t o = orient(p[i].x, p[i].y, p[j].x, p[j].y, p[k].x, p[k].y);
        if (o < 0) edge = false;
        if (o == 0) {
          // must lie on the closed segment [i, j]
          int64_t lox = std::min(p[i].x, p[j].x), hix = std::max(p[i].x, p[j].x);
          int64_t loy = std::min(p[i].y, p[j].y), hiy = std::max(p[i].y, p[j].y);
          if (p[k].x < lox || p[k].x > hix || p[k].y < loy || p[k].y > hiy)
            edge = false;
        }
      }
      if (edge) next[i] = (int)j;
    }
  }
  // all points collinear: both directions qualify for the extreme pair
  int64_t c = 0;
  int start = 0;  // p is sorted, so p[0] is the lexicographically smallest
  if (next[start] < 0) {
    hull_idx[0] = p[0].idx;
    return 1;
  }
  int cur = start;
  do {
    hull_idx[c++] = p[cur].idx;
    cur = next[cur];
    if (c > (int64_t)u) return -2;  // not a simple cycle: malformed input
  } while (cur != start && cur >= 0);
  return c;
}

// The whole method on one point set, in the paper's order (section 2 Steps
// 1-3, then section 3 case (2): the hull of the remaining points).
// Outputs: ext_idx[16]; m and poly_xy[32]; survivors (ascending) and their
// count; hull indices and their count.  surv_idx and hull_idx need room for n.
void oracle_cudapre(const float* xy, int64_t n, int angles, int64_t* ext_idx,
                    int32_t* m_out, int32_t* poly_xy, int64_t* surv_idx,
                    int64_t* n_surv, int64_t* hull_idx, int64_t* n_hull) {
  oracle_extremes(xy, n, angles, ext_idx);
  int64_t poly_idx[16];
  int m = n > 0 ? oracle_hull16(xy, ext_idx, poly_idx, poly_xy) : 0;
  *m_out = m;
  int64_t s = oracle_prefilter(xy, n, poly_xy, m, surv_idx);
  *n_surv = s;
  *n_hull = oracle_hull(xy, surv_idx, s, hull_idx);
}

// The whole method as oracle_cudapre, with the point loops split over
// `threads` host threads (0: all hardware threads), for the all-cores CPU
// baseline.  Step 1: each thread scans a contiguous range in increasing index
// with the same strict comparisons, and the ranges' winners are combined in
// range order keeping the earlier on equal values, so ties still go to the
// lowest index.  Step 3: each range's survivors, concatenated in range order
// (ascending).  The hull of the survivors: Andrew's chain per range, then
// once more over the union of the range hulls (every vertex of the whole
// hull is a vertex of the hull of its range, and equal coordinates keep the
// lowest index at both levels).  Returns the thread count used.
int oracle_cudapre_mt(const float* xy, int64_t n, int angles, int threads,
                      int64_t* ext_idx, int32_t* m_out, int32_t* poly_xy,
                      int64_t* surv_idx, int64_t* n_surv, int64_t* hull_idx,
                      int64_t* n_hull) {
  int T = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  if (T < 1) T = 1;
  if ((int64_t)T > n / 4096 + 1) T = (int)(n / 4096 + 1);
  std::vector<int64_t> lo(T + 1);
  for (int t = 0; t <= T; ++t) lo[t] = n * t / T;
  auto run = [&](auto&& fn) {
    std::vector<std::thread> th;
    for (int t = 0; t < T; ++t) th.emplace_back(fn, t);
    for (auto& x : th) x.join();
  };
  // Step 1
  Rot tab[4];
  angle_table(angles, tab);
  std::vector<int64_t> part_idx((size_t)T * 16, -1);
  std::vector<double> part_val((size_t)T * 16, 0.0);
  run([&](int t) {
    for (int g = 0; g < 4; ++g) {
      int64_t* pi = &part_idx[(size_t)t * 16 + 4 * g];
      double* pv = &part_val[(size_t)t * 16 + 4 * g];
      for (int64_t i = lo[t]; i < lo[t + 1]; ++i) {
        double x = (double)xy[2 * i];
        double y = (double)xy[2 * i + 1];
        double px = rot_x(x, y, tab[g]);
        double py = rot_y(x, y, tab[g]);
        if (pi[0] < 0 || px < pv[0]) { pv[0] = px; pi[0] = i; }
        if (pi[1] < 0 || px > pv[1]) { pv[1] = px; pi[1] = i; }
        if (pi[2] < 0 || py < pv[2]) { pv[2] = py; pi[2] = i; }
        if (pi[3] < 0 || py > pv[3]) { pv[3] = py; pi[3] = i; }
      }
    }
  });
  for (int k = 0; k < 16; ++k) {
    int64_t bi = -1;
    double bv = 0.0;
    for (int t = 0; t < T; ++t) {
      int64_t i = part_idx[(size_t)t * 16 + k];
      double v = part_val[(size_t)t * 16 + k];
      if (i < 0) continue;
      bool better = (k & 1) ? v > bv : v < bv;  // odd slots are maxima
      if (bi < 0 || better) { bi = i; bv = v; }
    }
    ext_idx[k] = bi;
  }
  // Step 2
  int64_t poly_idx[16];
  int m = n > 0 ? oracle_hull16(xy, ext_idx, poly_idx, poly_xy) : 0;
  *m_out = m;
  // Step 3
  std::vector<std::vector<int64_t>> surv(T);
  run([&](int t) {
    for (int64_t i = lo[t]; i < lo[t + 1]; ++i)
      if (!oracle_strictly_inside(poly_xy, m, to_i(xy[2 * i]), to_i(xy[2 * i + 1])))
        surv[t].push_back(i);
  });
  int64_t c = 0;
  for (int t = 0; t < T; ++t)
    for (int64_t i : surv[t]) surv_idx[c++] = i;
  *n_surv = c;
  // hull of the survivors: per range, then over the union of range hulls
  std::vector<std::vector<Pt>> part(T);
  run([&](int t) {
    std::vector<Pt> pts;
    pts.reserve(surv[t].size());
    for (int64_t i : surv[t]) pts.push_back({to_i(xy[2 * i]), to_i(xy[2 * i + 1]), i});
    part[t] = andrew(sorted_unique(std::move(pts)));
  });
  std::vector<Pt> all;
  for (int t = 0; t < T; ++t) all.insert(all.end(), part[t].begin(), part[t].end());
  std::vector<Pt> hull = andrew(sorted_unique(std::move(all)));
  for (size_t j = 0; j < hull.size(); ++j) hull_idx[j] = hull[j].idx;
  *n_hull = (int64_t)hull.size();
  return T;
}

// ---------------------------------------------------------------------------
// The 3D extension (section 5): six extremes (min/max of x, y, z) of the
// original set and of copies rotated about one axis, the convex polyhedron
// of those points, and the discard of the points strictly inside it.
// Readings where section 5 is silent:
//   * the rotation axis is z, with the angle table of 2D (cumulative 0, 30,
//     75, 120 degrees or absolute 0, 30, 45, 60): x' and y' exactly as in
//     2D, z' = z;
//   * slot 6g + k of group g: k = 0 argmin x', 1 argmax x', 2 argmin y',
//     3 argmax y', 4 argmin z', 5 argmax z'; ties go to the lowest index;
//   * points are float32 xyz, integer-valued with |v| <= 2^19, so every
//     plane test below is exact in int64 (normal components below 2^42,
//     offsets and tests below 2^63);
//   * the polyhedron is given by its facet planes (N, d), N an outward
//     normal with N.p <= d for every extreme point, reduced so that the
//     gcd of |Nx|, |Ny|, |Nz|, |d| is 1; fewer than four affinely
//     independent extremes give no facets and discard nothing;
//   * "inside" is strictly inside: N.p < d for every facet.

// O1-3D -- the 24 extremes; every group and axis computed independently.
void oracle3_extremes(const float* xyz, int64_t n, int angles, int64_t* out_idx) {
  Rot t[4];
  angle_table(angles, t);
  for (int g = 0; g < 4; ++g) {
    int64_t best[6];
    double val[6] = {0, 0, 0, 0, 0, 0};
    for (int k = 0; k < 6; ++k) best[k] = -1;
    for (int64_t i = 0; i < n; ++i) {
      double x = (double)xyz[3 * i];
      double y = (double)xyz[3 * i + 1];
      double z = (double)xyz[3 * i + 2];
      double v[3] = {rot_x(x, y, t[g]), rot_y(x, y, t[g]), z};
      for (int a = 0; a < 3; ++a) {
        if (best[2 * a] < 0 || v[a] < val[2 * a]) { val[2 * a] = v[a]; best[2 * a] = i; }
        if (best[2 * a + 1] < 0 || v[a] > val[2 * a + 1]) { val[2 * a + 1] = v[a]; best[2 * a + 1] = i; }
      }
    }
    for (int k = 0; k < 6; ++k) out_idx[6 * g + k] = best[k];
  }
}

namespace {

struct P3 {
  int64_t x, y, z, idx;
};

int64_t gcd_abs(int64_t a, int64_t b) {
  if (a < 0) a = -a;
  if (b < 0) b = -b;
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

}  // namespace

// O2-3D -- the facet planes of the convex polyhedron of the extremes, by
// the definition: the plane through three distinct, non-collinear extremes
// is a facet plane when every extreme lies on one closed side of it.  Each
// plane is written once (reduced, outward), in lexicographic order, as
// planes[4k..4k+3] = Nx, Ny, Nz, d.  Returns the facet count (at most
// max_planes; -1 if there are more).
int oracle3_facets(const float* xyz, const int64_t* ext_idx, int nslots, int64_t* planes, int max_planes) {
  std::vector<P3> pts;
  for (int k = 0; k < nslots; ++k) {
    int64_t i = ext_idx[k];
    if (i < 0) continue;
    P3 q = {(int64_t)xyz[3 * i], (int64_t)xyz[3 * i + 1], (int64_t)xyz[3 * i + 2], i};
    bool dup = false;
    for (const P3& r : pts)
      if (r.x == q.x && r.y == q.y && r.z == q.z) dup = true;
    if (!dup) pts.push_back(q);
  }
  std::vector<std::vector<int64_t>> found;
  size_t u = pts.size();
  for (size_t a = 0; a < u; ++a)
    for (size_t b = a + 1; b < u; ++b)
      for (size_t c = b + 1; c < u; ++c) {
        int64_t ux = pts[b].x - pts[a].x, uy = pts[b].y - pts[a].y, uz = pts[b].z - pts[a].z;
        int64_t vx = pts[c].x - pts[a].x, vy = pts[c].y - pts[a].y, vz = pts[c].z - pts[a].z;
        int64_t nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
        if (nx == 0 && ny == 0 && nz == 0) continue;  // collinear
        int64_t d = nx * pts[a].x + ny * pts[a].y + nz * pts[a].z;
        int pos = 0, neg = 0;
        for (size_t e = 0; e < u; ++e) {
          int64_t s = nx * pts[e].x + ny * pts[e].y + nz * pts[e].z - d;
          if (s > 0) ++pos;
          if (s < 0) ++neg;
        }
        if (pos == 0 && neg == 0) return 0;  // every extreme on one plane: no interior
        if (pos > 0 && neg > 0) continue;
        if (pos > 0) { nx = -nx; ny = -ny; nz = -nz; d = -d; }  // make every extreme satisfy N.p <= d
        int64_t g = gcd_abs(gcd_abs(nx, ny), gcd_abs(nz, d));
        std::vector<int64_t> pl = {nx / g, ny / g, nz / g, d / g};
        if (std::find(found.begin(), found.end(), pl) == found.end()) found.push_back(pl);
      }
  std::sort(found.begin(), found.end());
  if ((int)found.size() > max_planes) return -1;
  for (size_t k = 0; k < found.size(); ++k)
    for (int j = 0; j < 4; ++j) planes[4 * k + j] = found[k][j];
  return (int)found.size();
}

// O3-3D -- the points not strictly inside the polyhedron (all of them when
// it has no facets), ascending; returns their count.
int64_t oracle3_prefilter(const float* xyz, int64_t n, const int64_t* planes, int m, int64_t* surv_idx) {
  int64_t c = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t x = (int64_t)xyz[3 * i], y = (int64_t)xyz[3 * i + 1], z = (int64_t)xyz[3 * i + 2];
    bool inside = m > 0;
    for (int k = 0; k < m && inside; ++k)
      if (planes[4 * k] * x + planes[4 * k + 1] * y + planes[4 * k + 2] * z - planes[4 * k + 3] >= 0) inside = false;
    if (!inside) surv_idx[c++] = i;
  }
  return c;
}

// Returns 1 when every coordinate is finite, integer-valued and |v| <= 2^19.
int oracle3_check_domain(const float* xyz, int64_t n) {
  for (int64_t i = 0; i < 3 * n; ++i) {
    float v = xyz[i];
    if (!std::isfinite(v) || std::fabs(v) > 524288.0f || std::floor(v) != v) return 0;
  }
  return 1;
}

}  // extern "C"
