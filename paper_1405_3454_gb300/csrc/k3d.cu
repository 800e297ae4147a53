// k3d.cu -- the 3D extension of the method sketched in section 5: six
// extremes (min/max of x, y, z) of the point set and of copies rotated about
// one axis, the convex polyhedron of those points, and the discard of every
// point strictly inside it.  Entry point hull3_prefilter (include/cudapre.h).
//
// The rotation axis is z and the angle table is Step 1's (x' and y' exactly
// as in 2D, z' = z).  Points are float32 xyz, integer-valued with
// |v| <= 2^19, so every plane test is exact in int64: normal components stay
// below 2^42, offsets and tests below 2^63.
//
// k3_extremes   one pass over the points (three 16-byte loads per four
//               points); per thread and direction a float32 running best,
//               a tile of four points examined only when its float32 extreme
//               may reach the best within the direction's error band, and
//               candidates inside the band ordered by the binary64
//               definition, then by index; one exact partial per block.
// k3_finish     one block: the exact reduction of the partials (and the at
//               most three points after the last whole group of four), the
//               24 slots, the facet planes of the extremes by the definition
//               (a plane through three extremes with all of them on one
//               side, written once, reduced, outward), float32 plane
//               coefficients with a static error bound, the cell grid's
//               placement.
// k3_cells      the 64^3 cell codes (exact): inside every facet, outside
//               one, one facet uncertain, several.
// k3_filter     the inside test and compaction: the point's cell decides,
//               or its one uncertain facet in float32 with escalation to
//               int64 inside the bound, or every facet (EXACT mode: every
//               facet in int64 for every point).
#include <cfloat>

#include "internal.cuh"
#include "proj.cuh"

namespace cudapre {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int NSLOT3 = 24;
constexpr int MAXF3 = 48;        // facets of <= 18 distinct extremes: at most 32
constexpr int MAXP3 = 24;        // distinct extreme points
constexpr int T3 = 256;          // threads of the streaming kernels
constexpr int64_t MAX_B3 = 4096; // blocks (partial results) of the extreme search
constexpr float COORD3 = 524288.0f;  // 2^19
// groups of four points a thread loads at once: the float32 search, the
// plain binary64 search (register-bound), the inside test
constexpr int QU_EXT = 2, QU_EXACT = 1, QU_FLT = 2;

template <int ANG>
struct Dirs3 {
  static constexpr int NV = ANG == 0 ? 7 : 9;  // x, y, z, then x', y' of the rotated groups computed
  static constexpr int ND = 2 * NV;
};

// 3D value v -> its 2D value index (v = 2 is z)
__device__ __forceinline__ int v2of(int v) { return v < 2 ? v : v - 1; }

template <int ANG>
__device__ __forceinline__ float val3(int v, float x, float y, float z) {
  return v == 2 ? z : value32<ANG>(v2of(v), x, y);
}
template <int ANG>
__device__ __forceinline__ float band3(int v) {
  return v == 2 ? 0.0f : band_of<ANG>(v2of(v));
}
// binary64 definition of value v (z: exact)
template <int ANG>
__device__ __forceinline__ double val64_3(int v, float x, float y, float z) {
  return v == 2 ? (double)z : value64(ANG, v2of(v), x, y);
}

// Cell grid of the inside test: CG^3 cells of 2^k lattice points per axis
// from (gx, gy, gz), over the bounding box of the extremes (outside it a
// point is outside the polyhedron).  A cell's byte code, exact in int64:
// CELL3_IN every lattice point of the cell is strictly inside every facet;
// CELL3_OUT every point of the cell fails one facet; f + 1 only facet f can
// fail in the cell; CELL3_MANY several can.
constexpr int CG_LOG = 6;
constexpr int CG = 1 << CG_LOG;
constexpr int CELLS3 = CG * CG * CG;
constexpr uint8_t CELL3_IN = 0, CELL3_OUT = 254, CELL3_MANY = 255;

struct Poly3 {
  int32_t nf;           // facets (0: nothing is strictly inside)
  int32_t kc;           // log2 of the cell size
  int32_t gx, gy, gz;   // grid origin (a multiple of the cell size)
  int32_t pad_;
  uint32_t ext[NSLOT3];
  long long pl[MAXF3][4];  // Nx, Ny, Nz, d: strictly inside iff N.p < d for every facet
  float4 fc[MAXF3];        // float32 A, B, C, D: s = fma(A, x, fma(B, y, fma(C, z, D))) ~ N.p - d
  float fe[MAXF3];         // |s - (N.p - d)| <= fe
};

struct Ws3 {
  uint32_t status;
  uint32_t pad_;
  unsigned long long n_surv;
  unsigned long long n_escalated;
  Poly3 poly;
};

constexpr size_t WS3_HEADER = align_up(sizeof(Ws3), 256);

__device__ __forceinline__ void load_p3(const float* xyz, uint32_t i, float& x, float& y, float& z) {
  x = __ldg(xyz + 3 * (size_t)i);
  y = __ldg(xyz + 3 * (size_t)i + 1);
  z = __ldg(xyz + 3 * (size_t)i + 2);
}

// Is candidate a (float32 score sa, index ia) strictly better than b for
// direction d = 2v + k (k = 1 max, score = value; k = 0 min, score =
// -value)?  Outside the band the float32 scores decide, inside it the
// binary64 definition, then the lower index.
template <int ANG>
__device__ __forceinline__ bool better3(int d, float sa, uint32_t ia, float sb, uint32_t ib, const float* xyz) {
  if (ia == NONE) return false;
  if (ib == NONE) return true;
  if (ia == ib) return false;
  const float diff = sa - sb, band = band3<ANG>(d >> 1);
  if (diff > band) return true;
  if (diff < -band) return false;
  float ax, ay, az, bx, by, bz;
  load_p3(xyz, ia, ax, ay, az);
  load_p3(xyz, ib, bx, by, bz);
  double ea = val64_3<ANG>(d >> 1, ax, ay, az), eb = val64_3<ANG>(d >> 1, bx, by, bz);
  if (!(d & 1)) { ea = -ea; eb = -eb; }
  return ea > eb || (ea == eb && ia < ib);
}

// ----------------------------------------------------------------------------
// Step 1 in 3D.

// The rare path of direction d over the four points w[0..3] (indices i0 ..
// i0 + 3, in order): the running best (*best, *bidx) replaced by every point
// strictly better than it.  Out of line: the streaming loop stays small.
template <int ANG>
__device__ __noinline__ uint2 slow3(int d, float w0, float w1, float w2, float w3, uint32_t i0, float b, uint32_t bi,
                                    const float* xyz) {
  const float w[4] = {w0, w1, w2, w3};
  for (int p = 0; p < 4; ++p) {
    const float sc = (d & 1) ? w[p] : -w[p];
    if (better3<ANG>(d, sc, i0 + p, b, bi, xyz)) { b = sc; bi = i0 + p; }
  }
  return make_uint2(__float_as_uint(b), bi);  // (the running best, by value: it stays in registers)
}

template <int ANG, int FILTER>
__global__ void __launch_bounds__(T3, 2) k3_extremes(const float* __restrict__ xyz, int64_t n, const uint32_t* status,
                                                  BlockBest* bres) {
  constexpr int NV = Dirs3<ANG>::NV, ND = Dirs3<ANG>::ND;
  __shared__ float s_sc[ND][T3];
  __shared__ uint32_t s_ix[ND][T3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(status) != 0;
  float best[ND];
  uint32_t bidx[ND];
  float wthr[FILTER == HULL_FILTER_FP32 ? ND : 1];  // FP32 mode: the warp's best score minus the band
  double bd[FILTER == HULL_FILTER_FP32 ? 1 : ND];  // EXACT mode: the binary64 bests
#pragma unroll
  for (int d = 0; d < (FILTER == HULL_FILTER_FP32 ? ND : 1); ++d) wthr[d] = -FLT_MAX;
#pragma unroll
  for (int d = 0; d < ND; ++d) { best[d] = -FLT_MAX; bidx[d] = NONE; }
#pragma unroll
  for (int d = 0; d < (FILTER == HULL_FILTER_FP32 ? 1 : ND); ++d) bd[d] = -DBL_MAX;
  const int64_t nq = dead ? 0 : n / 4;
  const float4* Q = reinterpret_cast<const float4*>(xyz);
  const int64_t stride = (int64_t)gridDim.x * T3;
  // QU groups of four points per thread and iteration, all loads issued
  // before any is used (more bytes in flight per thread)
  constexpr int QU = FILTER == HULL_FILTER_FP32 ? QU_EXT : QU_EXACT;
  // whole warps iterate together (warp votes below); a lane past the end
  // repeats point group nq - 1 (a repeat never changes a best)
  for (int64_t qb = (int64_t)blockIdx.x * T3 + (tid & ~31); qb < nq; qb += QU * stride) {
    float4 A[QU], B[QU], C[QU];
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const int64_t q = min(qb + lane + u * stride, nq - 1);
      A[u] = __ldcs(Q + 3 * q); B[u] = __ldcs(Q + 3 * q + 1); C[u] = __ldcs(Q + 3 * q + 2);
    }
#pragma unroll
    for (int u = 0; u < QU; ++u) {
    if (qb + u * stride >= nq) break;
    const int64_t q = min(qb + lane + u * stride, nq - 1);
    const float4 a = A[u], b = B[u], c = C[u];
    const float px[4] = {a.x, a.w, b.z, c.y}, py[4] = {a.y, b.x, b.w, c.z}, pz[4] = {a.z, b.y, c.x, c.w};
    const uint32_t i0 = (uint32_t)(4 * q);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      float w[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) w[p] = val3<ANG>(v, px[p], py[p], pz[p]);
      if (FILTER == HULL_FILTER_FP32) {
        const float band = band3<ANG>(v);
        const float tmx = fmaxf(max3f(w[0], w[1], w[2]), w[3]);
        const float tmn = fminf(min3f(w[0], w[1], w[2]), w[3]);
        // the tile's extreme may reach the best within the band: the rare path
        // a lane enters the rare path only when its tile may reach the
        // warp's best within the band (wthr: warp-uniform), then updates its
        // own best exactly; the warp's threshold follows
        const bool hi = tmx >= wthr[2 * v + 1], lo = -tmn >= wthr[2 * v];
        if (__any_sync(FULL, hi)) {
          if (hi) {
            const uint2 r = slow3<ANG>(2 * v + 1, w[0], w[1], w[2], w[3], i0, best[2 * v + 1], bidx[2 * v + 1], xyz);
            best[2 * v + 1] = __uint_as_float(r.x);
            bidx[2 * v + 1] = r.y;
          }
          float m = best[2 * v + 1];
          for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, off));
          wthr[2 * v + 1] = m - band;
        }
        if (__any_sync(FULL, lo)) {
          if (lo) {
            const uint2 r = slow3<ANG>(2 * v, w[0], w[1], w[2], w[3], i0, best[2 * v], bidx[2 * v], xyz);
            best[2 * v] = __uint_as_float(r.x);
            bidx[2 * v] = r.y;
          }
          float m = best[2 * v];
          for (int off = 16; off; off >>= 1) m = fmaxf(m, __shfl_xor_sync(FULL, m, off));
          wthr[2 * v] = m - band;
        }
      } else {
        // the plain method: every point's binary64 value (the float32 score
        // kept beside it only serves the exact reductions below)
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const double e = val64_3<ANG>(v, px[p], py[p], pz[p]);
          if (bidx[2 * v + 1] == NONE || e > bd[2 * v + 1]) {
            bd[2 * v + 1] = e; best[2 * v + 1] = w[p]; bidx[2 * v + 1] = i0 + p;
          }
          if (bidx[2 * v] == NONE || -e > bd[2 * v]) {
            bd[2 * v] = -e; best[2 * v] = -w[p]; bidx[2 * v] = i0 + p;
          }
        }
      }
    }
    }
  }
  // the block's result per direction: every thread's candidate through
  // shared memory, one warp per direction (exact comparisons)
  __syncthreads();
#pragma unroll
  for (int d = 0; d < ND; ++d) { s_sc[d][tid] = best[d]; s_ix[d][tid] = bidx[d]; }
  __syncthreads();
  for (int d = warp; d < ND; d += T3 / 32) {
    float sc = s_sc[d][lane];
    uint32_t ix = s_ix[d][lane];
    for (int t = lane + 32; t < T3; t += 32)
      if (better3<ANG>(d, s_sc[d][t], s_ix[d][t], sc, ix, xyz)) { sc = s_sc[d][t]; ix = s_ix[d][t]; }
    for (int off = 16; off; off >>= 1) {
      const float so = __shfl_xor_sync(FULL, sc, off);
      const uint32_t io = __shfl_xor_sync(FULL, ix, off);
      if (better3<ANG>(d, so, io, sc, ix, xyz)) { sc = so; ix = io; }
    }
    if (lane == 0) {
      BlockBest r;
      r.idx = ix;
      r.pad_ = 0;
      r.s = -DBL_MAX;
      if (ix != NONE) {
        float x, y, z;
        load_p3(xyz, ix, x, y, z);
        const double e = val64_3<ANG>(d >> 1, x, y, z);
        r.s = (d & 1) ? e : -e;
      }
      bres[(size_t)blockIdx.x * ND + d] = r;
    }
  }
}

// ----------------------------------------------------------------------------
// Step 2 in 3D: the facet planes of the extremes' polyhedron.

__device__ long long gcd_ll(long long a, long long b) {
  a = a < 0 ? -a : a;
  b = b < 0 ? -b : b;
  while (b) {
    const long long t = a % b;
    a = b;
    b = t;
  }
  return a;
}

template <int ANG>
__global__ void __launch_bounds__(T3) k3_finish(const float* __restrict__ xyz, int64_t n, int64_t nblocks,
                                                 Ws3* W, const BlockBest* bres, uint32_t* ext_out) {
  constexpr int ND = Dirs3<ANG>::ND;
  __shared__ uint32_t s_dir[32];
  __shared__ uint32_t s_ext[NSLOT3];
  __shared__ long long s_px[MAXP3], s_py[MAXP3], s_pz[MAXP3];
  __shared__ int s_u, s_nf, s_flat;
  __shared__ long long s_pl[MAXF3 * 2][4];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dead = *reinterpret_cast<volatile uint32_t*>(&W->status) != 0;
  const int64_t nq = n / 4;
  // one warp per direction: the blocks' partials and the points after the
  // last group of four, by (binary64 score key, index)
  for (int d = warp; d < ND; d += T3 / 32) {
    unsigned long long ks = 0;
    uint32_t bi = NONE;
    auto take = [&](unsigned long long k, uint32_t i) {
      return i != NONE && (bi == NONE || k > ks || (k == ks && i < bi));
    };
    if (!dead) {
      for (int64_t e = lane; e < nblocks; e += 32) {
        const BlockBest b = bres[e * ND + d];
        const unsigned long long k = dkey(b.s);
        if (take(k, b.idx)) { ks = k; bi = b.idx; }
      }
      const int64_t t = 4 * nq + lane;
      if (lane < 3 && t < n) {
        float x, y, z;
        load_p3(xyz, (uint32_t)t, x, y, z);
        const double e = val64_3<ANG>(d >> 1, x, y, z);
        const unsigned long long k = dkey((d & 1) ? e : -e);
        if (take(k, (uint32_t)t)) { ks = k; bi = (uint32_t)t; }
      }
    }
    for (int off = 16; off; off >>= 1) {
      const uint32_t io = __shfl_xor_sync(FULL, bi, off);
      const unsigned long long ko = __shfl_xor_sync(FULL, ks, off);
      if (take(ko, io)) { ks = ko; bi = io; }
    }
    if (lane == 0) s_dir[d] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    // direction 2v + k of value v -> slot 6g + 2a + k (value v: 0 x, 1 y,
    // 2 z of group 0, then x', y' of the computed rotated groups)
    for (int k = 0; k < 2; ++k) {
      s_ext[0 + k] = s_dir[0 + k];
      s_ext[2 + k] = s_dir[2 + k];
      s_ext[4 + k] = s_dir[4 + k];
      for (int g = 1; g <= (ANG == 0 ? 2 : 3); ++g) {
        s_ext[6 * g + k] = s_dir[2 * (2 * g + 1) + k];      // x'
        s_ext[6 * g + 2 + k] = s_dir[2 * (2 * g + 2) + k];  // y'
      }
      for (int g = 1; g < 4; ++g) s_ext[6 * g + 4 + k] = s_dir[4 + k];  // z' = z
    }
    if (ANG == 0) {
      // 120 degrees from 30 degrees (x'(120) = -y'(30), y'(120) = x'(30))
      s_ext[18] = s_ext[9];
      s_ext[19] = s_ext[8];
      s_ext[20] = s_ext[6];
      s_ext[21] = s_ext[7];
    }
    if (dead || n == 0)
      for (int k = 0; k < NSLOT3; ++k) s_ext[k] = NONE;
    // distinct points: by index, then by coordinates, the lowest index kept
    // (the slot order decides nothing: the facets do not depend on it)
    int u = 0;
    uint32_t kept[NSLOT3];
    for (int k = 0; k < NSLOT3; ++k) {
      const uint32_t i = s_ext[k];
      if (i == NONE) continue;
      float x, y, z;
      load_p3(xyz, i, x, y, z);
      const long long X = (long long)x, Y = (long long)y, Z = (long long)z;
      int j = 0;
      while (j < u && !(s_px[j] == X && s_py[j] == Y && s_pz[j] == Z)) ++j;
      if (j == u) { s_px[u] = X; s_py[u] = Y; s_pz[u] = Z; kept[u] = i; ++u; }
      else if (i < kept[j]) kept[j] = i;
    }
    s_u = u;
    s_nf = 0;
    s_flat = 0;
  }
  __syncthreads();
  const int u = s_u;
  // every triple a < b < c of distinct points: a facet plane when all points
  // lie on one closed side; written by its canonical triple only (the first
  // two points of the plane and the first later one off their line)
  const int ntri = u * (u - 1) * (u - 2) / 6;
  for (int t = tid; t < ntri; t += T3) {
    int a = 0, b = 1, c = 2, r = t;
    // unrank t in lexicographic order
    for (a = 0;; ++a) {
      const int cnt = (u - 1 - a) * (u - 2 - a) / 2;
      if (r < cnt) break;
      r -= cnt;
    }
    for (b = a + 1;; ++b) {
      const int cnt = u - 1 - b;
      if (r < cnt) break;
      r -= cnt;
    }
    c = b + 1 + r;
    const long long ux = s_px[b] - s_px[a], uy = s_py[b] - s_py[a], uz = s_pz[b] - s_pz[a];
    const long long vx = s_px[c] - s_px[a], vy = s_py[c] - s_py[a], vz = s_pz[c] - s_pz[a];
    long long nx = uy * vz - uz * vy, ny = uz * vx - ux * vz, nz = ux * vy - uy * vx;
    if (nx == 0 && ny == 0 && nz == 0) continue;
    long long d = nx * s_px[a] + ny * s_py[a] + nz * s_pz[a];
    int pos = 0, neg = 0, z0 = -1, z1 = -1, z2 = -1;
    for (int e = 0; e < u; ++e) {
      const long long s = nx * s_px[e] + ny * s_py[e] + nz * s_pz[e] - d;
      pos += s > 0;
      neg += s < 0;
      if (s == 0) {
        if (z0 < 0) z0 = e;
        else if (z1 < 0) z1 = e;
        else if (z2 < 0) {
          const long long wx = s_px[e] - s_px[z0], wy = s_py[e] - s_py[z0], wz = s_pz[e] - s_pz[z0];
          const long long qx = s_px[z1] - s_px[z0], qy = s_py[z1] - s_py[z0], qz = s_pz[z1] - s_pz[z0];
          if (qy * wz - qz * wy != 0 || qz * wx - qx * wz != 0 || qx * wy - qy * wx != 0) z2 = e;
        }
      }
    }
    if (pos == 0 && neg == 0) { s_flat = 1; continue; }
    if (pos > 0 && neg > 0) continue;
    if (a != z0 || b != z1 || c != z2) continue;  // not this plane's canonical triple
    if (pos > 0) { nx = -nx; ny = -ny; nz = -nz; d = -d; }
    const long long g = gcd_ll(gcd_ll(nx, ny), gcd_ll(nz, d));
    const int k = atomicAdd(&s_nf, 1);
    if (k < MAXF3 * 2) {
      s_pl[k][0] = nx / g;
      s_pl[k][1] = ny / g;
      s_pl[k][2] = nz / g;
      s_pl[k][3] = d / g;
    }
  }
  __syncthreads();
  Poly3& P = W->poly;
  if (tid == 0) {
    int nf = s_flat ? 0 : s_nf;
    if (nf > MAXF3) {  // cannot happen for at most 18 distinct points
      atomicOr(&W->status, HULL_DEVICE_OVERFLOW);
      nf = 0;
    }
    // lexicographic order (the oracle's)
    for (int i = 1; i < nf; ++i)
      for (int j = i; j > 0; --j) {
        bool lt = false;
        for (int q = 0; q < 4; ++q)
          if (s_pl[j][q] != s_pl[j - 1][q]) { lt = s_pl[j][q] < s_pl[j - 1][q]; break; }
        if (!lt) break;
        for (int q = 0; q < 4; ++q) { const long long tq = s_pl[j][q]; s_pl[j][q] = s_pl[j - 1][q]; s_pl[j - 1][q] = tq; }
      }
    P.nf = nf;
    for (int k = 0; k < NSLOT3; ++k) {
      P.ext[k] = s_ext[k];
      if (ext_out) ext_out[k] = s_ext[k];
    }
  }
  __syncthreads();
  const int nf = P.nf;
  // float32 coefficients and the static error bound of
  //   s = fma(A', x, fma(B', y, fma(C', z, D'))),  A' = RN(Nx), ..., D' = RN(-d):
  // three fma roundings, each at most u |partial sum| <= u T, and the
  // coefficient roundings at most u (|Nx| + |Ny| + |Nz|) M + u |d| <= u T,
  // with T = (|A'| + |B'| + |C'|) M + |D'| (upward), u = 2^-24, M = 2^19:
  // E = 2 (4 + 2^-20) u T, computed with upward rounding (factor 2: margin).
  if (tid < nf) {
    const long long* q = s_pl[tid];
    P.pl[tid][0] = q[0]; P.pl[tid][1] = q[1]; P.pl[tid][2] = q[2]; P.pl[tid][3] = q[3];
    const float A = __ll2float_rn(q[0]), B = __ll2float_rn(q[1]), C = __ll2float_rn(q[2]), D = __ll2float_rn(-q[3]);
    P.fc[tid] = make_float4(A, B, C, D);
    const float aA = __ll2float_ru(q[0] < 0 ? -q[0] : q[0]), aB = __ll2float_ru(q[1] < 0 ? -q[1] : q[1]);
    const float aC = __ll2float_ru(q[2] < 0 ? -q[2] : q[2]), aD = __ll2float_ru(q[3] < 0 ? -q[3] : q[3]);
    float T = __fmul_ru(__fadd_ru(__fadd_ru(aA, aB), aC), COORD3);
    T = __fadd_ru(T, aD);
    P.fe[tid] = __fmul_ru(__fmul_ru(T, 0x1.000004p+3f), 0x1p-24f);  // 2 (4 + 2^-20) u T
  }
  // the cell grid: the smallest power-of-two cell size whose CG cells per
  // axis, from an origin aligned to it, cover the extremes' bounding box
  if (tid == 0) {
    long long lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      const long long* c = a == 0 ? s_px : (a == 1 ? s_py : s_pz);
      lo[a] = hi[a] = u > 0 ? c[0] : 0;
      for (int k = 1; k < u; ++k) { lo[a] = min(lo[a], c[k]); hi[a] = max(hi[a], c[k]); }
    }
    int kc = 0;
    auto origin = [](long long v, int k) { return (v >> k) << k; };  // floor to 2^k
    for (;; ++kc) {
      bool fits = true;
      for (int a = 0; a < 3; ++a) fits = fits && hi[a] - origin(lo[a], kc) < ((long long)CG << kc);
      if (fits) break;
    }
    P.kc = kc;
    P.gx = (int32_t)origin(lo[0], kc);
    P.gy = (int32_t)origin(lo[1], kc);
    P.gz = (int32_t)origin(lo[2], kc);
  }
}

// One thread per cell: its code (see Poly3), from the extreme values of
// N.p - d over the cell's corners (the plane test is linear), the corners
// clamped to the coordinate domain, so every product stays below 2^61.
// masks[c] (cells with code CELL3_MANY): bit f set when some point of the
// cell may fail facet f; every point of the cell is strictly inside the
// facets whose bit is clear.
__global__ void __launch_bounds__(T3) k3_cells(Ws3* W, uint8_t* codes, unsigned long long* masks) {
  __shared__ long long s_pl[MAXF3][4];
  __shared__ int s_meta[5];
  const int tid = threadIdx.x;
  if (*reinterpret_cast<volatile uint32_t*>(&W->status) != 0) return;
  const Poly3& P = W->poly;
  if (tid == 0) { s_meta[0] = P.nf; s_meta[1] = P.kc; s_meta[2] = P.gx; s_meta[3] = P.gy; s_meta[4] = P.gz; }
  for (int k = tid; k < 4 * MAXF3; k += T3) (&s_pl[0][0])[k] = (&P.pl[0][0])[k];
  __syncthreads();
  const int nf = s_meta[0];
  if (nf == 0) return;
  const int kc = s_meta[1];
  for (int c = blockIdx.x * T3 + tid; c < CELLS3; c += gridDim.x * T3) {
    const int ix = c & (CG - 1), iy = (c >> CG_LOG) & (CG - 1), iz = c >> (2 * CG_LOG);
    long long lo[3], hi[3];
    const long long base[3] = {(long long)s_meta[2] + ((long long)ix << kc), (long long)s_meta[3] + ((long long)iy << kc),
                               (long long)s_meta[4] + ((long long)iz << kc)};
    for (int a = 0; a < 3; ++a) {
      lo[a] = max(base[a], -(long long)COORD3);
      hi[a] = min(base[a] + (1ll << kc) - 1, (long long)COORD3);
    }
    uint8_t code = CELL3_IN;
    int unsure = 0, which = 0;
    unsigned long long mask = 0;
    for (int f = 0; f < nf && code != CELL3_OUT; ++f) {
      long long mx = -s_pl[f][3], mn = -s_pl[f][3];
      for (int a = 0; a < 3; ++a) {
        const long long p0 = s_pl[f][a] * lo[a], p1 = s_pl[f][a] * hi[a];
        mx += max(p0, p1);
        mn += min(p0, p1);
      }
      if (mn >= 0) code = CELL3_OUT;                  // every point fails facet f
      else if (mx >= 0) { ++unsure; which = f; mask |= 1ull << f; }  // some point may fail it
    }
    if (code != CELL3_OUT && lo[0] <= hi[0] && lo[1] <= hi[1] && lo[2] <= hi[2])
      code = unsure == 0 ? CELL3_IN : (unsure == 1 ? (uint8_t)(which + 1) : CELL3_MANY);
    if (lo[0] > hi[0] || lo[1] > hi[1] || lo[2] > hi[2]) code = CELL3_OUT;  // no point of the domain
    codes[c] = code;
    if (code == CELL3_MANY) masks[c] = mask;
  }
}

// ----------------------------------------------------------------------------
// Step 3 in 3D: the inside test and compaction of the survivors.

// The code of the point's cell (CELL3_OUT outside the grid): cell
// coordinates floor((v - g) 2^-kc) by round-down operations, exact for these
// integers.
__device__ __forceinline__ uint32_t cell_code(const uint8_t* codes, float gx, float gy, float gz, float sc, float x,
                                              float y, float z, int& cell) {
  const int cx = __float2int_rd(__fsub_rd(x, gx) * sc), cy = __float2int_rd(__fsub_rd(y, gy) * sc);
  const int cz = __float2int_rd(__fsub_rd(z, gz) * sc);
  cell = 0;
  if ((unsigned)(cx | cy | cz) >= (unsigned)CG) return CELL3_OUT;  // outside the extremes' bounding box
  cell = (cz << (2 * CG_LOG)) | (cy << CG_LOG) | cx;
  return __ldg(codes + cell);
}

// The facets of `mask` against one point (a CELL3_MANY cell: the point is
// strictly inside every other facet): 2 * escalations + (survives ? 1 : 0).
__device__ __noinline__ unsigned facets3_mask(const long long (*pl)[4], const float4* fc, const float* fe,
                                              unsigned long long mask, float x, float y, float z) {
  unsigned esc = 0;
  while (mask) {
    const int k = __ffsll((long long)mask) - 1;
    mask &= mask - 1;
    const float4 c = fc[k];
    const float s = fmaf(c.x, x, fmaf(c.y, y, fmaf(c.z, z, c.w)));
    const float e = fe[k];
    if (s < -e) continue;
    if (s > e) return 2 * esc + 1;
    ++esc;
    if (pl[k][0] * (long long)x + pl[k][1] * (long long)y + pl[k][2] * (long long)z - pl[k][3] >= 0)
      return 2 * esc + 1;
  }
  return 2 * esc;
}

// Every facet of the polyhedron against one point: 2 * escalations +
// (survives ? 1 : 0).  A facet the point fails ends the test.
template <int FILTER>
__device__ __noinline__ unsigned facets3(const long long (*pl)[4], const float4* fc, const float* fe, int nf, float x,
                                         float y, float z) {
  const long long X = (long long)x, Y = (long long)y, Z = (long long)z;
  unsigned esc = 0;
  for (int k = 0; k < nf; ++k) {
    if (FILTER == HULL_FILTER_FP32) {
      const float4 c = fc[k];
      const float s = fmaf(c.x, x, fmaf(c.y, y, fmaf(c.z, z, c.w)));
      const float e = fe[k];
      if (s < -e) continue;
      if (s > e) return 2 * esc + 1;
      ++esc;
    }
    if (pl[k][0] * X + pl[k][1] * Y + pl[k][2] * Z - pl[k][3] >= 0) return 2 * esc + 1;
  }
  return 2 * esc;
}

template <int FILTER>
__global__ void __launch_bounds__(T3) k3_filter(const float* __restrict__ xyz, int64_t n, Ws3* W,
                                                uint32_t* __restrict__ surv, const uint8_t* __restrict__ codes,
                                                const unsigned long long* __restrict__ masks) {
  __shared__ long long s_pl[MAXF3][4];
  __shared__ float4 s_fc[MAXF3];
  __shared__ float s_fe[MAXF3];
  __shared__ int s_nf;
  __shared__ float s_sp[4];
  const int tid = threadIdx.x, lane = tid & 31;
  if (*reinterpret_cast<volatile uint32_t*>(&W->status) != 0) return;
  const Poly3& P = W->poly;
  if (tid == 0) {
    s_nf = P.nf;
    s_sp[0] = (float)P.gx; s_sp[1] = (float)P.gy; s_sp[2] = (float)P.gz;
    s_sp[3] = __int_as_float((127 - P.kc) << 23);  // 2^-kc
  }
  for (int k = tid; k < MAXF3; k += T3) {
    s_pl[k][0] = P.pl[k][0]; s_pl[k][1] = P.pl[k][1]; s_pl[k][2] = P.pl[k][2]; s_pl[k][3] = P.pl[k][3];
    s_fc[k] = P.fc[k];
    s_fe[k] = P.fe[k];
  }
  __syncthreads();
  const int nf = s_nf;
  const float gx = s_sp[0], gy = s_sp[1], gz = s_sp[2], sc = s_sp[3];
  unsigned esc = 0;
  // survives: not strictly inside every facet.  FP32 mode: the point's cell
  // decides (exact cell code; cell coordinates floor((v - g) 2^-kc) by
  // round-down operations, exact for these integers), a cell with one
  // uncertain facet takes one float32 test with escalation, several the
  // full test; EXACT mode: every facet in int64.
  // survives: not strictly inside every facet.  FP32 mode: the point's cell
  // decides (exact cell code), a cell with one uncertain facet takes one
  // float32 test with escalation, several the full test; EXACT mode: every
  // facet in int64.
  auto survives = [&](float x, float y, float z) -> bool {
    if (nf == 0) return true;
    if (FILTER == HULL_FILTER_FP32) {
      int cell;
      const uint32_t code = cell_code(codes, gx, gy, gz, sc, x, y, z, cell);
      if (code == CELL3_IN) return false;
      if (code == CELL3_OUT) return true;
      if (code == CELL3_MANY) {
        const unsigned r = facets3_mask(s_pl, s_fc, s_fe, __ldg(masks + cell), x, y, z);
        esc += r >> 1;
        return r & 1;
      }
      if (code != CELL3_MANY) {
        const int f = (int)code - 1;
        const float4 c = s_fc[f];
        const float s = fmaf(c.x, x, fmaf(c.y, y, fmaf(c.z, z, c.w)));
        if (s < -s_fe[f]) return false;
        if (s > s_fe[f]) return true;
        ++esc;
        return s_pl[f][0] * (long long)x + s_pl[f][1] * (long long)y + s_pl[f][2] * (long long)z - s_pl[f][3] >= 0;
      }
    }
    const unsigned r = facets3<FILTER>(s_pl, s_fc, s_fe, nf, x, y, z);
    esc += r >> 1;
    return r & 1;
  };
  const int64_t nq = n / 4;
  const float4* Q = reinterpret_cast<const float4*>(xyz);
  const int64_t stride = (int64_t)gridDim.x * T3;
  // whole warps iterate together: the survivors of the warp's 4 x 32 points
  // are placed with one atomic
  constexpr int QU = QU_FLT;
  for (int64_t qb = (int64_t)blockIdx.x * T3 + (tid & ~31); qb < nq; qb += QU * stride) {
    float4 A[QU], B[QU], C[QU];
#pragma unroll
    for (int u = 0; u < QU; ++u) {
      const int64_t q = qb + lane + u * stride;
      if (q < nq) { A[u] = __ldcs(Q + 3 * q); B[u] = __ldcs(Q + 3 * q + 1); C[u] = __ldcs(Q + 3 * q + 2); }
    }
#pragma unroll
    for (int u = 0; u < QU; ++u) {
    const int64_t q = qb + lane + u * stride;
    bool keep[4] = {false, false, false, false};
    if (q < nq) {
      const float4 a = A[u], b = B[u], c = C[u];
      keep[0] = survives(a.x, a.y, a.z);
      keep[1] = survives(a.w, b.x, b.y);
      keep[2] = survives(b.z, b.w, c.x);
      keep[3] = survives(c.y, c.z, c.w);
    }
    const int mine = (int)keep[0] + keep[1] + keep[2] + keep[3];
    int pre = mine;
    for (int off = 1; off < 32; off <<= 1) {
      const int v = __shfl_up_sync(FULL, pre, off);
      if (lane >= off) pre += v;
    }
    const int total = __shfl_sync(FULL, pre, 31);
    if (total) {
      unsigned long long base = 0;
      if (lane == 31) base = atomicAdd(&W->n_surv, (unsigned long long)total);
      base = __shfl_sync(FULL, base, 31);
      unsigned long long pos = base + (unsigned long long)(pre - mine);
      for (int p = 0; p < 4; ++p)
        if (keep[p]) surv[pos++] = (uint32_t)(4 * q + p);
    }
    }
  }
  // the at most three points after the last group of four
  if (blockIdx.x == 0 && tid < (int)(n - 4 * nq)) {
    const uint32_t i = (uint32_t)(4 * nq + tid);
    float x, y, z;
    load_p3(xyz, i, x, y, z);
    if (survives(x, y, z)) surv[atomicAdd(&W->n_surv, 1ull)] = i;
  }
  for (int off = 16; off; off >>= 1) esc += __shfl_xor_sync(FULL, esc, off);
  if (lane == 0 && esc) atomicAdd(&W->n_escalated, (unsigned long long)esc);
}

__global__ void k3_validate(const float* __restrict__ xyz, int64_t n3, uint32_t* status) {
  bool bad = false;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n3; k += (int64_t)gridDim.x * blockDim.x) {
    const float v = __ldg(xyz + k);
    bad |= !(fabsf(v) <= COORD3) || truncf(v) != v;
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, HULL_DEVICE_DOMAIN);
}

__global__ void k3_count(const Ws3* W, int64_t* out) { *out = W->status ? 0 : (int64_t)W->n_surv; }

// Blocks of the streaming passes: resident ones (two per SM), fewer for
// small inputs (at least 16 groups of four points per thread).
int64_t blocks3(int64_t n) {
  const int64_t nq = n / 4;
  const int64_t want = (nq + 16 * T3 - 1) / (16 * T3);
  return std::max<int64_t>(1, std::min<int64_t>(want, std::min<int64_t>(MAX_B3, (int64_t)device_sm_count() * 2)));
}

constexpr size_t WS3_PARTIALS = align_up(sizeof(BlockBest) * 18 * (size_t)MAX_B3, 256);

size_t ws3_bytes(int64_t n) {
  (void)n;
  return WS3_HEADER + WS3_PARTIALS + align_up(CELLS3, 256) + sizeof(unsigned long long) * (size_t)CELLS3;
}

}  // namespace
}  // namespace cudapre

using namespace cudapre;

extern "C" {

size_t hull3_prefilter_workspace_bytes(int64_t n, const hull_options* opt) {
  (void)opt;
  return ws3_bytes(std::max<int64_t>(n, 0));
}

hull_status hull3_prefilter(const float* d_xyz, int64_t n, void* d_ws, size_t ws_bytes, uint32_t* d_survivor_idx,
                            int64_t* d_n_survivors, uint32_t* d_extreme_idx, const hull_options* opt, void* stream) {
  if (n < 0 || n > 0xFFFFFFFFll) return HULL_ERR_INVALID_ARG;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u) || !d_n_survivors) return HULL_ERR_INVALID_ARG;
  if (n > 0 && (!d_xyz || (reinterpret_cast<uintptr_t>(d_xyz) & 15u) || !d_survivor_idx)) return HULL_ERR_INVALID_ARG;
  hull_options o;
  hull_default_options(&o);
  if (opt) o = *opt;
  if (o.angles != HULL_ANGLES_CUMULATIVE && o.angles != HULL_ANGLES_ABSOLUTE) return HULL_ERR_UNSUPPORTED;
  if (o.filter != HULL_FILTER_EXACT && o.filter != HULL_FILTER_FP32) return HULL_ERR_UNSUPPORTED;
  if (o.no_prefilter) return HULL_ERR_UNSUPPORTED;
  if (ws_bytes < ws3_bytes(n)) return HULL_ERR_WORKSPACE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Ws3* W = static_cast<Ws3*>(d_ws);
  BlockBest* bres = reinterpret_cast<BlockBest*>(static_cast<char*>(d_ws) + WS3_HEADER);
  uint8_t* codes = static_cast<uint8_t*>(d_ws) + WS3_HEADER + WS3_PARTIALS;
  auto* masks = reinterpret_cast<unsigned long long*>(codes + align_up(CELLS3, 256));
  stage_mark(0, st);
  if (cudaMemsetAsync(W, 0, sizeof(Ws3), st) != cudaSuccess) return HULL_ERR_CUDA;
  if (o.validate && n > 0) {
    const int g = (int)std::min<int64_t>((3 * n + 255) / 256, (int64_t)device_sm_count() * 8);
    k3_validate<<<g, 256, 0, st>>>(d_xyz, 3 * n, &W->status);
    count_launches(1);
  }
  stage_mark(1, st);
  const int64_t G = blocks3(n);
  const int64_t Gf = std::max<int64_t>(1, std::min<int64_t>((n / 4 + T3 - 1) / T3, (int64_t)device_sm_count() * 4));
  // stage boundaries as the 2D calls: extremes | polyhedron | inside test
#define K3(A, F)                                                                          \
  do {                                                                                    \
    k3_extremes<A, F><<<(unsigned)G, T3, 0, st>>>(d_xyz, n, &W->status, bres);            \
    stage_mark(2, st);                                                                    \
    k3_finish<A><<<1, T3, 0, st>>>(d_xyz, n, G, W, bres, d_extreme_idx);                  \
    if (F == HULL_FILTER_FP32) k3_cells<<<CELLS3 / T3, T3, 0, st>>>(W, codes, masks);     \
    stage_mark(3, st);                                                                    \
    k3_filter<F><<<(unsigned)Gf, T3, 0, st>>>(d_xyz, n, W, d_survivor_idx, codes, masks); \
    stage_mark(4, st);                                                                    \
  } while (0)
  if (o.angles == HULL_ANGLES_CUMULATIVE) {
    if (o.filter == HULL_FILTER_FP32) K3(0, HULL_FILTER_FP32); else K3(0, HULL_FILTER_EXACT);
  } else {
    if (o.filter == HULL_FILTER_FP32) K3(1, HULL_FILTER_FP32); else K3(1, HULL_FILTER_EXACT);
  }
#undef K3
  k3_count<<<1, 1, 0, st>>>(W, d_n_survivors);
  count_launches(o.filter == HULL_FILTER_FP32 ? 5 : 4);
  stage_mark(5, st);
  stage_mark(6, st);
  return cudaGetLastError() == cudaSuccess ? HULL_OK : HULL_ERR_CUDA;
}

hull_status hull3_read_polyhedron(const void* d_ws, int32_t* h_nf, int64_t* h_planes, uint32_t* h_ext,
                                  int64_t* h_counts, void* stream) {
  if (!d_ws || !h_nf) return HULL_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Ws3 w;
  if (cudaMemcpyAsync(&w, d_ws, sizeof(Ws3), cudaMemcpyDeviceToHost, st) != cudaSuccess) return HULL_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return HULL_ERR_CUDA;
  *h_nf = w.poly.nf;
  for (int k = 0; k < w.poly.nf && k < MAXF3; ++k)
    if (h_planes)
      for (int q = 0; q < 4; ++q) h_planes[4 * k + q] = w.poly.pl[k][q];
  if (h_ext)
    for (int k = 0; k < NSLOT3; ++k) h_ext[k] = w.poly.ext[k];
  if (h_counts) {
    h_counts[0] = (int64_t)w.n_surv;
    h_counts[1] = (int64_t)w.n_escalated;
    h_counts[2] = (int64_t)w.status;
  }
  return HULL_OK;
}

}  // extern "C"
