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
//               coefficients with a static error bound, and an inscribed
//               sphere.
// k3_filter     the inside test and compaction: a point inside the sphere
//               is discarded at once; otherwise every facet in float32 with
//               escalation to int64 inside the bound (or int64 throughout in
//               EXACT mode), a point failing a facet survives.
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

struct Poly3 {
  int32_t nf;           // facets (0: nothing is strictly inside)
  int32_t sphere_on;
  float cx, cy, cz, r2; // inscribed sphere: (x-cx)^2+(y-cy)^2+(z-cz)^2 < r2 (float32, proven margin) => inside
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

template <int ANG, int FILTER>
__global__ void __launch_bounds__(T3, 2) k3_extremes(const float* __restrict__ xyz, int64_t n, const uint32_t* status,
                                                  BlockBest* bres) {
  constexpr int NV = Dirs3<ANG>::NV, ND = Dirs3<ANG>::ND;
  __shared__ float s_sc[T3 / 32][ND];
  __shared__ uint32_t s_ix[T3 / 32][ND];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(status) != 0;
  float best[ND];
  uint32_t bidx[ND];
  double bd[FILTER == HULL_FILTER_FP32 ? 1 : ND];  // EXACT mode: the binary64 bests
#pragma unroll
  for (int d = 0; d < ND; ++d) { best[d] = -FLT_MAX; bidx[d] = NONE; }
#pragma unroll
  for (int d = 0; d < (FILTER == HULL_FILTER_FP32 ? 1 : ND); ++d) bd[d] = -DBL_MAX;
  const int64_t nq = dead ? 0 : n / 4;
  const float4* Q = reinterpret_cast<const float4*>(xyz);
  for (int64_t q = (int64_t)blockIdx.x * T3 + tid; q < nq; q += (int64_t)gridDim.x * T3) {
    const float4 a = __ldcs(Q + 3 * q), b = __ldcs(Q + 3 * q + 1), c = __ldcs(Q + 3 * q + 2);
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
        // the tile's extreme may reach the best within the band: points in order
        if (tmx >= best[2 * v + 1] - band) {
#pragma unroll
          for (int p = 0; p < 4; ++p)
            if (better3<ANG>(2 * v + 1, w[p], i0 + p, best[2 * v + 1], bidx[2 * v + 1], xyz)) {
              best[2 * v + 1] = w[p];
              bidx[2 * v + 1] = i0 + p;
            }
        }
        if (-tmn >= best[2 * v] - band) {
#pragma unroll
          for (int p = 0; p < 4; ++p)
            if (better3<ANG>(2 * v, -w[p], i0 + p, best[2 * v], bidx[2 * v], xyz)) {
              best[2 * v] = -w[p];
              bidx[2 * v] = i0 + p;
            }
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
  // warp, then block: exact comparisons
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    float sc = best[d];
    uint32_t ix = bidx[d];
    for (int off = 16; off; off >>= 1) {
      const float so = __shfl_xor_sync(FULL, sc, off);
      const uint32_t io = __shfl_xor_sync(FULL, ix, off);
      if (better3<ANG>(d, so, io, sc, ix, xyz)) { sc = so; ix = io; }
    }
    if (lane == 0) { s_sc[warp][d] = sc; s_ix[warp][d] = ix; }
  }
  __syncthreads();
  if (tid < ND) {
    float sc = s_sc[0][tid];
    uint32_t ix = s_ix[0][tid];
    for (int w = 1; w < T3 / 32; ++w)
      if (better3<ANG>(tid, s_sc[w][tid], s_ix[w][tid], sc, ix, xyz)) { sc = s_sc[w][tid]; ix = s_ix[w][tid]; }
    BlockBest r;
    r.idx = ix;
    r.pad_ = 0;
    r.s = -DBL_MAX;
    if (ix != NONE) {
      float x, y, z;
      load_p3(xyz, ix, x, y, z);
      const double e = val64_3<ANG>(tid >> 1, x, y, z);
      r.s = (tid & 1) ? e : -e;
    }
    bres[(size_t)blockIdx.x * ND + tid] = r;
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
  // inscribed sphere around the mean of the distinct extremes, when that
  // integer point is strictly inside every facet (checked exactly): r^2 =
  // min over facets of (N.c - d)^2 / |N|^2 in binary64, shrunk by 2^-18 and
  // rounded down to float32 (the float32 distance test errs by far less)
  if (tid == 0) {
    P.sphere_on = 0;
    P.r2 = -1.0f;
    if (nf > 0) {
      double sx = 0, sy = 0, sz = 0;
      for (int k = 0; k < u; ++k) { sx += (double)s_px[k]; sy += (double)s_py[k]; sz += (double)s_pz[k]; }
      const long long cx = llrint(sx / u), cy = llrint(sy / u), cz = llrint(sz / u);
      double r2 = DBL_MAX;
      bool ok = true;
      for (int k = 0; k < nf && ok; ++k) {
        const long long* q = P.pl[k];
        const long long s = q[0] * cx + q[1] * cy + q[2] * cz - q[3];
        if (s >= 0) { ok = false; break; }
        const double nn = (double)q[0] * (double)q[0] + (double)q[1] * (double)q[1] + (double)q[2] * (double)q[2];
        r2 = fmin(r2, ((double)s * (double)s) / nn);
      }
      if (ok) {
        P.sphere_on = 1;
        P.cx = (float)cx;
        P.cy = (float)cy;
        P.cz = (float)cz;
        P.r2 = __double2float_rd(r2 * (1.0 - 0x1p-18));
      }
    }
  }
}

// ----------------------------------------------------------------------------
// Step 3 in 3D: the inside test and compaction of the survivors.

template <int FILTER>
__global__ void __launch_bounds__(T3) k3_filter(const float* __restrict__ xyz, int64_t n, Ws3* W,
                                                uint32_t* __restrict__ surv) {
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
    s_sp[0] = P.cx; s_sp[1] = P.cy; s_sp[2] = P.cz; s_sp[3] = P.sphere_on ? P.r2 : -1.0f;
  }
  for (int k = tid; k < MAXF3; k += T3) {
    s_pl[k][0] = P.pl[k][0]; s_pl[k][1] = P.pl[k][1]; s_pl[k][2] = P.pl[k][2]; s_pl[k][3] = P.pl[k][3];
    s_fc[k] = P.fc[k];
    s_fe[k] = P.fe[k];
  }
  __syncthreads();
  const int nf = s_nf;
  const float cx = s_sp[0], cy = s_sp[1], cz = s_sp[2], r2 = s_sp[3];
  unsigned esc = 0;
  // survives: not strictly inside every facet
  auto survives = [&](float x, float y, float z) -> bool {
    if (nf == 0) return true;
    if (FILTER == HULL_FILTER_FP32) {
      const float dx = x - cx, dy = y - cy, dz = z - cz;
      if (fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < r2) return false;
    }
    const long long X = (long long)x, Y = (long long)y, Z = (long long)z;
    for (int k = 0; k < nf; ++k) {
      if (FILTER == HULL_FILTER_FP32) {
        const float4 c = s_fc[k];
        const float s = fmaf(c.x, x, fmaf(c.y, y, fmaf(c.z, z, c.w)));
        const float e = s_fe[k];
        if (s < -e) continue;
        if (s > e) return true;
        ++esc;
      }
      if (s_pl[k][0] * X + s_pl[k][1] * Y + s_pl[k][2] * Z - s_pl[k][3] >= 0) return true;
    }
    return false;
  };
  const int64_t nq = n / 4;
  const float4* Q = reinterpret_cast<const float4*>(xyz);
  const int64_t stride = (int64_t)gridDim.x * T3;
  // whole warps iterate together: the survivors of the warp's 4 x 32 points
  // are placed with one atomic
  for (int64_t qb = (int64_t)blockIdx.x * T3 + (tid & ~31); qb < nq; qb += stride) {
    const int64_t q = qb + lane;
    bool keep[4] = {false, false, false, false};
    if (q < nq) {
      const float4 a = __ldcs(Q + 3 * q), b = __ldcs(Q + 3 * q + 1), c = __ldcs(Q + 3 * q + 2);
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
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(&W->n_surv, (unsigned long long)total);
    base = __shfl_sync(FULL, base, 31);
    unsigned long long pos = base + (unsigned long long)(pre - mine);
    for (int p = 0; p < 4; ++p)
      if (keep[p]) surv[pos++] = (uint32_t)(4 * q + p);
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

int64_t blocks3(int64_t n) {
  const int64_t nq = n / 4;
  const int64_t want = (nq + 64 * T3 - 1) / (64 * T3);  // about 64 groups of four per thread
  return std::max<int64_t>(1, std::min<int64_t>(want, std::min<int64_t>(MAX_B3, (int64_t)device_sm_count() * 8)));
}

size_t ws3_bytes(int64_t n) {
  (void)n;
  return WS3_HEADER + align_up(sizeof(BlockBest) * 18 * (size_t)MAX_B3, 256);
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
  stage_mark(0, st);
  if (cudaMemsetAsync(W, 0, sizeof(Ws3), st) != cudaSuccess) return HULL_ERR_CUDA;
  if (o.validate && n > 0) {
    const int g = (int)std::min<int64_t>((3 * n + 255) / 256, (int64_t)device_sm_count() * 8);
    k3_validate<<<g, 256, 0, st>>>(d_xyz, 3 * n, &W->status);
    count_launches(1);
  }
  stage_mark(1, st);
  const int64_t G = blocks3(n);
  const int64_t Gf = std::max<int64_t>(1, std::min<int64_t>((n / 4 + T3 - 1) / T3, (int64_t)device_sm_count() * 8));
  // stage boundaries as the 2D calls: extremes | polyhedron | inside test
#define K3(A, F)                                                                          \
  do {                                                                                    \
    k3_extremes<A, F><<<(unsigned)G, T3, 0, st>>>(d_xyz, n, &W->status, bres);            \
    stage_mark(2, st);                                                                    \
    k3_finish<A><<<1, T3, 0, st>>>(d_xyz, n, G, W, bres, d_extreme_idx);                  \
    stage_mark(3, st);                                                                    \
    k3_filter<F><<<(unsigned)Gf, T3, 0, st>>>(d_xyz, n, W, d_survivor_idx);               \
    stage_mark(4, st);                                                                    \
  } while (0)
  if (o.angles == HULL_ANGLES_CUMULATIVE) {
    if (o.filter == HULL_FILTER_FP32) K3(0, HULL_FILTER_FP32); else K3(0, HULL_FILTER_EXACT);
  } else {
    if (o.filter == HULL_FILTER_FP32) K3(1, HULL_FILTER_FP32); else K3(1, HULL_FILTER_EXACT);
  }
#undef K3
  k3_count<<<1, 1, 0, st>>>(W, d_n_survivors);
  count_launches(4);
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
