// k_extremes.cu -- Step 1 and Step 2 of the CudaPre method (arXiv 1405.3454,
// section 2): the 16 extreme points of the original and rotated point sets,
// then the convex polygon of those points by Andrew's monotone chain.  A
// streaming pass (k_extremes32 / k_extremes64) leaves one candidate per
// block and direction; a finishing kernel (one block per set) reduces them
// exactly and builds the polygon with its edge records, inner box and
// inscribed circle; k_cells builds the cell grid of the inside test.
//
// One pass over the points, streamed through shared memory by bulk copies.
// The paper's separate rotation kernels and per-direction reductions
// (section 4.2) become one fused projection + argreduction; no rotated copy
// is ever written.
//
// FP32 mode: each direction tracks a float32 value, an order-preserving
// multiple of the rotated coordinate that one fused multiply-add computes,
// with a proven error bound (internal.cuh); a tile of 8 points per thread is
// skipped for a direction when its float32 maximum cannot reach the block's
// best so far, and float32 values closer than the direction's band are
// ordered by the binary64 definition, so the chosen indices are exactly those
// of the definition.  EXACT mode evaluates the binary64 definition for every
// point.
#include <cfloat>

#include <utility>

#include "internal.cuh"
#include "proj.cuh"
#include "stream.cuh"

namespace cudapre {

namespace {

constexpr int BLOCK = 256;
constexpr int PAIRS_PER_THREAD = 4;  // 8 points per thread per step
constexpr int STEP = BLOCK * PAIRS_PER_THREAD;
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ float2 load_point(const float* xy, uint32_t i) {
  return __ldg(reinterpret_cast<const float2*>(xy) + i);
}

// Is candidate a (float32 score sa, index ia) strictly better than b for
// direction d?  Directions of group 0 compare exact float scores; rotated
// ones compare float32 scores outside the band and the binary64 definition
// inside it.  Antisymmetric for distinct indices, so butterfly reductions
// agree in every lane.
template <int ANG>
__device__ __forceinline__ bool better32(int d, float sa, uint32_t ia, float sb, uint32_t ib,
                                         const float* xy) {
  if (ia == NONE) return false;
  if (ib == NONE) return true;
  if (ia == ib) return false;
  if (d < 4) return sa > sb || (sa == sb && ia < ib);
  const float diff = sa - sb, band = band_of<ANG>(d >> 1);
  if (diff > band) return true;
  if (diff < -band) return false;
  const float2 pa = load_point(xy, ia), pb = load_point(xy, ib);
  const double ea = score64(ANG, d, pa.x, pa.y), eb = score64(ANG, d, pb.x, pb.y);
  return ea > eb || (ea == eb && ia < ib);
}

__device__ __forceinline__ void atomic_max_f(float* a, float v) {
  int* ai = reinterpret_cast<int*>(a);
  int old = *reinterpret_cast<volatile int*>(ai);
  while (__int_as_float(old) < v) {
    const int prev = atomicCAS(ai, old, __float_as_int(v));
    if (prev == old) break;
    old = prev;
  }
}
__device__ __forceinline__ void atomic_min_f(float* a, float v) {
  int* ai = reinterpret_cast<int*>(a);
  int old = *reinterpret_cast<volatile int*>(ai);
  while (__int_as_float(old) > v) {
    const int prev = atomicCAS(ai, old, __float_as_int(v));
    if (prev == old) break;
    old = prev;
  }
}

__device__ __forceinline__ float4 lds_vol4(const float* p) {
  float4 r;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.volatile.shared.v4.f32 {%0,%1,%2,%3}, [%4];"
               : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
               : "r"(a));
  return r;
}

// ----------------------------------------------------------------------------
// Step 2: the convex polygon of the extremes (Andrew's monotone chain, one
// warp), plus the per-edge records and the inner box used by Step 3.

__device__ void build_edges_and_box(Poly* P, int m, int lane, bool grid_on) {
  if (lane < m) {
    const int j = (lane + 1) % m;
    const long long ax = P->vx[lane], ay = P->vy[lane];
    const long long dx = (long long)P->vx[j] - ax, dy = (long long)P->vy[j] - ay;
    const long long A = -dy, B = dx, C = dy * ax - dx * ay;  // orient = A px + B py + C
    Edge e;
    e.A = __ll2float_rn(A);
    e.B = __ll2float_rn(B);
    e.C = __ll2float_rn(C);
    // Static bound of s = fma(A', px, fma(B', py, C')) against the exact
    // orientation for |px|, |py| <= M (primes: float32-rounded coefficients):
    //   |s - S'| <= u|A'|M + (2u + u^2)(|B'|M + |C'|)   (two fma roundings)
    //   |S' - S| <= u(|A| + |B|)M + u|C|               (coefficient roundings)
    // with u = 2^-24, M = 2^24, so uM = 1:
    //   E = |A'| + (2 + u)|B'| + (2 + u) u |C'| + |A| + |B| + u|C|,
    // evaluated in float32 rounding every step upward (a rigorous upper
    // bound; 2 + 2^-22 >= 2 + u), then doubled for safety.
    const float k2 = 2.0000002384185791f;  // 2 + 2^-22
    const float aA = __ll2float_ru(A < 0 ? -A : A), aB = __ll2float_ru(B < 0 ? -B : B);
    const float aC = __ll2float_ru(C < 0 ? -C : C);
    float E = __fadd_ru(fabsf(e.A), __fmul_ru(k2, fabsf(e.B)));
    E = __fadd_ru(E, __fmul_ru(__fmul_ru(k2, fabsf(e.C)), 0x1p-24f));
    E = __fadd_ru(E, __fadd_ru(aA, aB));
    E = __fadd_ru(E, __fmul_ru(aC, 0x1p-24f));
    e.E = 2.0f * E;
    e.ax = (int32_t)ax;
    e.ay = (int32_t)ay;
    e.dx = (int32_t)dx;
    e.dy = (int32_t)dy;
    P->e[lane] = e;
  }
  // Inner box: axis-aligned, around the centre of the bounding box with its
  // aspect (the vertex mean lies off-centre when the extremes crowd on one
  // side), grown until a corner meets an edge (float estimate),
  // rounded inward to integers and verified exactly (lane k checks edge k):
  // its 4 corners strictly inside make every point of the closed box
  // strictly inside.
  float box[4] = {1.0f, 0.0f, 1.0f, 0.0f};  // empty
  if (m >= 3) {
    int xl = P->vx[0], xh = P->vx[0], yl = P->vy[0], yh = P->vy[0];
    for (int k = 0; k < m; ++k) {
      xl = min(xl, P->vx[k]); xh = max(xh, P->vx[k]);
      yl = min(yl, P->vy[k]); yh = max(yh, P->vy[k]);
    }
    const float cx = (float)(0.5 * ((double)xl + (double)xh)), cy = (float)(0.5 * ((double)yl + (double)yh));
    const float wx = 0.5f * ((float)xh - (float)xl), wy = 0.5f * ((float)yh - (float)yl);
    float t = 1.0f;
    if (lane < m) {
      const int j = (lane + 1) % m;
      const float A = -((float)P->vy[j] - (float)P->vy[lane]), B = (float)P->vx[j] - (float)P->vx[lane];
      const float S = A * (cx - (float)P->vx[lane]) + B * (cy - (float)P->vy[lane]);
      for (int c = 0; c < 4; ++c) {
        const float sl = A * ((c & 1) ? wx : -wx) + B * ((c & 2) ? wy : -wy);
        if (sl < 0 && S > 0) t = fminf(t, S / -sl);
      }
    }
    for (int off = 16; off; off >>= 1) t = fminf(t, __shfl_xor_sync(FULL, t, off));
    t *= 0.98f;
    for (int it = 0; it < 60 && t > 1e-12f; ++it, t *= 0.5f) {
      const long long x0 = (long long)ceilf(cx - t * wx), x1 = (long long)floorf(cx + t * wx);
      const long long y0 = (long long)ceilf(cy - t * wy), y1 = (long long)floorf(cy + t * wy);
      if (x0 > x1 || y0 > y1) break;
      bool ok = true;
      if (lane < m) {
        const int j = (lane + 1) % m;
        for (int c = 0; c < 4; ++c)
          ok = ok && orient64(P->vx[lane], P->vy[lane], P->vx[j], P->vy[j], (c & 1) ? x1 : x0, (c & 2) ? y1 : y0) > 0;
      }
      if (__all_sync(FULL, ok)) {
        box[0] = (float)x0; box[1] = (float)x1; box[2] = (float)y0; box[3] = (float)y1;
        break;
      }
    }
  }
  // Inscribed circle around the box centre O: r^2 = min over the edges of
  // orient(O)^2 / (A^2 + B^2), orient exact in int64 and the quotient in
  // binary64, then shrunk by 2^-18 and rounded down to float32.  The float32
  // test fma(dx, dx, dy * dy) < cr2 under-estimates the true squared distance
  // by at most a factor (1 - 2^-24)^4, far inside that margin, so a point
  // that passes is at distance < r from O: strictly inside every edge.
  float cr2 = -1.0f;
  const bool has_box = m >= 3 && box[0] <= box[1];
  const long long cox = has_box ? (long long)floorf(0.5f * (box[0] + box[1])) : 0;
  const long long coy = has_box ? (long long)floorf(0.5f * (box[2] + box[3])) : 0;
  if (has_box) {
    double d2 = 1e300;
    if (lane < m) {
      const int j = (lane + 1) % m;
      const long long ax = P->vx[lane], ay = P->vy[lane];
      const long long dx = (long long)P->vx[j] - ax, dy = (long long)P->vy[j] - ay;
      const long long S = dx * (coy - ay) - dy * (cox - ax);  // > 0: O is strictly inside
      const double Sd = (double)S;
      d2 = (Sd * Sd) / (double)(dx * dx + dy * dy);
    }
    for (int off = 16; off; off >>= 1) d2 = fmin(d2, __shfl_xor_sync(FULL, d2, off));
    cr2 = __double2float_rd(d2 * (1.0 - 0x1p-18));
  }
  if (lane == 0) {
    P->ccx = (float)cox;
    P->ccy = (float)coy;
    P->cr2 = cr2;
    P->pad_ = 0;
    for (int c = 0; c < 4; ++c) P->box[c] = box[c];
    // An integer point strictly inside: the centre of a non-empty inner box.
    P->refine_on = box[0] <= box[1] ? 1 : 0;
    P->rox = P->refine_on ? (int)floorf(0.5f * (box[0] + box[1])) : 0;
    P->roy = P->refine_on ? (int)floorf(0.5f * (box[2] + box[3])) : 0;
    // Cell grid: smallest power-of-two cell sizes whose GRID cells, from an
    // origin aligned to the cell size, cover the bounding box.
    int xl = 0, xh = 0, yl = 0, yh = 0;
    for (int k = 0; k < m; ++k) {
      if (k == 0 || P->vx[k] < xl) xl = P->vx[k];
      if (k == 0 || P->vx[k] > xh) xh = P->vx[k];
      if (k == 0 || P->vy[k] < yl) yl = P->vy[k];
      if (k == 0 || P->vy[k] > yh) yh = P->vy[k];
    }
    int kx = 0, ky = 0;
    auto origin = [](int v, int k) { return (int)(((long long)v >> k) << k); };  // floor to 2^k
    while ((long long)xh - origin(xl, kx) >= ((long long)GRID << kx)) ++kx;
    while ((long long)yh - origin(yl, ky) >= ((long long)GRID << ky)) ++ky;
    P->kx = kx;
    P->ky = ky;
    P->gx0 = origin(xl, kx);
    P->gy0 = origin(yl, ky);
    if (!grid_on) {
      // no grid: every point of the domain falls in cell (0, 0), whose
      // entry lists every edge
      P->kx = P->ky = 30;
      P->gx0 = P->gy0 = -(1 << 25);
    }
  }
}

// ext: 16 extreme indices (NONE = absent) in shared memory; warp-wide.
__device__ void hull16_warp(const float* xy, const uint32_t* ext, Poly* P, bool grid_on) {
  __shared__ int s_x[NSLOT], s_y[NSLOT];
  __shared__ uint32_t s_i[NSLOT];
  __shared__ int s_hx[NSLOT + 1], s_hy[NSLOT + 1];
  __shared__ uint32_t s_hi[NSLOT + 1];
  __shared__ int s_m;
  const int lane = threadIdx.x & 31;
  uint32_t i = lane < NSLOT ? ext[lane] : NONE;
  const bool valid = i != NONE;
  int ix = 0, iy = 0;
  if (valid) {
    const float2 p = load_point(xy, i);
    ix = __float2int_rn(p.x);
    iy = __float2int_rn(p.y);
  }
  // Collapse duplicate indices and equal coordinates to the lowest index.
  bool dup = false;
  for (int j = 0; j < NSLOT; ++j) {
    const uint32_t ij = __shfl_sync(FULL, i, j);
    const int xj = __shfl_sync(FULL, ix, j), yj = __shfl_sync(FULL, iy, j);
    if (valid && ij != NONE && xj == ix && yj == iy && (ij < i || (ij == i && j < lane))) dup = true;
  }
  const bool keep = valid && !dup;
  // Rank by (x, y) among the kept points (coordinates are distinct now).
  int rank = 0;
  for (int j = 0; j < NSLOT; ++j) {
    const bool kj = __shfl_sync(FULL, keep, j);
    const int xj = __shfl_sync(FULL, ix, j), yj = __shfl_sync(FULL, iy, j);
    if (kj && (xj < ix || (xj == ix && yj < iy))) ++rank;
  }
  const int u = __popc(__ballot_sync(FULL, keep));
  if (keep) { s_x[rank] = ix; s_y[rank] = iy; s_i[rank] = i; }
  __syncwarp();
  if (lane == 0) {
    // Andrew's monotone chain; pop while the turn is not strictly left.
    int st[2 * NSLOT + 2];
    int k = 0;
    for (int a = 0; a < u; ++a) {
      while (k >= 2 && orient64(s_x[st[k - 2]], s_y[st[k - 2]], s_x[st[k - 1]], s_y[st[k - 1]],
                                s_x[a], s_y[a]) <= 0) --k;
      st[k++] = a;
    }
    const int lower = k + 1;
    for (int a = u - 2; a >= 0; --a) {
      while (k >= lower && orient64(s_x[st[k - 2]], s_y[st[k - 2]], s_x[st[k - 1]],
                                    s_y[st[k - 1]], s_x[a], s_y[a]) <= 0) --k;
      st[k++] = a;
    }
    int m = u <= 1 ? u : k - 1;  // last point repeats the first
    for (int a = 0; a < m; ++a) {
      s_hx[a] = s_x[st[a]];
      s_hy[a] = s_y[st[a]];
      s_hi[a] = s_i[st[a]];
    }
    s_m = m;
  }
  __syncwarp();
  const int m = s_m;
  if (lane < MAXV) {
    P->vx[lane] = lane < m ? s_hx[lane] : 0;
    P->vy[lane] = lane < m ? s_hy[lane] : 0;
    P->vidx[lane] = lane < m ? s_hi[lane] : NONE;
    P->ext[lane] = ext[lane];
  }
  if (lane == 0) P->m = m;
  __syncwarp();
  build_edges_and_box(P, m, lane, grid_on);
}

// ----------------------------------------------------------------------------
// FP32-filtered extreme search.
//
// The points stream through shared memory (stream.cuh): a producer warp
// issues bulk copies of 1024 pairs per stage and eight consumer warps take
// 8 points each per stage.  The running best of every thread and direction
// lives in shared memory: it is touched only when a tile can improve on the
// block's best, which is rare once the block-wide thresholds have risen.
// That rare path re-reads its tile from global memory (an L2 hit), so the
// streaming loop keeps no indexed arrays.  Each warp seeds the thresholds
// from its first tile with atomics; the loop has no block-wide barrier.

// Rare path, run by the whole warp when any lane's tile may improve on the
// block's best for value k (min if lo, max if hi).  Each lane picks its best
// tile point, a butterfly of exact comparisons picks the warp's, and lane 0
// merges it into the warp's running best (shared memory) and lowers the
// block threshold.  The tile is re-read from the stage in shared memory (the
// warp releases the stage only after this); f = first pair of the chunk in
// the set, cnt = its pairs.
template <int ANG>
__device__ __noinline__ void ext_slow(int k, bool lo, bool hi, int64_t f, int cnt, const float4* SP, int head,
                                      float* thr, float* wbest, uint32_t* widx, const float* xy) {
  const int tid = threadIdx.x, lane = tid & 31;
  float s_lo = -FLT_MAX, s_hi = -FLT_MAX;
  uint32_t i_lo = NONE, i_hi = NONE;
  const float t_lo = *reinterpret_cast<volatile float*>(&thr[2 * k]);
  const float t_hi = *reinterpret_cast<volatile float*>(&thr[2 * k + 1]);
  for (int j = 0; j < 8; ++j) {
    const int o = (j >> 1) * CONSUMERS + tid;
    const int oo = o < cnt ? o : 0;  // out of range: repeat a real point
    const int64_t q = f + oo;
    const float4 v = SP[oo];
    const float x = (j & 1) ? v.z : v.x, y = (j & 1) ? v.w : v.y;
    const uint32_t i = (uint32_t)(head + 2 * q) + (j & 1);
    const float val = value32<ANG>(k, x, y);
    if (lo && val <= t_lo && better32<ANG>(2 * k, -val, i, s_lo, i_lo, xy)) { s_lo = -val; i_lo = i; }
    if (hi && val >= t_hi && better32<ANG>(2 * k + 1, val, i, s_hi, i_hi, xy)) { s_hi = val; i_hi = i; }
  }
  for (int off = 16; off; off >>= 1) {
    const float a = __shfl_xor_sync(FULL, s_lo, off), b = __shfl_xor_sync(FULL, s_hi, off);
    const uint32_t ia = __shfl_xor_sync(FULL, i_lo, off), ib = __shfl_xor_sync(FULL, i_hi, off);
    if (better32<ANG>(2 * k, a, ia, s_lo, i_lo, xy)) { s_lo = a; i_lo = ia; }
    if (better32<ANG>(2 * k + 1, b, ib, s_hi, i_hi, xy)) { s_hi = b; i_hi = ib; }
  }
  if (lane == 0) {
    const float band = band_of<ANG>(k);
    if (better32<ANG>(2 * k, s_lo, i_lo, wbest[2 * k], widx[2 * k], xy)) {
      wbest[2 * k] = s_lo;
      widx[2 * k] = i_lo;
      atomic_min_f(&thr[2 * k], -s_lo + band);
    }
    if (better32<ANG>(2 * k + 1, s_hi, i_hi, wbest[2 * k + 1], widx[2 * k + 1], xy)) {
      wbest[2 * k + 1] = s_hi;
      widx[2 * k + 1] = i_hi;
      atomic_max_f(&thr[2 * k + 1], s_hi - band);
    }
  }
  __syncwarp();
}

template <int ANG>
__device__ __forceinline__ void ext_minmax(const float4& a, const float4& b, const float4& c, const float4& d,
                                           float* tmin, float* tmax) {
  // running min/max with three-input operations, two points at a time, so
  // only two points' values are live
  constexpr int NV = Dirs<ANG>::NV;
  float v[NV], w[NV];
  values32<ANG>(a.x, a.y, v);
#pragma unroll
  for (int k = 0; k < NV; ++k) { tmin[k] = v[k]; tmax[k] = v[k]; }
  auto pair = [&](float x0, float y0, float x1, float y1) {
    values32<ANG>(x0, y0, v);
    values32<ANG>(x1, y1, w);
#pragma unroll
    for (int k = 0; k < NV; ++k) { tmin[k] = min3f(tmin[k], v[k], w[k]); tmax[k] = max3f(tmax[k], v[k], w[k]); }
  };
  pair(a.z, a.w, b.x, b.y);
  pair(b.z, b.w, c.x, c.y);
  pair(c.z, c.w, d.x, d.y);
  values32<ANG>(d.z, d.w, v);
#pragma unroll
  for (int k = 0; k < NV; ++k) { tmin[k] = fminf(tmin[k], v[k]); tmax[k] = fmaxf(tmax[k], v[k]); }
}

// Warp-level seeding of the block thresholds from this warp's tile.
template <int ANG>
__device__ __forceinline__ void ext_seed(const float* tmin, const float* tmax, float* thr) {
  constexpr int NV = Dirs<ANG>::NV;
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float lo = tmin[k], hi = tmax[k];
    for (int off = 16; off; off >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(FULL, lo, off));
      hi = fmaxf(hi, __shfl_xor_sync(FULL, hi, off));
    }
    if (lane == 0) {
      const float band = band_of<ANG>(k);
      atomic_min_f(&thr[2 * k], lo + band);
      atomic_max_f(&thr[2 * k + 1], hi - band);
    }
  }
  __syncwarp();
}

// A block's result for one set (consumer warps): the binary64 score of every
// warp's candidate (one lane per direction), then an exact (score, index)
// reduction over the warps, into out[0 .. ND).  Out of line: it runs once per
// set and block, and keeps its registers out of the streaming loop.
template <int ANG>
__device__ __noinline__ void ext_block_result(const float* xy, const uint32_t* w_bidx, double* w_s64,
                                              BlockBest* out) {
  constexpr int ND = Dirs<ANG>::ND;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  consumers_sync();
  if (lane < ND) {
    const uint32_t i = w_bidx[warp * ND + lane];
    double sc = -DBL_MAX;
    if (i != NONE) {
      const float2 p = load_point(xy, i);
      sc = score64(ANG, lane, p.x, p.y);
    }
    w_s64[warp * ND + lane] = sc;
  }
  consumers_sync();
  if (tid < ND) {
    double bs = -DBL_MAX;
    unsigned long long bk = 0;
    uint32_t bi = NONE;
    for (int w = 0; w < CONSUMERS / 32; ++w) {
      const uint32_t i = w_bidx[w * ND + tid];
      const double sc = w_s64[w * ND + tid];
      const unsigned long long kk = dkey(sc);
      if (i != NONE && (bi == NONE || kk > bk || (kk == bk && i < bi))) { bs = sc; bk = kk; bi = i; }
    }
    BlockBest r;
    r.s = bs;
    r.idx = bi;
    r.pad_ = 0;
    out[tid] = r;
  }
  consumers_sync();
}

// Blocks per SM the streaming search is compiled for (registers per thread)
// and the stages of its shared-memory ring.
constexpr int EXT_MIN_BLOCKS = 2;
constexpr int64_t EXT_MIN_CHUNKS = 8;  // least chunks per block of a streaming search
constexpr int EXT_STAGES = 6;

// One set: partly dynamic shares (stream.cuh), one partial result per
// block.  A batch with units != null: static shares, then units claimed from
// *units (Split), one partial result per (share or unit, set).  Otherwise
// static shares of sp.ppb pairs, one partial result per (block, set).
template <int ANG>
__global__ void __launch_bounds__(STREAM_THREADS, EXT_MIN_BLOCKS) k_extremes32(Sets S, Split sp, uint32_t* gstatus,
                                                                   BlockBest* bres, uint32_t* units) {
  const int64_t ppb = sp.ppb;
  constexpr int NV = Dirs<ANG>::NV, ND = Dirs<ANG>::ND;
  extern __shared__ __align__(128) unsigned char dsm[];
  using SS = StreamSmemT<EXT_STAGES>;
  SS& SM = *reinterpret_cast<SS*>(dsm);
  __shared__ __align__(16) float thr[ND];  // trigger thresholds in value space
  __shared__ float w_best[CONSUMERS / 32][ND];   // per-warp running best (score space)
  __shared__ uint32_t w_bidx[CONSUMERS / 32][ND];
  __shared__ double w_s64[CONSUMERS / 32][ND];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dead = *reinterpret_cast<volatile uint32_t*>(gstatus) != 0;
  stream_init(SM);
  // one set: dynamic shares; a batch: the block's static share of the
  // virtual pair axis, set by set
  const bool dyn = S.S == 1;
  const int64_t P = S.pp_at(S.S);
  const int64_t v0 = (int64_t)blockIdx.x * ppb;
  const int64_t v1 = dead ? v0 : min(v0 + ppb, P);
  if (warp == PRODUCER_WARP) {
    if (dyn)
      stream_produce_dynamic(SM, reinterpret_cast<const float4*>(S.xy_of(0) + 2 * S.head_of(0)), S.npairs_of(0),
                             &S.h(0)->next_group[0], false, gstatus);
    else if (units)
      stream_produce_units(SM, S, sp, units, false, gstatus);
    else
      stream_produce_sets(SM, S, v0, v1, false, gstatus);
    return;
  }
  // a new set: clear the running bests and thresholds
  auto begin_set = [&]() {
    if (tid < CONSUMERS / 32 * ND) {
      (&w_best[0][0])[tid] = -FLT_MAX;
      (&w_bidx[0][0])[tid] = NONE;
    }
    if (tid < ND) thr[tid] = (tid & 1) ? -FLT_MAX : FLT_MAX;
    consumers_sync();
  };
  // one chunk in stage st: cnt pairs from pair f of the set (first: the
  // warp's first chunk of the set seeds the thresholds); the stage is
  // released after the rare path, which re-reads it
  auto chunk = [&](int st, int64_t f, int cnt, bool first, const float* xy, int head) {
    const float4* sp = SM.stage[st];
    const float4 a = sp[tid < cnt ? tid : 0];
    const float4 b = sp[tid + CONSUMERS < cnt ? tid + CONSUMERS : 0];
    const float4 cc = sp[tid + 2 * CONSUMERS < cnt ? tid + 2 * CONSUMERS : 0];
    const float4 d = sp[tid + 3 * CONSUMERS < cnt ? tid + 3 * CONSUMERS : 0];
    float tmin[NV], tmax[NV];
    ext_minmax<ANG>(a, b, cc, d, tmin, tmax);
    if (first) ext_seed<ANG>(tmin, tmax, thr);
    float t[ND];
#pragma unroll
    for (int q = 0; q < ND / 4; ++q) {
      const float4 v4 = lds_vol4(&thr[4 * q]);
      t[4 * q] = v4.x; t[4 * q + 1] = v4.y; t[4 * q + 2] = v4.z; t[4 * q + 3] = v4.w;
    }
    bool any = false;
#pragma unroll
    for (int kk = 0; kk < NV; ++kk) any |= (tmin[kk] <= t[2 * kk]) | (tmax[kk] >= t[2 * kk + 1]);
    if (__any_sync(FULL, any)) {  // rare: some lane's tile may improve a best
#pragma unroll
      for (int kk = 0; kk < NV; ++kk) {
        const bool lo2 = __any_sync(FULL, tmin[kk] <= t[2 * kk]), hi2 = __any_sync(FULL, tmax[kk] >= t[2 * kk + 1]);
        if (lo2 || hi2) ext_slow<ANG>(kk, lo2, hi2, f, cnt, sp, head, thr, w_best[warp], w_bidx[warp], xy);
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&SM.empty[st]);
  };
  if (dyn) {
    const float* xy = S.xy_of(0);
    const int head = S.head_of(0);
    const int64_t np = S.npairs_of(0);
    begin_set();
    for (int c = 0;; ++c) {
      const int id = stream_next_chunk(SM, c, gstatus);
      if (id < 0) break;
      const int64_t f = (int64_t)id * CHUNK;
      chunk(c % SS::STAGES, f, (int)min((int64_t)CHUNK, np - f), c == 0, xy, head);
    }
    ext_block_result<ANG>(xy, &w_bidx[0][0], &w_s64[0][0], bres + (size_t)blockIdx.x * ND);
    return;
  }
  if (units) {
    // the running bests carry over while the block stays in one set: each
    // segment's result (slot unit + set) is then the best over all of the
    // set's points this block has seen, still a candidate of that set
    int cur = -1;
    for (int c = 0;; ++c) {
      const ChunkMeta M = stream_next_meta(SM, c, gstatus);
      if (M.flags & META_END) break;
      const float* xy = S.xy_of(M.set);
      const bool fresh = M.set != cur;
      if (fresh) {
        begin_set();
        cur = M.set;
      }
      chunk(c % SS::STAGES, M.first, M.cnt, fresh && (M.flags & META_FIRST) != 0, xy, S.head_of(M.set));
      if (M.flags & META_LAST) {
        ext_block_result<ANG>(xy, &w_bidx[0][0], &w_s64[0][0], bres + ((size_t)M.unit + M.set) * ND);
      }
    }
    return;
  }
  int c = 0;
  bool stop = false;
  walk_segments(S, v0, v1, false, [&](int s, int64_t lo, int n) {
    const float* xy = S.xy_of(s);
    const int head = S.head_of(s);
    begin_set();
    const int nck = nchunks(n);
    for (int k = 0; k < nck; ++k, ++c) {
      const int st = c % SS::STAGES;
      if (!stop && !mbar_wait_status(&SM.full[st], (unsigned)((c / SS::STAGES) & 1), gstatus)) stop = true;
      if (stop) continue;
      const int f = k * CHUNK;
      chunk(st, lo + f, min(CHUNK, n - f), k == 0, xy, head);
    }
    ext_block_result<ANG>(xy, &w_bidx[0][0], &w_s64[0][0], bres + ((size_t)blockIdx.x + s) * ND);
  });
}

// ----------------------------------------------------------------------------
// EXACT mode: the binary64 definition for every point.

template <int ANG>
__global__ void __launch_bounds__(BLOCK) k_extremes64(Sets S, int64_t ppb, const uint32_t* gstatus,
                                                       BlockBest* blockres) {
  constexpr int NV = Dirs<ANG>::NV, ND = Dirs<ANG>::ND;
  __shared__ double s_red[BLOCK / 32][ND];
  __shared__ uint32_t s_redi[BLOCK / 32][ND];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(gstatus) != 0;
  double best[ND];
  uint32_t bidx[ND];

  auto offer = [&](float x, float y, uint32_t i) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      // group 0 is the original set: x' = x, y' = y exactly
      const double v = k == 0 ? (double)x : (k == 1 ? (double)y : value64(ANG, k, x, y));
      if (bidx[2 * k] == NONE || -v > best[2 * k] || (-v == best[2 * k] && i < bidx[2 * k])) {
        best[2 * k] = -v; bidx[2 * k] = i;
      }
      if (bidx[2 * k + 1] == NONE || v > best[2 * k + 1] || (v == best[2 * k + 1] && i < bidx[2 * k + 1])) {
        best[2 * k + 1] = v; bidx[2 * k + 1] = i;
      }
    }
  };

  const int64_t P = S.pp_at(S.S);
  const int64_t v0 = (int64_t)blockIdx.x * ppb;
  const int64_t v1 = dead ? v0 : min(v0 + ppb, P);
  walk_segments(S, v0, v1, false, [&](int s, int64_t lo, int n) {
#pragma unroll
    for (int d = 0; d < ND; ++d) { best[d] = -DBL_MAX; bidx[d] = NONE; }
    const int head = S.head_of(s);
    const float4* Pp = reinterpret_cast<const float4*>(S.xy_of(s) + 2 * head) + lo;
    const uint32_t ibase = (uint32_t)(head + 2 * lo);
    for (int f = 0; f < n; f += STEP) {
#pragma unroll
      for (int j = 0; j < PAIRS_PER_THREAD; ++j) {
        const int o = f + j * BLOCK + tid;
        if (o < n) {
          const float4 v = __ldcs(Pp + o);
          const uint32_t i = ibase + 2u * (uint32_t)o;
          offer(v.x, v.y, i);
          offer(v.z, v.w, i + 1);
        }
      }
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      double sc = best[d];
      uint32_t i = bidx[d];
      for (int off = 16; off; off >>= 1) {
        const double so = __shfl_xor_sync(FULL, sc, off);
        const uint32_t io = __shfl_xor_sync(FULL, i, off);
        if (io != NONE && (i == NONE || so > sc || (so == sc && io < i))) { sc = so; i = io; }
      }
      if (lane == 0) { s_red[warp][d] = sc; s_redi[warp][d] = i; }
    }
    __syncthreads();
    if (warp == 0) {
      for (int d = 0; d < ND; ++d) {
        double sc = lane < BLOCK / 32 ? s_red[lane][d] : -DBL_MAX;
        uint32_t i = lane < BLOCK / 32 ? s_redi[lane][d] : NONE;
        for (int off = 16; off; off >>= 1) {
          const double so = __shfl_xor_sync(FULL, sc, off);
          const uint32_t io = __shfl_xor_sync(FULL, i, off);
          if (io != NONE && (i == NONE || so > sc || (so == sc && io < i))) { sc = so; i = io; }
        }
        if (lane == 0) {
          BlockBest r;
          r.s = sc; r.idx = i; r.pad_ = 0;
          blockres[((size_t)blockIdx.x + s) * ND + d] = r;
        }
      }
    }
    __syncthreads();
  });
}

// ----------------------------------------------------------------------------
// Finishing kernel (one block): the exact reduction of all candidates, the
// 16 extremes, Step 2 (the polygon, its edge records and inner box) and the
// cell grid of the inside test.

template <int ANG, int FIN_THREADS>
__global__ void __launch_bounds__(FIN_THREADS) k_ext_finish(Sets S, Split sp, const uint32_t* gstatus,
                                                               const BlockBest* bres, uint32_t* ext_out,
                                                               uint16_t* cells_base, uint32_t* surv_idx,
                                                               unsigned long long* surv_key) {
  static_assert(FIN_THREADS % 32 == 0 && FIN_THREADS <= 1024, "whole warps");
  constexpr int ND = Dirs<ANG>::ND;
  __shared__ uint32_t s_ext[NSLOT];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int set = blockIdx.x;
  WsHeader* h = S.h(set);
  const float* xy = S.xy_of(set);
  const int64_t n = S.n_of(set);
  const int head = S.head_of(set);
  uint16_t* cells = cells_base + (size_t)set * (CELL_BYTES / 2);
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(gstatus) != 0 ||
                    *reinterpret_cast<volatile uint32_t*>(&h->status) != 0;
  // this set's partial results (Split): slots [e0, e1) of the static
  // shares that meet the set, then [f0, f1) of the units that meet it
  int64_t e0 = 0, e1 = 0, f0 = 0, f1 = 0;
  if (!dead && S.npairs_of(set) > 0) {
    const int64_t p0 = S.pp_at(set), p1 = S.pp_at(set + 1);
    if (p0 < sp.A) {
      e0 = p0 / sp.ppb + set;
      e1 = (min(p1, sp.A) - 1) / sp.ppb + set + 1;
    }
    if (p1 > sp.A) {
      f0 = sp.G + (max(p0, sp.A) - sp.A) / sp.U + set;
      f1 = sp.G + (p1 - 1 - sp.A) / sp.U + set + 1;
    }
  }
  const int64_t n_e = e1 - e0, n_all = n_e + (f1 - f0);
  // points outside the 16-byte pairs: the head point and an odd last point
  const bool lead = !dead && head == 1;
  const bool trail = !dead && n > head && ((n - head) & 1);
  // One warp per direction: its lanes take the set's block results (and the
  // loose points) in turn, then an exact butterfly by (score key, index).
  for (int d = warp; d < ND; d += FIN_THREADS / 32) {
    unsigned long long ks = 0;
    uint32_t bi = NONE;
    auto take = [&](unsigned long long k, uint32_t i) {
      return i != NONE && (bi == NONE || k > ks || (k == ks && i < bi));
    };
    for (int64_t q = lane; q < n_all; q += 32) {
      const int64_t e = q < n_e ? e0 + q : f0 + (q - n_e);
      const BlockBest b = bres[e * ND + d];
      const unsigned long long k = dkey(b.s);
      if (take(k, b.idx)) { ks = k; bi = b.idx; }
    }
    if (lane < 2 && (lane == 0 ? lead : trail)) {
      const uint32_t i = lane == 0 ? 0u : (uint32_t)(n - 1);
      const float2 p = load_point(xy, i);
      const unsigned long long k = dkey(score64(ANG, d, p.x, p.y));
      if (take(k, i)) { ks = k; bi = i; }
    }
    for (int off = 16; off; off >>= 1) {
      const uint32_t io = __shfl_xor_sync(FULL, bi, off);
      const unsigned long long ko = __shfl_xor_sync(FULL, ks, off);
      if (take(ko, io)) { ks = ko; bi = io; }
    }
    if (lane == 0) s_ext[d] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    if (ANG == 0) {
      // 120 degrees from 30 degrees: with the correctly rounded constants,
      // x'(120) = -y'(30) and y'(120) = x'(30) exactly.
      s_ext[12] = s_ext[7];  // argmin x'120 = argmax y'30
      s_ext[13] = s_ext[6];  // argmax x'120 = argmin y'30
      s_ext[14] = s_ext[4];  // argmin y'120 = argmin x'30
      s_ext[15] = s_ext[5];  // argmax y'120 = argmax x'30
    }
    if (dead) for (int k = 0; k < NSLOT; ++k) s_ext[k] = NONE;
  }
  __syncthreads();
  // Sets below GRID_MIN_POINTS get no cell grid (its construction would cost
  // more than the cell lookups save).
  const bool grid_on = n >= GRID_MIN_POINTS;
  if (warp == 0) {
    if (ext_out && lane < NSLOT) ext_out[(size_t)set * NSLOT + lane] = s_ext[lane];
    hull16_warp(xy, s_ext, &h->poly, grid_on);
  }
  __syncthreads();
  // The loose points' inside test (Step 3): exact against every edge.
  if (!dead && tid == 0) {
    const int mm = h->poly.m;
    for (int r = 0; r < 2; ++r) {
      if (!(r == 0 ? lead : trail)) continue;
      const uint32_t i = r == 0 ? 0u : (uint32_t)(n - 1);
      const float2 p = load_point(xy, i);
      const long long px = __float2ll_rn(p.x), py = __float2ll_rn(p.y);
      bool inside = mm >= 3;
      for (int k = 0; k < mm && inside; ++k) {
        const Edge& e = h->poly.e[k];
        inside = (long long)e.dx * (py - e.ay) - (long long)e.dy * (px - e.ax) > 0;
      }
      if (!inside) {
        const unsigned long long pos = atomicAdd(&h->n_surv, 1ull);
        surv_idx[S.off_at(set) + pos] = i;
        if (surv_key) surv_key[S.off_at(set) + pos] = point_key((int32_t)px, (int32_t)py);
      }
    }
  }
  // Sets below GRID_MIN_POINTS use one cell listing every edge (the cell
  // grid of larger sets is built by k_cells).
  const int m = h->poly.m;
  if (dead || m < 3) return;
  if (!grid_on && tid == 0) {
    cells[0] = (uint16_t)((1u << m) - 1u);
    reinterpret_cast<uint8_t*>(cells + GRID * GRID)[0] = (uint8_t)CELL_MULTI;
  }
}

// ----------------------------------------------------------------------------
// The cell grid of the inside test, in groups of CELL_ROWS rows spread over
// the blocks of a set.  For edge k the orientation is A x + B y + C (exact
// int64); its minimum over a cell is the minimum of A x over the cell's
// columns plus that of B y over its rows plus C (corners), likewise the
// maximum.  Bit k of a cell's mask: some point of the cell may fail edge k;
// a cell entirely outside edge k keeps only bit k.  Byte code: 0 inside,
// k + 1 only edge k, CELL_MULTI several edges.
constexpr int CELL_THREADS = 256;

// CELL_ROWS rows per group: a single set spreads 2-row groups over 64
// blocks (latency), a batch takes 8-row groups in one block per set.
template <int CELL_ROWS>
__global__ void __launch_bounds__(CELL_THREADS) k_cells(Sets S, const uint32_t* gstatus, uint16_t* cells_base) {
  // blockIdx.y takes every gridDim.y-th group of CELL_ROWS rows
  __shared__ long long s_ax[MAXV][GRID];       // per edge: min of A x per column
  __shared__ long long s_by[MAXV][CELL_ROWS];  // per edge: min of B y per row (this block's rows)
  __shared__ long long s_c[MAXV], s_span[MAXV];
  __shared__ int s_ra[CELL_ROWS], s_rb[CELL_ROWS];  // per row: columns inside every edge
  const int set = blockIdx.x, tid = threadIdx.x;
  const WsHeader* h = S.h(set);
  if (*reinterpret_cast<const volatile uint32_t*>(gstatus) || h->status) return;
  if (S.n_of(set) < GRID_MIN_POINTS) return;  // one cell listing every edge (finishing kernel)
  const Poly& P = h->poly;
  const int m = P.m;
  if (m < 3) return;
  uint16_t* cells = cells_base + (size_t)set * (CELL_BYTES / 2);
  const int kx = P.kx, ky = P.ky;
  for (int t = tid; t < m * GRID; t += CELL_THREADS) {
    const int k = t / GRID, c = t % GRID;
    const Edge& e = P.e[k];
    const long long A = -(long long)e.dy;
    const long long xa = (long long)P.gx0 + ((long long)c << kx), xb = xa + (1ll << kx) - 1;
    s_ax[k][c] = min(A * xa, A * xb);
    if (c == 0) {
      const long long B = e.dx;
      s_c[k] = (long long)e.dy * e.ax - (long long)e.dx * e.ay;
      // max - min over a cell: |A| (2^kx - 1) + |B| (2^ky - 1)
      s_span[k] = (A < 0 ? -A : A) * ((1ll << kx) - 1) + (B < 0 ? -B : B) * ((1ll << ky) - 1);
    }
  }
  for (int r0 = blockIdx.y * CELL_ROWS; r0 < GRID; r0 += gridDim.y * CELL_ROWS) {
    __syncthreads();
    for (int t = tid; t < m * CELL_ROWS; t += CELL_THREADS) {
      const int k = t / CELL_ROWS, row = t % CELL_ROWS;
      const long long B = P.e[k].dx;
      const long long ya = (long long)P.gy0 + ((long long)(r0 + row) << ky), yb = ya + (1ll << ky) - 1;
      s_by[k][row] = min(B * ya, B * yb);
    }
    if (tid < CELL_ROWS) { s_ra[tid] = 0; s_rb[tid] = GRID - 1; }
    __syncthreads();
    // Per row, the columns whose cells lie strictly inside every edge: the row
    // term is fixed and the column term min(A x) is monotone in the column
    // (increasing for A > 0, decreasing for A < 0), so "inside edge k" is a
    // half-line of columns, found by binary search; the row's interval is
    // their intersection.  Cells in it get code 0 at once.
    for (int t = tid; t < m * CELL_ROWS; t += CELL_THREADS) {
      const int k = t / CELL_ROWS, row = t % CELL_ROWS;
      const long long A = -(long long)P.e[k].dy;
      const long long rb = s_by[k][row] + s_c[k];
      if (A == 0) {
        if (s_ax[k][0] + rb <= 0) atomicMax(&s_ra[row], GRID);  // the whole row may fail edge k
      } else if (A > 0) {  // inside for columns >= the first passing one
        int lo = 0, hi = GRID;
        while (lo < hi) { const int mid = (lo + hi) >> 1; if (s_ax[k][mid] + rb > 0) hi = mid; else lo = mid + 1; }
        atomicMax(&s_ra[row], lo);
      } else {             // inside for columns <= the last passing one
        int lo = -1, hi = GRID - 1;
        while (lo < hi) { const int mid = (lo + hi + 1) >> 1; if (s_ax[k][mid] + rb > 0) lo = mid; else hi = mid - 1; }
        atomicMin(&s_rb[row], lo);
      }
    }
    __syncthreads();
    uint8_t* code8 = reinterpret_cast<uint8_t*>(cells + GRID * GRID);
    for (int t = tid; t < CELL_ROWS * GRID; t += CELL_THREADS) {
      const int cx = t & (GRID - 1), row = t >> GRID_LOG;
      const int c = (r0 + row) * GRID + cx;
      uint32_t mask = 0;
      if (cx < s_ra[row] || cx > s_rb[row]) {
        for (int k = 0; k < m; ++k) {
          const long long mn = s_ax[k][cx] + s_by[k][row] + s_c[k];
          if (mn + s_span[k] <= 0) { mask = 1u << k; break; }  // the cell's maximum
          if (mn <= 0) mask |= 1u << k;
        }
      }
      cells[c] = (uint16_t)mask;
      code8[c] = mask == 0 ? 0 : ((mask & (mask - 1)) == 0 ? (uint8_t)__ffs(mask) : (uint8_t)CELL_MULTI);
    }
  }
}

// Domain check (finite, integer-valued, |v| <= 2^24).
__global__ void k_validate(const float* __restrict__ xy, int64_t n2, uint32_t* status) {
  bool bad = false;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n2;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float v = __ldg(xy + k);
    bad |= !(fabsf(v) <= 16777216.0f) || truncf(v) != v;  // NaN fails the first test
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, HULL_DEVICE_DOMAIN);
}

template <typename K>
int occupancy(K kernel) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, BLOCK, 0) != cudaSuccess || b < 1) b = 1;
  return b;
}

}  // namespace

cudaError_t launch_validate(const float* xy, int64_t n, uint32_t* status, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int64_t want = (2 * n + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)device_sm_count() * 8);
  k_validate<<<grid, 256, 0, st>>>(xy, 2 * n, status);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_extremes(const Sets& S, int64_t pairs_bound, int angles, int filter, uint32_t* gstatus,
                            void* partials, uint16_t* cells, LaunchShape ls, uint32_t* ext_out, uint32_t* surv_idx,
                            unsigned long long* surv_key, cudaStream_t st, uint32_t* units) {
  const int64_t npairs = std::max<int64_t>(pairs_bound, 0);
  BlockBest* bres = static_cast<BlockBest*>(partials);
  const unsigned nsets = (unsigned)S.S;
  // blocks and pairs per block: at most one wave of resident blocks, each
  // share a whole number of chunks
  auto shape = [&](int occ) {
    const int64_t resident = (int64_t)device_sm_count() * std::max(occ, 1);
    int64_t G = ls.grid > 0 ? ls.grid : resident * stream_waves(S.S, npairs, resident, ls.waves);
    G = std::min<int64_t>(G, MAX_STREAM_BLOCKS);
    // small inputs: at least EXT_MIN_CHUNKS chunks per block (each block pays
    // a set-up, a threshold warm-up and a block result; the finishing kernel
    // one partial result per block)
    if (ls.grid <= 0) G = std::min<int64_t>(G, ((npairs + CHUNK - 1) / CHUNK + EXT_MIN_CHUNKS - 1) / EXT_MIN_CHUNKS);
    G = std::max<int64_t>(1, std::min<int64_t>(G, (npairs + CHUNK - 1) / CHUNK));
    int64_t ppb = (npairs + G - 1) / G;
    ppb = (ppb + CHUNK - 1) / CHUNK * CHUNK;
    if (ppb == 0) ppb = CHUNK;
    G = std::max<int64_t>(1, (npairs + ppb - 1) / ppb);
    return std::make_pair(G, ppb);
  };
  // The finishing kernel: one block per set, 1024 threads for a single set
  // (its cell grid in one pass), 256 for a batch (more sets resident).
#define FIN(A)                                                                                           \
  do {                                                                                                   \
    if (S.S == 1)                                                                                        \
      k_ext_finish<A, 1024><<<nsets, 1024, 0, st>>>(S, sp, gstatus, bres, ext_out, cells, surv_idx, surv_key); \
    else                                                                                                 \
      k_ext_finish<A, 256><<<nsets, 256, 0, st>>>(S, sp, gstatus, bres, ext_out, cells, surv_idx, surv_key);   \
  } while (0)
  if (filter == HULL_FILTER_FP32) {
    const size_t dsmem = sizeof(StreamSmemT<EXT_STAGES>);
    static bool attr[64][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr[dev][angles]) {
      cudaError_t e = angles == HULL_ANGLES_CUMULATIVE
                          ? cudaFuncSetAttribute(k_extremes32<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem)
                          : cudaFuncSetAttribute(k_extremes32<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
      if (e != cudaSuccess) return e;
      attr[dev][angles] = true;
    }
    int occ = 0;
    if (angles == HULL_ANGLES_CUMULATIVE)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_extremes32<0>, STREAM_THREADS, dsmem);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_extremes32<1>, STREAM_THREADS, dsmem);
    auto gp = shape(occ);
    Split sp{gp.second, npairs, 1, gp.first};
    uint32_t* un = nullptr;
    if (S.S > 1 && units) {
      // a batch: one wave of resident blocks, static shares of the first
      // DYN_STATIC_PCT percent of the pair axis, then units claimed
      // dynamically (partial slots: G + npairs / CHUNK + 1 + S at most)
      const int64_t resident = (int64_t)device_sm_count() * std::max(occ, 1);
      const int64_t G = ls.grid > 0 ? std::min<int64_t>(ls.grid, MAX_STREAM_BLOCKS) : resident;
      sp.G = G;
      sp.ppb = npairs * DYN_STATIC_PCT / 100 / G / CHUNK * CHUNK;
      sp.A = sp.ppb * G;
      if (sp.ppb == 0) { sp.ppb = CHUNK; sp.A = 0; }
      sp.U = unit_pairs(npairs - sp.A, G, EXT_UNIT_CHUNKS);
      gp.first = G;
      un = units;
    }
    if (angles == HULL_ANGLES_CUMULATIVE) {
      k_extremes32<0><<<(unsigned)gp.first, STREAM_THREADS, dsmem, st>>>(S, sp, gstatus, bres, un);
      stage_mark(2, st);
      FIN(0);
    } else {
      k_extremes32<1><<<(unsigned)gp.first, STREAM_THREADS, dsmem, st>>>(S, sp, gstatus, bres, un);
      stage_mark(2, st);
      FIN(1);
    }
  } else {
    const int occ = angles == HULL_ANGLES_CUMULATIVE ? occupancy(k_extremes64<0>) : occupancy(k_extremes64<1>);
    const auto gp = shape(occ);
    const Split sp{gp.second, npairs, 1, gp.first};
    if (angles == HULL_ANGLES_CUMULATIVE) {
      k_extremes64<0><<<(unsigned)gp.first, BLOCK, 0, st>>>(S, gp.second, gstatus, bres);
      stage_mark(2, st);
      FIN(0);
    } else {
      k_extremes64<1><<<(unsigned)gp.first, BLOCK, 0, st>>>(S, gp.second, gstatus, bres);
      stage_mark(2, st);
      FIN(1);
    }
  }
#undef FIN
  // one set: its rows over GRID / 2 blocks; a batch: one block per set
  if (S.S == 1)
    k_cells<2><<<dim3(nsets, GRID / 2), CELL_THREADS, 0, st>>>(S, gstatus, cells);
  else
    k_cells<8><<<dim3(nsets, 1), CELL_THREADS, 0, st>>>(S, gstatus, cells);
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace cudapre
