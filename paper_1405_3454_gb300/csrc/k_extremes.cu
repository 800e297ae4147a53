// k_extremes.cu -- Step 1 and Step 2 of the CudaPre method (arXiv 1405.3454,
// section 2): the 16 extreme points of the original and rotated point sets,
// then the convex polygon of those points by Andrew's monotone chain, all in
// one launch (the last block to finish runs the polygon stage).
//
// One pass over the points: each thread loads two points per 16-byte load and
// keeps, for every direction, its best candidate.  The paper's separate
// rotation kernels and per-direction reductions (section 4.2) become one
// fused projection + argreduction; no rotated copy is ever written.
//
// FP32 mode: projections are float32 (<= 2.5 from the binary64 definition);
// a tile of 8 points per thread is skipped for a direction when its float32
// maximum cannot reach the block's best so far, and float32 scores closer
// than BAND are ordered by the binary64 definition, so the chosen indices are
// exactly those of the definition.  EXACT mode evaluates the binary64
// definition for every point.
#include <cfloat>

#include "internal.cuh"

namespace cudapre {

namespace {

constexpr int BLOCK = 256;
constexpr int PAIRS_PER_THREAD = 4;  // 8 points per thread per step
constexpr int STEP = BLOCK * PAIRS_PER_THREAD;
constexpr unsigned FULL = 0xFFFFFFFFu;

template <int ANG>
struct Dirs {
  static constexpr int NV = ANG == 0 ? 6 : 8;  // projected values per point
  static constexpr int ND = 2 * NV;            // directions = extreme slots computed
};

// (cos, sin) of rotation group g.  Cumulative: 0, 30, 75, 120 degrees;
// absolute: 0, 30, 45, 60 degrees (section 2 Step 1, Figure 1).
__device__ __forceinline__ void rot_cs(int ang, int g, double& c, double& s) {
  if (g == 0) { c = 1.0; s = 0.0; return; }
  if (g == 1) { c = K_S3; s = 0.5; return; }
  if (ang == 0) {
    if (g == 2) { c = K_C75; s = K_S75; } else { c = -0.5; s = K_S3; }
  } else {
    if (g == 2) { c = K_H; s = K_H; } else { c = 0.5; s = K_S3; }
  }
}

// Binary64 definition of value v (group v/2, axis v%2):
//   axis 0: RN(RN(x*c) - RN(y*s)),  axis 1: RN(RN(x*s) + RN(y*c)).
__device__ __forceinline__ double value64(int ang, int v, float xf, float yf) {
  double c, s;
  rot_cs(ang, v >> 1, c, s);
  double x = (double)xf, y = (double)yf;
  if ((v & 1) == 0) return __dsub_rn(__dmul_rn(x, c), __dmul_rn(y, s));
  return __dadd_rn(__dmul_rn(x, s), __dmul_rn(y, c));
}

// Score of direction d = 2v + k: value for k = 1 (max), -value for k = 0.
__device__ __forceinline__ double score64(int ang, int d, float x, float y) {
  double v = value64(ang, d >> 1, x, y);
  return (d & 1) ? v : -v;
}

// Float32 values of one point (error <= 2.5 against value64, see E_PROJ).
template <int ANG>
__device__ __forceinline__ void values32(float x, float y, float* v) {
  v[0] = x;
  v[1] = y;
  const float hx = 0.5f * x, hy = 0.5f * y;
  v[2] = fmaf(x, F_S3, -hy);  // x s3 - y/2
  v[3] = fmaf(y, F_S3, hx);   // x/2 + y s3
  if (ANG == 0) {
    const float p = y * F_S75, q = y * F_C75;
    v[4] = fmaf(x, F_C75, -p);  // x c75 - y s75
    v[5] = fmaf(x, F_S75, q);   // x s75 + y c75
  } else {
    const float a = x * F_H, b = y * F_H;
    v[4] = a - b;               // (x - y) h
    v[5] = a + b;               // (x + y) h
    v[6] = fmaf(-y, F_S3, hx);  // x/2 - y s3
    v[7] = fmaf(x, F_S3, hy);   // x s3 + y/2
  }
}

template <int ANG>
__device__ __forceinline__ float value32(int v, float x, float y) {
  float t[Dirs<ANG>::NV];
  values32<ANG>(x, y, t);
  return t[v];
}

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
  const float diff = sa - sb;
  if (diff > BAND) return true;
  if (diff < -BAND) return false;
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

// Offer point (x, y, i) with float32 value `val` to direction d's running
// best of this thread; on a win, lower the block's trigger threshold.
template <int ANG>
__device__ __forceinline__ void offer32(int d, float val, float x, float y, uint32_t i,
                                        float& best, uint32_t& bidx, float* thr,
                                        const float* xy) {
  const float s = (d & 1) ? val : -val;
  bool take;
  if (bidx == NONE) {
    take = true;
  } else if (d < 4) {
    take = s > best || (s == best && i < bidx);
  } else {
    const float diff = s - best;
    if (diff > BAND) {
      take = true;
    } else if (diff < -BAND) {
      take = false;
    } else {
      const float2 pb = load_point(xy, bidx);
      const double e = score64(ANG, d, x, y), eb = score64(ANG, d, pb.x, pb.y);
      take = e > eb || (e == eb && i < bidx);
    }
  }
  if (take) {
    best = s;
    bidx = i;
    const float band = d < 4 ? 0.0f : BAND;
    if (d & 1) atomic_max_f(&thr[d], val - band);
    else atomic_min_f(&thr[d], val + band);
  }
}

// ----------------------------------------------------------------------------
// Step 2: the convex polygon of the extremes (Andrew's monotone chain, one
// warp), plus the per-edge records and the inner box used by Step 3.

__device__ void build_edges_and_box(Poly* P, int m, int lane) {
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
    // with u = 2^-24, M = 2^24; doubled for safety and rounded up.
    const double u = 0x1p-24, M = 16777216.0;
    const double bnd = u * fabs((double)e.A) * M +
                       (2.0 * u + u * u) * (fabs((double)e.B) * M + fabs((double)e.C)) +
                       u * (fabs((double)A) + fabs((double)B)) * M + u * fabs((double)C);
    e.E = __double2float_ru(2.0 * bnd);
    e.ax = (int32_t)ax;
    e.ay = (int32_t)ay;
    e.dx = (int32_t)dx;
    e.dy = (int32_t)dy;
    P->e[lane] = e;
  }
  if (lane == 0) {
    float box[4] = {1.0f, 0.0f, 1.0f, 0.0f};  // empty
    if (m >= 3) {
      // Axis-aligned box around the vertex mean with the aspect of the
      // bounding box, grown until a corner meets an edge (double), rounded
      // inward to integers and then verified exactly: its 4 corners strictly
      // inside make every point of the closed box strictly inside.
      double cx = 0, cy = 0;
      int xl = P->vx[0], xh = P->vx[0], yl = P->vy[0], yh = P->vy[0];
      for (int k = 0; k < m; ++k) {
        cx += P->vx[k];
        cy += P->vy[k];
        xl = min(xl, P->vx[k]); xh = max(xh, P->vx[k]);
        yl = min(yl, P->vy[k]); yh = max(yh, P->vy[k]);
      }
      cx /= m;
      cy /= m;
      const double wx = 0.5 * ((double)xh - xl), wy = 0.5 * ((double)yh - yl);
      double t = 1.0;
      for (int k = 0; k < m; ++k) {
        const int j = (k + 1) % m;
        const double A = -((double)P->vy[j] - P->vy[k]), B = (double)P->vx[j] - P->vx[k];
        const double S = A * (cx - P->vx[k]) + B * (cy - P->vy[k]);
        for (int c = 0; c < 4; ++c) {
          const double sl = A * ((c & 1) ? wx : -wx) + B * ((c & 2) ? wy : -wy);
          if (sl < 0 && S > 0) t = fmin(t, S / -sl);
        }
      }
      t *= 0.98;
      for (int it = 0; it < 60 && t > 1e-12; ++it, t *= 0.5) {
        const long long x0 = (long long)ceil(cx - t * wx), x1 = (long long)floor(cx + t * wx);
        const long long y0 = (long long)ceil(cy - t * wy), y1 = (long long)floor(cy + t * wy);
        if (x0 > x1 || y0 > y1) break;
        bool ok = true;
        for (int c = 0; c < 4 && ok; ++c) {
          const long long px = (c & 1) ? x1 : x0, py = (c & 2) ? y1 : y0;
          for (int k = 0; k < m && ok; ++k) {
            const int j = (k + 1) % m;
            ok = orient64(P->vx[k], P->vy[k], P->vx[j], P->vy[j], px, py) > 0;
          }
        }
        if (ok) {
          box[0] = (float)x0; box[1] = (float)x1; box[2] = (float)y0; box[3] = (float)y1;
          break;
        }
      }
    }
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
  }
}

// ext: 16 extreme indices (NONE = absent) in shared memory; warp-wide.
__device__ void hull16_warp(const float* xy, const uint32_t* ext, Poly* P) {
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
  build_edges_and_box(P, m, lane);
}

// ----------------------------------------------------------------------------
// Grid-level reduction of the per-block bests (binary64 scores, exact), run
// by the last block; then Step 2.

template <int ANG>
__device__ void finish_last_block(const float* xy, int64_t n, WsHeader* h,
                                  const BlockBest* blockres, uint32_t* ext_out) {
  constexpr int ND = Dirs<ANG>::ND;
  __shared__ uint32_t s_ext[NSLOT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int G = gridDim.x;
  for (int d = warp; d < ND; d += nwarps) {
    double bs = -DBL_MAX;
    uint32_t bi = NONE;
    for (int k = lane; k < G; k += 32) {
      const double s = __ldcg(&blockres[(size_t)k * ND + d].s);
      const uint32_t i = __ldcg(&blockres[(size_t)k * ND + d].idx);
      if (i != NONE && (bi == NONE || s > bs || (s == bs && i < bi))) { bs = s; bi = i; }
    }
    for (int off = 16; off; off >>= 1) {
      const double so = __shfl_xor_sync(FULL, bs, off);
      const uint32_t io = __shfl_xor_sync(FULL, bi, off);
      if (io != NONE && (bi == NONE || so > bs || (so == bs && io < bi))) { bs = so; bi = io; }
    }
    if (lane == 0) s_ext[d] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (ANG == 0) {
      // 120 degrees from 30 degrees: with the correctly rounded constants,
      // x'(120) = -y'(30) and y'(120) = x'(30) exactly.
      s_ext[12] = s_ext[7];  // argmin x'120 = argmax y'30
      s_ext[13] = s_ext[6];  // argmax x'120 = argmin y'30
      s_ext[14] = s_ext[4];  // argmin y'120 = argmin x'30
      s_ext[15] = s_ext[5];  // argmax y'120 = argmax x'30
    }
    if (h->status) for (int k = 0; k < NSLOT; ++k) s_ext[k] = NONE;
  }
  __syncthreads();
  if (warp == 0) {
    if (ext_out && lane < NSLOT) ext_out[lane] = s_ext[lane];
    hull16_warp(xy, s_ext, &h->poly);
  }
}

template <int ANG>
__device__ bool last_block_arrives(WsHeader* h) {
  __shared__ bool s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&h->done_blocks, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) __threadfence();
  return s_last;
}

// ----------------------------------------------------------------------------
// FP32-filtered extreme search.
//
// The running best of every thread and direction lives in shared memory: it
// is touched only when a tile can improve on the block's best, which is rare
// once the block-wide thresholds have risen.  The streaming loop therefore
// keeps only the current and the next tile in registers (8 points each), so
// four blocks fit on an SM and 32 bytes per thread are always in flight.

template <int ANG>
__global__ void __launch_bounds__(BLOCK, 3) k_extremes32(const float* __restrict__ xy, int64_t n,
                                                          int head, int64_t npairs, int64_t ppb,
                                                          WsHeader* h, BlockBest* blockres,
                                                          uint32_t* ext_out) {
  constexpr int NV = Dirs<ANG>::NV, ND = Dirs<ANG>::ND;
  __shared__ __align__(16) float thr[ND];  // trigger thresholds in value space
  __shared__ float s_best[ND][BLOCK];
  __shared__ uint32_t s_bidx[ND][BLOCK];
  __shared__ float s_red[BLOCK / 32][ND];
  __shared__ uint32_t s_redi[BLOCK / 32][ND];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dead = *reinterpret_cast<volatile uint32_t*>(&h->status) != 0;
#pragma unroll
  for (int d = 0; d < ND; ++d) { s_best[d][tid] = -FLT_MAX; s_bidx[d][tid] = NONE; }

  const float4* P = reinterpret_cast<const float4*>(xy + 2 * head);
  const int64_t p0 = (int64_t)blockIdx.x * ppb;
  const int64_t p1 = dead ? p0 : min(p0 + ppb, npairs);
  const int64_t nsteps = p1 > p0 ? (p1 - p0 + STEP - 1) / STEP : 0;

  float4 cur[PAIRS_PER_THREAD];
  auto load = [&](int64_t base, float4* v) {
#pragma unroll
    for (int j = 0; j < PAIRS_PER_THREAD; ++j) {
      const int64_t pp = base + j * BLOCK + tid;
      v[j] = __ldg(P + (pp < p1 ? pp : p0));  // out of range: repeat a real point
    }
  };
  if (nsteps > 0) load(p0, cur);
  for (int64_t st = 0; st < nsteps; ++st) {
    const int64_t base = p0 + st * BLOCK * PAIRS_PER_THREAD;
    float4 nxt[PAIRS_PER_THREAD];
    if (st + 1 < nsteps) load(base + STEP, nxt);
    float px[2 * PAIRS_PER_THREAD], py[2 * PAIRS_PER_THREAD];
#pragma unroll
    for (int j = 0; j < PAIRS_PER_THREAD; ++j) {
      px[2 * j] = cur[j].x; py[2 * j] = cur[j].y; px[2 * j + 1] = cur[j].z; py[2 * j + 1] = cur[j].w;
    }
    float tmin[NV], tmax[NV];
    {
      float v[NV];
      values32<ANG>(px[0], py[0], v);
#pragma unroll
      for (int k = 0; k < NV; ++k) { tmin[k] = v[k]; tmax[k] = v[k]; }
#pragma unroll
      for (int j = 1; j < 2 * PAIRS_PER_THREAD; ++j) {
        values32<ANG>(px[j], py[j], v);
#pragma unroll
        for (int k = 0; k < NV; ++k) { tmin[k] = fminf(tmin[k], v[k]); tmax[k] = fmaxf(tmax[k], v[k]); }
      }
    }
    if (st == 0) {
      // Seed the block's thresholds from the first tile of every thread.
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        float a = tmin[k], b = tmax[k];
        for (int off = 16; off; off >>= 1) {
          a = fminf(a, __shfl_xor_sync(FULL, a, off));
          b = fmaxf(b, __shfl_xor_sync(FULL, b, off));
        }
        if (lane == 0) { s_red[warp][2 * k] = a; s_red[warp][2 * k + 1] = b; }
      }
      __syncthreads();
      if (tid < ND) {
        float r = s_red[0][tid];
        for (int w = 1; w < BLOCK / 32; ++w) r = (tid & 1) ? fmaxf(r, s_red[w][tid]) : fminf(r, s_red[w][tid]);
        const float band = tid < 4 ? 0.0f : BAND;
        thr[tid] = (tid & 1) ? r - band : r + band;
      }
      __syncthreads();
    }
    float t[ND];
#pragma unroll
    for (int q = 0; q < ND / 4; ++q) {
      const float4 v = lds_vol4(&thr[4 * q]);
      t[4 * q] = v.x; t[4 * q + 1] = v.y; t[4 * q + 2] = v.z; t[4 * q + 3] = v.w;
    }
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      const bool lo = tmin[k] <= t[2 * k], hi = tmax[k] >= t[2 * k + 1];
      if (lo || hi) {
#pragma unroll 1
        for (int j = 0; j < 2 * PAIRS_PER_THREAD; ++j) {
          const float val = value32<ANG>(k, px[j], py[j]);
          const int64_t pp = base + (j >> 1) * BLOCK + tid;
          const uint32_t i = (uint32_t)(head + 2 * (pp < p1 ? pp : p0)) + (j & 1);
          if (lo && val <= *reinterpret_cast<volatile float*>(&thr[2 * k]))
            offer32<ANG>(2 * k, val, px[j], py[j], i, s_best[2 * k][tid], s_bidx[2 * k][tid], thr, xy);
          if (hi && val >= *reinterpret_cast<volatile float*>(&thr[2 * k + 1]))
            offer32<ANG>(2 * k + 1, val, px[j], py[j], i, s_best[2 * k + 1][tid], s_bidx[2 * k + 1][tid],
                         thr, xy);
        }
      }
    }
    if (st + 1 < nsteps) {
#pragma unroll
      for (int j = 0; j < PAIRS_PER_THREAD; ++j) cur[j] = nxt[j];
    }
  }
  // Points outside the 16-byte-aligned pairs: a leading point (block 0) and
  // a trailing point (last block).
  if (!dead && tid == 0) {
    const bool lead = blockIdx.x == 0 && head == 1;
    const bool trail = blockIdx.x == gridDim.x - 1 && ((n - head) & 1);
    for (int r = 0; r < 2; ++r) {
      if (!(r == 0 ? lead : trail)) continue;
      const uint32_t i = r == 0 ? 0u : (uint32_t)(n - 1);
      const float2 p = load_point(xy, i);
      float v[NV];
      values32<ANG>(p.x, p.y, v);
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        offer32<ANG>(2 * k, v[k], p.x, p.y, i, s_best[2 * k][tid], s_bidx[2 * k][tid], thr, xy);
        offer32<ANG>(2 * k + 1, v[k], p.x, p.y, i, s_best[2 * k + 1][tid], s_bidx[2 * k + 1][tid], thr, xy);
      }
    }
  }
  // Block reduction (warp butterfly, then across warps), exact.
#pragma unroll 1
  for (int d = 0; d < ND; ++d) {
    float s = s_best[d][tid];
    uint32_t i = s_bidx[d][tid];
    for (int off = 16; off; off >>= 1) {
      const float so = __shfl_xor_sync(FULL, s, off);
      const uint32_t io = __shfl_xor_sync(FULL, i, off);
      if (better32<ANG>(d, so, io, s, i, xy)) { s = so; i = io; }
    }
    if (lane == 0) { s_red[warp][d] = s; s_redi[warp][d] = i; }
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll 1
    for (int d = 0; d < ND; ++d) {
      float s = lane < BLOCK / 32 ? s_red[lane][d] : -FLT_MAX;
      uint32_t i = lane < BLOCK / 32 ? s_redi[lane][d] : NONE;
      for (int off = 16; off; off >>= 1) {
        const float so = __shfl_xor_sync(FULL, s, off);
        const uint32_t io = __shfl_xor_sync(FULL, i, off);
        if (better32<ANG>(d, so, io, s, i, xy)) { s = so; i = io; }
      }
      if (lane == 0) {
        BlockBest r;
        r.idx = i;
        r.pad_ = 0;
        if (i != NONE) {
          const float2 p = load_point(xy, i);
          r.s = score64(ANG, d, p.x, p.y);
        } else {
          r.s = -DBL_MAX;
        }
        blockres[(size_t)blockIdx.x * ND + d] = r;
      }
    }
  }
  if (last_block_arrives<ANG>(h)) finish_last_block<ANG>(xy, n, h, blockres, ext_out);
}

// ----------------------------------------------------------------------------
// EXACT mode: the binary64 definition for every point.

template <int ANG>
__global__ void __launch_bounds__(BLOCK) k_extremes64(const float* __restrict__ xy, int64_t n,
                                                       int head, int64_t npairs, int64_t ppb,
                                                       WsHeader* h, BlockBest* blockres,
                                                       uint32_t* ext_out) {
  constexpr int NV = Dirs<ANG>::NV, ND = Dirs<ANG>::ND;
  __shared__ double s_red[BLOCK / 32][ND];
  __shared__ uint32_t s_redi[BLOCK / 32][ND];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dead = *reinterpret_cast<volatile uint32_t*>(&h->status) != 0;
  double best[ND];
  uint32_t bidx[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) { best[d] = -DBL_MAX; bidx[d] = NONE; }

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

  const float4* P = reinterpret_cast<const float4*>(xy + 2 * head);
  const int64_t p0 = (int64_t)blockIdx.x * ppb;
  const int64_t p1 = dead ? p0 : min(p0 + ppb, npairs);
  for (int64_t base = p0; base < p1; base += STEP) {
#pragma unroll
    for (int j = 0; j < PAIRS_PER_THREAD; ++j) {
      const int64_t pp = base + j * BLOCK + tid;
      if (pp < p1) {
        const float4 v = __ldcs(P + pp);
        const uint32_t i = (uint32_t)(head + 2 * pp);
        offer(v.x, v.y, i);
        offer(v.z, v.w, i + 1);
      }
    }
  }
  if (!dead && tid == 0) {
    if (blockIdx.x == 0 && head == 1) { const float2 p = load_point(xy, 0); offer(p.x, p.y, 0); }
    if (blockIdx.x == gridDim.x - 1 && ((n - head) & 1)) {
      const float2 p = load_point(xy, (uint32_t)(n - 1));
      offer(p.x, p.y, (uint32_t)(n - 1));
    }
  }
#pragma unroll
  for (int d = 0; d < ND; ++d) {
    double s = best[d];
    uint32_t i = bidx[d];
    for (int off = 16; off; off >>= 1) {
      const double so = __shfl_xor_sync(FULL, s, off);
      const uint32_t io = __shfl_xor_sync(FULL, i, off);
      if (io != NONE && (i == NONE || so > s || (so == s && io < i))) { s = so; i = io; }
    }
    if (lane == 0) { s_red[warp][d] = s; s_redi[warp][d] = i; }
  }
  __syncthreads();
  if (warp == 0) {
    for (int d = 0; d < ND; ++d) {
      double s = lane < BLOCK / 32 ? s_red[lane][d] : -DBL_MAX;
      uint32_t i = lane < BLOCK / 32 ? s_redi[lane][d] : NONE;
      for (int off = 16; off; off >>= 1) {
        const double so = __shfl_xor_sync(FULL, s, off);
        const uint32_t io = __shfl_xor_sync(FULL, i, off);
        if (io != NONE && (i == NONE || so > s || (so == s && io < i))) { s = so; i = io; }
      }
      if (lane == 0) {
        BlockBest r;
        r.s = s; r.idx = i; r.pad_ = 0;
        blockres[(size_t)blockIdx.x * ND + d] = r;
      }
    }
  }
  if (last_block_arrives<ANG>(h)) finish_last_block<ANG>(xy, n, h, blockres, ext_out);
}

// Domain check (finite, integer-valued, |v| <= 2^24).
__global__ void k_validate(const float* __restrict__ xy, int64_t n2, WsHeader* h) {
  bool bad = false;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n2;
       k += (int64_t)gridDim.x * blockDim.x) {
    const float v = __ldg(xy + k);
    bad |= !(fabsf(v) <= 16777216.0f) || truncf(v) != v;  // NaN fails the first test
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&h->status, HULL_DEVICE_DOMAIN);
}

template <typename K>
int occupancy(K kernel) {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, BLOCK, 0) != cudaSuccess || b < 1) b = 1;
  return b;
}

}  // namespace

cudaError_t launch_validate(const float* xy, int64_t n, WsHeader* h, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const int64_t want = (2 * n + 255) / 256;
  const int grid = (int)std::min<int64_t>(want, (int64_t)device_sm_count() * 8);
  k_validate<<<grid, 256, 0, st>>>(xy, 2 * n, h);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_extremes(const float* xy, int64_t n, int angles, int filter, WsHeader* h,
                            BlockBest* blockres, int grid, int block, uint32_t* ext_out,
                            cudaStream_t st) {
  (void)block;
  const int head = (n > 0 && (reinterpret_cast<uintptr_t>(xy) & 15u)) ? 1 : 0;
  const int64_t npairs = n > head ? (n - head) / 2 : 0;
  int occ = 1;
  if (filter == HULL_FILTER_FP32)
    occ = angles == HULL_ANGLES_CUMULATIVE ? occupancy(k_extremes32<0>) : occupancy(k_extremes32<1>);
  else
    occ = angles == HULL_ANGLES_CUMULATIVE ? occupancy(k_extremes64<0>) : occupancy(k_extremes64<1>);
  int64_t G = grid > 0 ? grid : (int64_t)device_sm_count() * occ;
  G = std::max<int64_t>(1, std::min<int64_t>(G, (npairs + STEP - 1) / STEP));
  int64_t ppb = (npairs + G - 1) / G;
  ppb = (ppb + STEP - 1) / STEP * STEP;
  if (ppb == 0) ppb = STEP;
  G = std::max<int64_t>(1, (npairs + ppb - 1) / ppb);
  if (filter == HULL_FILTER_FP32) {
    if (angles == HULL_ANGLES_CUMULATIVE)
      k_extremes32<0><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, blockres, ext_out);
    else
      k_extremes32<1><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, blockres, ext_out);
  } else {
    if (angles == HULL_ANGLES_CUMULATIVE)
      k_extremes64<0><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, blockres, ext_out);
    else
      k_extremes64<1><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, blockres, ext_out);
  }
  count_launches(1);
  return cudaGetLastError();
}


}  // namespace cudapre
