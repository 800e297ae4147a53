// k_filter.cu -- Step 3 of the CudaPre method (arXiv 1405.3454, section 2):
// discard every point strictly inside the polygon of the extremes, and compact
// the survivors (their indices, plus their sort keys for the final hull).
//
// As in the paper each block first copies the polygon into shared memory and
// one thread tests several points.  The survivors are compacted in the same
// pass: a block-wide scan of per-thread counts and one atomic per block step.
//
// FP32 mode.  A point inside the exact inner box is discarded at once.  Else
// its cell of a GRID x GRID grid over the polygon's bounding box is found with
// two directed-rounding operations per coordinate; the cell's code lists the
// edges some point of the cell may fail (0: every point of the cell is
// strictly inside).  Only those edges are tested: s = fma(A, px, fma(B, py, C))
// with static bound E -- s > E certainly left, s < -E certainly not (the point
// survives), otherwise the exact int64 orientation decides (an escalation).
// Points beyond the grid are outside the bounding box and survive.
// EXACT mode (the plain method): the int64 orientation against every edge.
// Both modes give identical survivor sets.
#include "internal.cuh"

namespace cudapre {

namespace {

constexpr int BLOCK = 256;
constexpr int PAIRS = 4;  // 8 points per thread per step
constexpr int STEP = BLOCK * PAIRS;
constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int MAGIC = 0x4B000000;  // bit pattern of 2^23

__device__ __forceinline__ bool exact_left(const Edge& e, int ix, int iy) {
  const long long o = (long long)e.dx * (long long)(iy - e.ay) - (long long)e.dy * (long long)(ix - e.ax);
  return o > 0;
}

// ----------------------------------------------------------------------------
// Cell codes (one thread per cell).  For edge k the orientation is linear,
// A x + B y + C, so its minimum and maximum over the cell's integer points
// are at corners; everything is exact in int64.

__global__ void k_grid(WsHeader* h, uint16_t* cells) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= GRID * GRID) return;
  const Poly& P = h->poly;
  const int m = P.m;
  if (m < 3 || h->status) return;
  const int cx = c & (GRID - 1), cy = c >> GRID_LOG;
  const long long xa = (long long)P.gx0 + ((long long)cx << P.kx), xb = xa + (1ll << P.kx) - 1;
  const long long ya = (long long)P.gy0 + ((long long)cy << P.ky), yb = ya + (1ll << P.ky) - 1;
  uint32_t code = 0;
  for (int k = 0; k < m; ++k) {
    const Edge& e = P.e[k];
    const long long A = -(long long)e.dy, B = e.dx;
    const long long C = (long long)e.dy * e.ax - (long long)e.dx * e.ay;
    const long long mn = A * (A >= 0 ? xa : xb) + B * (B >= 0 ? ya : yb) + C;
    const long long mx = A * (A >= 0 ? xb : xa) + B * (B >= 0 ? yb : ya) + C;
    if (mx <= 0) { code = 1u << k; break; }  // every point fails edge k: one test decides
    if (mn <= 0) code |= 1u << k;
  }
  cells[c] = (uint16_t)code;
}

// ----------------------------------------------------------------------------

template <int FILTER>
struct Tester;

template <>
struct Tester<HULL_FILTER_FP32> {
  const Edge* E;
  const uint16_t* cells;
  float b0, b1, b2, b3, gx, gy, ix_scale, iy_scale;
  unsigned esc;
  __device__ __forceinline__ bool survives(float x, float y) {
    if (x >= b0 && x <= b1 && y >= b2 && y <= b3) return false;
    // exact cell coordinates: floor((x - gx) / 2^kx) from round-down
    // arithmetic (both steps are exact or round toward the floor)
    const float u = __fsub_rd(x, gx), v = __fsub_rd(y, gy);
    const int cx = __float_as_int(__fmaf_rd(u, ix_scale, 8388608.0f)) - MAGIC;
    const int cy = __float_as_int(__fmaf_rd(v, iy_scale, 8388608.0f)) - MAGIC;
    if ((unsigned)(cx | cy) >= (unsigned)GRID) return true;  // outside the bounding box
    uint32_t code = cells[(cy << GRID_LOG) | cx];
    while (code) {
      const int k = __ffs(code) - 1;
      code &= code - 1;
      const float4 c = *reinterpret_cast<const float4*>(&E[k].A);
      const float s = fmaf(c.x, x, fmaf(c.y, y, c.z));
      if (s > c.w) continue;
      if (s < -c.w) return true;
      ++esc;
      if (!exact_left(E[k], __float2int_rn(x), __float2int_rn(y))) return true;
    }
    return false;
  }
};

template <>
struct Tester<HULL_FILTER_EXACT> {
  const Edge* E;
  int m;
  unsigned esc;
  __device__ __forceinline__ bool survives(float x, float y) {
    const int ix = __float2int_rn(x), iy = __float2int_rn(y);
    for (int k = 0; k < m; ++k)
      if (!exact_left(E[k], ix, iy)) return true;
    return false;
  }
};

template <int FILTER, bool KEYS>
__global__ void __launch_bounds__(BLOCK, 4) k_filter(const float* __restrict__ xy, int64_t n, int head,
                                                      int64_t npairs, int64_t ppb, WsHeader* h,
                                                      const uint16_t* __restrict__ gcells,
                                                      uint32_t* __restrict__ surv_idx,
                                                      unsigned long long* __restrict__ surv_key) {
  __shared__ __align__(16) Edge s_e[MAXV];
  __shared__ __align__(16) uint16_t s_cells[FILTER == HULL_FILTER_FP32 ? GRID * GRID : 8];
  __shared__ float s_box[4];
  __shared__ int s_pm[5];
  __shared__ uint32_t s_wsum[BLOCK / 32];
  __shared__ unsigned long long s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (*reinterpret_cast<volatile uint32_t*>(&h->status) != 0) return;
  // Stage the polygon (and the cell grid) in shared memory (section 2, Step 3).
  if (tid < MAXV * (int)(sizeof(Edge) / 4))
    reinterpret_cast<uint32_t*>(s_e)[tid] = reinterpret_cast<const uint32_t*>(h->poly.e)[tid];
  if (tid < 4) s_box[tid] = h->poly.box[tid];
  if (tid == 0) {
    s_pm[0] = h->poly.m; s_pm[1] = h->poly.gx0; s_pm[2] = h->poly.gy0; s_pm[3] = h->poly.kx; s_pm[4] = h->poly.ky;
  }
  const int m_pre = h->poly.m;
  if (FILTER == HULL_FILTER_FP32 && m_pre >= 3) {
    const uint4* src = reinterpret_cast<const uint4*>(gcells);
    uint4* dst = reinterpret_cast<uint4*>(s_cells);
    for (int k = tid; k < GRID * GRID * 2 / 16; k += BLOCK) dst[k] = src[k];
  }
  __syncthreads();
  const int m = s_pm[0];
  Tester<FILTER> T;
  T.E = s_e;
  T.esc = 0;
  if constexpr (FILTER == HULL_FILTER_FP32) {
    T.cells = s_cells;
    T.b0 = s_box[0]; T.b1 = s_box[1]; T.b2 = s_box[2]; T.b3 = s_box[3];
    T.gx = (float)s_pm[1];
    T.gy = (float)s_pm[2];
    T.ix_scale = __int_as_float((127 - s_pm[3]) << 23);  // 2^-kx
    T.iy_scale = __int_as_float((127 - s_pm[4]) << 23);
  } else {
    T.m = m;
  }
  const bool all_survive = m < 3;

  const float4* P = reinterpret_cast<const float4*>(xy + 2 * head);
  const int64_t p0 = (int64_t)blockIdx.x * ppb;
  const int64_t p1 = min(p0 + ppb, npairs);
  // Points outside the aligned pairs go through the same compaction: block 0
  // takes the leading point, the last block the trailing one.
  const bool lead = blockIdx.x == 0 && head == 1;
  const bool trail = blockIdx.x == gridDim.x - 1 && ((n - head) & 1);
  const int64_t nsteps = p1 > p0 ? (p1 - p0 + STEP - 1) / STEP : 0;
  const int64_t total = nsteps + ((lead || trail) ? 1 : 0);
  // Steps run last-to-first: the extreme search streamed each block's range
  // first-to-last, so the tail of every range is still in L2.
  auto load = [&](int64_t s, float4* v) {
    const int64_t base = p0 + s * STEP;
#pragma unroll
    for (int j = 0; j < PAIRS; ++j) {
      const int64_t pp = base + j * BLOCK + tid;
      v[j] = pp < p1 ? __ldcs(P + pp) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  float4 cur[PAIRS];
  if (nsteps > 0) load(nsteps - 1, cur);
  for (int64_t it = 0; it < total; ++it) {
    const bool extra = it == nsteps;  // the step for the unaligned end points
    const int64_t s = nsteps - 1 - it;
    float4 nxt[PAIRS];
    if (!extra && s > 0) load(s - 1, nxt);
    uint32_t keep = 0;  // bit j: point slot j survives
    float px[2 * PAIRS], py[2 * PAIRS];
    uint32_t pid0 = 0;
    if (!extra) {
      const int64_t base = p0 + s * STEP;
#pragma unroll
      for (int j = 0; j < PAIRS; ++j) {
        px[2 * j] = cur[j].x; py[2 * j] = cur[j].y; px[2 * j + 1] = cur[j].z; py[2 * j + 1] = cur[j].w;
        const bool ok = base + j * BLOCK + tid < p1;
        if (ok && (all_survive || T.survives(cur[j].x, cur[j].y))) keep |= 1u << (2 * j);
        if (ok && (all_survive || T.survives(cur[j].z, cur[j].w))) keep |= 2u << (2 * j);
      }
      pid0 = (uint32_t)(head + 2 * (base + tid));
    } else if (tid < 2 && (tid == 0 ? lead : trail)) {
      const uint32_t i = tid == 0 ? 0u : (uint32_t)(n - 1);
      const float2 p = __ldg(reinterpret_cast<const float2*>(xy) + i);
      px[0] = p.x; py[0] = p.y;
      pid0 = i;
      if (all_survive || T.survives(p.x, p.y)) keep = 1u;
    }
    const int c = __popc(keep);
    if (__syncthreads_count(c) != 0) {
      // block-wide exclusive scan of the per-thread counts, one atomic
      int incl = c;
      for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += t;
      }
      if (lane == 31) s_wsum[warp] = incl;
      __syncthreads();
      if (tid == 0) {
        uint32_t run = 0;
        for (int w = 0; w < BLOCK / 32; ++w) { const uint32_t t = s_wsum[w]; s_wsum[w] = run; run += t; }
        s_base = atomicAdd(&h->n_surv, (unsigned long long)run);
      }
      __syncthreads();
      unsigned long long pos = s_base + s_wsum[warp] + (incl - c);
      while (keep) {
        const int j = __ffs(keep) - 1;
        keep &= keep - 1;
        // slot j is pair j/2 (index pid0 + 2*(j/2)*BLOCK) point j%2
        surv_idx[pos] = extra ? pid0 : pid0 + 2u * (uint32_t)((j >> 1) * BLOCK) + (uint32_t)(j & 1);
        if (KEYS) {
          float x = px[0], y = py[0];
#pragma unroll
          for (int q = 1; q < 2 * PAIRS; ++q) if (q == j) { x = px[q]; y = py[q]; }
          surv_key[pos] = point_key(__float2int_rn(x), __float2int_rn(y));
        }
        ++pos;
      }
      __syncthreads();  // s_wsum / s_base are reused by the next step
    }
    if (!extra && s > 0) {
#pragma unroll
      for (int j = 0; j < PAIRS; ++j) cur[j] = nxt[j];
    }
  }
  if (FILTER == HULL_FILTER_FP32) {
    unsigned e = T.esc;
    for (int off = 16; off; off >>= 1) e += __shfl_xor_sync(FULL, e, off);
    if (lane == 0 && e) atomicAdd(&h->n_escalated, (unsigned long long)e);
  }
}

__global__ void k_copy_count(const WsHeader* h, int64_t* out) {
  *out = h->status ? 0 : (int64_t)h->n_surv;
}

template <int FILTER, bool KEYS>
int filter_occupancy() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_filter<FILTER, KEYS>, BLOCK, 0) != cudaSuccess || b < 1)
    b = 1;
  return b;
}

}  // namespace

cudaError_t launch_filter(const float* xy, int64_t n, int filter, WsHeader* h, uint16_t* cells,
                          uint32_t* surv_idx, unsigned long long* surv_key, int grid, int block,
                          cudaStream_t st) {
  (void)block;
  if (n == 0) return cudaSuccess;
  const bool keys = surv_key != nullptr;
  if (filter == HULL_FILTER_FP32) {
    k_grid<<<GRID * GRID / 256, 256, 0, st>>>(h, cells);
    count_launches(1);
  }
  const int head = (reinterpret_cast<uintptr_t>(xy) & 15u) ? 1 : 0;
  const int64_t npairs = n > head ? (n - head) / 2 : 0;
  int occ = 1;
  if (filter == HULL_FILTER_FP32) occ = keys ? filter_occupancy<HULL_FILTER_FP32, true>() : filter_occupancy<HULL_FILTER_FP32, false>();
  else occ = keys ? filter_occupancy<HULL_FILTER_EXACT, true>() : filter_occupancy<HULL_FILTER_EXACT, false>();
  int64_t G = grid > 0 ? grid : (int64_t)device_sm_count() * occ;
  G = std::max<int64_t>(1, std::min<int64_t>(G, (npairs + STEP - 1) / STEP));
  int64_t ppb = (npairs + G - 1) / G;
  ppb = (ppb + STEP - 1) / STEP * STEP;
  if (ppb == 0) ppb = STEP;
  G = std::max<int64_t>(1, (npairs + ppb - 1) / ppb);
  if (filter == HULL_FILTER_FP32) {
    if (keys) k_filter<HULL_FILTER_FP32, true><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, cells, surv_idx, surv_key);
    else k_filter<HULL_FILTER_FP32, false><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, cells, surv_idx, surv_key);
  } else {
    if (keys) k_filter<HULL_FILTER_EXACT, true><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, cells, surv_idx, surv_key);
    else k_filter<HULL_FILTER_EXACT, false><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, cells, surv_idx, surv_key);
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_count(WsHeader* h, int64_t* out, cudaStream_t st) {
  k_copy_count<<<1, 1, 0, st>>>(h, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cudapre
