// k_filter.cu -- Step 3 of the CudaPre method (arXiv 1405.3454, section 2):
// discard every point strictly inside the polygon of the extremes, and compact
// the survivors (their indices, plus their sort keys for the final hull).
//
// As in the paper each block first copies the polygon into shared memory and
// one thread tests several points.  The survivors are compacted in the same
// pass through per-warp staging buffers in shared memory (one global atomic
// per buffer flush, no block-wide barrier in the streaming loop).
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
#include "stream.cuh"

namespace cudapre {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int MAGIC = 0x4B000000;  // bit pattern of 2^23

__device__ __forceinline__ bool exact_left(const Edge& e, int ix, int iy) {
  const long long o = (long long)e.dx * (long long)(iy - e.ay) - (long long)e.dy * (long long)(ix - e.ax);
  return o > 0;
}

// ----------------------------------------------------------------------------

template <int FILTER>
struct Tester;

// Every edge of the mask, float32 with exact escalation (cells near vertices
// and undecided float32 tests).  Returns 2 * escalations + (fails ? 1 : 0);
// a free function with register arguments.
__device__ __noinline__ unsigned fails_any(const Edge* E, uint32_t code, float x, float y) {
  unsigned esc = 0;
  while (code) {
    const int k = __ffs(code) - 1;
    code &= code - 1;
    const float4 c = *reinterpret_cast<const float4*>(&E[k].A);
    const float s = fmaf(c.x, x, fmaf(c.y, y, c.z));
    if (s > c.w) continue;
    if (s < -c.w) return 2 * esc + 1;
    ++esc;
    if (!exact_left(E[k], __float2int_rn(x), __float2int_rn(y))) return 2 * esc + 1;
  }
  return 2 * esc;
}

template <>
struct Tester<HULL_FILTER_FP32> {
  const Edge* E;
  const uint8_t* code8;      // shared memory
  const uint16_t* mask16;    // global memory (several-edge cells only)
  float gx, gy, ix_scale, iy_scale;
  unsigned esc;

  // Branch-free for the common cases: the cell lookup and the float32 test
  // of the cell's edge run for every point; only several-edge cells and
  // undecided float32 tests take a branch.
  __device__ __forceinline__ bool survives(float x, float y) {
    // exact cell coordinates: floor((x - gx) / 2^kx) from round-down
    // arithmetic (both steps are exact or round toward the floor)
    const float u = __fsub_rd(x, gx), v = __fsub_rd(y, gy);
    const int cx = __float_as_int(__fmaf_rd(u, ix_scale, 8388608.0f)) - MAGIC;
    const int cy = __float_as_int(__fmaf_rd(v, iy_scale, 8388608.0f)) - MAGIC;
    const bool in_grid = (unsigned)(cx | cy) < (unsigned)GRID;
    const int cell = in_grid ? ((cy << GRID_LOG) | cx) : 0;
    const uint32_t code = code8[cell];
    const int k = code != 0 && code != CELL_MULTI ? (int)code - 1 : 0;
    const float4 c = *reinterpret_cast<const float4*>(&E[k].A);
    const float s = fmaf(c.x, x, fmaf(c.y, y, c.z));
    const bool decided = s > c.w || s < -c.w;
    if (in_grid && code != 0 && (code == CELL_MULTI || !decided)) {
      const uint32_t mask = code == CELL_MULTI ? (uint32_t)__ldg(mask16 + cell) : 1u << k;
      const unsigned r = fails_any(E, mask, x, y);
      esc += r >> 1;
      return r & 1;
    }
    return !in_grid || (code != 0 && s < -c.w);
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

// Survivor output through a per-warp staging buffer in shared memory: per
// tile each lane counts its survivors, a warp scan places them, and a buffer
// that could overflow is first flushed by its warp with one global atomic and
// coalesced stores.  No block-wide barrier in the loop.
constexpr int WBUF = 128;  // >= 4 points x 32 lanes (a half tile)

template <bool KEYS>
struct WarpOut {
  uint32_t* s_idx;             // [WBUF] of this warp
  float2* s_xy;                // [WBUF] of this warp (coordinates, for the keys)
  int count;                   // warp-uniform fill level
  WsHeader* h;
  uint32_t* g_idx;
  unsigned long long* g_key;

  __device__ __forceinline__ void flush() {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    unsigned long long base = 0;
    if (lane == 0 && count) base = atomicAdd(&h->n_surv, (unsigned long long)count);
    base = __shfl_sync(FULL, base, 0);
    for (int k = lane; k < count; k += 32) {
      g_idx[base + k] = s_idx[k];
      if (KEYS) {
        const float2 p = s_xy[k];
        g_key[base + k] = point_key(__float2int_rn(p.x), __float2int_rn(p.y));
      }
    }
    __syncwarp();
    count = 0;
  }

  // Reserve room for this lane's c survivors; returns its first slot.
  __device__ __forceinline__ int reserve(int c) {
    const int lane = threadIdx.x & 31;
    int incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(FULL, incl, off);
      if (lane >= off) incl += t;
    }
    const int total = __shfl_sync(FULL, incl, 31);
    if (count + total > WBUF) flush();
    const int base = count + incl - c;
    count += total;
    return base;
  }

  __device__ __forceinline__ void put(int pos, uint32_t idx, float x, float y) {
    s_idx[pos] = idx;
    if (KEYS) s_xy[pos] = make_float2(x, y);
  }
};

using FilterStream = StreamSmemT<2>;

template <int FILTER, bool KEYS>
__global__ void __launch_bounds__(STREAM_THREADS, 3) k_filter(const float* __restrict__ xy, int64_t n, int head,
                                                               int64_t npairs, int64_t ppb, WsHeader* h,
                                                               const uint16_t* __restrict__ gcells,
                                                               uint32_t* __restrict__ surv_idx,
                                                               unsigned long long* __restrict__ surv_key) {
  extern __shared__ __align__(128) unsigned char dsm[];
  FilterStream& S = *reinterpret_cast<FilterStream*>(dsm);
  uint8_t* s_code = reinterpret_cast<uint8_t*>(dsm + sizeof(FilterStream));  // GRID*GRID (FP32)
  __shared__ __align__(16) Edge s_e[MAXV];
  __shared__ uint32_t s_oidx[CONSUMERS / 32][WBUF];
  __shared__ float2 s_oxy[KEYS ? CONSUMERS / 32 : 1][WBUF];
  __shared__ int s_pm[5];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (*reinterpret_cast<volatile uint32_t*>(&h->status) != 0) return;
  // Stage the polygon (and the cell grid) in shared memory (section 2, Step 3).
  if (tid < MAXV * (int)(sizeof(Edge) / 4))
    reinterpret_cast<uint32_t*>(s_e)[tid] = reinterpret_cast<const uint32_t*>(h->poly.e)[tid];
  if (tid == 0) {
    s_pm[0] = h->poly.m; s_pm[1] = h->poly.gx0; s_pm[2] = h->poly.gy0; s_pm[3] = h->poly.kx; s_pm[4] = h->poly.ky;
  }
  const int m_pre = h->poly.m;
  if (FILTER == HULL_FILTER_FP32 && m_pre >= 3) {
    const uint4* src = reinterpret_cast<const uint4*>(gcells + GRID * GRID);  // the byte codes
    uint4* dst = reinterpret_cast<uint4*>(s_code);
    for (int k = tid; k < GRID * GRID / 16; k += STREAM_THREADS) dst[k] = src[k];
  }
  stream_init(S);  // includes a block barrier
  const int m = s_pm[0];
  Tester<FILTER> T;
  T.E = s_e;
  T.esc = 0;
  if constexpr (FILTER == HULL_FILTER_FP32) {
    T.code8 = s_code;
    T.mask16 = gcells;
    T.gx = (float)s_pm[1];
    T.gy = (float)s_pm[2];
    T.ix_scale = __int_as_float((127 - s_pm[3]) << 23);  // 2^-kx
    T.iy_scale = __int_as_float((127 - s_pm[4]) << 23);
  } else {
    T.m = m;
  }
  const bool all_survive = m < 3;
  const float4* P = reinterpret_cast<const float4*>(xy + 2 * head);
  StreamRange R;
  R.p0 = (int64_t)blockIdx.x * ppb;
  R.p1 = min(R.p0 + ppb, npairs);
  R.nchunks = R.p1 > R.p0 ? (R.p1 - R.p0 + CHUNK - 1) / CHUNK : 0;
  // Chunks run last-to-first: the extreme search streamed each block's range
  // first-to-last, so the tail of every range is still in L2.
  R.reverse = true;

  if (warp == PRODUCER_WARP) {
    stream_produce(S, R, P, h);
    return;
  }
  WarpOut<KEYS> O;
  O.s_idx = s_oidx[warp];
  O.s_xy = s_oxy[KEYS ? warp : 0];
  O.count = 0;
  O.h = h;
  O.g_idx = surv_idx;
  O.g_key = surv_key;
  for (int64_t c = 0; c < R.nchunks; ++c) {
    const int s = (int)(c % FilterStream::STAGES);
    if (!mbar_wait(&S.full[s], (unsigned)((c / FilterStream::STAGES) & 1), h)) break;
    const int cnt = R.count(c);
    const int64_t f = R.first_pair(c);
    const float4* st = S.stage[s];
    float4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = st[tid + j * CONSUMERS];  // beyond cnt: ignored below
    __syncwarp();
    if (lane == 0) mbar_arrive(&S.empty[s]);
    uint32_t keep = 0;
    if (cnt == CHUNK) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (all_survive || T.survives(v[j].x, v[j].y)) keep |= 1u << (2 * j);
        if (all_survive || T.survives(v[j].z, v[j].w)) keep |= 2u << (2 * j);
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (tid + j * CONSUMERS < cnt) {
          if (all_survive || T.survives(v[j].x, v[j].y)) keep |= 1u << (2 * j);
          if (all_survive || T.survives(v[j].z, v[j].w)) keep |= 2u << (2 * j);
        }
      }
    }
    const uint32_t i0 = (uint32_t)(head + 2 * (f + tid));
    // two half tiles of 4 points each, so one half never exceeds WBUF
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const uint32_t kh = (keep >> (4 * half)) & 15u;
      int pos = O.reserve(__popc(kh));
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const int j = 4 * half + jj;
        if (kh & (1u << jj)) {
          const float4& q = v[j >> 1];
          O.put(pos++, i0 + 2u * (uint32_t)((j >> 1) * CONSUMERS) + (uint32_t)(j & 1), (j & 1) ? q.z : q.x,
                (j & 1) ? q.w : q.y);
        }
      }
    }
  }
  // Points outside the aligned pairs: block 0 takes the leading point, the
  // last block the trailing one (lanes 0 and 1 of warp 0).
  if (warp == 0) {
    const bool lead = blockIdx.x == 0 && head == 1;
    const bool trail = blockIdx.x == gridDim.x - 1 && ((n - head) & 1);
    bool k = false;
    uint32_t i = 0;
    float2 p = make_float2(0.f, 0.f);
    if ((lane == 0 && lead) || (lane == 1 && trail)) {
      i = lane == 0 ? 0u : (uint32_t)(n - 1);
      p = __ldg(reinterpret_cast<const float2*>(xy) + i);
      k = all_survive || T.survives(p.x, p.y);
    }
    const int pos = O.reserve(k ? 1 : 0);
    if (k) O.put(pos, i, p.x, p.y);
  }
  O.flush();
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
size_t filter_dsmem() {
  return sizeof(FilterStream) + (FILTER == HULL_FILTER_FP32 ? (size_t)GRID * GRID : 0);
}

template <int FILTER, bool KEYS>
cudaError_t filter_launch(const float* xy, int64_t n, int head, int64_t npairs, int grid, WsHeader* h,
                          uint16_t* cells, uint32_t* surv_idx, unsigned long long* surv_key, cudaStream_t st) {
  static bool attr[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t dsmem = filter_dsmem<FILTER, KEYS>();
  if (dev >= 0 && dev < 64 && !attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_filter<FILTER, KEYS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_filter<FILTER, KEYS>, STREAM_THREADS, dsmem);
  occ = std::max(occ, 1);
  int64_t G = grid > 0 ? grid : (int64_t)device_sm_count() * occ;
  G = std::max<int64_t>(1, std::min<int64_t>(G, (npairs + CHUNK - 1) / CHUNK));
  int64_t ppb = (npairs + G - 1) / G;
  ppb = (ppb + CHUNK - 1) / CHUNK * CHUNK;
  if (ppb == 0) ppb = CHUNK;
  G = std::max<int64_t>(1, (npairs + ppb - 1) / ppb);
  k_filter<FILTER, KEYS><<<(unsigned)G, STREAM_THREADS, dsmem, st>>>(xy, n, head, npairs, ppb, h, cells, surv_idx,
                                                                       surv_key);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_filter(const float* xy, int64_t n, int filter, WsHeader* h, uint16_t* cells,
                          uint32_t* surv_idx, unsigned long long* surv_key, int grid, int block,
                          cudaStream_t st) {
  (void)block;
  if (n == 0) return cudaSuccess;
  const bool keys = surv_key != nullptr;
  const int head = (reinterpret_cast<uintptr_t>(xy) & 15u) ? 1 : 0;
  const int64_t npairs = n > head ? (n - head) / 2 : 0;
  if (filter == HULL_FILTER_FP32)
    return keys ? filter_launch<HULL_FILTER_FP32, true>(xy, n, head, npairs, grid, h, cells, surv_idx, surv_key, st)
                : filter_launch<HULL_FILTER_FP32, false>(xy, n, head, npairs, grid, h, cells, surv_idx, surv_key, st);
  return keys ? filter_launch<HULL_FILTER_EXACT, true>(xy, n, head, npairs, grid, h, cells, surv_idx, surv_key, st)
              : filter_launch<HULL_FILTER_EXACT, false>(xy, n, head, npairs, grid, h, cells, surv_idx, surv_key, st);
}

cudaError_t launch_copy_count(WsHeader* h, int64_t* out, cudaStream_t st) {
  k_copy_count<<<1, 1, 0, st>>>(h, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cudapre
