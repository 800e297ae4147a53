// k_filter.cu -- Step 3 of the CudaPre method (arXiv 1405.3454, section 2):
// discard every point strictly inside the polygon of the extremes, and compact
// the survivors (their indices, plus their sort keys for the final hull).
//
// As in the paper each block first copies the polygon into shared memory;
// one thread tests several points.  The survivors are compacted in the same
// pass: a block-wide scan of per-thread counts and one atomic per block step.
//
// FP32 mode (per point): inside the exact inner box -> discarded; else per
// edge s = fma(A, px, fma(B, py, C)) with static bound E: s > E certainly
// left of the edge, s < -E certainly not (survives), otherwise the exact
// int64 orientation decides (counted as an escalation).  EXACT mode: the int64
// orientation for every edge.  Both give identical survivor sets.
#include "internal.cuh"

namespace cudapre {

namespace {

constexpr int BLOCK = 256;
constexpr int PAIRS = 4;  // 8 points per thread per step
constexpr int STEP = BLOCK * PAIRS;
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ bool exact_left(const Edge& e, int ix, int iy) {
  const long long o = (long long)e.dx * (long long)(iy - e.ay) - (long long)e.dy * (long long)(ix - e.ax);
  return o > 0;
}

template <int FILTER>
__device__ __forceinline__ bool survives(float x, float y, int m, const float* box,
                                         const Edge* E, unsigned& esc) {
  if (m < 3) return true;
  if (FILTER == HULL_FILTER_FP32) {
    if (x >= box[0] && x <= box[1] && y >= box[2] && y <= box[3]) return false;
    for (int k = 0; k < m; ++k) {
      const float4 c = *reinterpret_cast<const float4*>(&E[k].A);
      const float s = fmaf(c.x, x, fmaf(c.y, y, c.z));
      if (s > c.w) continue;
      if (s < -c.w) return true;
      ++esc;
      if (!exact_left(E[k], __float2int_rn(x), __float2int_rn(y))) return true;
    }
    return false;
  } else {
    const int ix = __float2int_rn(x), iy = __float2int_rn(y);
    for (int k = 0; k < m; ++k)
      if (!exact_left(E[k], ix, iy)) return true;
    return false;
  }
}

template <int FILTER, bool KEYS>
__global__ void __launch_bounds__(BLOCK) k_filter(const float* __restrict__ xy, int64_t n, int head,
                                                   int64_t npairs, int64_t ppb, WsHeader* h,
                                                   uint32_t* __restrict__ surv_idx,
                                                   unsigned long long* __restrict__ surv_key) {
  __shared__ __align__(16) Edge s_e[MAXV];
  __shared__ float s_box[4];
  __shared__ int s_m;
  __shared__ uint32_t s_wsum[BLOCK / 32];
  __shared__ unsigned long long s_base;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (*reinterpret_cast<volatile uint32_t*>(&h->status) != 0) return;
  // Stage the polygon in shared memory (section 2, Step 3).
  if (tid < MAXV * (int)(sizeof(Edge) / 4))
    reinterpret_cast<uint32_t*>(s_e)[tid] = reinterpret_cast<const uint32_t*>(h->poly.e)[tid];
  if (tid < 4) s_box[tid] = h->poly.box[tid];
  if (tid == 0) s_m = h->poly.m;
  __syncthreads();
  const int m = s_m;
  const float box[4] = {s_box[0], s_box[1], s_box[2], s_box[3]};
  unsigned esc = 0;

  const float4* P = reinterpret_cast<const float4*>(xy + 2 * head);
  const int64_t p0 = (int64_t)blockIdx.x * ppb;
  const int64_t p1 = min(p0 + ppb, npairs);
  // Extra points outside the aligned pairs go through the same compaction:
  // block 0 takes the leading point, the last block the trailing one.
  const bool lead = blockIdx.x == 0 && head == 1;
  const bool trail = blockIdx.x == gridDim.x - 1 && ((n - head) & 1);
  const int64_t nsteps = p1 > p0 ? (p1 - p0 + STEP - 1) / STEP : 0;
  const int64_t total_steps = nsteps + ((lead || trail) ? 1 : 0);
  for (int64_t st = 0; st < total_steps; ++st) {
    uint32_t keep = 0;  // bit j: point slot j survives
    float px[2 * PAIRS], py[2 * PAIRS];
    uint32_t pid[PAIRS];
    if (st < nsteps) {
      const int64_t base = p0 + st * STEP;
#pragma unroll
      for (int j = 0; j < PAIRS; ++j) {
        const int64_t pp = base + j * BLOCK + tid;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pp < p1) v = __ldcs(P + pp);
        px[2 * j] = v.x; py[2 * j] = v.y; px[2 * j + 1] = v.z; py[2 * j + 1] = v.w;
        pid[j] = (uint32_t)(head + 2 * pp);
        if (pp < p1) {
          if (survives<FILTER>(v.x, v.y, m, box, s_e, esc)) keep |= 1u << (2 * j);
          if (survives<FILTER>(v.z, v.w, m, box, s_e, esc)) keep |= 2u << (2 * j);
        }
      }
    } else if (tid < 2) {
      // the extra step: thread 0 the leading point, thread 1 the trailing one
      const bool mine = tid == 0 ? lead : trail;
      if (mine) {
        const uint32_t i = tid == 0 ? 0u : (uint32_t)(n - 1);
        const float2 p = __ldg(reinterpret_cast<const float2*>(xy) + i);
        px[0] = p.x; py[0] = p.y;
        pid[0] = i;
        if (survives<FILTER>(p.x, p.y, m, box, s_e, esc)) keep = 1u;
      }
    }
    const int c = __popc(keep);
    if (__syncthreads_count(c) == 0) continue;
    // block-wide exclusive scan of the per-thread counts
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
      const uint32_t i = (st < nsteps) ? pid[j >> 1] + (j & 1) : pid[0];
      surv_idx[pos] = i;
      if (KEYS) {
        // j is dynamic here; select through a small switch-free gather
        float x = px[0], y = py[0];
#pragma unroll
        for (int q = 1; q < 2 * PAIRS; ++q) if (q == j) { x = px[q]; y = py[q]; }
        surv_key[pos] = point_key(__float2int_rn(x), __float2int_rn(y));
      }
      ++pos;
    }
    __syncthreads();  // s_wsum / s_base reused by the next step
  }
  if (FILTER == HULL_FILTER_FP32) {
    unsigned e = esc;
    for (int off = 16; off; off >>= 1) e += __shfl_xor_sync(FULL, e, off);
    if (lane == 0 && e) atomicAdd(&h->n_escalated, (unsigned long long)e);
  }
}

__global__ void k_copy_count(const WsHeader* h, int64_t* out) {
  *out = h->status ? 0 : (int64_t)h->n_surv;
}

}  // namespace

cudaError_t launch_filter(const float* xy, int64_t n, int filter, WsHeader* h, uint32_t* surv_idx,
                          unsigned long long* surv_key, int grid, int block, cudaStream_t st) {
  (void)block;
  if (n == 0) return cudaSuccess;
  const int head = (reinterpret_cast<uintptr_t>(xy) & 15u) ? 1 : 0;
  const int64_t npairs = n > head ? (n - head) / 2 : 0;
  int64_t G = grid > 0 ? grid : (int64_t)device_sm_count() * 4;
  G = std::max<int64_t>(1, std::min<int64_t>(G, (npairs + STEP - 1) / STEP));
  int64_t ppb = (npairs + G - 1) / G;
  ppb = (ppb + STEP - 1) / STEP * STEP;
  if (ppb == 0) ppb = STEP;
  G = std::max<int64_t>(1, (npairs + ppb - 1) / ppb);
  const bool keys = surv_key != nullptr;
  if (filter == HULL_FILTER_FP32) {
    if (keys) { k_filter<HULL_FILTER_FP32, true><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, surv_idx, surv_key); count_launches(1); }
    else { k_filter<HULL_FILTER_FP32, false><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, surv_idx, surv_key); count_launches(1); }
  } else {
    if (keys) { k_filter<HULL_FILTER_EXACT, true><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, surv_idx, surv_key); count_launches(1); }
    else { k_filter<HULL_FILTER_EXACT, false><<<(unsigned)G, BLOCK, 0, st>>>(xy, n, head, npairs, ppb, h, surv_idx, surv_key); count_launches(1); }
  }
  return cudaGetLastError();
}

cudaError_t launch_copy_count(WsHeader* h, int64_t* out, cudaStream_t st) {
  k_copy_count<<<1, 1, 0, st>>>(h, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cudapre
