// k_sort.cu -- device LSD radix sort of the survivors' (x, y) keys with their
// point indices, the first half of the final-hull stage (section 3, case (2):
// the hull of the remaining points; the paper ran Qhull on the CPU there).
//
// The element count is read from device memory (the compaction counter), so
// the whole sequence needs no host round trip and can be captured in a CUDA
// graph.  Keys are 52 bits; 7 passes of 8-bit digits.  Each pass is
// reduce-then-scan: per-tile digit counts, a per-digit scan over tiles, and a
// stable scatter in which each warp ranks its own 512-element slice.
#include "internal.cuh"

namespace cudapre {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int SBLOCK = 256;
constexpr int WARPS = SBLOCK / 32;
constexpr int PER_WARP = SORT_TILE / WARPS;  // 512
constexpr int ROWS = PER_WARP / 32;          // 16
static_assert(SORT_TILE == SBLOCK * ROWS, "tile shape");

// Element count of the large path: 0 (nothing to do) when the one-block
// path takes the set.
__device__ __forceinline__ int64_t dev_count(const WsHeader* h, const unsigned long long* count) {
  if (*reinterpret_cast<const volatile uint32_t*>(&h->status)) return 0;
  const int64_t m = (int64_t)*reinterpret_cast<const volatile unsigned long long*>(count);
  return m > SMALL_MAX ? m : 0;
}

__device__ __forceinline__ uint32_t digit(unsigned long long k, int pass) {
  return (uint32_t)(k >> (8 * pass)) & 255u;
}

// Digit histograms of all passes in one read (they do not depend on order).
__global__ void __launch_bounds__(SBLOCK) k_hist_all(const unsigned long long* __restrict__ keys,
                                                      WsHeader* h, const unsigned long long* count) {
  __shared__ uint32_t hs[SORT_PASSES][256];
  for (int k = threadIdx.x; k < SORT_PASSES * 256; k += SBLOCK) (&hs[0][0])[k] = 0;
  __syncthreads();
  const int64_t m = dev_count(h, count);
  for (int64_t j = (int64_t)blockIdx.x * SBLOCK + threadIdx.x; j < m; j += (int64_t)gridDim.x * SBLOCK) {
    const unsigned long long k = keys[j];
#pragma unroll
    for (int p = 0; p < SORT_PASSES; ++p) atomicAdd(&hs[p][digit(k, p)], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < SORT_PASSES * 256; k += SBLOCK) {
    const uint32_t c = (&hs[0][0])[k];
    if (c) atomicAdd(&(&h->hist[0][0])[k], c);
  }
}

// Per-tile digit counts: tilecnt[d * NT + t].
__global__ void __launch_bounds__(SBLOCK) k_tile_count(const unsigned long long* __restrict__ keys,
                                                        const WsHeader* h, const unsigned long long* count,
                                                        int pass, int64_t NT, uint32_t* __restrict__ tilecnt) {
  __shared__ uint32_t hs[256];
  const int64_t m = dev_count(h, count);
  const int64_t nt = (m + SORT_TILE - 1) / SORT_TILE;
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    hs[threadIdx.x] = 0;
    __syncthreads();
    const int64_t b = t * SORT_TILE;
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < ROWS; ++r) {
      const int64_t j = b + (int64_t)r * SBLOCK + threadIdx.x;
      const uint32_t d = j < m ? digit(keys[j], pass) : 256u;
      const unsigned peers = __match_any_sync(FULL, d);
      if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&hs[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    tilecnt[(int64_t)threadIdx.x * NT + t] = hs[threadIdx.x];
    __syncthreads();
  }
}

// Exclusive scan over tiles of one digit's counts, offset by the number of
// elements with a smaller digit.  One block per digit.
__global__ void __launch_bounds__(1024) k_tile_scan(const WsHeader* h, const unsigned long long* count,
                                                     int pass, int64_t NT, uint32_t* __restrict__ tilecnt) {
  __shared__ uint32_t s_w[32];
  __shared__ uint32_t s_carry;
  const int d = blockIdx.x;
  const int64_t m = dev_count(h, count);
  const int64_t nt = (m + SORT_TILE - 1) / SORT_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) {
    uint32_t base = 0;
    for (int e = 0; e < d; ++e) base += h->hist[pass][e];
    s_carry = base;
  }
  __syncthreads();
  uint32_t* row = tilecnt + (int64_t)d * NT;
  for (int64_t c0 = 0; c0 < nt; c0 += 1024) {
    const int64_t t = c0 + threadIdx.x;
    const uint32_t v = t < nt ? row[t] : 0u;
    uint32_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
      const uint32_t u = __shfl_up_sync(FULL, incl, off);
      if (lane >= off) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint32_t w = s_w[lane];
      uint32_t wi = w;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t u = __shfl_up_sync(FULL, wi, off);
        if (lane >= off) wi += u;
      }
      s_w[lane] = wi - w;  // exclusive prefix of warp totals
    }
    __syncthreads();
    const uint32_t carry = s_carry;
    if (t < nt) row[t] = carry + s_w[warp] + incl - v;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = carry + s_w[warp] + incl;
    __syncthreads();
  }
}

// Stable scatter of one pass.  Warp w owns elements [t*T + w*512, +512) of
// tile t, read in rows of 32 (so order is (warp, row, lane) = index order).
__global__ void __launch_bounds__(SBLOCK) k_tile_scatter(const unsigned long long* __restrict__ kin,
                                                          const uint32_t* __restrict__ vin,
                                                          unsigned long long* __restrict__ kout,
                                                          uint32_t* __restrict__ vout,
                                                          const WsHeader* h, const unsigned long long* count,
                                                          int pass, int64_t NT,
                                                          const uint32_t* __restrict__ tilecnt) {
  __shared__ uint32_t wc[WARPS][256];
  const int64_t m = dev_count(h, count);
  const int64_t nt = (m + SORT_TILE - 1) / SORT_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    for (int k = threadIdx.x; k < WARPS * 256; k += SBLOCK) (&wc[0][0])[k] = 0;
    __syncthreads();
    const int64_t b = t * SORT_TILE + (int64_t)warp * PER_WARP;
    unsigned long long kk[ROWS];
    uint32_t vv[ROWS];
    uint32_t dd[ROWS];
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int64_t j = b + r * 32 + lane;
      if (j < m) { kk[r] = kin[j]; vv[r] = vin[j]; dd[r] = digit(kk[r], pass); }
      else { kk[r] = 0; vv[r] = 0; dd[r] = 256u; }
    }
    // warp-local digit counts
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const unsigned peers = __match_any_sync(FULL, dd[r]);
      if (dd[r] < 256u && lane == __ffs(peers) - 1) wc[warp][dd[r]] += (uint32_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {
      // per digit: global offset of this tile, then prefix over warps
      const int d = threadIdx.x;
      uint32_t run = tilecnt[(int64_t)d * NT + t];
#pragma unroll
      for (int w = 0; w < WARPS; ++w) { const uint32_t c = wc[w][d]; wc[w][d] = run; run += c; }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const unsigned peers = __match_any_sync(FULL, dd[r]);
      if (dd[r] < 256u) {
        const uint32_t pos = wc[warp][dd[r]] + (uint32_t)__popc(peers & lt);
        kout[pos] = kk[r];
        vout[pos] = vv[r];
      }
      __syncwarp();
      if (dd[r] < 256u && lane == __ffs(peers) - 1) wc[warp][dd[r]] += (uint32_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
  }
}

}  // namespace

cudaError_t launch_sort(int64_t cap, WsHeader* h, const unsigned long long* count,
                        unsigned long long* keys_a, uint32_t* vals_a, unsigned long long* keys_b,
                        uint32_t* vals_b, uint32_t* tilecnt, cudaStream_t st) {
  const int64_t NT = sort_tiles(cap);
  const int sms = device_sm_count();
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(NT, (int64_t)sms * 8));
  const unsigned gh = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cap + SBLOCK - 1) / SBLOCK, (int64_t)sms * 8));
  k_hist_all<<<gh, SBLOCK, 0, st>>>(keys_a, h, count);
  count_launches(1);
  unsigned long long* kin = keys_a;
  uint32_t* vin = vals_a;
  unsigned long long* kout = keys_b;
  uint32_t* vout = vals_b;
  for (int p = 0; p < SORT_PASSES; ++p) {
    k_tile_count<<<g, SBLOCK, 0, st>>>(kin, h, count, p, NT, tilecnt);
    count_launches(1);
    k_tile_scan<<<256, 1024, 0, st>>>(h, count, p, NT, tilecnt);
    count_launches(1);
    k_tile_scatter<<<g, SBLOCK, 0, st>>>(kin, vin, kout, vout, h, count, p, NT, tilecnt);
    count_launches(1);
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  // SORT_PASSES is odd: the sorted data ends in (keys_b, vals_b).
  return cudaGetLastError();
}

}  // namespace cudapre
