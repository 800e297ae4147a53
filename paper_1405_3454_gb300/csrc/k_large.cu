// k_large.cu -- the hull of a survivor set too large for the one-block path:
// device LSD radix sort of the (x, y) keys with their point indices, then
// Andrew's monotone chain over the sorted keys, chunked (section 3, case (2):
// the hull of the points that remain; the paper ran Qhull on the CPU there).
//
// One cooperative launch does the whole stage for a list of jobs (one per
// point set), its phases separated by a grid barrier: the sort is 7 passes
// of 8-bit digits over the 52-bit keys, each reduce-then-scan (per-tile digit
// counts, a per-digit scan over tiles, a stable scatter in which each warp
// ranks its own 512-element slice); the chain is chunked -- level 0 chains
// every sorted chunk of CHAIN_C0 keys, each later level concatenates
// CHAIN_FAN consecutive chunk chains (still sorted) and chains them again,
// until one chunk is left.  A hull vertex of the whole set is a vertex of
// every chunk chain that contains it, so the last chain is the hull.  Stacks
// are written in place over the consumed input (a push never overtakes the
// read cursor); among equal keys the lowest index is kept.
//
// Every size is read on the device.  A job whose count is at most SMALL_MAX
// (the one-block path has written its result) or whose status word is set
// is skipped by every block alike.  Barrier waits are bounded: on expiry the
// kernel records HULL_DEVICE_TIMEOUT and returns.
#include "internal.cuh"

namespace cudapre {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int LBLOCK = 256;
constexpr int WARPS = LBLOCK / 32;
constexpr int PER_WARP = SORT_TILE / WARPS;  // 512
constexpr int ROWS = PER_WARP / 32;          // 16
static_assert(SORT_TILE == LBLOCK * ROWS, "tile shape");
constexpr long long BAR_LIMIT_CYCLES = 1ll << 31;  // about one second

// Grid barrier over the cooperative launch; false when the wait expired.
__device__ bool grid_sync(uint32_t* bar, uint32_t* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile uint32_t* gen = bar + 1;
    const uint32_t g = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) + 1u == gridDim.x) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g) {
        if (clock64() - t0 > BAR_LIMIT_CYCLES) {
          atomicOr(status, HULL_DEVICE_TIMEOUT);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return (*reinterpret_cast<volatile uint32_t*>(status) & HULL_DEVICE_TIMEOUT) == 0;
}

__device__ __forceinline__ uint32_t digit(unsigned long long k, int pass) {
  return (uint32_t)(k >> (8 * pass)) & 255u;
}

__device__ __forceinline__ long long cross_k(unsigned long long o, unsigned long long a, unsigned long long b) {
  // differences of lattice coordinates within +-2^24 fit in 32 bits
  const int ox = key_x(o), oy = key_y(o);
  return (long long)(key_x(a) - ox) * (key_y(b) - oy) - (long long)(key_y(a) - oy) * (key_x(b) - ox);
}

// One monotone chain kept as an in-place stack K[base..base+n), V likewise.
// UPPER = false: lower chain (pop while the turn is not strictly left);
// UPPER = true: upper chain walked left to right (pop while not strictly right).
template <bool UPPER>
struct Stack {
  unsigned long long* K;
  uint32_t* V;
  int64_t base;
  int64_t n;
  unsigned long long t1, t2;  // top and second keys (valid when n >= 1 / 2)

  __device__ __forceinline__ void init(unsigned long long* k, uint32_t* v, int64_t b) {
    K = k; V = v; base = b; n = 0; t1 = t2 = 0;
  }
  __device__ __forceinline__ void push(unsigned long long key, uint32_t idx) {
    if (n >= 1 && key == t1) {  // equal coordinates: keep the lowest index
      const uint32_t old = V[base + n - 1];
      if (idx < old) V[base + n - 1] = idx;
      return;
    }
    while (n >= 2) {
      const long long c = cross_k(t2, t1, key);
      if (UPPER ? (c < 0) : (c > 0)) break;
      --n;
      t1 = t2;
      if (n >= 2) t2 = K[base + n - 2];
    }
    K[base + n] = key;
    V[base + n] = idx;
    ++n;
    t2 = t1;
    t1 = key;
  }
};

struct SortSmem {
  uint32_t hs[SORT_PASSES][256];
  uint32_t wc[WARPS][256];
  uint32_t sw[WARPS];
  uint32_t carry;
};

// Digit histograms of all passes in one read (they do not depend on order).
__device__ void hist_all(SortSmem& S, const unsigned long long* keys, int64_t m, uint32_t* hist) {
  for (int k = threadIdx.x; k < SORT_PASSES * 256; k += LBLOCK) (&S.hs[0][0])[k] = 0;
  __syncthreads();
  for (int64_t j = (int64_t)blockIdx.x * LBLOCK + threadIdx.x; j < m; j += (int64_t)gridDim.x * LBLOCK) {
    const unsigned long long k = keys[j];
#pragma unroll
    for (int p = 0; p < SORT_PASSES; ++p) atomicAdd(&S.hs[p][digit(k, p)], 1u);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < SORT_PASSES * 256; k += LBLOCK) {
    const uint32_t c = (&S.hs[0][0])[k];
    if (c) atomicAdd(hist + k, c);
  }
}

// Per-tile digit counts of one pass: tilecnt[d * NT + t].
__device__ void tile_count(SortSmem& S, const unsigned long long* keys, int64_t m, int pass, int64_t NT,
                           uint32_t* tilecnt) {
  const int64_t nt = (m + SORT_TILE - 1) / SORT_TILE;
  const int lane = threadIdx.x & 31;
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    S.hs[0][threadIdx.x] = 0;
    __syncthreads();
    const int64_t b = t * SORT_TILE;
    for (int r = 0; r < ROWS; ++r) {
      const int64_t j = b + (int64_t)r * LBLOCK + threadIdx.x;
      const uint32_t d = j < m ? digit(keys[j], pass) : 256u;
      const unsigned peers = __match_any_sync(FULL, d);
      if (d < 256u && lane == __ffs(peers) - 1) atomicAdd(&S.hs[0][d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    tilecnt[(int64_t)threadIdx.x * NT + t] = S.hs[0][threadIdx.x];
    __syncthreads();
  }
}

// Exclusive scan over tiles of each digit's counts, offset by the number of
// elements with a smaller digit.  Digits are spread over the blocks.
__device__ void tile_scan(SortSmem& S, int64_t m, int pass, int64_t NT, const uint32_t* hist, uint32_t* tilecnt) {
  const int64_t nt = (m + SORT_TILE - 1) / SORT_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = blockIdx.x; d < 256; d += gridDim.x) {
    if (threadIdx.x == 0) {
      uint32_t base = 0;
      for (int e = 0; e < d; ++e) base += hist[pass * 256 + e];
      S.carry = base;
    }
    __syncthreads();
    uint32_t* row = tilecnt + (int64_t)d * NT;
    for (int64_t c0 = 0; c0 < nt; c0 += LBLOCK) {
      const int64_t t = c0 + threadIdx.x;
      const uint32_t v = t < nt ? row[t] : 0u;
      uint32_t incl = v;
      for (int off = 1; off < 32; off <<= 1) {
        const uint32_t u = __shfl_up_sync(FULL, incl, off);
        if (lane >= off) incl += u;
      }
      if (lane == 31) S.sw[warp] = incl;
      __syncthreads();
      uint32_t wpre = 0, tot = 0;
      for (int w = 0; w < WARPS; ++w) {
        const uint32_t x = S.sw[w];
        if (w < warp) wpre += x;
        tot += x;
      }
      const uint32_t carry = S.carry;
      if (t < nt) row[t] = carry + wpre + incl - v;
      __syncthreads();
      if (threadIdx.x == 0) S.carry = carry + tot;
      __syncthreads();
    }
  }
}

// Stable scatter of one pass.  Warp w owns elements [t*T + w*512, +512) of
// tile t, read in rows of 32 (so order is (warp, row, lane) = index order).
__device__ void tile_scatter(SortSmem& S, const unsigned long long* kin, const uint32_t* vin,
                             unsigned long long* kout, uint32_t* vout, int64_t m, int pass, int64_t NT,
                             const uint32_t* tilecnt) {
  const int64_t nt = (m + SORT_TILE - 1) / SORT_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    for (int k = threadIdx.x; k < WARPS * 256; k += LBLOCK) (&S.wc[0][0])[k] = 0;
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
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const unsigned peers = __match_any_sync(FULL, dd[r]);
      if (dd[r] < 256u && lane == __ffs(peers) - 1) S.wc[warp][dd[r]] += (uint32_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    {
      const int d = threadIdx.x;
      uint32_t run = tilecnt[(int64_t)d * NT + t];
#pragma unroll
      for (int w = 0; w < WARPS; ++w) { const uint32_t c = S.wc[w][d]; S.wc[w][d] = run; run += c; }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const unsigned peers = __match_any_sync(FULL, dd[r]);
      if (dd[r] < 256u) {
        const uint32_t pos = S.wc[warp][dd[r]] + (uint32_t)__popc(peers & lt);
        kout[pos] = kk[r];
        vout[pos] = vv[r];
      }
      __syncwarp();
      if (dd[r] < 256u && lane == __ffs(peers) - 1) S.wc[warp][dd[r]] += (uint32_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
  }
}

// Level 0: virtual thread g chains sorted elements [g*C0, min((g+1)*C0, m));
// the lower chain in place in (Ks, Vs), the upper chain into (Ku, Vu) at the
// same offsets; counts to cnt_lo[g], cnt_up[g].
__device__ void chain0(unsigned long long* Ks, uint32_t* Vs, unsigned long long* Ku, uint32_t* Vu, int64_t m,
                       uint32_t* cnt_lo, uint32_t* cnt_up) {
  const int64_t nch = (m + CHAIN_C0 - 1) / CHAIN_C0;
  for (int64_t g = (int64_t)blockIdx.x * LBLOCK + threadIdx.x; g < nch; g += (int64_t)gridDim.x * LBLOCK) {
    const int64_t start = g * CHAIN_C0;
    const int64_t end = min(start + (int64_t)CHAIN_C0, m);
    Stack<false> lo;
    Stack<true> up;
    lo.init(Ks, Vs, start);
    up.init(Ku, Vu, start);
    for (int64_t j = start; j < end; ++j) {
      const unsigned long long k = Ks[j];
      const uint32_t v = Vs[j];
      lo.push(k, v);
      up.push(k, v);
    }
    cnt_lo[g] = (uint32_t)lo.n;
    cnt_up[g] = (uint32_t)up.n;
  }
}

// Later level: group g merges the chains of chunks [g*FAN, (g+1)*FAN) of the
// previous level (span `span` each); virtual thread 2g does the lower
// chains, 2g+1 the upper ones.
__device__ void chainN(unsigned long long* Ks, uint32_t* Vs, unsigned long long* Ku, uint32_t* Vu, int64_t m,
                       const uint32_t* cin_lo, const uint32_t* cin_up, uint32_t* cout_lo, uint32_t* cout_up,
                       int64_t nch_prev, int64_t span) {
  const int64_t ng = (nch_prev + CHAIN_FAN - 1) / CHAIN_FAN;
  for (int64_t t = (int64_t)blockIdx.x * LBLOCK + threadIdx.x; t < 2 * ng; t += (int64_t)gridDim.x * LBLOCK) {
    const int64_t g = t >> 1;
    const int64_t c0 = g * CHAIN_FAN;
    const int64_t c1 = min(c0 + (int64_t)CHAIN_FAN, nch_prev);
    if (!(t & 1)) {
      Stack<false> s;
      s.init(Ks, Vs, c0 * span);
      for (int64_t c = c0; c < c1; ++c) {
        const int64_t b = c * span, cnt = cin_lo[c];
        for (int64_t j = 0; j < cnt; ++j) s.push(Ks[b + j], Vs[b + j]);
      }
      cout_lo[g] = (uint32_t)s.n;
    } else {
      Stack<true> s;
      s.init(Ku, Vu, c0 * span);
      for (int64_t c = c0; c < c1; ++c) {
        const int64_t b = c * span, cnt = cin_up[c];
        for (int64_t j = 0; j < cnt; ++j) s.push(Ku[b + j], Vu[b + j]);
      }
      cout_up[g] = (uint32_t)s.n;
    }
  }
}

// The hull counter-clockwise from the lexicographic minimum: the lower chain
// left to right, then the upper chain right to left, without repeating the
// two end points.
__device__ void chain_emit(const uint32_t* Vs, const uint32_t* Vu, const uint32_t* cnt_lo, const uint32_t* cnt_up,
                           uint32_t* out_idx, int64_t* out_n) {
  const int64_t a = cnt_lo[0], b = cnt_up[0];
  const int64_t gt = (int64_t)blockIdx.x * LBLOCK + threadIdx.x, gs = (int64_t)gridDim.x * LBLOCK;
  if (a <= 1) {
    if (gt == 0) {
      out_idx[0] = Vs[0];
      *out_n = 1;
    }
    return;
  }
  for (int64_t k = gt; k < a - 1; k += gs) out_idx[k] = Vs[k];
  // upper vertex k (1 <= k <= b-1) goes to a-1 + (b-1-k)
  for (int64_t k = 1 + gt; k <= b - 1; k += gs) out_idx[(a - 1) + (b - 1 - k)] = Vu[k];
  if (gt == 0) *out_n = (a - 1) + (b - 1);
}

__global__ void __launch_bounds__(LBLOCK) k_large(const LargeJob* __restrict__ table, const int* njobs_dev,
                                                   LargeJob single, uint32_t* bar, uint32_t* bar_status) {
  __shared__ SortSmem S;
  const int njobs = table ? *reinterpret_cast<const volatile int*>(njobs_dev) : 1;
  for (int jb = 0; jb < njobs; ++jb) {
    const LargeJob J = table ? table[jb] : single;
    if (*reinterpret_cast<const volatile uint32_t*>(&J.h->status)) continue;
    const int64_t m = (int64_t)*reinterpret_cast<const volatile unsigned long long*>(J.count);
    if (m <= SMALL_MAX) continue;
    const int64_t NT = sort_tiles(J.cap);
    hist_all(S, J.ka, m, &J.h->hist[0][0]);
    if (!grid_sync(bar, bar_status)) return;
    unsigned long long *kin = J.ka, *kout = J.kb;
    uint32_t *vin = J.va, *vout = J.vb;
    for (int p = 0; p < SORT_PASSES; ++p) {
      tile_count(S, kin, m, p, NT, J.tilecnt);
      if (!grid_sync(bar, bar_status)) return;
      tile_scan(S, m, p, NT, &J.h->hist[0][0], J.tilecnt);
      if (!grid_sync(bar, bar_status)) return;
      tile_scatter(S, kin, vin, kout, vout, m, p, NT, J.tilecnt);
      if (!grid_sync(bar, bar_status)) return;
      unsigned long long* tk = kin; kin = kout; kout = tk;
      uint32_t* tv = vin; vin = vout; vout = tv;
    }
    // sorted in (kin, vin); upper chains go to (kout, vout)
    const int64_t nch0 = (std::max<int64_t>(J.cap, 1) + CHAIN_C0 - 1) / CHAIN_C0;
    uint32_t* lo[2] = {J.cnt, J.cnt + 2 * nch0};
    uint32_t* up[2] = {J.cnt + nch0, J.cnt + 3 * nch0};
    chain0(kin, vin, kout, vout, m, lo[0], up[0]);
    if (!grid_sync(bar, bar_status)) return;
    int64_t nch = (m + CHAIN_C0 - 1) / CHAIN_C0, span = CHAIN_C0;
    int par = 0;
    while (nch > 1) {
      chainN(kin, vin, kout, vout, m, lo[par], up[par], lo[par ^ 1], up[par ^ 1], nch, span);
      if (!grid_sync(bar, bar_status)) return;
      par ^= 1;
      nch = (nch + CHAIN_FAN - 1) / CHAIN_FAN;
      span *= CHAIN_FAN;
    }
    chain_emit(vin, vout, lo[par], up[par], J.out_idx, J.out_n);
    // the next job reuses nothing of this one, but its histogram phase must
    // not overtake this one's emission on shared barrier state: no barrier
    // needed (the buffers differ and the barrier counter is balanced).
  }
}

}  // namespace

int chain_levels(int64_t cap) {
  int64_t nch = (std::max<int64_t>(cap, 1) + CHAIN_C0 - 1) / CHAIN_C0;
  int levels = 1;
  while (nch > 1) { nch = (nch + CHAIN_FAN - 1) / CHAIN_FAN; ++levels; }
  return levels;
}

cudaError_t launch_large(const LargeJob* table, const int* njobs, const LargeJob& single, uint32_t* bar,
                         uint32_t* bar_status, cudaStream_t st) {
  static int occ_cache[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (occ_cache[dev] == 0) {
    int occ = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_large, LBLOCK, 0);
    if (e != cudaSuccess) return e;
    occ_cache[dev] = std::max(1, std::min(occ, 4));
  }
  const unsigned G = (unsigned)(device_sm_count() * occ_cache[dev]);
  LargeJob one = single;
  const LargeJob* tab = table;
  const int* nj = njobs;
  uint32_t* b = bar;
  uint32_t* bs = bar_status;
  void* args[] = {(void*)&tab, (void*)&nj, (void*)&one, (void*)&b, (void*)&bs};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_large, dim3(G), dim3(LBLOCK), args, 0, st);
  count_launches(1);
  return e;
}

}  // namespace cudapre
