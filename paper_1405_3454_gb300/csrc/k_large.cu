// k_large.cu -- the hull of a survivor set too large for the one-block path:
// device LSD radix sort of the (x, y) keys with their point indices, then
// Andrew's monotone chain over the sorted keys, chunked (section 3, case (2):
// the hull of the points that remain; the paper ran Qhull on the CPU there).
//
// Two cooperative launches do the whole stage for a list of jobs (one per
// point set): the sort, then the chains, each phase's steps separated by a
// grid barrier.  The sort runs one
// sweep per 8-bit digit of the 52-bit keys that varies among them (at most
// 7): each sweep reads and writes every element once, tiles finding their
// output offsets by decoupled look-back (see sort_pass).  The chain is
// chunked: level 0 chains every sorted chunk of CHAIN_C0 keys, each later
// level concatenates CHAIN_FAN consecutive chunk chains (still sorted) and
// chains them again, until one chunk is left.  A hull vertex of the whole
// set is a vertex of every chunk chain that contains it, so the last chain
// is the hull.  Among equal keys the lowest index is kept.  Each chunk (or
// group of chunk chains) is one warp's: it reads its input coalesced into
// shared memory, its lanes chain short runs of it in parallel, and lane 0
// (and lane 16, for the other side) walks only the vertices of those runs'
// chains (see window_chain).
//
// Every size is read on the device.  A job whose count is at most SMALL_MAX
// (the small-set path has written its result) or whose status word is set
// is skipped by every block alike.  Barrier and look-back waits are
// bounded: on expiry the kernel records HULL_DEVICE_TIMEOUT and returns.
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

// ----------------------------------------------------------------------------
// One-sweep LSD radix sort.  Every pass reads each (key, index) once and
// writes it once.  A block claims tiles of SORT_TILE elements in order from
// a counter; per tile it ranks the elements by digit (per-warp counts, the
// lanes sharing a digit found by nine ballots; one warp per 512-element
// slice, so ranks are stable), publishes
// the tile's per-digit counts in the tile's status words, and finds how many
// elements of each digit all earlier tiles hold by looking back over their
// status words (decoupled look-back: a word holds either the tile's own
// count or the inclusive prefix through that tile; the walk adds counts until
// it meets a prefix).  The tile is then reordered by digit in shared memory
// and written out in that order, so consecutive threads write consecutive
// addresses.  Status words carry the pass number, so one clearing per job
// serves every pass.  A pass whose digit is the same for every key moves
// nothing and is skipped: a bit varies among the keys iff both the OR of the
// keys and the OR of their complements have it.  The digit histograms of
// all passes are counted in one read of the keys before the first pass,
// with the two ORs.

constexpr unsigned long long ST_AGG = 1ull << 62;     // the word holds the tile's own count
constexpr unsigned long long ST_PREFIX = 2ull << 62;  // ... the inclusive prefix through the tile
constexpr int ST_TAG_SHIFT = 58;                      // 4-bit pass tag (pass + 1)
constexpr unsigned long long ST_COUNT = (1ull << ST_TAG_SHIFT) - 1;
constexpr int LOOK = 8;  // status words of earlier tiles read at once in the look-back

__device__ __forceinline__ unsigned long long st_word(unsigned long long state, int pass, unsigned long long c) {
  return state | ((unsigned long long)(pass + 1) << ST_TAG_SHIFT) | c;
}

// Shared memory of the sort (dynamic): the tile reordered by digit, and the
// per-warp / per-digit bookkeeping.  The histogram phase reuses the key area.
struct SortSmem {
  unsigned long long keys[SORT_TILE];
  uint32_t vals[SORT_TILE];
  uint32_t wc[WARPS][256];     // per warp: digit counts, then their exclusive prefix over warps
  uint32_t lstart[256];        // first position of each digit in the reordered tile
  long long delta[256];        // output position - position in the reordered tile, per digit
  uint32_t excl[256];          // elements of all keys with a smaller digit (this pass)
  uint32_t wsum[WARPS];
  uint32_t tile;
};

// The launch's dynamic shared memory, named inside each phase function: the
// phases are out of line, and a struct passed by reference would reach them
// as a generic pointer (generic accesses, and global loads kept in order
// with the shared-memory stores they might alias).
template <class T>
__device__ __forceinline__ T& dyn_smem() {
  extern __shared__ __align__(16) unsigned char k_large_smem[];
  return *reinterpret_cast<T*>(k_large_smem);
}

// Passes whose digit varies among the keys, as a bit mask (bit p: pass p).
__device__ __forceinline__ unsigned live_passes(const WsHeader* h) {
  const unsigned long long v = h->key_or & h->key_nor;
  unsigned mask = 0;
  for (int p = 0; p < SORT_PASSES; ++p)
    if ((v >> (8 * p)) & 255ull) mask |= 1u << p;
  return mask;
}

// One read of the keys: the digit histograms of every pass (a histogram
// does not depend on the order of the keys, so each pass's is known before
// any pass runs), the OR of the keys and of their complements, and the job's
// tile status words cleared.
__device__ __noinline__ void hist_read(const unsigned long long* keys, int64_t m, WsHeader* h,
                                       unsigned long long* status, int64_t nstatus) {
  SortSmem& S = dyn_smem<SortSmem>();
  // HCOPIES sub-histograms per pass (warp w counts into copy w % HCOPIES) in
  // the key area, to spread the shared-memory atomics
  constexpr int HCOPIES = 4;
  constexpr int HN = SORT_PASSES * HCOPIES * 256;
  static_assert(HN * 4 <= (int)sizeof(S.keys), "sub-histograms fit");
  uint32_t* hs = reinterpret_cast<uint32_t*>(S.keys);
  for (int k = threadIdx.x; k < HN; k += LBLOCK) hs[k] = 0;
  __syncthreads();
  uint32_t* mine = hs + ((threadIdx.x >> 5) % HCOPIES) * 256;
  const int64_t gt = (int64_t)blockIdx.x * LBLOCK + threadIdx.x, gs = (int64_t)gridDim.x * LBLOCK;
  unsigned long long o = 0, no = 0;
  for (int64_t j = gt; j < m; j += gs) {
    const unsigned long long k = __ldcs(keys + j);
    o |= k;
    no |= ~k;
#pragma unroll
    for (int p = 0; p < SORT_PASSES; ++p) atomicAdd(&mine[p * HCOPIES * 256 + digit(k, p)], 1u);
  }
  for (int off = 16; off; off >>= 1) {
    o |= __shfl_xor_sync(FULL, o, off);
    no |= __shfl_xor_sync(FULL, no, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicOr(&h->key_or, o);
    atomicOr(&h->key_nor, no);
  }
  for (int64_t j = gt; j < nstatus; j += gs) status[j] = 0ull;
  __syncthreads();
  for (int k = threadIdx.x; k < SORT_PASSES * 256; k += LBLOCK) {
    const int p = k >> 8, d = k & 255;
    uint32_t c = 0;
#pragma unroll
    for (int q = 0; q < HCOPIES; ++q) c += hs[(p * HCOPIES + q) * 256 + d];
    if (c) atomicAdd(&h->hist[p][d], c);
  }
  __syncthreads();
}

// Exclusive block scan of one value per thread (LBLOCK == 256 threads).
__device__ __forceinline__ uint32_t block_excl_scan(SortSmem& S, uint32_t v) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t u = __shfl_up_sync(FULL, incl, off);
    if (lane >= off) incl += u;
  }
  if (lane == 31) S.wsum[warp] = incl;
  __syncthreads();
  uint32_t pre = 0;
  for (int w = 0; w < warp; ++w) pre += S.wsum[w];
  __syncthreads();
  return pre + incl - v;
}

// One pass over m elements from (kin, vin) to (kout, vout).  Returns false
// when a look-back wait gave up (nothing more is written).
__device__ __noinline__ bool sort_pass(const unsigned long long* kin, const uint32_t* vin,
                                       unsigned long long* kout, uint32_t* vout, int64_t m, int pass,
                                       const uint32_t* hist, uint32_t* tile_next, unsigned long long* status,
                                       uint32_t* gstatus) {
  SortSmem& S = dyn_smem<SortSmem>();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, d0 = threadIdx.x;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t nt = (m + SORT_TILE - 1) / SORT_TILE;
  // elements with a smaller digit, over the whole set (thread d0 = digit d0)
  {
    const uint32_t c = hist[pass * 256 + d0];
    S.excl[d0] = block_excl_scan(S, c);
  }
  bool ok = true;
  for (;;) {
    if (threadIdx.x == 0) S.tile = atomicAdd(tile_next + pass, 1u);
    for (int k = threadIdx.x; k < WARPS * 256; k += LBLOCK) (&S.wc[0][0])[k] = 0;
    __syncthreads();
    const int64_t t = S.tile;
    if (t >= nt) break;
    // load the warp's slice in rows of 32 and rank each element among the
    // earlier elements of its warp with the same digit
    const int64_t b = t * SORT_TILE + (int64_t)warp * PER_WARP;
    unsigned long long kk[ROWS];
    uint32_t vv[ROWS];
    uint32_t rk2[ROWS / 2];  // ranks (< 4096), two per word
    unsigned valid = 0;      // bit r: row r holds an element
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const int64_t j = b + r * 32 + lane;
      if (j < m) { kk[r] = kin[j]; vv[r] = vin[j]; valid |= 1u << r; }
      else { kk[r] = 0; vv[r] = 0; }
    }
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      const uint32_t d = ((valid >> r) & 1u) ? digit(kk[r], pass) : 256u;
      // lanes with the same digit (9 bits: 256 marks a lane past the end)
      unsigned peers = FULL;
#pragma unroll
      for (int bt = 0; bt < 9; ++bt) {
        const bool on = (d >> bt) & 1u;
        const unsigned bal = __ballot_sync(FULL, on);
        peers &= on ? bal : ~bal;
      }
      const uint32_t c = d < 256u ? S.wc[warp][d] : 0u;
      const uint32_t rank = c + (uint32_t)__popc(peers & lt);
      if (r & 1) rk2[r >> 1] |= rank << 16; else rk2[r >> 1] = rank;
      __syncwarp();
      if (d < 256u && lane == __ffs(peers) - 1) S.wc[warp][d] = c + (uint32_t)__popc(peers);
      __syncwarp();
    }
    __syncthreads();
    // thread d0: the tile's count of digit d0, the warps' offsets within it
    uint32_t cnt = 0;
#pragma unroll
    for (int w = 0; w < WARPS; ++w) { const uint32_t c = S.wc[w][d0]; S.wc[w][d0] = cnt; cnt += c; }
    unsigned long long* my = status + (size_t)t * 256 + d0;
    // publish the count at once, so later tiles need not wait for our look-back
    atomicExch(my, t == 0 ? st_word(ST_PREFIX, pass, cnt) : st_word(ST_AGG, pass, cnt));
    const uint32_t ls = block_excl_scan(S, cnt);
    S.lstart[d0] = ls;
    __syncthreads();
    // reorder the tile by digit in shared memory (stable)
#pragma unroll
    for (int r = 0; r < ROWS; ++r) {
      if ((valid >> r) & 1u) {
        const uint32_t d = digit(kk[r], pass);
        const uint32_t pos = S.lstart[d] + S.wc[warp][d] + ((rk2[r >> 1] >> (16 * (r & 1))) & 0xFFFFu);
        S.keys[pos] = kk[r];
        S.vals[pos] = vv[r];
      }
    }
    // (the tile's data now lives in shared memory only: the look-back holds
    // no element registers)
    // look back over the earlier tiles' words for this digit
    // (LOOK words at a time, loaded together: tile q, q - 1, ...; the walk
    // consumes them in order and stops at the first prefix; a word not yet
    // published is read again)
    unsigned long long before = 0;
    if (t > 0) {
      int64_t q = t - 1;
      const long long t0 = clock64();
      bool done = false;
      while (!done) {
        unsigned long long w[LOOK];
#pragma unroll
        for (int k = 0; k < LOOK; ++k)
          w[k] = q - k >= 0 ? *reinterpret_cast<volatile unsigned long long*>(status + (size_t)(q - k) * 256 + d0)
                            : 0ull;
        int used = 0;
        bool stall = false;
#pragma unroll
        for (int k = 0; k < LOOK; ++k) {
          if (done || stall) continue;
          if ((int)((w[k] >> ST_TAG_SHIFT) & 15u) == pass + 1 && (w[k] & (3ull << 62))) {
            before += w[k] & ST_COUNT;
            ++used;
            if (w[k] & ST_PREFIX) done = true;
          } else {
            stall = true;
          }
        }
        q -= used;
        if (!done && stall && clock64() - t0 > BAR_LIMIT_CYCLES) {
          atomicOr(gstatus, HULL_DEVICE_TIMEOUT);
          ok = false;
          break;
        }
      }
      if (ok) atomicExch(my, st_word(ST_PREFIX, pass, before + cnt));
    }
    S.delta[d0] = (long long)S.excl[d0] + (long long)before - (long long)ls;
    const int okb = __syncthreads_and(ok ? 1 : 0);
    if (!okb) return false;
    // write it out in that order: each digit's run goes to consecutive addresses
    const int tn = (int)min((int64_t)SORT_TILE, m - t * SORT_TILE);
    for (int j = threadIdx.x; j < tn; j += LBLOCK) {
      const unsigned long long k = S.keys[j];
      const int64_t pos = (int64_t)j + S.delta[digit(k, pass)];
      kout[pos] = k;
      vout[pos] = S.vals[j];
    }
    __syncthreads();
  }
  return ok;
}

// ----------------------------------------------------------------------------
// The chains, one warp per chunk (level 0) or per group of chunk chains.
//
// A window of at most CHAIN_C0 + 2 entries (sorted keys with their indices)
// is chained in two levels: each of nl lanes chains S consecutive entries of
// it (S = max(ceil(entries / nl), RUN_MIN)) on a small stack of window
// entries, then one lane pushes the vertices of those run chains, in order,
// onto the chunk's running stack.  An entry off its run's chain lies on or
// above (lower chain; below for the upper one) the chain of a subset holding
// it, so it is no strict vertex of any larger set's chain either; the first
// and the last entry of every run stay.  At level 0 lanes 0-15 do a chunk's
// lower chain and lanes 16-31 its upper chain on the same instruction stream
// (the turn's sense is a run-time sign), so lanes 0 and 16 walk the two
// chains side by side; later levels do the same with a group's lower and
// upper chains.  The
// running stack keeps its last RING entries in shared memory (slot e % RING,
// tagged with e); an entry leaving the ring while it is still on the stack
// is written to its final place in global memory (entry e at base + e), and
// finish() writes the rest, so only deep stacks touch global memory before
// the end.
constexpr int RUN_MIN = 8;                               // entries of a run at least
constexpr int RUN_CAP = 16 * ((CHAIN_C0 + 2 + 15) / 16);  // run entries of a side (16 or 32 lanes)
constexpr int RING = 64;
static_assert((RING & (RING - 1)) == 0, "ring slots by mask");

struct WarpChain {
  unsigned long long k[CHAIN_C0];  // the chunk's elements (level 0) or the window (later levels)
  unsigned long long rk[2][RING];  // per side: ring of the running stack's last entries
  int64_t rpos[2][RING];           // ... the entry each slot holds
  uint32_t v[CHAIN_C0];
  uint32_t rv[2][RING];
  int runn[32];                    // run chain lengths, by lane
  int64_t off[2][CHAIN_FAN + 1];   // later levels, per side: the group's chain offsets
  uint16_t pos[2][CHAIN_C0 + 2];   // level 0, per side: the window's entries as positions in k / v
  uint16_t run[2][RUN_CAP];        // per side: run chains (window entries), run i's from i * S
};
struct ChainSmem {
  WarpChain w[WARPS];
};

// The running stack of one chain: push by one lane, init and finish by the
// warp.  sg = +1: lower chain (pop while the turn is not strictly left);
// sg = -1: upper chain (pop while it is not strictly right).
struct RunStack {
  unsigned long long* K;  // output: entry e at K[base + e], V[base + e]
  uint32_t* V;
  unsigned long long* rk;  // this side's ring
  uint32_t* rv;
  int64_t* rpos;
  int64_t base;
  int64_t n;                  // entries
  unsigned long long k1, k2;  // top and second keys
  uint32_t v1;                // top index
  long long sg;

  __device__ __forceinline__ void init(WarpChain& W, int side, unsigned long long* k, uint32_t* v, int64_t b,
                                       long long sign) {
    K = k; V = v; base = b; n = 0; k1 = k2 = 0; v1 = 0; sg = sign;
    rk = W.rk[side]; rv = W.rv[side]; rpos = W.rpos[side];
  }
  // a tag no entry position (nor n - RING) can take; warp-wide
  static __device__ __forceinline__ void clear(WarpChain& W, int side) {
    for (int i = threadIdx.x & 31; i < RING; i += 32) W.rpos[side][i] = INT64_MIN;
  }
  static __device__ __forceinline__ int slot(int64_t e) { return (int)((uint64_t)e & (RING - 1)); }
  // entry e (< n): from its ring slot, else from global memory (it left the
  // ring while on the stack, so it was written there)
  __device__ __forceinline__ void entry(int64_t e, unsigned long long& k, uint32_t& v) const {
    const int q = slot(e);
    if (rpos[q] == e) { k = rk[q]; v = rv[q]; }
    else { k = K[base + e]; v = V[base + e]; }
  }
  __device__ __forceinline__ void push(unsigned long long key, uint32_t val) {
    if (n > 0 && key == k1) {  // equal coordinates: the lowest index stands
      if (val < v1) {
        v1 = val;
        const int q = slot(n - 1);
        if (rpos[q] == n - 1) rv[q] = val;
        else V[base + n - 1] = val;
      }
      return;
    }
    while (n >= 2 && sg * cross_k(k2, k1, key) <= 0) {
      --n;
      k1 = k2;
      unsigned long long kk;
      entry(n - 1, kk, v1);
      if (n >= 2) { uint32_t vv; entry(n - 2, k2, vv); }
    }
    const int q = slot(n);
    if (rpos[q] == n - RING) {  // a stack entry leaves the ring
      K[base + n - RING] = rk[q];
      V[base + n - RING] = rv[q];
    }
    rk[q] = key;
    rv[q] = val;
    rpos[q] = n;
    ++n;
    k2 = k1;
    k1 = key;
    v1 = val;
  }
  // warp-wide, after the last push (by lane `owner`): the entries still in
  // the ring to global memory; returns n
  __device__ __forceinline__ int64_t finish(int owner) {
    const int64_t nn = __shfl_sync(FULL, n, owner);
    unsigned long long* KK = reinterpret_cast<unsigned long long*>(__shfl_sync(FULL, (unsigned long long)K, owner));
    uint32_t* VV = reinterpret_cast<uint32_t*>(__shfl_sync(FULL, (unsigned long long)V, owner));
    const int64_t bb = __shfl_sync(FULL, base, owner);
    unsigned long long* RK = reinterpret_cast<unsigned long long*>(__shfl_sync(FULL, (unsigned long long)rk, owner));
    uint32_t* RV = reinterpret_cast<uint32_t*>(__shfl_sync(FULL, (unsigned long long)rv, owner));
    int64_t* RP = reinterpret_cast<int64_t*>(__shfl_sync(FULL, (unsigned long long)rpos, owner));
    for (int64_t e = max(nn - RING, (int64_t)0) + (threadIdx.x & 31); e < nn; e += 32) {
      const int q = slot(e);
      if (RP[q] == e) { KK[bb + e] = RK[q]; VV[bb + e] = RV[q]; }
    }
    __syncwarp();
    return nn;
  }
};

// Lane-level chain of window entries [lo, lo + len) onto q (window entries);
// returns its length.  Entry e is element ps[e], or element eb + e when ps
// is null.
__device__ __forceinline__ int run_chain(const WarpChain& W, const uint16_t* ps, int eb, int lo, int len,
                                         uint16_t* q, long long sg) {
  auto el = [&](int e) { return ps ? (int)ps[e] : eb + e; };
  int n = 0;
  unsigned long long k1 = 0, k2 = 0;
  for (int t = 0; t < len; ++t) {
    const int e = lo + t;
    const int p = el(e);
    const unsigned long long key = W.k[p];
    if (n > 0 && key == k1) {  // equal coordinates: keep the lower index
      if (W.v[p] < W.v[el(q[n - 1])]) q[n - 1] = (uint16_t)e;
      continue;
    }
    while (n >= 2 && sg * cross_k(k2, k1, key) <= 0) {
      --n;
      k1 = k2;
      if (n >= 2) k2 = W.k[el(q[n - 2])];
    }
    q[n++] = (uint16_t)e;
    k2 = k1;
    k1 = key;
  }
  return n;
}

// One window of `len` (<= CHAIN_C0 + 2) entries of side `side` onto R, by
// the nl lanes from lane0 (all lanes call it; each lane's arguments are its
// group's); lane0 walks and owns R.  Entry e is element ps[e], or element
// eb + e when ps is null.
__device__ __forceinline__ void window_chain(WarpChain& W, int side, const uint16_t* ps, int eb, int lane0, int nl,
                                             int len, RunStack& R) {
  const int lane = threadIdx.x & 31, li = lane - lane0;
  const int S = max((len + nl - 1) / nl, RUN_MIN);
  const int lo = min(li * S, len), n = max(min(S, len - lo), 0);
  uint16_t* run = W.run[side];
  W.runn[lane] = n > 0 ? run_chain(W, ps, eb, lo, n, run + li * S, R.sg) : 0;
  __syncwarp();
  if (li == 0) {
    const int nr = (len + S - 1) / S;
    for (int l = 0; l < nr; ++l) {
      const int c = W.runn[lane0 + l];
      for (int i = 0; i < c; ++i) {
        const int e = run[l * S + i];
        const int p = ps ? (int)ps[e] : eb + e;
        R.push(W.k[p], W.v[p]);
      }
    }
  }
  __syncwarp();
}

// First position of the run of keys equal to W.k[e] (within the chunk);
// after chain0's first step its slot holds the run's lowest index.
__device__ __forceinline__ int run_start(const WarpChain& W, int e) {
  while (e > 0 && W.k[e - 1] == W.k[e]) --e;
  return e;
}

// Level 0: warp w chains sorted elements [t*C0, min((t+1)*C0, m)) for its
// chunks t; the lower chain in place in (Ks, Vs), the upper chain into (Ku,
// Vu) at the same offsets; counts to cnt_lo[t], cnt_up[t].  Only the lowest
// point of an x column can be a lower-chain vertex and only its highest an
// upper-chain vertex (every other point of the column lies between them on a
// vertical segment), so the lower chain takes the first point of every
// column of the chunk and the upper chain the last key of every column
// (with the lowest index among its copies).  The whole hull's lower chain
// must still end, and its upper chain start, at the lexicographic maximum
// resp. minimum (the emission joins them there), so every chunk also gives
// its last key to the lower chain and its first point to the upper one.
__device__ __noinline__ void chain0(unsigned long long* Ks, uint32_t* Vs, unsigned long long* Ku,
                                    uint32_t* Vu, int64_t m, uint32_t* cnt_lo, uint32_t* cnt_up) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  WarpChain& W = dyn_smem<ChainSmem>().w[warp];
  const int64_t nch = (m + CHAIN_C0 - 1) / CHAIN_C0;
  for (int64_t t = (int64_t)blockIdx.x * WARPS + warp; t < nch; t += (int64_t)gridDim.x * WARPS) {
    const int64_t tb = t * CHAIN_C0;
    const int tn = (int)min((int64_t)CHAIN_C0, m - tb);
    // the chunk in rows of 32, eight rows' loads in flight at a time
    constexpr int R8 = 8;
    for (int r0 = 0; r0 < CHAIN_C0 / 32; r0 += R8) {
      unsigned long long kk[R8];
      uint32_t vv[R8];
#pragma unroll
      for (int r = 0; r < R8; ++r) {
        const int e = (r0 + r) * 32 + lane;
        if (e < tn) { kk[r] = Ks[tb + e]; vv[r] = Vs[tb + e]; }
      }
#pragma unroll
      for (int r = 0; r < R8; ++r) {
        const int e = (r0 + r) * 32 + lane;
        if (e < tn) { W.k[e] = kk[r]; W.v[e] = vv[r]; }
      }
    }
    RunStack::clear(W, 0);
    RunStack::clear(W, 1);
    __syncwarp();
    // Equal keys are adjacent but their indices in no order (survivors come
    // in compaction order): the first slot of every run of equal keys takes
    // the run's lowest index, and the candidates below are run starts.
    for (int e0 = 0; e0 < tn; e0 += 32) {
      const int e = e0 + lane;
      if (e < tn && e > 0 && W.k[e - 1] == W.k[e] && (e == tn - 1 || W.k[e + 1] != W.k[e])) {
        int s = e;
        uint32_t mv = W.v[e];
        while (s > 0 && W.k[s - 1] == W.k[e]) {
          --s;
          mv = min(mv, W.v[s]);
        }
        W.v[s] = mv;
      }
    }
    __syncwarp();
    // lower list: the first point of every column, then the chunk's last key;
    // upper list: the chunk's first point, then the last key of every column
    int Llo = 0, Lup = 1;
    if (lane == 0) W.pos[1][0] = 0;
    for (int e0 = 0; e0 < tn; e0 += 32) {
      const int e = e0 + lane;
      const int x = e < tn ? key_x(W.k[e]) : 0;
      const bool flo = e < tn && (e == 0 || key_x(W.k[e - 1]) != x);
      const bool fup = e < tn && (e == tn - 1 || key_x(W.k[e + 1]) != x);
      const unsigned blo = __ballot_sync(FULL, flo), bup = __ballot_sync(FULL, fup);
      if (flo) W.pos[0][Llo + __popc(blo & lt)] = (uint16_t)e;
      if (fup) W.pos[1][Lup + __popc(bup & lt)] = (uint16_t)run_start(W, e);
      Llo += __popc(blo);
      Lup += __popc(bup);
    }
    if (lane == 0) W.pos[0][Llo] = (uint16_t)run_start(W, tn - 1);
    ++Llo;
    __syncwarp();
    const int side = lane >> 4;
    RunStack R;
    R.init(W, side, side ? Ku : Ks, side ? Vu : Vs, tb, side ? -1 : 1);
    window_chain(W, side, W.pos[side], 0, side * 16, 16, side ? Lup : Llo, R);
    const int64_t nlo = R.finish(0);
    const int64_t nup = R.finish(16);
    if (lane == 0) {
      cnt_lo[t] = (uint32_t)nlo;
      cnt_up[t] = (uint32_t)nup;
    }
    __syncwarp();
  }
}

// One group of a later level: the chains of chunks [c0, c1) of the previous
// level (span `span` each, counts cin_lo / cin_up), concatenated in order
// (still sorted), chained again in place from c0 * span by one warp, lanes
// 0-15 the lower chains and lanes 16-31 the upper ones side by side, window
// by window (each side's window takes half of the chunk area).  An unread
// entry j of a side's concatenation sits at or after c0 * span + j, and the
// stack's entry e is written at c0 * span + e with e below the entries read
// so far, so no write reaches input not yet read.
__device__ __forceinline__ void merge_group(WarpChain& W, unsigned long long* Ks, uint32_t* Vs,
                                            unsigned long long* Ku, uint32_t* Vu, const uint32_t* cin_lo,
                                            const uint32_t* cin_up, int64_t c0, int64_t c1, int64_t span,
                                            uint32_t* out_lo, uint32_t* out_up) {
  constexpr int WCAP = CHAIN_C0 / 2;
  const int lane = threadIdx.x & 31, side = lane >> 4, li = lane & 15;
  const int nc = (int)(c1 - c0);  // at most CHAIN_FAN == 32
  for (int sd = 0; sd < 2; ++sd) {  // the chain offsets of both sides (warp-wide scans)
    const int64_t cnt = lane < nc ? (int64_t)(sd ? cin_up : cin_lo)[c0 + lane] : 0;
    int64_t incl = cnt;
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t u = __shfl_up_sync(FULL, incl, off);
      if (lane >= off) incl += u;
    }
    if (lane == 0) W.off[sd][0] = 0;
    if (lane < nc) W.off[sd][lane + 1] = incl;
  }
  RunStack::clear(W, 0);
  RunStack::clear(W, 1);
  __syncwarp();
  unsigned long long* K = side ? Ku : Ks;
  uint32_t* V = side ? Vu : Vs;
  const int64_t total = W.off[side][nc];
  const int64_t tmax = max(W.off[0][nc], W.off[1][nc]);
  RunStack R;
  R.init(W, side, K, V, c0 * span, side ? -1 : 1);
  const int eb = side * WCAP;
  for (int64_t w0 = 0; w0 < tmax; w0 += WCAP) {
    const int len = (int)max(min((int64_t)WCAP, total - w0), (int64_t)0);
    for (int c = 0; c < nc; ++c) {
      const int64_t oc = W.off[side][c];
      const int64_t a = max(oc, w0), b = min(W.off[side][c + 1], w0 + len);
      const int64_t src = (c0 + c) * span - oc;
      for (int64_t j = a + li; j < b; j += 16) {
        W.k[eb + (j - w0)] = K[src + j];
        W.v[eb + (j - w0)] = V[src + j];
      }
    }
    __syncwarp();
    window_chain(W, side, nullptr, eb, side * 16, 16, len, R);
  }
  const int64_t nlo = R.finish(0), nup = R.finish(16);
  if (lane == 0) {
    *out_lo = (uint32_t)nlo;
    *out_up = (uint32_t)nup;
  }
  __syncwarp();
}

// Later level: group g merges the chains of chunks [g*FAN, (g+1)*FAN) of the
// previous level, one warp per group.
__device__ __noinline__ void chainN(unsigned long long* Ks, uint32_t* Vs, unsigned long long* Ku,
                                    uint32_t* Vu, const uint32_t* cin_lo, const uint32_t* cin_up, uint32_t* cout_lo,
                                    uint32_t* cout_up, int64_t nch_prev, int64_t span) {
  const int warp = threadIdx.x >> 5;
  WarpChain& W = dyn_smem<ChainSmem>().w[warp];
  const int64_t ng = (nch_prev + CHAIN_FAN - 1) / CHAIN_FAN;
  for (int64_t g = (int64_t)blockIdx.x * WARPS + warp; g < ng; g += (int64_t)gridDim.x * WARPS) {
    const int64_t c0 = g * CHAIN_FAN;
    const int64_t c1 = min(c0 + (int64_t)CHAIN_FAN, nch_prev);
    merge_group(W, Ks, Vs, Ku, Vu, cin_lo, cin_up, c0, c1, span, cout_lo + g, cout_up + g);
  }
}

// The hull counter-clockwise from the lexicographic minimum: the lower chain
// left to right, then the upper chain right to left, without repeating the
// two end points.
__device__ __noinline__ void chain_emit(const uint32_t* Vs, const uint32_t* Vu, const uint32_t* cnt_lo, const uint32_t* cnt_up,
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

// phase 0: the histograms and the sort passes of every job; phase 1: the
// chains and the emission of every job (a launch of its own, so that each
// phase gets the dynamic shared memory it needs and the sort keeps the rest
// of the SM's memory as L1).
__global__ void __launch_bounds__(LBLOCK, 2) k_large(const LargeJob* __restrict__ table, const int* njobs_dev,
                                                   LargeJob single, uint32_t* bar, uint32_t* bar_status, int phase) {
  if (*reinterpret_cast<const volatile uint32_t*>(bar_status) & HULL_DEVICE_TIMEOUT) return;
  const int njobs = table ? *reinterpret_cast<const volatile int*>(njobs_dev) : 1;
  for (int jb = 0; jb < njobs; ++jb) {
    const LargeJob J = table ? table[jb] : single;
    if (*reinterpret_cast<const volatile uint32_t*>(&J.h->status)) continue;
    const int64_t m = (int64_t)*reinterpret_cast<const volatile unsigned long long*>(J.count);
    if (m <= SMALL_MAX) continue;
    if (phase == 0) {
      const int64_t nt = (m + SORT_TILE - 1) / SORT_TILE;
      hist_read(J.ka, m, J.h, J.tilecnt, nt * 256);
      if (!grid_sync(bar, bar_status)) return;
      const unsigned live = live_passes(J.h);  // the passes that move anything
      unsigned long long *kin = J.ka, *kout = J.kb;
      uint32_t *vin = J.va, *vout = J.vb;
      for (int p = 0; p < SORT_PASSES; ++p) {
        if (!((live >> p) & 1u)) continue;
        const bool ok = sort_pass(kin, vin, kout, vout, m, p, &J.h->hist[0][0], J.h->tile_next, J.tilecnt,
                                  bar_status);
        if (!grid_sync(bar, bar_status) || !ok) return;
        unsigned long long* tk = kin; kin = kout; kout = tk;
        uint32_t* tv = vin; vin = vout; vout = tv;
      }
      // the next job uses other buffers and its own counters; the barrier
      // words are balanced, so it needs no barrier first
      continue;
    }
    // sorted in (kin, vin): the buffer the last live pass wrote; upper
    // chains go to (kout, vout)
    const bool odd = __popc(live_passes(J.h)) & 1;
    unsigned long long *kin = odd ? J.kb : J.ka, *kout = odd ? J.ka : J.kb;
    uint32_t *vin = odd ? J.vb : J.va, *vout = odd ? J.va : J.vb;
    const int64_t nch0 = (std::max<int64_t>(J.cap, 1) + CHAIN_C0 - 1) / CHAIN_C0;
    uint32_t* lo[2] = {J.cnt, J.cnt + 2 * nch0};
    uint32_t* up[2] = {J.cnt + nch0, J.cnt + 3 * nch0};
    chain0(kin, vin, kout, vout, m, lo[0], up[0]);
    if (!grid_sync(bar, bar_status)) return;
    int64_t nch = (m + CHAIN_C0 - 1) / CHAIN_C0, span = CHAIN_C0;
    int par = 0;
    while (nch > 1) {
      chainN(kin, vin, kout, vout, lo[par], up[par], lo[par ^ 1], up[par ^ 1], nch, span);
      if (!grid_sync(bar, bar_status)) return;
      par ^= 1;
      nch = (nch + CHAIN_FAN - 1) / CHAIN_FAN;
      span *= CHAIN_FAN;
    }
    chain_emit(vin, vout, lo[par], up[par], J.out_idx, J.out_n);
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
  static int occ_cache[64][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  const size_t dsm[2] = {sizeof(SortSmem), sizeof(ChainSmem)};
  if (occ_cache[dev][0] == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_large, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)std::max(dsm[0], dsm[1]));
    if (e != cudaSuccess) return e;
    for (int ph = 0; ph < 2; ++ph) {
      int occ = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_large, LBLOCK, dsm[ph]);
      if (e != cudaSuccess) return e;
      occ_cache[dev][ph] = std::max(1, std::min(occ, 4));
    }
  }
  LargeJob one = single;
  const LargeJob* tab = table;
  const int* nj = njobs;
  uint32_t* b = bar;
  uint32_t* bs = bar_status;
  for (int ph = 0; ph < 2; ++ph) {
    const unsigned G = (unsigned)(device_sm_count() * occ_cache[dev][ph]);
    int phase = ph;
    void* args[] = {(void*)&tab, (void*)&nj, (void*)&one, (void*)&b, (void*)&bs, (void*)&phase};
    const cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_large, dim3(G), dim3(LBLOCK), args, dsm[ph], st);
    count_launches(1);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cudapre
