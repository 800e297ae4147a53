// stream.cuh -- bulk-copy (TMA engine) streaming of a block's range of 16-byte
// point pairs into a ring of shared-memory stages, for the two passes over
// the points (the extreme search and the inside test).
//
// One producer warp (its lane 0) issues cp.async.bulk copies of CHUNK pairs
// per stage; the copy engine signals the stage's "full" mbarrier with the
// transferred byte count.  Consumer warps wait on "full", copy their pairs to
// registers and arrive on the stage's "empty" mbarrier as soon as they no
// longer read the stage (the inside test at once, the extreme search after
// its rare path), so the producer can refill it while they compute.  Every
// wait is bounded: on timeout the kernel records HULL_DEVICE_TIMEOUT and
// stops streaming.
#pragma once

#include <algorithm>

#include "internal.cuh"

namespace cudapre {

constexpr int CONSUMERS = 256;               // consumer threads (8 warps)
constexpr int PRODUCER_WARP = CONSUMERS / 32;
constexpr int STREAM_THREADS = CONSUMERS + 32;
constexpr int CHUNK = 4 * CONSUMERS;         // pairs per stage (4 per consumer thread)
constexpr long long WAIT_LIMIT_CYCLES = 1ll << 31;  // about one second
// A large batch's streaming passes launch up to BATCH_WAVES waves of resident
// blocks: the block scheduler then hands the shares out as SMs free up, which
// evens out sets of unequal cost per point.  Every block keeps at least
// WAVE_MIN_CHUNKS chunks; one set takes one wave (equal cost per point).
constexpr int BATCH_WAVES = 4;
constexpr int64_t WAVE_MIN_CHUNKS = 32;
constexpr int64_t MAX_STREAM_BLOCKS = 4096;  // partial-result slots per call
// One set streams with partly dynamic shares: every block first takes a
// static run of DYN_STATIC_PCT percent of an equal share, then producers
// claim groups of DYN_GROUP chunks of the rest from a counter in the set's
// header, so blocks that draw more bandwidth take more chunks (equal static
// shares ended up to 2x apart in time on a 2^28-point set).
constexpr int DYN_GROUP = 4;
constexpr int DYN_STATIC_PCT = 75;
// Largest unit of a batch's dynamic streaming, in chunks: the inside test
// keeps no state across units; the extreme search carries its running bests
// across units of one set, but starts afresh (and re-seeds) on each new set.
constexpr int64_t FILTER_UNIT_CHUNKS = 64;
constexpr int64_t EXT_UNIT_CHUNKS = 64;

inline int stream_waves(int sets, int64_t npairs, int64_t resident_blocks, int max_waves = 0) {
  if (sets <= 1) return 1;
  const int64_t w = npairs / (resident_blocks * WAVE_MIN_CHUNKS * CHUNK);
  return (int)std::max<int64_t>(1, std::min<int64_t>(max_waves > 0 ? max_waves : BATCH_WAVES, w));
}

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity; false (and the timeout
// bit set in *status) when it does not complete within `limit` cycles.
__device__ __forceinline__ bool mbar_wait_limit(unsigned long long* bar, unsigned parity, uint32_t* status,
                                                long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > limit) {
      atomicOr(status, HULL_DEVICE_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ bool mbar_wait_status(unsigned long long* bar, unsigned parity, uint32_t* status) {
  return mbar_wait_limit(bar, parity, status, WAIT_LIMIT_CYCLES);
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// What a stage holds when a batch streams by units (see
// stream_produce_units): the chunk's set, its unit, its first pair within
// the set and its pairs, and whether it opens / closes its segment (the
// part of one set inside one unit) or ends the stream.
constexpr int META_FIRST = 1, META_LAST = 2, META_END = 4;
struct ChunkMeta {
  int set;
  int unit;
  int first;
  int cnt;
  int flags;
};

// Shared state of one block's stream with NS stages.
template <int NS>
struct StreamSmemT {
  static constexpr int STAGES = NS;
  float4 stage[NS][CHUNK];
  unsigned long long full[NS];
  unsigned long long empty[NS];
  int id[NS];  // dynamic shares: the chunk in the stage, -1 = end of the stream
  ChunkMeta meta[NS];
};

// How a streaming pass splits the virtual pair axis [0, P) over its G
// blocks: block b first takes the static share [b ppb, min((b + 1) ppb, A)),
// then the blocks claim units of U pairs of [A, P) from a counter.  Results
// of (block b, set s) of the static part go to slot b + s, those of (unit u,
// set s) to slot G + u + s: every slot is one (share or unit, set) pair,
// because shares and units are contiguous, in axis order, and the static
// part comes first.
struct Split {
  int64_t ppb;  // pairs of a static share
  int64_t A;    // end of the static part (a multiple of ppb, or P)
  int64_t U;    // pairs of a unit of the dynamic part
  int64_t G;    // blocks
};

// A batch's streaming passes split the virtual pair axis into units of
// `upairs` pairs (a whole number of chunks) that blocks claim one at a time
// from a counter, so blocks whose sets cost more per point simply claim
// fewer units.  Unit u's results for set s go to slot u + s: units are
// contiguous and claimed in axis order, so the pair (u, s) -> u + s is one
// to one (a later unit never meets an earlier set).
inline int64_t unit_pairs(int64_t npairs, int64_t blocks, int64_t max_chunks) {
  const int64_t nck = (npairs + CHUNK - 1) / CHUNK;
  const int64_t per = nck / (8 * std::max<int64_t>(blocks, 1));  // about 8 units per block at least
  return std::max<int64_t>(1, std::min<int64_t>(max_chunks, per)) * CHUNK;
}

// The segments of a block's share [v0, v1) of the virtual pair axis, one
// per set it meets, in order (or in reverse): f(s, first local pair, pairs).
// Producer and consumers walk the same sequence; each splits a segment into
// chunks of CHUNK pairs anchored at the segment's first pair (chunk k of
// nchunks(n), visited first-to-last or last-to-first).
template <class F>
__device__ __forceinline__ void walk_segments(const Sets& S, int64_t v0, int64_t v1, bool reverse, F&& f) {
  if (v0 >= v1) return;
  if (!reverse) {
    int s = S.set_of_pair(v0);
    int64_t p = v0;
    for (;;) {
      const int64_t a = S.pp_at(s);
      const int64_t hi = min(v1, S.pp_at(s + 1));
      f(s, p - a, (int)(hi - p));
      p = hi;
      if (p >= v1) break;
      ++s;
      while (S.pp_at(s + 1) <= p) ++s;  // skip sets without pairs
    }
  } else {
    int s = S.set_of_pair(v1 - 1);
    int64_t p = v1;
    for (;;) {
      const int64_t a = S.pp_at(s);
      const int64_t lo = max(v0, a);
      f(s, lo - a, (int)(p - lo));
      p = lo;
      if (p <= v0) break;
      --s;
      while (s > 0 && S.pp_at(s) >= p) --s;  // the set holding pair p - 1
    }
  }
}

__device__ __forceinline__ int nchunks(int n) { return (n + CHUNK - 1) / CHUNK; }
// First pair (relative to the segment) and pair count of visit k.
__device__ __forceinline__ int chunk_first(int k, int nck, bool reverse) {
  return (reverse ? nck - 1 - k : k) * CHUNK;
}

// Named barrier of the consumer warps only (the producer warp runs ahead).
__device__ __forceinline__ void consumers_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(CONSUMERS) : "memory");
}

// Producer (lane 0 of the producer warp) over a walk of segments: every
// chunk into the next stage, waiting for a free stage each time; then it
// waits until the copies it issued have landed.
template <class SS>
__device__ __forceinline__ void stream_produce_sets(SS& SM, const Sets& S, int64_t v0, int64_t v1, bool reverse,
                                                    uint32_t* status) {
  constexpr int STAGES = SS::STAGES;
  if ((threadIdx.x & 31) != 0) return;
  int c = 0;
  bool stop = false;
  walk_segments(S, v0, v1, reverse, [&](int s, int64_t lo, int n) {
    const float4* P = reinterpret_cast<const float4*>(S.xy_of(s) + 2 * S.head_of(s)) + lo;
    const int nck = nchunks(n);
    for (int k = 0; k < nck && !stop; ++k, ++c) {
      const int st = c % STAGES;
      const int ph = c / STAGES;
      if (ph > 0 && !mbar_wait_status(&SM.empty[st], (unsigned)((ph - 1) & 1), status)) { stop = true; break; }
      if (*reinterpret_cast<volatile uint32_t*>(status) & HULL_DEVICE_TIMEOUT) { stop = true; break; }
      const int f = chunk_first(k, nck, reverse);
      const unsigned bytes = (unsigned)min(CHUNK, n - f) * 16u;
      mbar_arrive_tx(&SM.full[st], bytes);
      bulk_g2s(&SM.stage[st][0], P + f, bytes, &SM.full[st]);
    }
  });
  for (int d = c > STAGES ? c - STAGES : 0; d < c; ++d)
    mbar_wait_status(&SM.full[d % STAGES], (unsigned)((d / STAGES) & 1), status);
}

// Producer (lane 0 of the producer warp) with partly dynamic shares over
// the nck chunks of one set (npairs pairs from P).  Logical chunk k is
// chunk k, or nck - 1 - k when `reverse`.  Block b first streams logical
// chunks [b q, (b + 1) q), q = DYN_STATIC_PCT percent of nck / gridDim.x,
// then claims groups of the rest from *next (one claim kept in flight; every
// claimed group is streamed, so every chunk is streamed by exactly one
// block).  Each chunk's number goes into the stage before its "full" barrier
// is armed; -1 (a plain arrival) ends the stream.
template <class SS>
__device__ __forceinline__ void stream_produce_dynamic(SS& SM, const float4* P, int64_t npairs, uint32_t* next,
                                                       bool reverse, uint32_t* status) {
  constexpr int STAGES = SS::STAGES;
  if ((threadIdx.x & 31) != 0) return;
  const int nck = (int)((npairs + CHUNK - 1) / CHUNK);
  const int q = (int)((int64_t)nck * DYN_STATIC_PCT / 100 / gridDim.x);
  const int pool = q * (int)gridDim.x;  // first logical chunk of the shared pool
  const int ngroups = (nck - pool + DYN_GROUP - 1) / DYN_GROUP;
  const bool dead = *reinterpret_cast<volatile uint32_t*>(status) != 0;
  uint32_t nxt = dead ? (uint32_t)ngroups : atomicAdd(next, 1u);
  int k = dead ? nck : (int)blockIdx.x * q, kend = dead ? nck : k + q;
  int c = 0;
  for (;; ++c) {
    const int st = c % STAGES;
    const int ph = c / STAGES;
    if (ph > 0 && !mbar_wait_status(&SM.empty[st], (unsigned)((ph - 1) & 1), status)) break;
    if (k >= kend) {
      k = nxt < (uint32_t)ngroups ? pool + (int)nxt * DYN_GROUP : nck;
      kend = min(k + DYN_GROUP, nck);
      if (k < nck) nxt = atomicAdd(next, 1u);
    }
    if (k >= nck || (*reinterpret_cast<volatile uint32_t*>(status) & HULL_DEVICE_TIMEOUT)) {
      SM.id[st] = -1;
      mbar_arrive(&SM.full[st]);
      ++c;
      break;
    }
    const int id = reverse ? nck - 1 - k : k;
    ++k;
    const unsigned bytes = (unsigned)min((int64_t)CHUNK, npairs - (int64_t)id * CHUNK) * 16u;
    SM.id[st] = id;
    mbar_arrive_tx(&SM.full[st], bytes);
    bulk_g2s(&SM.stage[st][0], P + (int64_t)id * CHUNK, bytes, &SM.full[st]);
  }
  // c stages were armed (the end marker included): the last ones must land
  for (int d = c > STAGES ? c - STAGES : 0; d < c; ++d)
    mbar_wait_status(&SM.full[d % STAGES], (unsigned)((d / STAGES) & 1), status);
}

// Producer (lane 0 of the producer warp) of a batch streaming by units:
// this block's static share of [0, sp.A) first (unit number blockIdx.x),
// then units of [sp.A, P) claimed from *next (unit number G + u; last unit
// first when `reverse`) until none is left.  Each chunk of each segment (the
// part of one set inside a share or unit) is described in its stage's meta;
// a stage flagged META_END (a plain arrival) ends the stream.
template <class SS>
__device__ __forceinline__ void stream_produce_units(SS& SM, const Sets& S, const Split& sp, uint32_t* next,
                                                     bool reverse, uint32_t* status) {
  constexpr int STAGES = SS::STAGES;
  if ((threadIdx.x & 31) != 0) return;
  const int64_t P = S.pp_at(S.S);
  const int64_t nunits = P > sp.A ? (P - sp.A + sp.U - 1) / sp.U : 0;
  int c = 0;
  bool stop = *reinterpret_cast<volatile uint32_t*>(status) != 0;
  auto stream_range = [&](int64_t v0, int64_t v1, int64_t unit) {
    walk_segments(S, v0, v1, reverse, [&](int s, int64_t lo, int n) {
      const float4* Pp = reinterpret_cast<const float4*>(S.xy_of(s) + 2 * S.head_of(s)) + lo;
      const int nck = nchunks(n);
      for (int q = 0; q < nck && !stop; ++q, ++c) {
        const int st = c % STAGES;
        const int ph = c / STAGES;
        if (ph > 0 && !mbar_wait_status(&SM.empty[st], (unsigned)((ph - 1) & 1), status)) { stop = true; break; }
        if (*reinterpret_cast<volatile uint32_t*>(status) & HULL_DEVICE_TIMEOUT) { stop = true; break; }
        const int f = chunk_first(q, nck, reverse);
        const int cnt = min(CHUNK, n - f);
        ChunkMeta& M = SM.meta[st];
        M.set = s;
        M.unit = (int)unit;
        M.first = (int)(lo + f);
        M.cnt = cnt;
        M.flags = (q == 0 ? META_FIRST : 0) | (q == nck - 1 ? META_LAST : 0);
        mbar_arrive_tx(&SM.full[st], (unsigned)cnt * 16u);
        bulk_g2s(&SM.stage[st][0], Pp + f, (unsigned)cnt * 16u, &SM.full[st]);
      }
    });
  };
  if (!stop && sp.A > 0) {
    const int64_t v0 = (int64_t)blockIdx.x * sp.ppb;
    stream_range(v0, min(v0 + sp.ppb, sp.A), blockIdx.x);
  }
  while (!stop) {
    const int64_t k = (int64_t)atomicAdd(next, 1u);
    if (k >= nunits) break;
    const int64_t u = reverse ? nunits - 1 - k : k;
    const int64_t v0 = sp.A + u * sp.U;
    stream_range(v0, min(v0 + sp.U, P), sp.G + u);
  }
  // the end marker (after a timeout the consumers stop by themselves)
  {
    const int st = c % STAGES;
    const int ph = c / STAGES;
    if (ph == 0 || mbar_wait_status(&SM.empty[st], (unsigned)((ph - 1) & 1), status)) {
      SM.meta[st].flags = META_END;
      mbar_arrive(&SM.full[st]);
      ++c;
    }
  }
  for (int d = c > STAGES ? c - STAGES : 0; d < c; ++d)
    mbar_wait_status(&SM.full[d % STAGES], (unsigned)((d / STAGES) & 1), status);
}

// Consumers' side of streaming by units: wait for stage c and read its
// meta; a copy with META_END when the stream ends or the wait gave up.
template <class SS>
__device__ __forceinline__ ChunkMeta stream_next_meta(SS& SM, int c, uint32_t* status) {
  const int st = c % SS::STAGES;
  ChunkMeta M;
  if (!mbar_wait_status(&SM.full[st], (unsigned)((c / SS::STAGES) & 1), status)) {
    M.set = 0; M.unit = 0; M.first = 0; M.cnt = 0; M.flags = META_END;
    return M;
  }
  const volatile ChunkMeta& V = SM.meta[st];
  M.set = V.set; M.unit = V.unit; M.first = V.first; M.cnt = V.cnt; M.flags = V.flags;
  return M;
}

// Consumers' side of dynamic shares: wait for stage c and read its chunk
// number; -1 at the end of the stream or when the wait gave up.
template <class SS>
__device__ __forceinline__ int stream_next_chunk(SS& SM, int c, uint32_t* status) {
  const int st = c % SS::STAGES;
  if (!mbar_wait_status(&SM.full[st], (unsigned)((c / SS::STAGES) & 1), status)) return -1;
  return *reinterpret_cast<volatile int*>(&SM.id[st]);
}

template <class SS>
__device__ __forceinline__ void stream_init(SS& S) {
  if (threadIdx.x == 0) {
    for (int s = 0; s < SS::STAGES; ++s) {
      mbar_init(&S.full[s], 1);
      mbar_init(&S.empty[s], CONSUMERS / 32);
    }
    mbar_init_fence();
  }
  __syncthreads();
}

}  // namespace cudapre
