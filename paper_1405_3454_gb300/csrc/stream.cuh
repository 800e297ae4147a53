// stream.cuh -- bulk-copy (TMA engine) streaming of a block's range of 16-byte
// point pairs into a ring of shared-memory stages, for the two passes over
// the points (the extreme search and the inside test).
//
// One producer warp (its lane 0) issues cp.async.bulk copies of CHUNK pairs
// per stage; the copy engine signals the stage's "full" mbarrier with the
// transferred byte count.  Consumer warps wait on "full", copy their pairs to
// registers and arrive on the stage's "empty" mbarrier at once, so the
// producer can refill it while they compute.  Every wait is bounded: on
// timeout the kernel records HULL_DEVICE_TIMEOUT and stops streaming.
#pragma once

#include "internal.cuh"

namespace cudapre {

constexpr int CONSUMERS = 256;               // consumer threads (8 warps)
constexpr int PRODUCER_WARP = CONSUMERS / 32;
constexpr int STREAM_THREADS = CONSUMERS + 32;
constexpr int CHUNK = 4 * CONSUMERS;         // pairs per stage (4 per consumer thread)
constexpr long long WAIT_LIMIT_CYCLES = 1ll << 31;  // about one second

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
// bit set) when it does not complete within WAIT_LIMIT_CYCLES.
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, WsHeader* h) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
      atomicOr(&h->status, HULL_DEVICE_TIMEOUT);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Shared state of one block's stream with NS stages.
template <int NS>
struct StreamSmemT {
  static constexpr int STAGES = NS;
  float4 stage[NS][CHUNK];
  unsigned long long full[NS];
  unsigned long long empty[NS];
};

// Chunk c of a block's pair range [p0, p1) in processing order; `reverse`
// walks the range last chunk first.
struct StreamRange {
  int64_t p0, p1, nchunks;
  bool reverse;
  __device__ __forceinline__ int64_t first_pair(int64_t c) const {
    const int64_t k = reverse ? nchunks - 1 - c : c;
    return p0 + k * CHUNK;
  }
  __device__ __forceinline__ int count(int64_t c) const {
    const int64_t f = first_pair(c);
    return (int)min((int64_t)CHUNK, p1 - f);
  }
};

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

// Producer (lane 0 of the producer warp): issue every chunk, waiting for a
// free stage each time; then wait until the copies it issued have landed.
template <class SS>
__device__ __forceinline__ void stream_produce(SS& S, const StreamRange& R, const float4* P, WsHeader* h) {
  constexpr int STAGES = SS::STAGES;
  if ((threadIdx.x & 31) != 0) return;
  int64_t c = 0;
  for (; c < R.nchunks; ++c) {
    const int s = (int)(c % STAGES);
    const int64_t k = c / STAGES;
    if (k > 0 && !mbar_wait(&S.empty[s], (unsigned)((k - 1) & 1), h)) break;
    if (*reinterpret_cast<volatile uint32_t*>(&h->status) & HULL_DEVICE_TIMEOUT) break;
    const unsigned bytes = (unsigned)R.count(c) * 16u;
    mbar_arrive_tx(&S.full[s], bytes);
    bulk_g2s(&S.stage[s][0], P + R.first_pair(c), bytes, &S.full[s]);
  }
  // drain: the last min(c, STAGES) copies must complete before the block exits
  for (int64_t d = c > STAGES ? c - STAGES : 0; d < c; ++d)
    mbar_wait(&S.full[d % STAGES], (unsigned)((d / STAGES) & 1), h);
}

}  // namespace cudapre
