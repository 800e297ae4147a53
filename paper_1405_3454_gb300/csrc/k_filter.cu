// k_filter.cu -- Step 3 of the CudaPre method (arXiv 1405.3454, section 2):
// discard every point strictly inside the polygon of the extremes, and compact
// the survivors (their indices, plus their sort keys for the final hull).
//
// As in the paper each block first copies the polygon into shared memory and
// one thread tests several points.  The survivors are compacted in the same
// pass through per-warp staging buffers in shared memory (one global atomic
// per buffer flush, no block-wide barrier in the streaming loop; see WarpOut
// for the reserving variant of hull_compute on large sets).
//
// FP32 mode.  A point inside the polygon's inscribed circle (float32 test with
// a proven margin) or inside the inner box around the circle's centre (a
// box verified in int64; the float32 compares below are exact) is discarded
// at once.  One set takes whichever of the two holds more lattice points
// (the streaming loop is compiled for each, and a launch runs one); a batch
// takes their union in one loop for all of its sets.  Every other point goes, with its
// coordinates, to a per-warp queue; 32 queued points at a time take the full
// test.  Its cell of a GRID x GRID grid over the polygon's bounding box is
// found with two directed-rounding operations per coordinate; the cell's code
// lists the edges some point of the cell may fail (0: every point of the cell
// is strictly inside).  Only those edges are tested: s = fma(A, px, fma(B, py,
// C)) with static bound E -- s > E certainly left, s < -E certainly not (the
// point survives), otherwise the exact int64 orientation decides (an
// escalation).  Points beyond the grid are outside the bounding box and
// survive.
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

// ----------------------------------------------------------------------------
// Survivor output: a per-warp staging buffer of (index, sort key) in shared
// memory, filled while the point's coordinates are still in registers.  No
// block-wide barrier in the streaming loop.
//
// Exact mode (the survivor set of hull_prefilter, and batches): a full
// buffer is flushed with one global atomic (its base in the compacted
// output) and coalesced stores.
//
// Reserving mode (hull_compute on one set, where the survivors only feed
// the hull): flushes are exactly WFLUSH entries, so each warp reserves the
// slots of its next flush right after the current one and the atomic's
// latency is hidden behind a buffer's worth of points; the body is written
// by a bulk copy from shared memory.  The warp's last reserved block is
// filled after its final entries with copies of one of its survivors (same
// index and key): the hull kernels keep one of equal points, so copies of a
// point change no hull, and h->n_fill counts them.  On the 2^28-point disk
// this took the pass from 0.411 to 0.387 ms and added 2.6% copies.
constexpr int WBUF = 320;
constexpr int WFLUSH = RESERVE_FLUSH;        // entries per reserving-mode flush
static_assert(WFLUSH + 32 <= WBUF, "a push adds at most 32");
constexpr int WROW_IDX = WBUF + 4;  // a row's slots: room to shift by up to 3 entries
constexpr int WROW_KEY = WBUF + 2;
static_assert(WROW_IDX * 4 % 16 == 0 && WROW_KEY * 8 % 16 == 0, "rows start on 16-byte boundaries");

// Entries [0, count) of a warp's row move to [s, s + count) (s < 4), last
// chunk of 32 first, so nothing is overwritten before it is read.
template <class T>
__device__ __forceinline__ void warp_shift_right(T* buf, int count, int s) {
  if (s == 0) return;
  const int lane = threadIdx.x & 31;
  for (int c0 = ((count - 1) >> 5) << 5; c0 >= 0; c0 -= 32) {
    const int k = c0 + lane;
    T v{};
    if (k < count) v = buf[k];
    __syncwarp();
    if (k < count) buf[k + s] = v;
    __syncwarp();
  }
}

// Warp-wide: entries [0, count) of buf go to dst[0, count) of global
// memory.  buf is shifted so that buf and dst agree modulo 16 bytes; lanes
// store the entries before the first and after the last 16-byte boundary of
// dst, lane 0 the body in one bulk copy.  Returns whether it issued one.
template <class T>
__device__ __forceinline__ bool warp_store_bulk(T* buf, int count, T* dst) {
  constexpr int PER = 16 / (int)sizeof(T);
  const int lane = threadIdx.x & 31;
  const int s = (int)(((uintptr_t)dst / sizeof(T)) & (PER - 1));  // dst's entries past a 16-byte boundary
  warp_shift_right(buf, count, s);
  const int head = min((PER - s) & (PER - 1), count);
  const int body = (count - head) & ~(PER - 1);
  const int t0 = head + body;
  if (lane < head) dst[lane] = buf[s + lane];
  if (lane < count - t0) dst[t0 + lane] = buf[s + t0 + lane];
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (body > 0 && lane == 0)
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst + head),
                 "r"((unsigned)__cvta_generic_to_shared(buf + s + head)), "r"((unsigned)(body * sizeof(T)))
                 : "memory");
  return body > 0;
}

template <bool KEYS, bool RES = false>
struct WarpOut {
  uint32_t* s_idx;            // [WROW_IDX] of this warp
  unsigned long long* s_key;  // [WROW_KEY] of this warp (KEYS only)
  int count;                  // warp-uniform fill level
  WsHeader* h;
  uint32_t* g_idx;
  unsigned long long* g_key;
  bool has_res;               // warp-uniform: lane 0 holds a reserved block
  unsigned long long nres;    // lane 0: base of the reserved block
  uint32_t fill_i;            // lane 0: a survivor of this warp (reserving mode)
  unsigned long long fill_k;

  __device__ __forceinline__ void init() {
    count = 0;
    has_res = false;
    nres = 0;
    fill_i = 0;
    fill_k = 0;
  }

  // entries [0, n) to base by bulk copy; the row is free again on return
  __device__ __forceinline__ void store_bulk(int n, unsigned long long base) {
    bool issued = warp_store_bulk(s_idx, n, g_idx + base);
    if (KEYS) issued |= warp_store_bulk(s_key, n, g_key + base);
    if ((threadIdx.x & 31) == 0 && issued) {
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __syncwarp();
  }

  // reserving mode: the first WFLUSH entries to the reserved block
  __device__ __forceinline__ void flush_full() {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    unsigned long long base = 0;
    if (has_res) {
      base = __shfl_sync(FULL, nres, 0);
      if (lane == 0) nres = atomicAdd(&h->n_surv, (unsigned long long)WFLUSH);  // the next block, used later
    } else {
      if (lane == 0) {
        base = atomicAdd(&h->n_surv, 2ull * WFLUSH);
        nres = base + WFLUSH;
      }
      base = __shfl_sync(FULL, base, 0);
      has_res = true;
    }
    if (lane == 0) {
      fill_i = s_idx[0];
      if (KEYS) fill_k = s_key[0];
    }
    // the (at most 31) entries past WFLUSH wait in registers: the shift
    // before the bulk copy overwrites their first slots
    const int left = count - WFLUSH;
    uint32_t li = 0;
    unsigned long long lk = 0;
    if (lane < left) {
      li = s_idx[WFLUSH + lane];
      if (KEYS) lk = s_key[WFLUSH + lane];
    }
    __syncwarp();
    store_bulk(WFLUSH, base);
    if (lane < left) {
      s_idx[lane] = li;
      if (KEYS) s_key[lane] = lk;
    }
    __syncwarp();
    count = left;
  }

  // everything out (the end of a set)
  __device__ __forceinline__ void flush() {
    const int lane = threadIdx.x & 31;
    __syncwarp();
    if (RES && has_res) {
      const unsigned long long base = __shfl_sync(FULL, nres, 0);
      const uint32_t fi = __shfl_sync(FULL, fill_i, 0);
      const unsigned long long fk = __shfl_sync(FULL, fill_k, 0);
      if (count) store_bulk(count, base);
      for (int k = count + lane; k < WFLUSH; k += 32) {
        g_idx[base + k] = fi;
        if (KEYS) g_key[base + k] = fk;
      }
      if (lane == 0 && count < WFLUSH) atomicAdd(&h->n_fill, (unsigned long long)(WFLUSH - count));
      has_res = false;
    } else {
      unsigned long long base = 0;
      if (lane == 0 && count) base = atomicAdd(&h->n_surv, (unsigned long long)count);
      base = __shfl_sync(FULL, base, 0);
      for (int k = lane; k < count; k += 32) {
        g_idx[base + k] = s_idx[k];
        if (KEYS) g_key[base + k] = s_key[k];
      }
    }
    __syncwarp();
    count = 0;
  }

  // the end of the kernel: bulk copies must have been written, not only read
  __device__ __forceinline__ void drain_copies() {
    if (RES && (threadIdx.x & 31) == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
  }

  // At most one survivor per lane (ballot placement).
  __device__ __forceinline__ void push(bool keep, uint32_t idx, float x, float y) {
    const unsigned bal = __ballot_sync(FULL, keep);
    if (!bal) return;
    if (!RES && count + 32 > WBUF) flush();
    if (keep) {
      const int pos = count + __popc(bal & ((1u << (threadIdx.x & 31)) - 1u));
      s_idx[pos] = idx;
      if (KEYS) s_key[pos] = point_key(__float2int_rn(x), __float2int_rn(y));
    }
    count += __popc(bal);
    if (RES && count >= WFLUSH) flush_full();
  }
};

// ----------------------------------------------------------------------------
// The FP32-filtered inside test.
//
// Streaming pass: a point inside the polygon's inscribed circle (float32
// test with a proven margin) is discarded at once; every other point is
// queued, with its coordinates and index, in a per-warp ring in shared
// memory.  Whenever 32 are queued, each lane takes one and runs the full
// test: cell lookup, then the float32 edge test(s) with exact escalation.
// No point is read from memory twice.

// The quick discard of the streaming loop.
constexpr int QUICK_CIRCLE = 0, QUICK_BOX = 1, QUICK_UNION = 2;

// Blocks per SM the inside test is compiled for, and its ring's stages.
constexpr int FLT_MIN_BLOCKS = 3;
constexpr int64_t FLT_MIN_CHUNKS = 4;  // least chunks per block of an inside test
constexpr int FLT_STAGES = 2;
using FilterStream = StreamSmemT<FLT_STAGES>;
// Points per thread between two drains of the queue (8 = once per chunk).
constexpr int FLT_DRAIN_POINTS = 2;
constexpr int QCAP = 31 + 32 * FLT_DRAIN_POINTS;  // left over + pushed between drains (a per-warp stack)

struct Cells {
  const uint8_t* code8;    // GRID*GRID byte codes (global memory, L1-cached)
  const uint16_t* mask16;  // GRID*GRID edge masks (several-edge cells)
  float gx, gy, sx, sy;

  // Byte code of the point's cell; 256 when outside the grid.
  __device__ __forceinline__ uint32_t code(float x, float y, int& cell) const {
    // exact cell coordinates: floor((x - gx) / 2^kx) from round-down
    // arithmetic (both steps are exact or round toward the floor)
    const float u = __fsub_rd(x, gx), v = __fsub_rd(y, gy);
    const int cx = __float_as_int(__fmaf_rd(u, sx, 8388608.0f)) - MAGIC;
    const int cy = __float_as_int(__fmaf_rd(v, sy, 8388608.0f)) - MAGIC;
    const bool in_grid = (unsigned)(cx | cy) < (unsigned)GRID;
    cell = in_grid ? ((cy << GRID_LOG) | cx) : 0;
    return in_grid ? (uint32_t)__ldg(code8 + cell) : 256u;
  }
};

// Rare outcomes of the full test, out of line: a cell listing several edges,
// or a float32 single-edge test inside its error bound (exact int64).
__device__ __noinline__ unsigned full_test_rare(const Edge* E, const uint16_t* mask16, uint32_t code, int cell,
                                                float x, float y) {
  if (code == CELL_MULTI) return fails_any(E, __ldg(mask16 + cell), x, y);
  const Edge& e = E[code - 1];
  return 2 + (exact_left(e, __float2int_rn(x), __float2int_rn(y)) ? 0u : 1u);
}

// Full inside test of one point: cell lookup, float32 edge test(s), exact
// escalation.  Returns 2 * escalations + (survives ? 1 : 0).  The common
// outcomes (inside cell, outside the grid, one edge decided in float32) take
// no branch.
__device__ __forceinline__ unsigned full_test(const Edge* E, const Cells& C, float x, float y) {
  int cell;
  const uint32_t code = C.code(x, y, cell);
  const float4 c = *reinterpret_cast<const float4*>(&E[(code - 1) & (MAXV - 1)].A);
  const float sv = fmaf(c.x, x, fmaf(c.y, y, c.z));
  const bool single = code - 1u < (uint32_t)(CELL_MULTI - 1);  // 1 .. 254
  const bool undecided = single && !(sv > c.w) && !(sv < -c.w);
  if (code == CELL_MULTI || undecided) return full_test_rare(E, C.mask16, code, cell, x, y);
  return (code == 256u || (single && sv < -c.w)) ? 1u : 0u;
}

// RES: reserving mode (one set with keys, see WarpOut).
// units != null: a batch streaming by units of ppb pairs (stream.cuh).
template <bool KEYS, bool RES>
__global__ void __launch_bounds__(STREAM_THREADS, FLT_MIN_BLOCKS) k_filter32(Sets S, int64_t ppb, uint32_t* gstatus,
                                                                 const uint16_t* __restrict__ cells_base,
                                                                 uint32_t* __restrict__ surv_idx,
                                                                 unsigned long long* __restrict__ surv_key,
                                                                 uint32_t* units) {
  extern __shared__ __align__(128) unsigned char dsm[];
  FilterStream& SM = *reinterpret_cast<FilterStream*>(dsm);
  __shared__ __align__(16) Edge s_e[MAXV];
  __shared__ __align__(8) float2 s_qxy[CONSUMERS / 32][QCAP];
  __shared__ uint32_t s_qi[CONSUMERS / 32][QCAP];
  __shared__ __align__(16) unsigned long long s_okey[CONSUMERS / 32][KEYS ? WROW_KEY : 2];
  __shared__ __align__(16) uint32_t s_oidx[CONSUMERS / 32][WROW_IDX];
  __shared__ float s_box[4];
  __shared__ int s_pm[5];
  __shared__ float s_circ[3];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const bool dead = *reinterpret_cast<volatile uint32_t*>(gstatus) != 0;
  stream_init(SM);
  // One set: dynamic shares, claimed last chunk first (the extreme search
  // claimed them first to last, so the chunks it streamed last are still in
  // L2).  A batch: static shares of the virtual pair axis, blocks and chunks
  // last-to-first for the same reason.
  const bool dyn = RES || S.S == 1;  // the reserving mode serves one set only
  const int64_t P = S.pp_at(S.S);
  const int64_t v0 = (int64_t)(gridDim.x - 1 - blockIdx.x) * ppb;
  const int64_t v1 = dead ? v0 : min(v0 + ppb, P);
  if (warp == PRODUCER_WARP) {
    if (dyn) {
      stream_produce_dynamic(SM, reinterpret_cast<const float4*>(S.xy_of(0) + 2 * S.head_of(0)), S.npairs_of(0),
                             &S.h(0)->next_group[1], true, gstatus);
    } else if constexpr (!RES) {
      if (units)
        stream_produce_units(SM, S, Split{CHUNK, 0, ppb, (int64_t)gridDim.x}, units, true, gstatus);
      else
        stream_produce_sets(SM, S, v0, v1, true, gstatus);
    }
    return;
  }
  WarpOut<KEYS, RES> O;
  O.s_idx = s_oidx[warp];
  O.s_key = s_okey[warp];
  O.init();
  float2* qxy = s_qxy[warp];
  uint32_t* qi = s_qi[warp];
  int qn = 0;  // warp-uniform fill of the queue (used as a stack)
  unsigned esc = 0;
  bool all_survive = true;
  Cells C;
  // the quick discard of the set: the circle of centre (ccx, ccy) and
  // squared radius cr2, and the box |x - ccx| <= hx, |y - ccy| <= hy
  float ccx = 0.0f, ccy = 0.0f, cr2 = -1.0f, hx = -1.0f, hy = -1.0f;
  uint32_t ibase = 0;
  WsHeader* h = nullptr;
  // Full test of the `count` (<= 32) most recently queued points, one per lane.
  auto drain = [&](int count) {
    const bool mine = lane < count;
    const int slot = qn - count + lane;
    float2 p = make_float2(0.0f, 0.0f);
    uint32_t i = 0;
    bool keep = false;
    if (mine) {
      p = qxy[slot];
      i = qi[slot];
      if (all_survive) {
        keep = true;
      } else {
        const unsigned r = full_test(s_e, C, p.x, p.y);
        esc += r >> 1;
        keep = r & 1;
      }
    }
    qn -= count;
    O.push(keep, i, p.x, p.y);
  };
  // a new set (first pair lo of its segment): its polygon, inscribed circle
  // and cell grid (section 2, Step 3: the polygon goes to shared memory),
  // its output
  auto begin_set = [&](int set, int64_t lo) {
    consumers_sync();
    h = S.h(set);
    if (tid < MAXV * (int)(sizeof(Edge) / 4))
      reinterpret_cast<uint32_t*>(s_e)[tid] = reinterpret_cast<const uint32_t*>(h->poly.e)[tid];
    if (tid == 0) {
      s_pm[0] = h->poly.m; s_pm[1] = h->poly.gx0; s_pm[2] = h->poly.gy0; s_pm[3] = h->poly.kx; s_pm[4] = h->poly.ky;
      s_circ[0] = h->poly.ccx; s_circ[1] = h->poly.ccy; s_circ[2] = h->poly.cr2;
      for (int k = 0; k < 4; ++k) s_box[k] = h->poly.box[k];
    }
    consumers_sync();
    all_survive = s_pm[0] < 3;
    const uint16_t* cells = cells_base + (size_t)set * (CELL_BYTES / 2);
    C.code8 = reinterpret_cast<const uint8_t*>(cells + GRID * GRID);
    C.mask16 = cells;
    C.gx = (float)s_pm[1];
    C.gy = (float)s_pm[2];
    C.sx = __int_as_float((127 - s_pm[3]) << 23);  // 2^-kx
    C.sy = __int_as_float((127 - s_pm[4]) << 23);
    ccx = s_circ[0];
    ccy = s_circ[1];
    cr2 = all_survive ? -1.0f : s_circ[2];
    // Half-widths of the part of the inner box [x0, x1] x [y0, y1] centred on
    // (ccx, ccy), in integers, at most 2^24 - 1: then for lattice points
    // fl(|x - ccx|) <= hx implies the exact |x - ccx| <= hx (a difference
    // that rounds is above 2^24), so x0 <= x <= x1.  Negative when there is
    // no box or the centre lies outside it.
    auto half = [](float c, float lo, float hi) {
      const long long w = min((long long)c - (long long)lo, (long long)hi - (long long)c);
      return (float)min(w, (long long)COORD_MAX - 1);
    };
    const bool box_ok = !all_survive && s_box[0] <= s_box[1] && s_box[2] <= s_box[3];
    hx = box_ok ? half(ccx, s_box[0], s_box[1]) : -1.0f;
    hy = box_ok ? half(ccy, s_box[2], s_box[3]) : -1.0f;
    O.h = h;
    O.g_idx = surv_idx + S.off_at(set);
    O.g_key = KEYS ? surv_key + S.off_at(set) : nullptr;
    esc = 0;
    ibase = (uint32_t)(S.head_of(set) + 2 * lo) + 2u * (uint32_t)tid;
  };
  // one chunk in stage st: cnt pairs from pair f of the segment, with the
  // quick discard QUICK (QUICK_CIRCLE, QUICK_BOX or QUICK_UNION)
  auto chunk_q = [&](auto QUICK, int st, int f, int cnt) {
    constexpr int Q = decltype(QUICK)::value;
    const float4* sp = SM.stage[st];
    float4 v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = sp[tid + j * CONSUMERS];  // beyond cnt: ignored below
    __syncwarp();
    if (lane == 0) mbar_arrive(&SM.empty[st]);
    const uint32_t i0 = ibase + 2u * (uint32_t)f;
    const int lim = cnt - tid;
#pragma unroll
    for (int j0 = 0; j0 < 8; j0 += FLT_DRAIN_POINTS) {
#pragma unroll
      for (int j = j0; j < j0 + FLT_DRAIN_POINTS; ++j) {
        const float x = (j & 1) ? v[j >> 1].z : v[j >> 1].x, y = (j & 1) ? v[j >> 1].w : v[j >> 1].y;
        const float dx = x - ccx, dy = y - ccy;
        bool in;
        if constexpr (Q == QUICK_CIRCLE) in = fmaf(dx, dx, dy * dy) < cr2;
        else if constexpr (Q == QUICK_BOX) in = (fabsf(dx) <= hx) & (fabsf(dy) <= hy);
        else in = (fmaf(dx, dx, dy * dy) < cr2) | ((fabsf(dx) <= hx) & (fabsf(dy) <= hy));
        const bool need = (j >> 1) * CONSUMERS < lim && !in;
        const unsigned bal = __ballot_sync(FULL, need);
        const int slot = qn + __popc(bal & lt);
        if (need) {
          qxy[slot] = make_float2(x, y);
          qi[slot] = i0 + 2u * (uint32_t)((j >> 1) * CONSUMERS) + (uint32_t)(j & 1);
        }
        qn += __popc(bal);
      }
      __syncwarp();
      while (qn >= 32) drain(32);
    }
  };
  // the end of a set: queued points, buffered survivors, counters
  auto end_set = [&]() {
    __syncwarp();
    if (qn > 0) drain(qn);
    O.flush();
    for (int off = 16; off; off >>= 1) esc += __shfl_xor_sync(FULL, esc, off);
    if (lane == 0 && esc) atomicAdd(&h->n_escalated, (unsigned long long)esc);
  };
  using Union = std::integral_constant<int, QUICK_UNION>;
  auto chunk = [&](int st, int f, int cnt) { chunk_q(Union{}, st, f, cnt); };
  if (dyn) {
    const int64_t np = S.npairs_of(0);
    begin_set(0, 0);
    auto run = [&](auto QUICK) {
      for (int c = 0;; ++c) {
        const int id = stream_next_chunk(SM, c, gstatus);
        if (id < 0) break;
        const int f = id * CHUNK;
        chunk_q(QUICK, c % FilterStream::STAGES, f, (int)min((int64_t)CHUNK, np - f));
      }
    };
    // the box's lattice points against the circle's (about pi r^2)
    if (hx >= 0.0f && hy >= 0.0f && (2.0f * hx + 1.0f) * (2.0f * hy + 1.0f) > 3.14159f * cr2)
      run(std::integral_constant<int, QUICK_BOX>{});
    else
      run(std::integral_constant<int, QUICK_CIRCLE>{});
    end_set();
    O.drain_copies();
    return;
  }
  if constexpr (!RES) {
    if (units) {
      for (int c = 0;; ++c) {
        const ChunkMeta M = stream_next_meta(SM, c, gstatus);
        if (M.flags & META_END) break;
        if (M.flags & META_FIRST) begin_set(M.set, 0);
        chunk(c % FilterStream::STAGES, M.first, M.cnt);
        if (M.flags & META_LAST) end_set();
      }
      return;
    }
    int c = 0;
    bool stop = false;
    walk_segments(S, v0, v1, true, [&](int set, int64_t lo, int n) {
      begin_set(set, lo);
      const int nck = nchunks(n);
      for (int k = 0; k < nck; ++k, ++c) {
        const int st = c % FilterStream::STAGES;
        if (!stop && !mbar_wait_status(&SM.full[st], (unsigned)((c / FilterStream::STAGES) & 1), gstatus)) stop = true;
        if (stop) continue;
        const int f = chunk_first(k, nck, true);
        chunk(st, f, min(CHUNK, n - f));
      }
      end_set();
    });
  }
}

// ----------------------------------------------------------------------------
// The plain inside test (int64 orientation against every edge), same stream.

template <bool KEYS>
__global__ void __launch_bounds__(STREAM_THREADS, 3) k_filter_exact(Sets S, int64_t ppb, uint32_t* gstatus,
                                                                     uint32_t* __restrict__ surv_idx,
                                                                     unsigned long long* __restrict__ surv_key) {
  extern __shared__ __align__(128) unsigned char dsm[];
  FilterStream& SM = *reinterpret_cast<FilterStream*>(dsm);
  __shared__ __align__(16) Edge s_e[MAXV];
  __shared__ __align__(16) unsigned long long s_okey[CONSUMERS / 32][KEYS ? WROW_KEY : 2];
  __shared__ __align__(16) uint32_t s_oidx[CONSUMERS / 32][WROW_IDX];
  __shared__ int s_m;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool dead = *reinterpret_cast<volatile uint32_t*>(gstatus) != 0;
  stream_init(SM);
  const int64_t P = S.pp_at(S.S);
  // blocks take their shares last-to-first: the first ones to run read what
  // the extreme search read last (still in L2)
  const int64_t v0 = (int64_t)(gridDim.x - 1 - blockIdx.x) * ppb;
  const int64_t v1 = dead ? v0 : min(v0 + ppb, P);
  if (warp == PRODUCER_WARP) {
    stream_produce_sets(SM, S, v0, v1, true, gstatus);
    return;
  }
  Tester<HULL_FILTER_EXACT> T;
  T.E = s_e;
  T.m = 0;
  T.esc = 0;
  bool all_survive = true;
  WarpOut<KEYS> O;
  O.s_idx = s_oidx[warp];
  O.s_key = s_okey[warp];
  O.init();
  int c = 0;
  bool stop = false;
  walk_segments(S, v0, v1, true, [&](int set, int64_t lo, int n) {
    consumers_sync();
    WsHeader* h = S.h(set);
    if (tid < MAXV * (int)(sizeof(Edge) / 4))
      reinterpret_cast<uint32_t*>(s_e)[tid] = reinterpret_cast<const uint32_t*>(h->poly.e)[tid];
    if (tid == 0) s_m = h->poly.m;
    consumers_sync();
    T.m = s_m;
    all_survive = s_m < 3;
    O.h = h;
    O.g_idx = surv_idx + S.off_at(set);
    O.g_key = KEYS ? surv_key + S.off_at(set) : nullptr;
    const uint32_t ibase = (uint32_t)(S.head_of(set) + 2 * lo) + 2u * (uint32_t)tid;
    const int nck = nchunks(n);
    for (int k = 0; k < nck; ++k, ++c) {
      const int st = c % FilterStream::STAGES;
      if (!stop && !mbar_wait_status(&SM.full[st], (unsigned)((c / FilterStream::STAGES) & 1), gstatus)) stop = true;
      if (stop) continue;
      const int f = chunk_first(k, nck, true);
      const int cnt = min(CHUNK, n - f);
      const float4* sp = SM.stage[st];
      float4 v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = sp[tid + j * CONSUMERS];
      __syncwarp();
      if (lane == 0) mbar_arrive(&SM.empty[st]);
      const uint32_t i0 = ibase + 2u * (uint32_t)f;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const float x = (j & 1) ? v[j >> 1].z : v[j >> 1].x, y = (j & 1) ? v[j >> 1].w : v[j >> 1].y;
        const bool keep = tid + (j >> 1) * CONSUMERS < cnt && (all_survive || T.survives(x, y));
        O.push(keep, i0 + 2u * (uint32_t)((j >> 1) * CONSUMERS) + (uint32_t)(j & 1), x, y);
      }
    }
    O.flush();
  });
}

__global__ void k_all_keys(const float* __restrict__ xy, int64_t n, WsHeader* h, unsigned long long* __restrict__ keys,
                           uint32_t* __restrict__ vals) {
  if (*reinterpret_cast<volatile uint32_t*>(&h->status) != 0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float2 p = __ldcs(reinterpret_cast<const float2*>(xy) + i);
    keys[i] = point_key(__float2int_rn(p.x), __float2int_rn(p.y));
    vals[i] = (uint32_t)i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) h->n_surv = (unsigned long long)n;
}

__global__ void k_copy_count(const WsHeader* h, int64_t* out) {
  *out = h->status ? 0 : (int64_t)h->n_surv;
}

template <class K>
cudaError_t stream_launch(K kernel, bool& attr_done, size_t dsmem, int64_t npairs, const LaunchShape& ls, int sets,
                          int64_t& G, int64_t& ppb, bool by_units = false) {
  const int grid = ls.grid;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsmem);
    if (e != cudaSuccess) return e;
    attr_done = true;
  }
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, STREAM_THREADS, dsmem);
  occ = std::max(occ, 1);
  const int64_t resident = (int64_t)device_sm_count() * occ;
  if (by_units) {
    // one wave of resident blocks claiming units of ppb pairs
    const int64_t G0 = grid > 0 ? std::min<int64_t>(grid, MAX_STREAM_BLOCKS) : resident;
    ppb = unit_pairs(npairs, G0, ls.unit_chunks > 0 ? ls.unit_chunks : FILTER_UNIT_CHUNKS);
    G = std::max<int64_t>(1, std::min<int64_t>(G0, (npairs + ppb - 1) / ppb));
    return cudaSuccess;
  }
  G = grid > 0 ? grid : resident * stream_waves(sets, npairs, resident, ls.waves);
  G = std::min<int64_t>(G, MAX_STREAM_BLOCKS);
  // small inputs: at least FLT_MIN_CHUNKS chunks per block
  if (grid <= 0) G = std::min<int64_t>(G, ((npairs + CHUNK - 1) / CHUNK + FLT_MIN_CHUNKS - 1) / FLT_MIN_CHUNKS);
  G = std::max<int64_t>(1, std::min<int64_t>(G, (npairs + CHUNK - 1) / CHUNK));
  ppb = (npairs + G - 1) / G;
  ppb = (ppb + CHUNK - 1) / CHUNK * CHUNK;
  if (ppb == 0) ppb = CHUNK;
  G = std::max<int64_t>(1, (npairs + ppb - 1) / ppb);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_filter(const Sets& S, int64_t pairs_bound, int filter, uint32_t* gstatus, uint16_t* cells,
                          uint32_t* surv_idx, unsigned long long* surv_key, LaunchShape ls, cudaStream_t st,
                          bool reserve, uint32_t* units) {
  const int64_t npairs = std::max<int64_t>(pairs_bound, 0);
  if (npairs == 0) return cudaSuccess;  // every point is a loose point (finishing kernel)
  const bool keys = surv_key != nullptr;
  static bool attr[64][5] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  int64_t G = 1, ppb = CHUNK;
  cudaError_t e;
  const size_t ds = sizeof(FilterStream);
  const bool by_units = S.S > 1 && units != nullptr;
  uint32_t* un = by_units ? units : nullptr;
  if (filter == HULL_FILTER_FP32) {
    if (keys) {
      if ((e = stream_launch(k_filter32<true, false>, attr[dev][0], ds, npairs, ls, S.S, G, ppb, by_units)) !=
          cudaSuccess)
        return e;
      // reserving mode only within the capacity the caller's layout added
      if (reserve && S.S == 1 && G * (CONSUMERS / 32) <= RESERVE_WARPS) {
        if ((e = stream_launch(k_filter32<true, true>, attr[dev][4], ds, npairs, ls, S.S, G, ppb)) != cudaSuccess)
          return e;
        k_filter32<true, true><<<(unsigned)G, STREAM_THREADS, ds, st>>>(S, ppb, gstatus, cells, surv_idx, surv_key,
                                                                         nullptr);
      } else {
        k_filter32<true, false><<<(unsigned)G, STREAM_THREADS, ds, st>>>(S, ppb, gstatus, cells, surv_idx, surv_key,
                                                                          un);
      }
    } else {
      if ((e = stream_launch(k_filter32<false, false>, attr[dev][1], ds, npairs, ls, S.S, G, ppb, by_units)) !=
          cudaSuccess)
        return e;
      k_filter32<false, false><<<(unsigned)G, STREAM_THREADS, ds, st>>>(S, ppb, gstatus, cells, surv_idx, surv_key,
                                                                         un);
    }
  } else {
    if (keys) {
      if ((e = stream_launch(k_filter_exact<true>, attr[dev][2], ds, npairs, ls, S.S, G, ppb)) != cudaSuccess) return e;
      k_filter_exact<true><<<(unsigned)G, STREAM_THREADS, ds, st>>>(S, ppb, gstatus, surv_idx, surv_key);
    } else {
      if ((e = stream_launch(k_filter_exact<false>, attr[dev][3], ds, npairs, ls, S.S, G, ppb)) != cudaSuccess) return e;
      k_filter_exact<false><<<(unsigned)G, STREAM_THREADS, ds, st>>>(S, ppb, gstatus, surv_idx, surv_key);
    }
  }
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_all_keys(const float* xy, int64_t n, WsHeader* h, unsigned long long* keys, uint32_t* vals,
                            cudaStream_t st) {
  const int64_t g = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)device_sm_count() * 8));
  k_all_keys<<<(unsigned)g, 256, 0, st>>>(xy, n, h, keys, vals);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_copy_count(WsHeader* h, int64_t* out, cudaStream_t st) {
  k_copy_count<<<1, 1, 0, st>>>(h, out);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cudapre
