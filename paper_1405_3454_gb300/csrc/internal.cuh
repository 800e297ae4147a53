// internal.cuh -- device-side layout, constants and helpers shared by the
// kernels of the CudaPre implementation (arXiv 1405.3454).  Not part of the
// public ABI (include/cudapre.h).
#pragma once

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/cudapre.h"

namespace cudapre {

// ----------------------------------------------------------------------------
// Projection constants: correctly rounded closed forms (section 2, Step 1).
//   K_S3 = sqrt(3)/2, K_C75 = (sqrt(6)-sqrt(2))/4, K_S75 = (sqrt(6)+sqrt(2))/4,
//   K_H = sqrt(2)/2.  cos(radians(t)) would be off by one ulp for 30 degrees.
constexpr double K_S3 = 0x1.bb67ae8584caap-1;
constexpr double K_C75 = 0x1.0907dc1930690p-2;
constexpr double K_S75 = 0x1.ee8dd4748bf15p-1;
constexpr double K_H = 0x1.6a09e667f3bcdp-1;
constexpr float F_S3 = (float)K_S3;
constexpr float F_C75 = (float)K_C75;
constexpr float F_S75 = (float)K_S75;
constexpr float F_H = (float)K_H;

// Float32 values of the extreme search.  Each tracked value is a positive
// multiple k of a rotated coordinate (the order of the points is unchanged),
// chosen so that one fused multiply-add computes it:
//   30 and 60 degrees: k = 2, e.g. 2 x'(30) = fma(x, 2 s3, -y);
//   75 degrees:        k = 1/c75, x'(75)/c75 = fma(y, -tan75, x);
//   45 degrees:        k = 1/h,   x'(45)/h = x - y.
// For |x|, |y| <= 2^24 the float32 value is within 3 (30, 45 and 60 degrees)
// or 6 (75 degrees) of k times the binary64 definition: coefficient rounding
// (|y| * half an ulp of the coefficient) plus the final rounding (half an ulp
// of a result below 2^26 resp. 2^27).  Two candidates whose float32 values
// differ by more than BAND_LO = 16 resp. BAND_HI = 32 -- over twice the sum of
// their errors -- are ordered by the float32 values; otherwise the binary64
// definition decides.
constexpr float BAND_LO = 16.0f;
constexpr float BAND_HI = 32.0f;
constexpr float F_2S3 = (float)(2.0 * K_S3);
// tan(75 degrees) = 2 + sqrt(3), correctly rounded to float
constexpr float F_T75 = 0x1.ddb3d8p+1f;

constexpr int MAXV = 16;          // polygon vertices (16 extremes at most)
constexpr int NSLOT = 16;         // extreme slots
constexpr uint32_t NONE = 0xFFFFFFFFu;
constexpr int32_t COORD_MAX = 1 << 24;

// ----------------------------------------------------------------------------
// Step-2 polygon as the inside test consumes it.
struct Edge {
  float A, B, C, E;     // float32 s = fma(A, px, fma(B, py, C)), |s - orient| <= E
  int32_t ax, ay;       // exact tail vertex
  int32_t dx, dy;       // exact edge vector
};

// Cell grid over the polygon's bounding box for the inside test: GRID x GRID
// cells of 2^kx by 2^ky lattice points from (gx0, gy0).  Cell code = bit mask
// of the edges that some point of the cell may fail; 0 = every point of the
// cell is strictly inside (discard without a test).
constexpr int GRID_LOG = 7;
constexpr int64_t GRID_MIN_POINTS = 1 << 16;  // smaller sets use one cell listing every edge
constexpr int GRID = 1 << GRID_LOG;
// Cell storage in the workspace: GRID*GRID uint16 edge masks, then GRID*GRID
// byte codes (0: inside, k + 1: only edge k, CELL_MULTI: see the mask).
constexpr int CELL_MULTI = 255;
constexpr size_t CELL_BYTES = (size_t)GRID * GRID * 3;

struct Poly {
  int32_t m;            // vertex count (0..16); < 3 discards nothing
  int32_t gx0, gy0;     // cell grid origin (multiples of the cell sizes)
  int32_t kx, ky;       // log2 of the cell sizes
  int32_t rox, roy;     // integer point strictly inside (centre of the inner box)
  int32_t refine_on;    // 1 when (rox, roy) is valid
  // Inscribed circle for a quick discard: every point whose float32
  // (x - ccx)^2 + (y - ccy)^2, computed as fma(dx, dx, dy * dy), is below
  // cr2 is strictly inside the polygon; cr2 = -1 when there is none.
  float ccx, ccy, cr2;
  int32_t pad_;
  float box[4];         // closed inner box x0, x1, y0, y1 (integer-valued);
                        // every point of it is strictly inside; x0 > x1 if empty
  int32_t vx[MAXV], vy[MAXV];
  uint32_t vidx[MAXV];  // point index of each vertex
  uint32_t ext[NSLOT];  // the 16 extreme indices (slot order of the ABI)
  Edge e[MAXV];
};

// Per-block partial result of the extreme search: binary64 score (sign
// applied so that larger is better) and point index.
struct BlockBest {
  double s;
  uint32_t idx;
  uint32_t pad_;
};

// Workspace header (offset 0 of every workspace); zeroed by each call.
struct WsHeader {
  uint32_t status;        // HULL_DEVICE_* bits
  uint32_t next_group[2];  // dynamic shares of one set: chunk-group counters of Step 1 and Step 3
  unsigned long long n_surv;      // survivors written by the inside test
  unsigned long long n_escalated; // float32 decisions escalated to int64
  unsigned long long n_fill;      // copies of survivors filling reserved slots (hull_compute on one set)
  uint32_t bar_count, bar_gen;  // grid barrier of the cooperative large-set kernel
  uint32_t hist[8][256];  // radix-sort digit histograms (all passes)
  uint32_t tile_next[8];  // radix sort: next tile to claim, per pass
  unsigned long long key_or, key_nor;  // radix sort: OR of the keys and of their complements
  unsigned long long n_surv2;  // survivors left by the refinement round
  uint32_t n_lower, n_upper;   // small-set hull: vertices of the lower / upper chain
  float refine_r2;             // refinement: squared radius of a disk inside the winners' polygon (or -1)
  int32_t refine_cx, refine_cy;  // and its centre
  uint32_t refine_pad_;
  Poly poly;
  unsigned long long rbin[1024];  // refinement: per angular bin, packed farthest survivor
};

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
constexpr size_t HEADER_BYTES = align_up(sizeof(WsHeader), 256);

// ----------------------------------------------------------------------------
// Exact helpers.

__host__ __device__ inline long long orient64(long long ax, long long ay, long long bx,
                                              long long by, long long px, long long py) {
  return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

// Sort key of an integer point: x and y shifted to [0, 2^25] and packed
// (x in bits 26..51, y in bits 0..25), so key order is (x, y) order.
__host__ __device__ inline unsigned long long point_key(int32_t ix, int32_t iy) {
  return ((unsigned long long)(uint32_t)(ix + COORD_MAX) << 26) |
         (unsigned long long)(uint32_t)(iy + COORD_MAX);
}
__host__ __device__ inline int32_t key_x(unsigned long long k) {
  return (int32_t)(k >> 26) - COORD_MAX;
}
__host__ __device__ inline int32_t key_y(unsigned long long k) {
  return (int32_t)(k & ((1ull << 26) - 1)) - COORD_MAX;
}

// ----------------------------------------------------------------------------
// The point sets of one call.  A single set (hull_prefilter, hull_compute)
// travels by value with no device tables; a batch keeps its S+1 element
// offsets (the caller's) and its S+1 pair prefix in device memory.  Set s
// holds points [off(s), off(s+1)) of xy; its float4 pairs start at its
// first 16-byte aligned point (the "head" point before it, if any, and an
// odd trailing point are handled by the finishing kernel).  The pairs of all
// sets, concatenated, form the virtual pair axis that the streaming passes
// split evenly over their blocks.
struct Sets {
  const float* xy;
  const int64_t* off;    // S+1 element offsets, or null: one set of n1 points
  const int64_t* start;  // S first rows of the sets in xy, or null: off
  const int64_t* pp;     // S+1 prefix of the sets' pair counts, or null
  int64_t n1;
  int S;
  char* hdr;             // S headers, HEADER_BYTES apart

  // off(s): where set s's part of every per-point workspace array begins
  // (the prefix of the set sizes); start(s): its first point in xy.
  __host__ __device__ int64_t off_at(int s) const { return off ? off[s] : (s == 0 ? 0 : n1); }
  __host__ __device__ int64_t start_at(int s) const { return start ? start[s] : off_at(s); }
  __host__ __device__ const float* xy_of(int s) const { return xy + 2 * start_at(s); }
  __host__ __device__ int64_t n_of(int s) const { return off_at(s + 1) - off_at(s); }
  __host__ __device__ int head_of(int s) const {
    return (n_of(s) > 0 && (reinterpret_cast<uintptr_t>(xy_of(s)) & 15u)) ? 1 : 0;
  }
  __host__ __device__ int64_t npairs_of(int s) const {
    const int64_t n = n_of(s);
    const int h = head_of(s);
    return n > h ? (n - h) / 2 : 0;
  }
  __host__ __device__ int64_t pp_at(int s) const { return pp ? pp[s] : (s == 0 ? 0 : npairs_of(0)); }
  __host__ __device__ WsHeader* h(int s) const {
    return reinterpret_cast<WsHeader*>(hdr + (size_t)s * HEADER_BYTES);
  }
  // The set holding virtual pair p (0 <= p < total pairs).
  __device__ int set_of_pair(int64_t p) const {
    if (!pp) return 0;
    int lo = 0, hi = S - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pp[mid] <= p) lo = mid; else hi = mid - 1;
    }
    return lo;
  }
};

// ----------------------------------------------------------------------------
// Launch shapes and per-device facts.
int device_sm_count();

// Launch shape of the streaming passes (hull_options; 0 = built-in choice):
// blocks, waves of a batch's static shares, chunks of a batch's units.
struct LaunchShape {
  int grid;
  int waves;
  int unit_chunks;
};

// Process-wide count of kernels enqueued by this library (instrumentation).
void count_launches(int k);
// Stage boundary b of the current call for an attached stage timer
// (instrumentation; nothing when no timer is attached).
void stage_mark(int b, cudaStream_t st);

// Launchers (one per translation unit); all enqueue on `st`.  `gstatus` is
// the status word every step checks first (the header's for one set, the
// batch word for a batch); a nonzero word skips the work.
cudaError_t launch_validate(const float* xy, int64_t n, uint32_t* status, cudaStream_t st);
// Steps 1-2 for every set: the streaming search (pairs_bound >= the total
// pairs of all sets), then one finishing block per set (the 16 extremes,
// the polygon, the cell grid, and the inside test of the points outside the
// 16-byte pairs, whose survivors go to surv_idx / surv_key at the set's
// offset).  `partials` holds (blocks + S) x 16 block results.
// A batch passes `units` (a zeroed counter): its FP32 streaming search
// claims units of the pair axis dynamically, and `partials` then needs
// npairs / 1024 + 1 + S slots.
cudaError_t launch_extremes(const Sets& S, int64_t pairs_bound, int angles, int filter, uint32_t* gstatus,
                            void* partials, uint16_t* cells, LaunchShape ls, uint32_t* ext_out, uint32_t* surv_idx,
                            unsigned long long* surv_key, cudaStream_t st, uint32_t* units = nullptr);
// hull_compute on one set of at least RESERVE_MIN_POINTS points gives its
// per-point buffers RESERVE_WARPS * RESERVE_FLUSH extra entries, so the
// inside test may reserve survivor slots ahead (k_filter.cu): every warp
// then writes at most RESERVE_FLUSH copies beyond its survivors.
// Survivor positions stay below 2^32 (they are packed into 32 bits), so
// the largest sets do without.
constexpr int64_t RESERVE_MIN_POINTS = 1ll << 24;
constexpr int64_t RESERVE_WARPS = 4096;
constexpr int RESERVE_FLUSH = 256;
inline bool compute_reserves(int64_t n) {
  return n >= RESERVE_MIN_POINTS && n <= 0xFFFFFFFFll - RESERVE_WARPS * RESERVE_FLUSH;
}
inline int64_t compute_capacity(int64_t n) {
  return std::max<int64_t>(n, 1) + (compute_reserves(n) ? RESERVE_WARPS * RESERVE_FLUSH : 0);
}

// Step 3 for every set: survivors (set-local indices, keys when surv_key is
// not null) at the set's offset, counted in its header.
// (a batch passes `units`, a zeroed counter: the FP32 pass then claims
// units of the pair axis dynamically)
cudaError_t launch_filter(const Sets& S, int64_t pairs_bound, int filter, uint32_t* gstatus, uint16_t* cells,
                          uint32_t* surv_idx, unsigned long long* surv_key, LaunchShape ls, cudaStream_t st,
                          bool reserve = false, uint32_t* units = nullptr);
// The large path (sort + chunked chain) of one point set; it runs only when
// *count > SMALL_MAX and the set's status word is clear.
struct LargeJob {
  WsHeader* h;                      // status word and digit histograms of the set
  const unsigned long long* count;  // survivors to sort (device)
  unsigned long long* ka;           // survivor keys / indices (capacity cap)
  uint32_t* va;
  unsigned long long* kb;           // second buffer pair (capacity cap)
  uint32_t* vb;
  unsigned long long* tilecnt;      // 256 * sort_tiles(cap) tile status words of the sort
  uint32_t* cnt;                    // 4 * ceil(cap / CHAIN_C0)
  uint32_t* out_idx;                // hull vertex indices (local to the set)
  int64_t* out_n;
  int64_t cap;
};
// Two cooperative launches (the sort, then the chains) over
// `table[0 .. *njobs)` (njobs in device memory), or over `single` when table
// is null; bar = two zeroed words for the grid barrier, bar_status = where a
// barrier timeout is recorded.
cudaError_t launch_large(const LargeJob* table, const int* njobs, const LargeJob& single, uint32_t* bar,
                         uint32_t* bar_status, cudaStream_t st);
cudaError_t launch_copy_count(WsHeader* h, int64_t* out, cudaStream_t st);
// Every point as a survivor (the paper's case (1), no preprocessing): its
// key and index, and the count n.
cudaError_t launch_all_keys(const float* xy, int64_t n, WsHeader* h, unsigned long long* keys, uint32_t* vals,
                            cudaStream_t st);

constexpr int REFINE_BINS = 1024;         // angular bins of the refinement round
constexpr int SMALL_MAX = 8192;           // survivor sets up to this size: one-block hull
constexpr int TINY_MAX = 1024;            // ... up to this size: one short kernel

// The refinement round for every set; tp = S+1 work-tile prefix (batch).
cudaError_t launch_refine(const Sets& S, const uint32_t* gstatus, int64_t* tp, const unsigned long long* keys_in,
                          const uint32_t* vals_in, unsigned long long* keys_out, uint32_t* vals_out, int4* tri,
                          int64_t cap, cudaStream_t st);
// State of the small-set hull between its launches (in the workspace).
constexpr int SMALL_NCH = 32;
struct SmallWs {
  int active;  // 1 when prune/emit have work
  int u;       // distinct points
  int C;       // chunk capacity
  int pad_;
  int cnt[2][SMALL_NCH];
  int base[2][SMALL_NCH + 1];
  int2 pts[SMALL_MAX];
  uint32_t uid[SMALL_MAX];
  uint16_t chain[2][SMALL_MAX];
  uint8_t keep[2][SMALL_MAX];
  uint8_t flag[SMALL_MAX];  // whole-GPU path: bit 0 lower-chain vertex, bit 1 upper
};

cudaError_t launch_small_hull(const Sets& S, const uint32_t* gstatus, int which, const unsigned long long* keys,
                              const uint32_t* vals, SmallWs* sw, uint32_t* out, int64_t* out_n, cudaStream_t st);

// Sizes used by the sort and chain stages.
constexpr int SORT_TILE = 4096;           // elements per sort tile
constexpr int SORT_PASSES = 7;            // 8-bit digits over the 52-bit key
constexpr int CHAIN_C0 = 512;             // sorted elements per level-0 chunk (one warp each)
constexpr int CHAIN_FAN = 32;             // chunks merged per later-level group

__host__ __device__ inline int64_t sort_tiles(int64_t cap) { return (cap + SORT_TILE - 1) / SORT_TILE; }
// Per-set regions of the sort-tile and chain-count arrays, from the set's
// element offset: 256 * sort_tiles(n_s) resp. 4 * ceil(n_s / CHAIN_C0)
// entries fit between consecutive sets' starts (0 for set 0).
__host__ __device__ inline size_t tiles_at(int64_t off, int s) { return 256 * (size_t)(off / SORT_TILE + s); }
__host__ __device__ inline size_t chains_at(int64_t off, int s) { return 4 * (size_t)(off / CHAIN_C0 + s); }
int chain_levels(int64_t cap);

// Instrumentation: one bounded wait that runs out (k_selftest.cu).
cudaError_t launch_wait_selftest(uint32_t* status, long long limit, cudaStream_t st);

// Batch-only steps (k_batch.cu).
cudaError_t launch_batch_setup(const Sets& S, int64_t n_total, int64_t n_xy, uint32_t* bstatus, int64_t* pp,
                               cudaStream_t st);
cudaError_t launch_batch_jobs(const Sets& S, const uint32_t* bstatus, int which, unsigned long long* ka, uint32_t* va,
                              unsigned long long* kb, uint32_t* vb, unsigned long long* tilecnt, uint32_t* cnt, uint32_t* out,
                              int64_t* out_n, LargeJob* jobs, int* njobs, cudaStream_t st);
cudaError_t launch_batch_emit(const Sets& S, uint32_t* bstatus, const int64_t* hcnt, const uint32_t* hstage,
                              int64_t* hull_offsets, int64_t* hull_idx, cudaStream_t st);

}  // namespace cudapre
