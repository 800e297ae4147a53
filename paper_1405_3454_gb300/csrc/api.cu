// api.cu -- the C ABI (include/cudapre.h): argument checks, workspace layout
// and the launch sequence of each entry point.  Host code only enqueues; no
// step of the method runs on the host.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace cudapre {

int device_sm_count() {
  static int cache[64];
  static std::mutex mu;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  std::lock_guard<std::mutex> lk(mu);
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 152;
    cache[dev] = v;
  }
  return cache[dev];
}

namespace {
std::atomic<long long> g_launches{0};
}  // namespace

void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

}  // namespace cudapre

// Stage timer (instrumentation only): CUDA events at stage boundaries.
struct hull_timer {
  int cap = 0;
  int calls = 0;
  std::vector<cudaEvent_t> ev;  // cap x (HULL_STAGES + 1)
};

namespace cudapre {
namespace {
thread_local hull_timer* g_timer = nullptr;

}  // namespace

// Marks boundary `b` (0..HULL_STAGES) of the current call.
void stage_mark(int b, cudaStream_t st) {
  hull_timer* t = g_timer;
  if (!t || t->calls >= t->cap) return;
  cudaEventRecord(t->ev[(size_t)t->calls * (HULL_STAGES + 1) + b], st);
  if (b == HULL_STAGES) ++t->calls;
}

namespace {

void mark(int b, cudaStream_t st) { stage_mark(b, st); }

constexpr int64_t MAX_N = 0xFFFFFFFFll;  // indices are uint32
constexpr int64_t MAX_BLOCKS = 4096;     // per-block partials of the extreme search

struct Layout {
  size_t header = 0, blockres = 0, cells = 0, tri = 0, small = 0, keys_a = 0, vals_a = 0, keys_b = 0, vals_b = 0, tilecnt = 0,
         cnt = 0, total = 0;
};

Layout layout(int64_t n, bool full) {
  Layout L;
  size_t off = HEADER_BYTES;
  L.header = 0;
  L.blockres = off;
  off += align_up(sizeof(BlockBest) * NSLOT * (MAX_BLOCKS + 1), 256);
  L.cells = off;
  off += align_up(CELL_BYTES, 256);
  if (full) {
    const int64_t cap = compute_capacity(n);
    L.tri = off; off += align_up(sizeof(int4) * 2 * REFINE_BINS, 256);
    L.small = off; off += align_up(sizeof(SmallWs), 256);
    L.keys_a = off; off += align_up(8 * (size_t)cap, 256);
    L.vals_a = off; off += align_up(4 * (size_t)cap, 256);
    L.keys_b = off; off += align_up(8 * (size_t)cap, 256);
    L.vals_b = off; off += align_up(4 * (size_t)cap, 256);
    L.tilecnt = off; off += align_up(8 * 256 * (size_t)sort_tiles(cap), 256);
    const int64_t nch0 = (cap + CHAIN_C0 - 1) / CHAIN_C0;
    L.cnt = off; off += align_up(4 * 4 * (size_t)nch0, 256);
  }
  L.total = off;
  return L;
}

// Workspace of hull_batch (S sets, n_total points): a 256-byte batch word
// block, then the per-set headers and tables, then the per-point buffers
// (each set's part at its element offset).
struct BatchLayout {
  size_t bhdr = 0, hdr = 0, pp = 0, tp = 0, jobs = 0, hcnt = 0, blockres = 0, cells = 0, tri = 0, small = 0,
         keys_a = 0, vals_a = 0, keys_b = 0, vals_b = 0, tilecnt = 0, cnt = 0, hstage = 0, total = 0;
};

BatchLayout batch_layout(int64_t n_total, int32_t S) {
  BatchLayout L;
  const size_t s = (size_t)std::max<int32_t>(S, 0);
  const size_t n = (size_t)std::max<int64_t>(n_total, 1);
  size_t off = 0;
  auto put = [&](size_t& at, size_t bytes) { at = off; off += align_up(bytes, 256); };
  put(L.bhdr, 256);
  put(L.hdr, HEADER_BYTES * s);
  put(L.pp, 8 * (s + 1));
  put(L.tp, 8 * (s + 1));
  put(L.jobs, sizeof(LargeJob) * s);
  put(L.hcnt, 8 * s);
  // partial results: per (block, set) of a static split, or per (unit, set)
  put(L.blockres, sizeof(BlockBest) * NSLOT * ((size_t)MAX_BLOCKS + s + n / 2048 + 2));
  put(L.cells, CELL_BYTES * s);
  put(L.tri, sizeof(int4) * 2 * REFINE_BINS * s);
  put(L.small, sizeof(SmallWs) * s);
  put(L.keys_a, 8 * n);
  put(L.vals_a, 4 * n);
  put(L.keys_b, 8 * n);
  put(L.vals_b, 4 * n);
  put(L.tilecnt, 8 * 256 * (n / SORT_TILE + s + 1));
  put(L.cnt, 4 * 4 * (n / CHAIN_C0 + s + 1));
  put(L.hstage, 4 * n);
  L.total = off;
  return L;
}

// The batch word block: status, then the grid barrier of the large path.
struct BatchWords {
  uint32_t status;
  uint32_t bar_count, bar_gen;
  int njobs;             // sets that take the large-set hull path
  uint32_t next_unit[2];  // units claimed by the streaming search and by the inside test
};

hull_status check_opts(const hull_options* o) {
  if (!o) return HULL_OK;
  if (o->angles != HULL_ANGLES_CUMULATIVE && o->angles != HULL_ANGLES_ABSOLUTE) return HULL_ERR_UNSUPPORTED;
  if (o->filter != HULL_FILTER_EXACT && o->filter != HULL_FILTER_FP32) return HULL_ERR_UNSUPPORTED;
  if (o->block < 0 || o->grid < 0 || o->grid > MAX_BLOCKS) return HULL_ERR_INVALID_ARG;
  if (o->refine != 0 && o->refine != 1) return HULL_ERR_UNSUPPORTED;
  if (o->no_prefilter != 0 && o->no_prefilter != 1) return HULL_ERR_UNSUPPORTED;
  if (o->waves < 0 || o->waves > 16 || o->unit_chunks < 0 || o->unit_chunks > 1024) return HULL_ERR_INVALID_ARG;
  for (int k = 0; k < 7; ++k) if (o->reserved[k] != 0) return HULL_ERR_UNSUPPORTED;
  return HULL_OK;
}

hull_options opts_or_default(const hull_options* o) {
  hull_options d;
  hull_default_options(&d);
  return o ? *o : d;
}

hull_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HULL_OK : HULL_ERR_CUDA; }

LaunchShape shape_of(const hull_options& o) { return LaunchShape{o.grid, o.waves, o.unit_chunks}; }

#define HULL_TRY(expr)                               \
  do {                                               \
    cudaError_t e_ = (expr);                         \
    if (e_ != cudaSuccess) return HULL_ERR_CUDA;     \
  } while (0)

Sets single_set(const float* d_xy, int64_t n, char* ws) {
  Sets S;
  S.xy = d_xy;
  S.off = nullptr;
  S.start = nullptr;
  S.pp = nullptr;
  S.n1 = n;
  S.S = 1;
  S.hdr = ws;
  return S;
}

// Steps 1-3 shared by hull_prefilter and hull_compute.
hull_status run_prefilter(const float* d_xy, int64_t n, char* ws, const Layout& L,
                          uint32_t* surv_idx, unsigned long long* surv_key, uint32_t* ext_out,
                          const hull_options& o, cudaStream_t st, bool reserve = false) {
  WsHeader* h = reinterpret_cast<WsHeader*>(ws + L.header);
  const Sets S = single_set(d_xy, n, ws + L.header);
  mark(0, st);
  HULL_TRY(cudaMemsetAsync(h, 0, sizeof(WsHeader), st));
  if (o.validate) HULL_TRY(launch_validate(d_xy, n, &h->status, st));
  mark(1, st);
  const int64_t npairs = S.npairs_of(0);
  uint16_t* cells = reinterpret_cast<uint16_t*>(ws + L.cells);
  HULL_TRY(launch_extremes(S, npairs, o.angles, o.filter, &h->status, ws + L.blockres, cells, shape_of(o), ext_out,
                           surv_idx, surv_key, st));  // marks boundary 2 between its two kernels
  mark(3, st);
  HULL_TRY(launch_filter(S, npairs, o.filter, &h->status, cells, surv_idx, surv_key, shape_of(o), st, reserve));
  mark(4, st);
  return HULL_OK;
}

hull_status check_common(const float* d_xy, int64_t n, void* d_ws) {
  if (n < 0 || n > MAX_N) return HULL_ERR_INVALID_ARG;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return HULL_ERR_INVALID_ARG;
  if (n > 0 && (!d_xy || (reinterpret_cast<uintptr_t>(d_xy) & 7u))) return HULL_ERR_INVALID_ARG;
  return HULL_OK;
}

}  // namespace
}  // namespace cudapre

using namespace cudapre;

extern "C" {

int32_t hull_abi_version(void) { return 1; }

void hull_default_options(hull_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->angles = HULL_ANGLES_CUMULATIVE;
  opt->filter = HULL_FILTER_FP32;
  opt->refine = 1;
}

void hull_constants(double* out) {
  if (!out) return;
  out[0] = K_S3;
  out[1] = K_C75;
  out[2] = K_S75;
  out[3] = K_H;
}

const char* hull_strerror(hull_status s) {
  switch (s) {
    case HULL_OK: return "HULL_OK";
    case HULL_ERR_INVALID_ARG: return "HULL_ERR_INVALID_ARG: invalid argument";
    case HULL_ERR_DOMAIN: return "HULL_ERR_DOMAIN: input outside the integer [-2^24, 2^24] domain";
    case HULL_ERR_WORKSPACE: return "HULL_ERR_WORKSPACE: workspace too small";
    case HULL_ERR_CUDA: return "HULL_ERR_CUDA: CUDA runtime or launch error";
    case HULL_ERR_TIMEOUT: return "HULL_ERR_TIMEOUT: a bounded device wait expired";
    case HULL_ERR_BUDGET: return "HULL_ERR_BUDGET: request exceeds the memory budget";
    case HULL_ERR_UNSUPPORTED: return "HULL_ERR_UNSUPPORTED: unsupported option";
  }
  return "unknown hull_status";
}

size_t hull_prefilter_workspace_bytes(int64_t n, const hull_options* opt) {
  (void)opt;
  return layout(std::max<int64_t>(n, 0), false).total;
}

size_t hull_workspace_bytes(int64_t n, const hull_options* opt) {
  (void)opt;
  return layout(std::max<int64_t>(n, 0), true).total;
}

hull_status hull_prefilter(const float* d_xy, int64_t n, void* d_ws, size_t ws_bytes,
                           uint32_t* d_survivor_idx, int64_t* d_n_survivors,
                           uint32_t* d_extreme_idx, const hull_options* opt, void* stream) {
  hull_status s = check_common(d_xy, n, d_ws);
  if (s != HULL_OK) return s;
  if ((s = check_opts(opt)) != HULL_OK) return s;
  if (!d_n_survivors || (n > 0 && !d_survivor_idx)) return HULL_ERR_INVALID_ARG;
  if (opt && opt->no_prefilter) return HULL_ERR_UNSUPPORTED;
  const Layout L = layout(n, false);
  if (ws_bytes < L.total) return HULL_ERR_WORKSPACE;
  const hull_options o = opts_or_default(opt);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  s = run_prefilter(d_xy, n, ws, L, d_survivor_idx, nullptr, d_extreme_idx, o, st);
  if (s != HULL_OK) return s;
  s = cuda_status(launch_copy_count(reinterpret_cast<WsHeader*>(ws), d_n_survivors, st));
  mark(5, st);
  mark(6, st);
  return s;
}

hull_status hull_compute(const float* d_xy, int64_t n, void* d_ws, size_t ws_bytes,
                         uint32_t* d_hull_idx, int64_t* d_n_hull, const hull_options* opt,
                         void* stream) {
  hull_status s = check_common(d_xy, n, d_ws);
  if (s != HULL_OK) return s;
  if ((s = check_opts(opt)) != HULL_OK) return s;
  if (!d_n_hull || (n > 0 && !d_hull_idx)) return HULL_ERR_INVALID_ARG;
  const Layout L = layout(n, true);
  if (ws_bytes < L.total) return HULL_ERR_WORKSPACE;
  const hull_options o = opts_or_default(opt);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  WsHeader* h = reinterpret_cast<WsHeader*>(ws);
  auto* ka = reinterpret_cast<unsigned long long*>(ws + L.keys_a);
  auto* va = reinterpret_cast<uint32_t*>(ws + L.vals_a);
  auto* kb = reinterpret_cast<unsigned long long*>(ws + L.keys_b);
  auto* vb = reinterpret_cast<uint32_t*>(ws + L.vals_b);
  if (o.no_prefilter) {
    // the paper's case (1): every point goes to the hull stage
    mark(0, st);
    HULL_TRY(cudaMemsetAsync(h, 0, sizeof(WsHeader), st));
    if (o.validate) HULL_TRY(launch_validate(d_xy, n, &h->status, st));
    mark(1, st);
    mark(2, st);
    mark(3, st);
    HULL_TRY(launch_all_keys(d_xy, n, h, ka, va, st));
    mark(4, st);
  } else {
    // the survivor buffers have room for reserved slots (compute_capacity)
    s = run_prefilter(d_xy, n, ws, L, va, ka, nullptr, o, st, compute_reserves(n));
    if (s != HULL_OK) return s;
  }
  const int64_t cap = compute_capacity(n);
  // The hull of the survivors.  With refinement the survivors in (ka, va)
  // are thinned into (kb, vb) first.  Sets up to SMALL_MAX points take the
  // small-set path; larger ones two cooperative launches of the device radix
  // sort (7 passes, ending in the other buffer) and the chunked chain (its
  // upper chains in the input).
  const bool refine = o.refine != 0 && !o.no_prefilter;
  const Sets S = single_set(d_xy, n, ws);
  unsigned long long* kin = ka;
  uint32_t* vin = va;
  unsigned long long* kot = kb;
  uint32_t* vot = vb;
  const unsigned long long* count = &h->n_surv;
  if (refine) {
    HULL_TRY(launch_refine(S, &h->status, nullptr, ka, va, kb, vb, reinterpret_cast<int4*>(ws + L.tri), cap, st));
    kin = kb; vin = vb; kot = ka; vot = va;
    count = &h->n_surv2;
  }
  HULL_TRY(launch_small_hull(S, &h->status, refine ? 1 : 0, kin, vin, reinterpret_cast<SmallWs*>(ws + L.small),
                             d_hull_idx, d_n_hull, st));
  LargeJob J;
  J.h = h;
  J.count = count;
  J.ka = kin; J.va = vin; J.kb = kot; J.vb = vot;
  J.tilecnt = reinterpret_cast<unsigned long long*>(ws + L.tilecnt);
  J.cnt = reinterpret_cast<uint32_t*>(ws + L.cnt);
  J.out_idx = d_hull_idx;
  J.out_n = d_n_hull;
  J.cap = cap;
  mark(5, st);
  HULL_TRY(launch_large(nullptr, nullptr, J, &h->bar_count, &h->status, st));
  mark(6, st);
  return HULL_OK;
}

size_t hull_batch_workspace_bytes(int64_t n_total, int32_t S, const hull_options* opt) {
  (void)opt;
  return batch_layout(n_total, S).total;
}

hull_status hull_batch(const float* d_xy, const int64_t* d_offsets, int32_t S, int64_t n_total, void* d_ws,
                       size_t ws_bytes, int64_t* d_hull_idx, int64_t* d_hull_offsets, const hull_options* opt,
                       void* stream) {
  return hull_batch_ranges(d_xy, n_total, nullptr, d_offsets, S, n_total, d_ws, ws_bytes, d_hull_idx,
                           d_hull_offsets, opt, stream);
}

hull_status hull_batch_ranges(const float* d_xy, int64_t n_xy, const int64_t* d_starts, const int64_t* d_offsets,
                              int32_t S, int64_t n_total, void* d_ws, size_t ws_bytes, int64_t* d_hull_idx,
                              int64_t* d_hull_offsets, const hull_options* opt, void* stream) {
  if (S < 0 || n_total < 0 || n_total > ((int64_t)1 << 40) || n_xy < 0) return HULL_ERR_INVALID_ARG;
  if (!d_offsets || !d_hull_offsets || !d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u))
    return HULL_ERR_INVALID_ARG;
  if (n_total > 0 && (!d_xy || (reinterpret_cast<uintptr_t>(d_xy) & 7u) || !d_hull_idx)) return HULL_ERR_INVALID_ARG;
  if (!d_starts && n_xy != n_total) return HULL_ERR_INVALID_ARG;
  hull_status s;
  if ((s = check_opts(opt)) != HULL_OK) return s;
  if (opt && opt->no_prefilter) return HULL_ERR_UNSUPPORTED;
  const BatchLayout L = batch_layout(n_total, S);
  if (ws_bytes < L.total) return HULL_ERR_WORKSPACE;
  const hull_options o = opts_or_default(opt);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(d_ws);
  BatchWords* bw = reinterpret_cast<BatchWords*>(ws + L.bhdr);
  // the words and per-set counters that must start at zero
  HULL_TRY(cudaMemsetAsync(ws, 0, L.hdr + HEADER_BYTES * (size_t)S, st));
  if (S == 0) {
    HULL_TRY(cudaMemsetAsync(d_hull_offsets, 0, sizeof(int64_t), st));
    return HULL_OK;
  }
  Sets SS;
  SS.xy = d_xy;
  SS.off = d_offsets;
  SS.start = d_starts;
  SS.pp = reinterpret_cast<const int64_t*>(ws + L.pp);
  SS.n1 = 0;
  SS.S = S;
  SS.hdr = ws + L.hdr;
  uint32_t* bstatus = &bw->status;
  auto* ka = reinterpret_cast<unsigned long long*>(ws + L.keys_a);
  auto* va = reinterpret_cast<uint32_t*>(ws + L.vals_a);
  auto* kb = reinterpret_cast<unsigned long long*>(ws + L.keys_b);
  auto* vb = reinterpret_cast<uint32_t*>(ws + L.vals_b);
  auto* hstage = reinterpret_cast<uint32_t*>(ws + L.hstage);
  auto* hcnt = reinterpret_cast<int64_t*>(ws + L.hcnt);
  uint16_t* cells = reinterpret_cast<uint16_t*>(ws + L.cells);
  // The streaming search keeps several waves of static shares (its per-set
  // work is heavier than the inside test's); the inside test claims units.
  const bool ext_units = false;
  mark(0, st);
  if (o.validate) HULL_TRY(launch_validate(d_xy, n_xy, bstatus, st));
  HULL_TRY(launch_batch_setup(SS, n_total, n_xy, bstatus, reinterpret_cast<int64_t*>(ws + L.pp), st));
  mark(1, st);
  const int64_t pairs_bound = n_total / 2;
  HULL_TRY(launch_extremes(SS, pairs_bound, o.angles, o.filter, bstatus, ws + L.blockres, cells, shape_of(o), nullptr, va,
                           ka, st, ext_units ? &bw->next_unit[0] : nullptr));  // marks boundary 2 between its two kernels
  mark(3, st);
  HULL_TRY(launch_filter(SS, pairs_bound, o.filter, bstatus, cells, va, ka, shape_of(o), st, false, &bw->next_unit[1]));
  mark(4, st);
  const int64_t cap = std::max<int64_t>(n_total, 1);
  const bool refine = o.refine != 0;
  unsigned long long* kin = ka;
  uint32_t* vin = va;
  unsigned long long* kot = kb;
  uint32_t* vot = vb;
  if (refine) {
    HULL_TRY(launch_refine(SS, bstatus, reinterpret_cast<int64_t*>(ws + L.tp), ka, va, kb, vb,
                           reinterpret_cast<int4*>(ws + L.tri), cap, st));
    kin = kb; vin = vb; kot = ka; vot = va;
  }
  const int which = refine ? 1 : 0;
  HULL_TRY(launch_small_hull(SS, bstatus, which, kin, vin, reinterpret_cast<SmallWs*>(ws + L.small), hstage, hcnt,
                             st));
  LargeJob* jobs = reinterpret_cast<LargeJob*>(ws + L.jobs);
  HULL_TRY(launch_batch_jobs(SS, bstatus, which, kin, vin, kot, vot, reinterpret_cast<unsigned long long*>(ws + L.tilecnt),
                             reinterpret_cast<uint32_t*>(ws + L.cnt), hstage, hcnt, jobs, &bw->njobs, st));
  mark(5, st);
  LargeJob none{};
  HULL_TRY(launch_large(jobs, &bw->njobs, none, &bw->bar_count, bstatus, st));
  HULL_TRY(launch_batch_emit(SS, bstatus, hcnt, hstage, d_hull_offsets, d_hull_idx, st));
  mark(6, st);
  return HULL_OK;
}

hull_status hull_selftest_wait(void* d_ws, int64_t limit_cycles, void* stream) {
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255u)) return HULL_ERR_INVALID_ARG;
  if (limit_cycles < 1 || limit_cycles > ((int64_t)1 << 31)) return HULL_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t* status = reinterpret_cast<uint32_t*>(d_ws);  // the first word of every workspace
  HULL_TRY(cudaMemsetAsync(status, 0, sizeof(uint32_t), st));
  HULL_TRY(launch_wait_selftest(status, limit_cycles, st));
  return HULL_OK;
}

hull_status hull_read_counters(const void* d_ws, int64_t* h_n_survivors, int64_t* h_n_escalated,
                               void* stream) {
  if (!d_ws) return HULL_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  WsHeader hh;
  HULL_TRY(cudaMemcpyAsync(&hh, d_ws, sizeof(WsHeader), cudaMemcpyDeviceToHost, st));
  HULL_TRY(cudaStreamSynchronize(st));
  if (h_n_survivors) *h_n_survivors = (int64_t)(hh.n_surv - hh.n_fill);
  if (h_n_escalated) *h_n_escalated = (int64_t)hh.n_escalated;
  return HULL_OK;
}

hull_status hull_read_stats(const void* d_ws, hull_stats* h_out, void* stream) {
  if (!d_ws || !h_out) return HULL_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  WsHeader hh;
  HULL_TRY(cudaMemcpyAsync(&hh, d_ws, sizeof(WsHeader), cudaMemcpyDeviceToHost, st));
  HULL_TRY(cudaStreamSynchronize(st));
  h_out->n_survivors = (int64_t)(hh.n_surv - hh.n_fill);
  h_out->n_escalated = (int64_t)hh.n_escalated;
  h_out->n_refined = (int64_t)hh.n_surv2;
  h_out->polygon_vertices = hh.poly.m;
  h_out->device_status = hh.status;
  return HULL_OK;
}

hull_status hull_read_polygon(const void* d_ws, int32_t* h_m, int32_t* h_xy, uint32_t* h_idx,
                              void* stream) {
  if (!d_ws || !h_m || !h_xy) return HULL_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  WsHeader hh;
  HULL_TRY(cudaMemcpyAsync(&hh, d_ws, sizeof(WsHeader), cudaMemcpyDeviceToHost, st));
  HULL_TRY(cudaStreamSynchronize(st));
  *h_m = hh.poly.m;
  for (int k = 0; k < hh.poly.m && k < MAXV; ++k) {
    h_xy[2 * k] = hh.poly.vx[k];
    h_xy[2 * k + 1] = hh.poly.vy[k];
    if (h_idx) h_idx[k] = hh.poly.vidx[k];
  }
  return HULL_OK;
}

hull_status hull_batch_read_set(const void* d_ws, int64_t n_total, int32_t S, int32_t s, hull_set_info* h_out,
                                void* stream) {
  if (!d_ws || !h_out || S < 0 || n_total < 0 || s < 0 || s >= S) return HULL_ERR_INVALID_ARG;
  const BatchLayout L = batch_layout(n_total, S);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  WsHeader hh;
  const char* src = static_cast<const char*>(d_ws) + L.hdr + (size_t)s * HEADER_BYTES;
  HULL_TRY(cudaMemcpyAsync(&hh, src, sizeof(WsHeader), cudaMemcpyDeviceToHost, st));
  HULL_TRY(cudaStreamSynchronize(st));
  std::memset(h_out, 0, sizeof(*h_out));
  const int m = std::max(0, std::min(hh.poly.m, MAXV));
  h_out->polygon_vertices = m;
  for (int k = 0; k < m; ++k) {
    h_out->polygon_xy[2 * k] = hh.poly.vx[k];
    h_out->polygon_xy[2 * k + 1] = hh.poly.vy[k];
    h_out->polygon_idx[k] = hh.poly.vidx[k];
  }
  for (int k = 0; k < NSLOT; ++k) h_out->extreme_idx[k] = hh.poly.ext[k];
  h_out->n_survivors = (int64_t)(hh.n_surv - hh.n_fill);
  h_out->n_escalated = (int64_t)hh.n_escalated;
  h_out->n_refined = (int64_t)hh.n_surv2;
  h_out->device_status = hh.status;
  return HULL_OK;
}

hull_status hull_get_device_status(const void* d_ws, uint32_t* h_bits, void* stream) {
  if (!d_ws) return HULL_ERR_INVALID_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  uint32_t bits = 0;
  HULL_TRY(cudaMemcpyAsync(&bits, d_ws, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  HULL_TRY(cudaStreamSynchronize(st));
  if (h_bits) *h_bits = bits;
  if (bits & HULL_DEVICE_DOMAIN) return HULL_ERR_DOMAIN;
  if (bits & HULL_DEVICE_TIMEOUT) return HULL_ERR_TIMEOUT;
  if (bits & HULL_DEVICE_OFFSETS) return HULL_ERR_INVALID_ARG;
  if (bits) return HULL_ERR_CUDA;
  return HULL_OK;
}

hull_timer* hull_timer_create(int32_t max_calls) {
  if (max_calls <= 0) return nullptr;
  hull_timer* t = new hull_timer();
  t->cap = max_calls;
  t->ev.resize((size_t)max_calls * (HULL_STAGES + 1));
  for (auto& e : t->ev) {
    if (cudaEventCreate(&e) != cudaSuccess) {
      e = nullptr;
      hull_timer_destroy(t);
      return nullptr;
    }
  }
  return t;
}

void hull_timer_destroy(hull_timer* t) {
  if (!t) return;
  if (g_timer == t) g_timer = nullptr;
  for (auto e : t->ev) if (e) cudaEventDestroy(e);
  delete t;
}

void hull_timer_attach(hull_timer* t) { g_timer = t; }

hull_status hull_timer_read(hull_timer* t, float* h_ms, int32_t* h_calls) {
  if (!t || !h_ms) return HULL_ERR_INVALID_ARG;
  for (int s = 0; s < HULL_STAGES; ++s) h_ms[s] = 0.0f;
  for (int c = 0; c < t->calls; ++c) {
    cudaEvent_t* e = &t->ev[(size_t)c * (HULL_STAGES + 1)];
    HULL_TRY(cudaEventSynchronize(e[HULL_STAGES]));
    for (int s = 0; s < HULL_STAGES; ++s) {
      float ms = 0.0f;
      HULL_TRY(cudaEventElapsedTime(&ms, e[s], e[s + 1]));
      h_ms[s] += ms;
    }
  }
  if (h_calls) *h_calls = t->calls;
  t->calls = 0;
  return HULL_OK;
}

int64_t hull_launch_count(void) { return (int64_t)g_launches.load(); }

}  // extern "C"
