// k_batch.cu -- the kernels that only a batch of point sets needs: checking
// the caller's set offsets and laying out the virtual pair axis, the job
// table of the large-set hull path, and the final packing of every set's
// hull into one array of global point indices.  Each set goes through the
// same steps of the method (section 2, Steps 1-3, then the hull of the
// survivors) as a single set.
#include "internal.cuh"

namespace cudapre {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int TB = 1024;

// Exclusive block scan of int64 values in chunks of TB; returns nothing,
// calls put(s, exclusive prefix) for s < n, and the total at the end.
template <class Get, class Put>
__device__ int64_t block_prefix(int n, Get get, Put put) {
  __shared__ int64_t s_w[TB / 32];
  __shared__ int64_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int s0 = 0; s0 < n; s0 += TB) {
    const int s = s0 + threadIdx.x;
    const int64_t v = s < n ? get(s) : 0;
    int64_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t u = __shfl_up_sync(FULL, incl, off);
      if (lane >= off) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    int64_t wpre = 0, tot = 0;
    for (int w = 0; w < TB / 32; ++w) {
      const int64_t x = s_w[w];
      if (w < warp) wpre += x;
      tot += x;
    }
    const int64_t carry = s_carry;
    if (s < n) put(s, carry + wpre + incl - v);
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + tot;
    __syncthreads();
  }
  const int64_t total = s_carry;
  __syncthreads();
  return total;
}

// Offsets check (off[0] == 0, non-decreasing, off[S] == n_total; with
// start rows, every set within the n_xy points) and the prefix of the sets'
// 16-byte pair counts.  Bad offsets set HULL_DEVICE_OFFSETS in the batch
// status and every later step skips.
__global__ void __launch_bounds__(TB) k_batch_setup(Sets S, int64_t n_total, int64_t n_xy, uint32_t* bstatus,
                                                    int64_t* pp) {
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = (S.off[0] != 0 || S.off[S.S] != n_total) ? 1 : 0;
  __syncthreads();
  bool bad = false;
  for (int s = threadIdx.x; s < S.S; s += TB) {
    const int64_t n = S.off[s + 1] - S.off[s];
    bad |= n < 0 || n > 0xFFFFFFFFll;
    if (S.start) bad |= S.start[s] < 0 || S.start[s] > n_xy - n;
  }
  if (bad) atomicOr(&s_bad, 1);
  __syncthreads();
  const bool ok = s_bad == 0;
  if (!ok && threadIdx.x == 0) atomicOr(bstatus, HULL_DEVICE_OFFSETS);
  Sets T = S;
  T.pp = nullptr;
  const int64_t total = block_prefix(
      S.S, [&](int s) { return ok ? T.npairs_of(s) : (int64_t)0; }, [&](int s, int64_t v) { pp[s] = v; });
  if (threadIdx.x == 0) pp[S.S] = total;
}

// Large-path jobs: the sets whose survivors after the refinement round
// (which = 1) or after Step 3 (which = 0) exceed the one-block hull, listed
// in jobs[0 .. *njobs) in any order.
__global__ void k_batch_jobs(Sets S, const uint32_t* bstatus, int which, unsigned long long* ka, uint32_t* va,
                             unsigned long long* kb, uint32_t* vb, unsigned long long* tilecnt, uint32_t* cnt, uint32_t* out,
                             int64_t* out_n, LargeJob* jobs, int* njobs) {
  if (*reinterpret_cast<const volatile uint32_t*>(bstatus)) return;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S.S; s += gridDim.x * blockDim.x) {
    const int64_t o = S.off_at(s);
    WsHeader* h = S.h(s);
    if (h->status) continue;
    if ((which == 0 ? h->n_surv : h->n_surv2) <= (unsigned long long)SMALL_MAX) continue;
    LargeJob J;
    J.h = h;
    J.count = which == 0 ? &h->n_surv : &h->n_surv2;
    J.ka = ka + o; J.va = va + o; J.kb = kb + o; J.vb = vb + o;
    J.tilecnt = tilecnt + tiles_at(o, s);
    J.cnt = cnt + chains_at(o, s);
    J.out_idx = out + o;
    J.out_n = out_n + s;
    J.cap = S.n_of(s) > 0 ? S.n_of(s) : 1;
    jobs[atomicAdd(njobs, 1)] = J;
  }
}

// Hull offsets (exclusive prefix of the sets' hull sizes) and the batch
// status (every set's status word or-ed in).
__global__ void __launch_bounds__(TB) k_batch_offsets(Sets S, uint32_t* bstatus, const int64_t* hcnt,
                                                      int64_t* hoff) {
  __shared__ uint32_t s_or;
  if (threadIdx.x == 0) s_or = 0;
  __syncthreads();
  uint32_t st = 0;
  for (int s = threadIdx.x; s < S.S; s += TB) st |= S.h(s)->status;
  if (st) atomicOr(&s_or, st);
  __syncthreads();
  const bool dead = (*reinterpret_cast<volatile uint32_t*>(bstatus) | s_or) != 0;
  if (threadIdx.x == 0 && s_or) atomicOr(bstatus, s_or);
  const int64_t total = block_prefix(
      S.S, [&](int s) { return dead ? (int64_t)0 : hcnt[s]; }, [&](int s, int64_t v) { hoff[s] = v; });
  if (threadIdx.x == 0) hoff[S.S] = total;
}

// Global indices: hull vertex k of set s goes to hull_idx[hoff[s] + k] as
// start(s) + (its index within the set).
__global__ void k_batch_gather(Sets S, const uint32_t* hstage, const int64_t* hoff, int64_t* hull_idx) {
  for (int s = blockIdx.x; s < S.S; s += gridDim.x) {
    const int64_t b = hoff[s], c = hoff[s + 1] - b, o = S.off_at(s), g = S.start_at(s);
    for (int64_t k = threadIdx.x; k < c; k += blockDim.x) hull_idx[b + k] = g + (int64_t)hstage[o + k];
  }
}

}  // namespace

cudaError_t launch_batch_setup(const Sets& S, int64_t n_total, int64_t n_xy, uint32_t* bstatus, int64_t* pp,
                               cudaStream_t st) {
  k_batch_setup<<<1, TB, 0, st>>>(S, n_total, n_xy, bstatus, pp);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_jobs(const Sets& S, const uint32_t* bstatus, int which, unsigned long long* ka, uint32_t* va,
                              unsigned long long* kb, uint32_t* vb, unsigned long long* tilecnt, uint32_t* cnt, uint32_t* out,
                              int64_t* out_n, LargeJob* jobs, int* njobs, cudaStream_t st) {
  const unsigned g = (unsigned)std::min<int64_t>(((int64_t)S.S + 255) / 256, 1024);
  k_batch_jobs<<<g, 256, 0, st>>>(S, bstatus, which, ka, va, kb, vb, tilecnt, cnt, out, out_n, jobs, njobs);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_batch_emit(const Sets& S, uint32_t* bstatus, const int64_t* hcnt, const uint32_t* hstage,
                              int64_t* hull_offsets, int64_t* hull_idx, cudaStream_t st) {
  k_batch_offsets<<<1, TB, 0, st>>>(S, bstatus, hcnt, hull_offsets);
  const unsigned g = (unsigned)std::min<int64_t>(S.S, (int64_t)device_sm_count() * 8);
  k_batch_gather<<<g, 256, 0, st>>>(S, hstage, hull_offsets, hull_idx);
  count_launches(2);
  return cudaGetLastError();
}

}  // namespace cudapre
