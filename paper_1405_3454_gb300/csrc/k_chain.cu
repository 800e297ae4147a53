// k_chain.cu -- Andrew's monotone chain over the sorted survivors, the second
// half of the final-hull stage (section 3, case (2): the hull of the points
// that remain after the preprocessing).
//
// Chunked: level 0 runs the lower and the upper chain of every sorted chunk
// of CHAIN_C0 keys; each later level concatenates CHAIN_FAN consecutive
// chunk chains (still sorted) and chains them again, until one chunk is
// left.  A hull vertex of the whole set is a vertex of every chunk chain
// that contains it, so the final chain is the hull of the union.  Stacks are
// written in place over the consumed input (a push never overtakes the read
// cursor).  Equal keys are adjacent (sorted input; chunk seams), and the
// lowest index is kept among them.  Every size is read on the device.
#include "internal.cuh"

namespace cudapre {

namespace {

// Element count of the large path: 0 (nothing to do) when the one-block
// path takes the set.
__device__ __forceinline__ int64_t dev_count(const WsHeader* h, const unsigned long long* count) {
  if (*reinterpret_cast<const volatile uint32_t*>(&h->status)) return 0;
  const int64_t m = (int64_t)*reinterpret_cast<const volatile unsigned long long*>(count);
  return m > SMALL_MAX ? m : 0;
}

__device__ __forceinline__ long long cross_k(unsigned long long o, unsigned long long a,
                                             unsigned long long b) {
  const long long ox = key_x(o), oy = key_y(o);
  return ((long long)key_x(a) - ox) * ((long long)key_y(b) - oy) -
         ((long long)key_y(a) - oy) * ((long long)key_x(b) - ox);
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

// Level 0: thread g chains sorted elements [g*C0, min((g+1)*C0, m)).
// Lower chain in place in (Ks, Vs); upper chain into (Ku, Vu) at the same
// offsets.  Counts to cnt_lo[g], cnt_up[g].
__global__ void k_chain0(unsigned long long* Ks, uint32_t* Vs, unsigned long long* Ku, uint32_t* Vu,
                         const WsHeader* h, const unsigned long long* count, uint32_t* cnt_lo, uint32_t* cnt_up, int64_t nch) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= nch) return;
  const int64_t m = dev_count(h, count);
  const int64_t start = g * CHAIN_C0;
  if (start >= m) return;
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

// Later level: group g merges the chains of chunks [g*FAN, (g+1)*FAN) of the
// previous level (span `span_prev` each).  Thread 2g+0 does the lower
// chains, 2g+1 the upper ones.
__global__ void k_chainN(unsigned long long* Ks, uint32_t* Vs, unsigned long long* Ku, uint32_t* Vu,
                         const WsHeader* h, const unsigned long long* count, const uint32_t* cin_lo, const uint32_t* cin_up,
                         uint32_t* cout_lo, uint32_t* cout_up, int64_t nch_prev, int64_t span_prev,
                         int64_t ngroups) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = t >> 1;
  const bool upper = t & 1;
  if (g >= ngroups) return;
  const int64_t m = dev_count(h, count);
  const int64_t c0 = g * CHAIN_FAN;
  if (c0 * span_prev >= m) return;
  const int64_t c1 = min(c0 + (int64_t)CHAIN_FAN, nch_prev);
  if (!upper) {
    Stack<false> s;
    s.init(Ks, Vs, c0 * span_prev);
    for (int64_t c = c0; c < c1 && c * span_prev < m; ++c) {
      const int64_t b = c * span_prev, cnt = cin_lo[c];
      for (int64_t j = 0; j < cnt; ++j) s.push(Ks[b + j], Vs[b + j]);
    }
    cout_lo[g] = (uint32_t)s.n;
  } else {
    Stack<true> s;
    s.init(Ku, Vu, c0 * span_prev);
    for (int64_t c = c0; c < c1 && c * span_prev < m; ++c) {
      const int64_t b = c * span_prev, cnt = cin_up[c];
      for (int64_t j = 0; j < cnt; ++j) s.push(Ku[b + j], Vu[b + j]);
    }
    cout_up[g] = (uint32_t)s.n;
  }
}

// Hull counter-clockwise from the lexicographic minimum: the lower chain
// left to right, then the upper chain right to left, without repeating the
// two end points.
__global__ void k_chain_final(const uint32_t* Vs, const uint32_t* Vu, const WsHeader* h,
                              const unsigned long long* count, const uint32_t* cnt_lo,
                              const uint32_t* cnt_up, uint32_t* out_idx, int64_t* out_n) {
  const int64_t m = dev_count(h, count);
  if (m == 0) return;  // the one-block path wrote the result
  const int64_t a = cnt_lo[0], b = cnt_up[0];
  int64_t pos = 0;
  if (a == 1) {
    out_idx[pos++] = Vs[0];
  } else {
    for (int64_t k = 0; k + 1 < a; ++k) out_idx[pos++] = Vs[k];
    for (int64_t k = b - 1; k >= 1; --k) out_idx[pos++] = Vu[k];
  }
  *out_n = pos;
}

}  // namespace

int chain_levels(int64_t cap) {
  int64_t nch = (std::max<int64_t>(cap, 1) + CHAIN_C0 - 1) / CHAIN_C0;
  int levels = 1;
  while (nch > 1) { nch = (nch + CHAIN_FAN - 1) / CHAIN_FAN; ++levels; }
  return levels;
}

// cnt holds four arrays of nch0 entries: lower/upper for even and odd levels.
cudaError_t launch_chain(int64_t cap, WsHeader* h, const unsigned long long* count,
                         unsigned long long* keys_s, uint32_t* vals_s, unsigned long long* keys_u,
                         uint32_t* vals_u, uint32_t* cnt, uint32_t* out_idx, int64_t* out_n,
                         cudaStream_t st) {
  const int64_t nch0 = (std::max<int64_t>(cap, 1) + CHAIN_C0 - 1) / CHAIN_C0;
  uint32_t* lo[2] = {cnt, cnt + 2 * nch0};
  uint32_t* up[2] = {cnt + nch0, cnt + 3 * nch0};
  const int TB = 128;
  k_chain0<<<(unsigned)((nch0 + TB - 1) / TB), TB, 0, st>>>(keys_s, vals_s, keys_u, vals_u, h, count, lo[0], up[0], nch0);
  count_launches(1);
  int64_t nch = nch0, span = CHAIN_C0;
  int par = 0;
  while (nch > 1) {
    const int64_t ng = (nch + CHAIN_FAN - 1) / CHAIN_FAN;
    const int64_t threads = 2 * ng;
    k_chainN<<<(unsigned)((threads + TB - 1) / TB), TB, 0, st>>>(keys_s, vals_s, keys_u, vals_u, h, count,
                                                                 lo[par], up[par], lo[par ^ 1], up[par ^ 1],
                                                                 nch, span, ng);
    count_launches(1);
    par ^= 1;
    nch = ng;
    span *= CHAIN_FAN;
  }
  k_chain_final<<<1, 1, 0, st>>>(vals_s, vals_u, h, count, lo[par], up[par], out_idx, out_n);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cudapre
