// k_hull_small.cu -- the hull of a survivor set of at most SMALL_MAX points:
// the final step of the method, the hull of the points that remain (section
// 3, case (2)).
//
// A batch's sets of at most TINY_MAX points:
// tiny     (one block per set) bitonic sort, then Andrew's lower and upper
//          monotone chains in two levels.
// One set uses the whole GPU, without sorting (its chain walk would be one
// thread's sequence of dependent steps):
// classify (one warp per survivor v) v is a vertex of the lower chain iff
//          no point with equal coordinates has a lower index, and either v is
//          the lexicographically smallest or largest point, or the most
//          counter-clockwise incoming direction v - a over every point a
//          before v (in (x, y) order) turns strictly left into the most
//          clockwise outgoing direction b - v over every point b after v;
//          the upper chain is the same with the turns mirrored.  The
//          directions of each reduction lie in a half-plane, so the cross
//          product orders them.
// rank     (one warp per vertex) its position: how many vertices of its chain
//          come before it in (x, y) order.
// A batch gives each set one block (many sets at once):
// prep     sort the survivors by (x, y, index) in registers and shared
//          memory, keep the first of each run of equal coordinates (the
//          lowest index), split them into 32 chunks and run the lower and
//          upper chain of each chunk;
// prune    (one warp per chunk-chain vertex) the test of classify over the
//          32 chunk chains, each by binary search (the extremes over one
//          convex chain are unimodal);
// emit     the lower hull left to right, then the upper hull right to left.
#include <type_traits>

#include "internal.cuh"

namespace cudapre {

namespace {

constexpr int SB = 1024;      // threads

constexpr int NCH = SMALL_NCH;  // chunks (one warp each)
constexpr unsigned FULL = 0xFFFFFFFFu;

// Cross product of two difference vectors of lattice points within +-2^24
// (32-bit components; one widening multiply per product).
__device__ __forceinline__ long long cr(int ax, int ay, int bx, int by) {
  return (long long)ax * by - (long long)ay * bx;
}

// Exclusive block scan of one int per thread; writes the total to *tot.
__device__ __forceinline__ int block_scan(int v, int* s_w, int* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int incl = v;
  for (int off = 1; off < 32; off <<= 1) {
    const int t = __shfl_up_sync(FULL, incl, off);
    if (lane >= off) incl += t;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = s_w[lane];
    int wi = w;
    for (int off = 1; off < 32; off <<= 1) {
      const int t = __shfl_up_sync(FULL, wi, off);
      if (lane >= off) wi += t;
    }
    s_w[lane] = wi - w;
    if (lane == 31) *tot = wi;
  }
  __syncthreads();
  const int r = s_w[warp] + incl - v;
  __syncthreads();
  return r;
}

struct Pts {
  const int* x;
  const int* y;
};

// Chain of chunk c (positions into the unique arrays) for sign S (+1 lower,
// -1 upper), computed by one thread, in place from `base`.
// Chain of chunk [lo, hi) (positions into the unique arrays) for sign sg
// (+1 lower, -1 upper), computed by one thread into st; the top two stack
// points stay in registers.  Lower and upper chains of one chunk run in two
// lanes of one warp on the same instruction stream.
__device__ int chunk_chain(Pts P, int lo, int hi, uint16_t* st, long long sg) {
  int n = 0;
  int x1 = 0, y1 = 0, x2 = 0, y2 = 0;
  for (int p = lo; p < hi; ++p) {
    const int px = P.x[p], py = P.y[p];
    while (n >= 2) {
      const long long c = sg * cr(x1 - x2, y1 - y2, px - x2, py - y2);
      if (c > 0) break;
      --n;
      x1 = x2; y1 = y2;
      if (n >= 2) { const int a = st[n - 2]; x2 = P.x[a]; y2 = P.y[a]; }
    }
    st[n++] = (uint16_t)p;
    x2 = x1; y2 = y1;
    x1 = px; y1 = py;
  }
  return n;
}

__device__ __forceinline__ int64_t count_of(const WsHeader* h, const unsigned long long* c) {
  if (*reinterpret_cast<const volatile uint32_t*>(&h->status)) return 0;
  return (int64_t)*reinterpret_cast<const volatile unsigned long long*>(c);
}

// prep: sort, dedupe, chunk chains -> SmallWs (global).
__global__ void __launch_bounds__(SB, 1) k_small_prep(Sets S, const uint32_t* gstatus, int which,
                                                       const unsigned long long* __restrict__ kin_base,
                                                       const uint32_t* __restrict__ vin_base, SmallWs* sw_base,
                                                       uint32_t* __restrict__ out_base, int64_t* out_n_base) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_w[32];
  __shared__ int s_tot;
  __shared__ int s_cnt[2][NCH];
  const int tid = threadIdx.x;
  const int set = blockIdx.x;
  const WsHeader* h = S.h(set);
  const int64_t o = S.off_at(set);
  const unsigned long long* kin = kin_base + o;
  const uint32_t* vin = vin_base + o;
  uint32_t* out = out_base + o;
  int64_t* out_n = out_n_base + set;
  SmallWs* sw = sw_base + set;
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(gstatus) != 0;
  const int64_t m64 = dead ? 0 : count_of(h, which == 0 ? &h->n_surv : &h->n_surv2);
  if (m64 > SMALL_MAX || m64 <= TINY_MAX) {  // the large path, the tiny kernel, or nothing to do
    if (tid == 0) {
      sw->active = 0;
      if (m64 == 0) *out_n = 0;
    }
    return;
  }
  const int m = (int)m64;
  int P2 = 2;
  while (P2 < m) P2 <<= 1;
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(sm);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + SMALL_MAX);
  uint16_t* chain = reinterpret_cast<uint16_t*>(si + SMALL_MAX);  // [2][SMALL_MAX]
  // Bitonic sort by (key, index) of P2 = 2^p elements (2048..8192), element
  // i = r * SB + tid held in registers by thread tid (r < P2 / SB): partner
  // distances below 32 are exchanged by warp shuffles, distances of SB and
  // more stay in the thread, only 32..SB/2 go through shared memory.
  {
    constexpr int EMAX = SMALL_MAX / SB;
    const int NE = P2 / SB;
    unsigned long long qk[EMAX];
    uint32_t qv[EMAX];
#pragma unroll
    for (int r = 0; r < EMAX; ++r) {
      const int i = r * SB + tid;
      qk[r] = (r < NE && i < m) ? kin[i] : ~0ull;
      qv[r] = (r < NE && i < m) ? vin[i] : ~0u;
    }
    for (int k = 2; k <= P2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        if (j >= SB) {  // partner in the same thread: element r ^ (j / SB)
          auto in_thread = [&](auto JR) {
            constexpr int jr = decltype(JR)::value;
#pragma unroll
            for (int r = 0; r < EMAX; ++r) {
              const int l = r ^ jr;
              if (l > r && l < EMAX && r < NE) {
                const int i = r * SB + tid;
                const bool asc = (i & k) == 0;
                const bool gt = qk[r] > qk[l] || (qk[r] == qk[l] && qv[r] > qv[l]);
                if (gt == asc) {
                  const unsigned long long tk = qk[r]; qk[r] = qk[l]; qk[l] = tk;
                  const uint32_t tv = qv[r]; qv[r] = qv[l]; qv[l] = tv;
                }
              }
            }
          };
          const int jr = j / SB;  // 1, 2 or 4
          if (jr == 1) in_thread(std::integral_constant<int, 1>{});
          else if (jr == 2) in_thread(std::integral_constant<int, 2>{});
          else in_thread(std::integral_constant<int, 4>{});
          continue;
        }
        if (j >= 32) {  // through shared memory
#pragma unroll
          for (int r = 0; r < EMAX; ++r)
            if (r < NE) { sk[r * SB + tid] = qk[r]; si[r * SB + tid] = qv[r]; }
          __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < EMAX; ++r) {
          if (r < NE) {
            const int i = r * SB + tid;
            unsigned long long pk;
            uint32_t pv;
            if (j >= 32) {
              pk = sk[i ^ j];
              pv = si[i ^ j];
            } else {
              pk = __shfl_xor_sync(FULL, qk[r], j);
              pv = __shfl_xor_sync(FULL, qv[r], j);
            }
            const bool asc = (i & k) == 0;
            const bool lower = (i & j) == 0;  // the smaller index of the pair
            const bool pgt = pk > qk[r] || (pk == qk[r] && pv > qv[r]);  // partner is larger
            // the lower element keeps the minimum when ascending
            const bool take = lower == asc ? !pgt : pgt;
            if (take) { qk[r] = pk; qv[r] = pv; }
          }
        }
        if (j >= 32) __syncthreads();
      }
    }
#pragma unroll
    for (int r = 0; r < EMAX; ++r)
      if (r < NE) { sk[r * SB + tid] = qk[r]; si[r * SB + tid] = qv[r]; }
    __syncthreads();
  }
  // dedupe: first of each run of equal keys (lowest index) -> unique arrays
  constexpr int E = SMALL_MAX / SB;  // elements per thread (blocked)
  unsigned long long rk[E];
  uint32_t ri[E];
  int c = 0;
#pragma unroll
  for (int e = 0; e < E; ++e) {
    const int i = tid * E + e;
    rk[e] = i < m ? sk[i] : ~0ull;
    ri[e] = i < m ? si[i] : 0u;
    const bool first = i < m && (i == 0 || sk[i - 1] != rk[e]);
    if (!first) rk[e] = ~0ull;
    c += first;
  }
  __syncthreads();
  int pos = block_scan(c, s_w, &s_tot);
  const int u = s_tot;
  int* ux = reinterpret_cast<int*>(sm);  // aliases sk (all reads done)
  int* uy = ux + SMALL_MAX;
  uint32_t* uid = reinterpret_cast<uint32_t*>(uy + SMALL_MAX);  // aliases si
#pragma unroll
  for (int e = 0; e < E; ++e) {
    if (rk[e] != ~0ull) {
      ux[pos] = key_x(rk[e]);
      uy[pos] = key_y(rk[e]);
      uid[pos] = ri[e];
      ++pos;
    }
  }
  __syncthreads();
  if (u == 1) {
    if (tid == 0) { out[0] = uid[0]; *out_n = 1; sw->active = 0; }
    return;
  }
  const Pts P{ux, uy};
  // chunk chains: warp w, lane 0 lower / lane 1 upper
  const int C = (u + NCH - 1) / NCH;
  {
    const int w = tid >> 5, lane = tid & 31;
    const int lo = min(w * C, u), hi = min(lo + C, u);
    if (lane < 2) s_cnt[lane][w] = chunk_chain(P, lo, hi, chain + lane * SMALL_MAX + w * C, lane == 0 ? 1 : -1);
  }
  __syncthreads();
  // publish to global
  for (int i = tid; i < u; i += SB) {
    sw->pts[i] = make_int2(ux[i], uy[i]);
    sw->uid[i] = uid[i];
  }
  for (int w = 0; w < NCH; ++w) {
    for (int k = tid; k < s_cnt[0][w]; k += SB) sw->chain[0][w * C + k] = chain[w * C + k];
    for (int k = tid; k < s_cnt[1][w]; k += SB) sw->chain[1][w * C + k] = chain[SMALL_MAX + w * C + k];
  }
  if (tid < 2) {
    int run = 0;
    for (int w = 0; w < NCH; ++w) {
      sw->cnt[tid][w] = s_cnt[tid][w];
      sw->base[tid][w] = run;
      run += s_cnt[tid][w];
    }
    sw->base[tid][NCH] = run;
  }
  if (tid == 0) { sw->u = u; sw->C = C; sw->active = 1; }
}

// tiny: the whole hull of a set with at most TINY_MAX survivors in one
// block.  A bitonic sort of (key, index) (partners closer than 32 by warp
// shuffles, farther ones through shared memory), then Andrew's chains in two
// levels: the lower and upper chain of each of TCH chunks of the sorted
// points in parallel (one lane each), then one walk over the chunk chains'
// vertices in order.  A point off its chunk's chain is no vertex of the
// set's chain, so the second walk sees the same vertices as a walk over all
// points, in far fewer steps.  Equal keys are adjacent with the lowest index
// first; both walks skip a point equal to the top of their stack.
constexpr int TB = 256;
constexpr int TCH = 32;                 // chunks of the first level
constexpr int TE = TINY_MAX / TB;       // sort elements per thread

// Chain walk over the positions pos(0 .. len) of the sorted points (sign sg:
// +1 lower, -1 upper) into q; returns its length.  Pops while the turn is
// not strictly left (lower) / right (upper); the top two entries stay in
// registers.
template <class Pos>
__device__ __forceinline__ int chain_walk(const int2* sp, int len, Pos pos, uint16_t* q, long long sg) {
  int n = 0;
  int x1 = 0, y1 = 0, x2 = 0, y2 = 0;
  for (int t = 0; t < len; ++t) {
    const int p = pos(t);
    const int2 cur = sp[p];
    if (n > 0 && cur.x == x1 && cur.y == y1) continue;  // equal points: the first (lowest index) stands
    while (n >= 2) {
      if (sg * cr(x1 - x2, y1 - y2, cur.x - x2, cur.y - y2) > 0) break;
      --n;
      x1 = x2; y1 = y2;
      if (n >= 2) { const int2 u = sp[q[n - 2]]; x2 = u.x; y2 = u.y; }
    }
    q[n++] = (uint16_t)p;
    x2 = x1; y2 = y1;
    x1 = cur.x; y1 = cur.y;
  }
  return n;
}

__global__ void __launch_bounds__(TB) k_small_tiny(Sets S, const uint32_t* gstatus, int which,
                                                    const unsigned long long* __restrict__ kin_base,
                                                    const uint32_t* __restrict__ vin_base,
                                                    uint32_t* __restrict__ out_base, int64_t* out_n_base) {
  __shared__ unsigned long long sk[TINY_MAX];
  __shared__ uint32_t si[TINY_MAX];
  __shared__ uint16_t sc[2][TINY_MAX];  // chunk chains, chunk c's from c * C
  __shared__ uint16_t sq[2][TINY_MAX];  // the set's chains
  __shared__ int s_cc[2][TCH];
  __shared__ int s_n[2];
  const int tid = threadIdx.x;
  const int set = blockIdx.x;
  const WsHeader* h = S.h(set);
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(gstatus) != 0;
  const int64_t m64 = dead ? 0 : count_of(h, which == 0 ? &h->n_surv : &h->n_surv2);
  if (m64 == 0) {  // nothing survives (or the call is dead): an empty hull
    if (tid == 0) out_n_base[set] = 0;
    return;
  }
  if (m64 > TINY_MAX) return;
  const int m = (int)m64;
  const int64_t o = S.off_at(set);
  int P2 = 2;
  while (P2 < m) P2 <<= 1;
  {
    // element i = r * TB + tid in registers; padding sorts last
    const int NE = (P2 + TB - 1) / TB;
    unsigned long long qk[TE];
    uint32_t qv[TE];
#pragma unroll
    for (int r = 0; r < TE; ++r) {
      const int i = r * TB + tid;
      qk[r] = (r < NE && i < m) ? kin_base[o + i] : ~0ull;
      qv[r] = (r < NE && i < m) ? vin_base[o + i] : ~0u;
    }
    for (int k = 2; k <= P2; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        if (j >= TB) {  // partner in the same thread: element r ^ (j / TB)
          auto in_thread = [&](auto JR) {
            constexpr int jr = decltype(JR)::value;
#pragma unroll
            for (int r = 0; r < TE; ++r) {
              const int l = r ^ jr;
              if (l > r && l < TE && r < NE) {
                const bool asc = ((r * TB + tid) & k) == 0;
                const bool gt = qk[r] > qk[l] || (qk[r] == qk[l] && qv[r] > qv[l]);
                if (gt == asc) {
                  const unsigned long long tk = qk[r]; qk[r] = qk[l]; qk[l] = tk;
                  const uint32_t tv = qv[r]; qv[r] = qv[l]; qv[l] = tv;
                }
              }
            }
          };
          static_assert(TE <= 4, "in-thread partners at distances TB and 2 TB");
          if (j == TB) in_thread(std::integral_constant<int, 1>{});
          else in_thread(std::integral_constant<int, 2>{});
          continue;
        }
        if (j >= 32) {
#pragma unroll
          for (int r = 0; r < TE; ++r)
            if (r < NE) { sk[r * TB + tid] = qk[r]; si[r * TB + tid] = qv[r]; }
          __syncthreads();
        }
#pragma unroll
        for (int r = 0; r < TE; ++r) {
          if (r < NE) {
            const int i = r * TB + tid;
            unsigned long long pk;
            uint32_t pv;
            if (j >= 32) {
              pk = (i ^ j) < P2 ? sk[i ^ j] : ~0ull;
              pv = (i ^ j) < P2 ? si[i ^ j] : ~0u;
            } else {
              pk = __shfl_xor_sync(FULL, qk[r], j);
              pv = __shfl_xor_sync(FULL, qv[r], j);
            }
            const bool asc = (i & k) == 0;
            const bool lower = (i & j) == 0;
            const bool pgt = pk > qk[r] || (pk == qk[r] && pv > qv[r]);
            const bool take = lower == asc ? !pgt : pgt;
            if (take && i < P2) { qk[r] = pk; qv[r] = pv; }
          }
        }
        if (j >= 32) __syncthreads();
      }
    }
    // sorted keys decoded to coordinates in place of the keys
    int2* sp = reinterpret_cast<int2*>(sk);
#pragma unroll
    for (int r = 0; r < TE; ++r) {
      const int i = r * TB + tid;
      if (r < NE && i < m) { sp[i] = make_int2(key_x(qk[r]), key_y(qk[r])); si[i] = qv[r]; }
    }
    __syncthreads();
  }
  const int2* sp = reinterpret_cast<const int2*>(sk);
  // first level: warp 0 the lower chains, warp 1 the upper chains, lane c chunk c
  const int C = (m + TCH - 1) / TCH;
  if (tid < 64) {
    const int c = tid & 31, s = tid >> 5;
    const int lo = min(c * C, m), len = min(C, m - lo);
    s_cc[s][c] = len > 0 ? chain_walk(sp, len, [&](int t) { return lo + t; }, sc[s] + c * C, s == 0 ? 1 : -1) : 0;
  }
  __syncthreads();
  // second level: thread 0 the lower chain, thread 32 the upper chain, over
  // the chunk chains in order
  if (tid == 0 || tid == 32) {
    const int s = tid >> 5;
    int total = 0;
    for (int c = 0; c < TCH; ++c) total += s_cc[s][c];
    int c = 0, k = 0;  // the walk's cursor: chunk c, entry k
    s_n[s] = chain_walk(sp, total, [&](int) {
      while (k == s_cc[s][c]) { ++c; k = 0; }
      return (int)sc[s][c * C + k++];
    }, sq[s], s == 0 ? 1 : -1);
  }
  __syncthreads();
  uint32_t* out = out_base + o;
  const int a = s_n[0], b = s_n[1];
  if (a == 1) {  // every survivor has the same coordinates
    if (tid == 0) { out[0] = si[sq[0][0]]; out_n_base[set] = 1; }
    return;
  }
  for (int k = tid; k < a - 1; k += TB) out[k] = si[sq[0][k]];
  for (int k = 1 + tid; k <= b - 1; k += TB) out[(a - 1) + (b - 1 - k)] = si[sq[1][k]];
  if (tid == 0) out_n_base[set] = (int64_t)(a - 1) + (b - 1);
}

// Unique points read through the read-only path.
struct GPts {
  const int2* p;
  __device__ __forceinline__ int2 at(int i) const { return __ldg(p + i); }
};

// Over chain ch[0..k) of points all before v: the most counter-clockwise
// incoming direction v - a (sign S); returns the point.
template <int S>
__device__ int g_best_in(GPts P, const uint16_t* ch, int k, long long vx, long long vy) {
  int lo = 0, hi = k - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int2 a = P.at(__ldg(ch + mid)), b = P.at(__ldg(ch + mid + 1));
    const long long c = S * cr(vx - a.x, vy - a.y, vx - b.x, vy - b.y);
    if (c > 0) lo = mid + 1; else hi = mid;
  }
  return __ldg(ch + lo);
}

// Over chain ch[0..k) of points all after v: the most clockwise outgoing
// direction b - v (sign S); returns the point.
template <int S>
__device__ int g_best_out(GPts P, const uint16_t* ch, int k, long long vx, long long vy) {
  int lo = 0, hi = k - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int2 a = P.at(__ldg(ch + mid)), b = P.at(__ldg(ch + mid + 1));
    const long long c = S * cr(a.x - vx, a.y - vy, b.x - vx, b.y - vy);
    if (c < 0) lo = mid + 1; else hi = mid;
  }
  return __ldg(ch + lo);
}

template <int S>
__device__ __forceinline__ void prune_one(const SmallWs* sw, int s, int j) {
  const int lane = threadIdx.x & 31;
  const int u = sw->u, C = sw->C;
  const int* cnt = sw->cnt[s];
  const int* base = sw->base[s];
  int w = 0;
  while (w + 1 < NCH && base[w + 1] <= j) ++w;
  const int k = j - base[w];
  const uint16_t* ch = sw->chain[s];
  const GPts P{sw->pts};
  const int v = ch[w * C + k];
  if (v == 0 || v == u - 1) {
    if (lane == 0) const_cast<SmallWs*>(sw)->keep[s][j] = 1;
    return;
  }
  const int2 pv = P.at(v);
  const long long vx = pv.x, vy = pv.y;
  // lane c: chunk c's most counter-clockwise incoming / most clockwise outgoing direction
  long long ix = 0, iy = 0, ox = 0, oy = 0;
  bool hin = false, hout = false;
  const int c = lane;
  if (c < w && cnt[c] > 0) {
    const int2 a = P.at(g_best_in<S>(P, ch + c * C, cnt[c], vx, vy));
    ix = vx - a.x; iy = vy - a.y; hin = true;
  } else if (c == w) {
    if (k > 0) { const int2 a = P.at(ch[w * C + k - 1]); ix = vx - a.x; iy = vy - a.y; hin = true; }
    if (k + 1 < cnt[w]) { const int2 b = P.at(ch[w * C + k + 1]); ox = b.x - vx; oy = b.y - vy; hout = true; }
  } else if (c > w && cnt[c] > 0) {
    const int2 b = P.at(g_best_out<S>(P, ch + c * C, cnt[c], vx, vy));
    ox = b.x - vx; oy = b.y - vy; hout = true;
  }
  for (int off = 16; off; off >>= 1) {
    const long long jx = __shfl_xor_sync(FULL, ix, off), jy = __shfl_xor_sync(FULL, iy, off);
    const bool jh = __shfl_xor_sync(FULL, hin, off);
    if (jh && (!hin || S * cr(ix, iy, jx, jy) > 0)) { ix = jx; iy = jy; hin = true; }
    const long long px = __shfl_xor_sync(FULL, ox, off), py = __shfl_xor_sync(FULL, oy, off);
    const bool ph = __shfl_xor_sync(FULL, hout, off);
    if (ph && (!hout || S * cr(ox, oy, px, py) < 0)) { ox = px; oy = py; hout = true; }
  }
  if (lane == 0) const_cast<SmallWs*>(sw)->keep[s][j] = (hin && hout && S * cr(ix, iy, ox, oy) > 0) ? 1 : 0;
}

// prune: one warp per chunk-chain vertex (lower ones first, then upper).
__global__ void __launch_bounds__(256) k_small_prune(const SmallWs* sw_base) {
  const SmallWs* sw = sw_base + blockIdx.x;  // one set per grid column
  if (!*reinterpret_cast<const volatile int*>(&sw->active)) return;
  const int nl = sw->base[0][NCH], total = nl + sw->base[1][NCH];
  const int warps = (gridDim.y * blockDim.x) >> 5;
  for (int g = (blockIdx.y * blockDim.x + threadIdx.x) >> 5; g < total; g += warps) {
    if (g < nl) prune_one<1>(sw, 0, g);
    else prune_one<-1>(sw, 1, g - nl);
  }
}

// emit: the lower hull left to right without its last point, then the upper
// hull right to left without its first and last points.
__global__ void __launch_bounds__(SB, 1) k_small_emit(Sets S, const SmallWs* sw_base, uint32_t* __restrict__ out_base,
                                                       int64_t* out_n_base) {
  __shared__ int s_w[32];
  __shared__ int s_tot;
  __shared__ int s_lower;
  const int tid = threadIdx.x;
  const int set = blockIdx.x;
  const SmallWs* sw = sw_base + set;
  uint32_t* out = out_base + S.off_at(set);
  int64_t* out_n = out_n_base + set;
  if (!*reinterpret_cast<const volatile int*>(&sw->active)) return;
  const int C = sw->C;
  for (int s = 0; s < 2; ++s) {
    const int total = sw->base[s][NCH];
    const int per = (total + SB - 1) / SB;
    const int j0 = min(tid * per, total), j1 = min(j0 + per, total);
    int cnt = 0;
    for (int j = j0; j < j1; ++j) cnt += sw->keep[s][j];
    int o = block_scan(cnt, s_w, &s_tot);
    const int a = s_tot;  // vertices of this chain, both end points included
    const int la = s == 0 ? a : s_lower;
    int w = 0;
    for (int j = j0; j < j1; ++j) {
      if (!sw->keep[s][j]) continue;
      while (w + 1 < NCH && sw->base[s][w + 1] <= j) ++w;
      const int v = sw->chain[s][w * C + (j - sw->base[s][w])];
      if (s == 0) {
        if (o < a - 1) out[o] = sw->uid[v];
      } else if (o >= 1) {
        // upper vertex o (1 .. a-1) -> after the la-1 lower vertices, reversed
        out[(la - 1) + (a - 1 - o)] = sw->uid[v];
      }
      ++o;
    }
    if (tid == 0) {
      if (s == 0) s_lower = a;
      else *out_n = (int64_t)la + (int64_t)a - 2;
    }
    __syncthreads();
  }
}

// Cross product of two directions given by 32-bit components (each product
// is one widening multiply).
__device__ __forceinline__ long long crs(int bx, int by, int dx, int dy) {
  return (long long)bx * dy - (long long)by * dx;
}

constexpr int CW = 8;  // warps per block of classify and rank

__global__ void __launch_bounds__(CW * 32) k_small_classify(Sets S, const uint32_t* gstatus, int which,
                                                             const unsigned long long* __restrict__ kin_base,
                                                             const uint32_t* __restrict__ vin_base,
                                                             SmallWs* sw_base) {
  const int set = blockIdx.x;
  WsHeader* h = S.h(set);
  if (*reinterpret_cast<const volatile uint32_t*>(gstatus)) return;
  const int64_t m64 = count_of(h, which == 0 ? &h->n_surv : &h->n_surv2);
  if (m64 == 0 || m64 > SMALL_MAX) return;
  const int m = (int)m64;
  const int64_t o = S.off_at(set);
  const unsigned long long* K = kin_base + o;
  const uint32_t* V = vin_base + o;
  SmallWs* sw = sw_base + set;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.y * CW;
  for (int v = blockIdx.y * CW + (threadIdx.x >> 5); v < m; v += warps) {
    const unsigned long long kv = __ldg(K + v);
    const uint32_t iv = __ldg(V + v);
    const int vx = key_x(kv), vy = key_y(kv);
    // per lane: best incoming (lower: most CCW, upper: most CW) and best
    // outgoing (lower: most CW, upper: most CCW) directions.  They start at
    // unreachable directions that every real one beats (real components are
    // within 2^25): (1, -2^26) is clockwise, (-1, 2^26) counter-clockwise of
    // every direction of the half-plane; no branch depends on the lane.
    constexpr int BIG = 1 << 26;
    int lix = 1, liy = -BIG, uix = -1, uiy = BIG;  // incoming
    int lox = -1, loy = BIG, uox = 1, uoy = -BIG;  // outgoing
    bool dup = false;
    for (int a = lane; a < m; a += 32) {
      const unsigned long long ka = __ldg(K + a);
      if (ka == kv) {  // equal coordinates (rare): the lowest index stands for them, and of
                       // copies of one point (same index) the first position
        const uint32_t ia = __ldg(V + a);
        dup |= ia < iv || (ia == iv && a < v);
        continue;
      }
      const bool before = ka < kv;
      const int ax = key_x(ka), ay = key_y(ka);
      // incoming v - a (a before v) or outgoing a - v (a after v)
      const int dx = before ? vx - ax : ax - vx, dy = before ? vy - ay : ay - vy;
      const int bl_x = before ? lix : lox, bl_y = before ? liy : loy;
      const int bu_x = before ? uix : uox, bu_y = before ? uiy : uoy;
      // lower: incoming keeps the most CCW, outgoing the most CW (upper: mirrored)
      const long long cl = crs(bl_x, bl_y, dx, dy), cu = crs(bu_x, bu_y, dx, dy);
      const bool tl = before ? cl > 0 : cl < 0, tu = before ? cu < 0 : cu > 0;
      if (before) {
        lix = tl ? dx : lix; liy = tl ? dy : liy;
        uix = tu ? dx : uix; uiy = tu ? dy : uiy;
      } else {
        lox = tl ? dx : lox; loy = tl ? dy : loy;
        uox = tu ? dx : uox; uoy = tu ? dy : uoy;
      }
    }
    for (int off = 16; off; off >>= 1) {
      int x1 = __shfl_xor_sync(FULL, lix, off), y1 = __shfl_xor_sync(FULL, liy, off);
      if (crs(lix, liy, x1, y1) > 0) { lix = x1; liy = y1; }
      x1 = __shfl_xor_sync(FULL, uix, off); y1 = __shfl_xor_sync(FULL, uiy, off);
      if (crs(uix, uiy, x1, y1) < 0) { uix = x1; uiy = y1; }
      x1 = __shfl_xor_sync(FULL, lox, off); y1 = __shfl_xor_sync(FULL, loy, off);
      if (crs(lox, loy, x1, y1) < 0) { lox = x1; loy = y1; }
      x1 = __shfl_xor_sync(FULL, uox, off); y1 = __shfl_xor_sync(FULL, uoy, off);
      if (crs(uox, uoy, x1, y1) > 0) { uox = x1; uoy = y1; }
      dup |= __shfl_xor_sync(FULL, dup, off);
    }
    // no point before (after) v: the incoming (outgoing) best is still its start
    const bool hin = !(lix == 1 && liy == -BIG), hout = !(lox == -1 && loy == BIG);
    if (lane == 0) {
      uint8_t f = 0;
      if (!dup) {
        const bool end = !hin || !hout;
        if (end || crs(lix, liy, lox, loy) > 0) f |= 1;
        if (end || crs(uix, uiy, uox, uoy) < 0) f |= 2;
      }
      sw->flag[v] = f;
      if (f & 1) atomicAdd(&h->n_lower, 1u);
      if (f & 2) atomicAdd(&h->n_upper, 1u);
    }
  }
}

__global__ void __launch_bounds__(CW * 32) k_small_rank(Sets S, const uint32_t* gstatus, int which,
                                                         const unsigned long long* __restrict__ kin_base,
                                                         const uint32_t* __restrict__ vin_base,
                                                         const SmallWs* sw_base, uint32_t* __restrict__ out_base,
                                                         int64_t* out_n_base) {
  const int set = blockIdx.x;
  const WsHeader* h = S.h(set);
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(gstatus) != 0;
  const int64_t m64 = dead ? 0 : count_of(h, which == 0 ? &h->n_surv : &h->n_surv2);
  if (m64 == 0) {  // nothing survives (or the call is dead): an empty hull
    if (blockIdx.y == 0 && threadIdx.x == 0) out_n_base[set] = 0;
    return;
  }
  if (m64 > SMALL_MAX) return;
  const int m = (int)m64;
  const int64_t o = S.off_at(set);
  const unsigned long long* K = kin_base + o;
  const uint32_t* V = vin_base + o;
  const uint8_t* F = sw_base[set].flag;
  uint32_t* out = out_base + o;
  const int la = (int)h->n_lower, lb = (int)h->n_upper;
  const int lane = threadIdx.x & 31;
  const int warps = gridDim.y * CW;
  if (blockIdx.y == 0 && threadIdx.x == 0) out_n_base[set] = la <= 1 ? 1 : (int64_t)(la - 1) + (lb - 1);
  for (int v = blockIdx.y * CW + (threadIdx.x >> 5); v < m; v += warps) {
    const uint8_t f = F[v];
    if (!f) continue;
    const unsigned long long kv = __ldg(K + v);
    int rl = 0, ru = 0;
    for (int a = lane; a < m; a += 32) {
      const uint8_t fa = F[a];
      const unsigned long long ka = __ldg(K + a);
      if (fa && ka < kv) { rl += fa & 1; ru += fa >> 1; }
    }
    for (int off = 16; off; off >>= 1) {
      rl += __shfl_xor_sync(FULL, rl, off);
      ru += __shfl_xor_sync(FULL, ru, off);
    }
    if (lane == 0) {
      const uint32_t iv = __ldg(V + v);
      if (la <= 1) {  // every survivor has the same coordinates
        out[0] = iv;
      } else {
        if ((f & 1) && rl < la - 1) out[rl] = iv;
        if ((f & 2) && ru >= 1) out[(la - 1) + (lb - 1 - ru)] = iv;
      }
    }
  }
}

}  // namespace

size_t small_hull_smem() {
  return SMALL_MAX * (sizeof(unsigned long long) + sizeof(uint32_t) + 2 * sizeof(uint16_t));
}

cudaError_t launch_small_hull(const Sets& S, const uint32_t* gstatus, int which, const unsigned long long* keys,
                              const uint32_t* vals, SmallWs* sw, uint32_t* out, int64_t* out_n, cudaStream_t st) {
  const unsigned nsets = (unsigned)S.S;
  if (S.S == 1) {  // the whole GPU on one set: a warp for every possible survivor
    const unsigned gy = (unsigned)(SMALL_MAX / CW);
    k_small_classify<<<dim3(1, gy), CW * 32, 0, st>>>(S, gstatus, which, keys, vals, sw);
    k_small_rank<<<dim3(1, gy), CW * 32, 0, st>>>(S, gstatus, which, keys, vals, sw, out, out_n);
    count_launches(2);
    return cudaGetLastError();
  }
  k_small_tiny<<<nsets, TB, 0, st>>>(S, gstatus, which, keys, vals, out, out_n);
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = small_hull_smem();
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_small_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  k_small_prep<<<nsets, SB, smem, st>>>(S, gstatus, which, keys, vals, sw, out, out_n);
  k_small_prune<<<dim3(nsets, 8), 256, 0, st>>>(sw);
  k_small_emit<<<nsets, SB, 0, st>>>(S, sw, out, out_n);
  count_launches(4);
  return cudaGetLastError();
}

}  // namespace cudapre
