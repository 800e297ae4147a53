// k_hull_small.cu -- Andrew's monotone chain for a small survivor set (up to
// SMALL_MAX points) in one thread block: the final step of the method, the
// hull of the points that remain (section 3, case (2)).
//
// 1. Load the survivors into shared memory and bitonic-sort them by
//    (x, y, index); keep the first of each run of equal coordinates, which
//    has the lowest index.
// 2. Split the sorted points into 32 chunks; one lane per chunk runs the
//    lower and one the upper monotone chain of its chunk.
// 3. A chunk-chain vertex v is a vertex of the whole lower hull iff every
//    earlier point a and later point b make a strict left turn a -> v -> b.
//    Equivalently, the most counter-clockwise incoming direction v - a turns
//    strictly left into the most clockwise outgoing direction b - v.  Over
//    one chunk's convex chain these extremes are unimodal, so each is a
//    binary search; all candidates are tested in parallel.  The upper hull is
//    the same test with the orientation sign flipped.
// 4. Write the lower hull left to right, then the upper hull right to left.
#include "internal.cuh"

namespace cudapre {

namespace {

constexpr int SB = 1024;      // threads
constexpr int NCH = 32;       // chunks (one warp each)
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ long long cr(long long ax, long long ay, long long bx, long long by) {
  return ax * by - ay * bx;
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
template <int S>
__device__ int chunk_chain(Pts P, int lo, int hi, uint16_t* st) {
  int n = 0;
  for (int p = lo; p < hi; ++p) {
    const long long px = P.x[p], py = P.y[p];
    while (n >= 2) {
      const int a = st[n - 2], b = st[n - 1];
      const long long c = S * cr(P.x[b] - (long long)P.x[a], P.y[b] - (long long)P.y[a], px - P.x[a], py - P.y[a]);
      if (c > 0) break;
      --n;
    }
    st[n++] = (uint16_t)p;
  }
  return n;
}

// Over chain ch[0..k) of points all before v: the most counter-clockwise
// incoming direction v - a (sign S), as an index into ch.
template <int S>
__device__ int best_in(Pts P, const uint16_t* ch, int k, long long vx, long long vy) {
  int lo = 0, hi = k - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int a = ch[mid], b = ch[mid + 1];
    // is v - b counter-clockwise of v - a ?
    const long long c = S * cr(vx - P.x[a], vy - P.y[a], vx - P.x[b], vy - P.y[b]);
    if (c > 0) lo = mid + 1; else hi = mid;
  }
  return ch[lo];
}

// Over chain ch[0..k) of points all after v: the most clockwise outgoing
// direction b - v (sign S).
template <int S>
__device__ int best_out(Pts P, const uint16_t* ch, int k, long long vx, long long vy) {
  int lo = 0, hi = k - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    const int a = ch[mid], b = ch[mid + 1];
    // is b - v clockwise of a - v ?
    const long long c = S * cr(P.x[a] - vx, P.y[a] - vy, P.x[b] - vx, P.y[b] - vy);
    if (c < 0) lo = mid + 1; else hi = mid;
  }
  return ch[lo];
}

// Marks keep[j] for every candidate j (chunk-chain vertices, chunk-major).
template <int S>
__device__ void prune(Pts P, int u, int C, const uint16_t* ch, const int* cnt, const int* cbase, int total,
                      uint8_t* keep) {
  for (int j = threadIdx.x; j < total; j += SB) {
    int w = 0;
    while (w + 1 < NCH && cbase[w + 1] <= j) ++w;
    const int k = j - cbase[w];
    const uint16_t* own = ch + w * C;
    const int v = own[k];
    if (v == 0 || v == u - 1) { keep[j] = 1; continue; }
    const long long vx = P.x[v], vy = P.y[v];
    // most counter-clockwise incoming direction
    long long ix = 0, iy = 0;
    bool have_in = false;
    auto offer_in = [&](int a) {
      const long long dx = vx - P.x[a], dy = vy - P.y[a];
      if (!have_in || S * cr(ix, iy, dx, dy) > 0) { ix = dx; iy = dy; have_in = true; }
    };
    if (k > 0) offer_in(own[k - 1]);
    for (int c = 0; c < w; ++c)
      if (cnt[c] > 0) offer_in(best_in<S>(P, ch + c * C, cnt[c], vx, vy));
    long long ox = 0, oy = 0;
    bool have_out = false;
    auto offer_out = [&](int b) {
      const long long dx = P.x[b] - vx, dy = P.y[b] - vy;
      if (!have_out || S * cr(ox, oy, dx, dy) < 0) { ox = dx; oy = dy; have_out = true; }
    };
    if (k + 1 < cnt[w]) offer_out(own[k + 1]);
    for (int c = w + 1; c < NCH; ++c)
      if (cnt[c] > 0) offer_out(best_out<S>(P, ch + c * C, cnt[c], vx, vy));
    keep[j] = (have_in && have_out && S * cr(ix, iy, ox, oy) > 0) ? 1 : 0;
  }
}

__device__ __forceinline__ int64_t count_of(const WsHeader* h, const unsigned long long* c) {
  if (*reinterpret_cast<const volatile uint32_t*>(&h->status)) return 0;
  return (int64_t)*reinterpret_cast<const volatile unsigned long long*>(c);
}

__global__ void __launch_bounds__(SB, 1) k_small_hull(const unsigned long long* __restrict__ kin,
                                                       const uint32_t* __restrict__ vin,
                                                       const unsigned long long* count, const WsHeader* h,
                                                       uint32_t* __restrict__ out, int64_t* out_n) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_w[32];
  __shared__ int s_tot;
  __shared__ int s_cnt[2][NCH], s_base[2][NCH + 1];
  __shared__ int s_lower;
  const int tid = threadIdx.x;
  const int64_t m64 = count_of(h, count);
  if (m64 > SMALL_MAX) return;  // the large path handles it
  if (m64 == 0) {
    if (tid == 0) *out_n = 0;
    return;
  }
  const int m = (int)m64;
  int P2 = 2;
  while (P2 < m) P2 <<= 1;
  unsigned long long* sk = reinterpret_cast<unsigned long long*>(sm);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + SMALL_MAX);
  uint16_t* chain = reinterpret_cast<uint16_t*>(si + SMALL_MAX);  // [2][SMALL_MAX]
  uint8_t* keep = reinterpret_cast<uint8_t*>(chain + 2 * SMALL_MAX);  // [2][SMALL_MAX]
  for (int i = tid; i < P2; i += SB) {
    sk[i] = i < m ? kin[i] : ~0ull;
    si[i] = i < m ? vin[i] : ~0u;
  }
  __syncthreads();
  // 1. bitonic sort by (key, index)
  for (int k = 2; k <= P2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < P2; i += SB) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = sk[i], b = sk[l];
          const uint32_t ai = si[i], bi = si[l];
          const bool gt = a > b || (a == b && ai > bi);
          if (gt == ((i & k) == 0)) { sk[i] = b; sk[l] = a; si[i] = bi; si[l] = ai; }
        }
      }
      __syncthreads();
    }
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
  int* ux = reinterpret_cast<int*>(sm);             // aliases sk (all reads done)
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
    if (tid == 0) { out[0] = uid[0]; *out_n = 1; }
    return;
  }
  const Pts P{ux, uy};
  // 2. chunk chains: warp w, lane 0 lower / lane 1 upper
  const int C = (u + NCH - 1) / NCH;
  {
    const int w = tid >> 5, lane = tid & 31;
    const int lo = min(w * C, u), hi = min(lo + C, u);
    if (lane == 0) s_cnt[0][w] = chunk_chain<1>(P, lo, hi, chain + w * C);
    if (lane == 1) s_cnt[1][w] = chunk_chain<-1>(P, lo, hi, chain + SMALL_MAX + w * C);
  }
  __syncthreads();
  if (tid < 2) {
    int run = 0;
    for (int w = 0; w < NCH; ++w) { s_base[tid][w] = run; run += s_cnt[tid][w]; }
    s_base[tid][NCH] = run;
  }
  __syncthreads();
  // 3. global hull vertices among the chunk-chain vertices
  prune<1>(P, u, C, chain, s_cnt[0], s_base[0], s_base[0][NCH], keep);
  prune<-1>(P, u, C, chain + SMALL_MAX, s_cnt[1], s_base[1], s_base[1][NCH], keep + SMALL_MAX);
  __syncthreads();
  // 4. compact: the lower hull left to right without its last point, then
  //    the upper hull right to left without its first and last points
  for (int s = 0; s < 2; ++s) {
    const int total = s_base[s][NCH];
    const int per = (total + SB - 1) / SB;
    const int j0 = min(tid * per, total), j1 = min(j0 + per, total);
    int cnt = 0;
    for (int j = j0; j < j1; ++j) cnt += keep[s * SMALL_MAX + j];
    int o = block_scan(cnt, s_w, &s_tot);
    const int a = s_tot;  // vertices of this chain, both end points included
    const int la = s == 0 ? a : s_lower;
    for (int j = j0; j < j1; ++j) {
      if (!keep[s * SMALL_MAX + j]) continue;
      int w = 0;
      while (w + 1 < NCH && s_base[s][w + 1] <= j) ++w;
      const int v = chain[s * SMALL_MAX + w * C + (j - s_base[s][w])];
      if (s == 0) {
        if (o < a - 1) out[o] = uid[v];
      } else if (o >= 1) {
        // upper vertex o (1 .. a-1) -> after the la-1 lower vertices, reversed
        out[(la - 1) + (a - 1 - o)] = uid[v];
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

}  // namespace

size_t small_hull_smem() {
  return SMALL_MAX * (sizeof(unsigned long long) + sizeof(uint32_t) + 2 * sizeof(uint16_t) + 2);
}

cudaError_t launch_small_hull(const unsigned long long* keys, const uint32_t* vals,
                              const unsigned long long* count, const WsHeader* h, uint32_t* out,
                              int64_t* out_n, cudaStream_t st) {
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const size_t smem = small_hull_smem();
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(k_small_hull, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  k_small_hull<<<1, SB, smem, st>>>(keys, vals, count, h, out, out_n);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace cudapre
