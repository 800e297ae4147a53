// k_refine.cu -- a second, finer discard round on the survivors before the
// final hull (the paper's idea of section 2 applied again: points strictly
// inside a polygon whose vertices are input points cannot be hull vertices).
//
// Around an integer point O strictly inside the Step-2 polygon the survivors
// are binned by a monotone pseudo-angle; each bin keeps its farthest point
// (the "winner").  Consecutive winners w, w' and O span triangles; a survivor
// strictly inside the triangle (O, w, w') of its bin is strictly inside the
// hull of the input (O is interior, w and w' are input points) and is
// dropped.  The triangle test is exact (int64 orientations); the binning may
// round any way it likes -- it only decides which triangle is tried.  On the
// uniform disk this leaves a few thousand of ~18 million survivors.
#include "internal.cuh"

namespace cudapre {

namespace {

constexpr int RBLOCK = 256;
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ int64_t count_of(const WsHeader* h, const unsigned long long* c) {
  if (*reinterpret_cast<const volatile uint32_t*>(&h->status)) return 0;
  return (int64_t)*reinterpret_cast<const volatile unsigned long long*>(c);
}

// Diamond angle of (qx, qy) in [0, 4), monotone in the polar angle.
__device__ __forceinline__ int bin_of(float qx, float qy) {
  const float ax = fabsf(qx), ay = fabsf(qy);
  const float t = __fdividef(ay, fmaxf(ax + ay, 1e-30f));  // in [0, 1]
  float a;
  if (qx >= 0.0f) a = qy >= 0.0f ? t : 4.0f - t;
  else a = qy >= 0.0f ? 2.0f - t : 2.0f + t;
  int b = (int)(a * (REFINE_BINS / 4.0f));
  return min(max(b, 0), REFINE_BINS - 1);
}

constexpr int RU = 8;            // survivors per thread per work tile
constexpr int RT = RU * RBLOCK;  // survivors per work tile

// Work tiles over the sets' survivor counts: tile t of set s covers its
// survivors [(t - tp[s]) RT, ...).  One set: tp == null and the tiles of set
// 0 follow from its count.
struct Tiles {
  const int64_t* tp;
  int S;
  __device__ int64_t total(const Sets& SS, const uint32_t* gstatus) const {
    if (*reinterpret_cast<const volatile uint32_t*>(gstatus)) return 0;
    if (tp) return tp[S];
    const WsHeader* h = SS.h(0);
    return (count_of(h, &h->n_surv) + RT - 1) / RT;
  }
  __device__ int set_of(int64_t t) const {
    if (!tp) return 0;
    int lo = 0, hi = S - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tp[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
  }
  __device__ int64_t first(int s) const { return tp ? tp[s] : 0; }
};

// Pass 1: per bin, the survivor farthest from O (packed squared distance and
// survivor position; ties go to the larger position, any choice is valid).
// A block accumulates in shared memory while its tiles stay in one set.
__global__ void __launch_bounds__(RBLOCK) k_refine_bins(Sets S, Tiles T, const uint32_t* gstatus,
                                                         const unsigned long long* __restrict__ keys_base) {
  __shared__ unsigned long long s_bin[REFINE_BINS];
  const int64_t nt = T.total(S, gstatus);
  int cur = -1;
  WsHeader* h = nullptr;
  float ox = 0.0f, oy = 0.0f;
  bool on = false;
  int64_t m = 0;
  const unsigned long long* keys = nullptr;
  auto flush = [&]() {
    __syncthreads();
    if (cur >= 0)
      for (int k = threadIdx.x; k < REFINE_BINS; k += RBLOCK)
        if (s_bin[k]) atomicMax(&h->rbin[k], s_bin[k]);
    __syncthreads();
  };
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const int s = T.set_of(t);
    if (s != cur) {
      flush();
      for (int k = threadIdx.x; k < REFINE_BINS; k += RBLOCK) s_bin[k] = 0;
      cur = s;
      h = S.h(s);
      ox = (float)h->poly.rox;
      oy = (float)h->poly.roy;
      on = h->poly.refine_on;
      m = count_of(h, &h->n_surv);
      keys = keys_base + S.off_at(s);
      __syncthreads();
    }
    if (!on) continue;
    const int64_t j0 = (t - T.first(s)) * RT + threadIdx.x;
    unsigned long long kv[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) kv[u] = j0 + u * RBLOCK < m ? keys[j0 + u * RBLOCK] : 0ull;
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int64_t j = j0 + u * RBLOCK;
      if (j < m) {
        const float qx = (float)key_x(kv[u]) - ox, qy = (float)key_y(kv[u]) - oy;
        const float r2 = fmaf(qx, qx, qy * qy);
        const unsigned long long packed = ((unsigned long long)__float_as_uint(r2) << 32) | (uint32_t)j;
        atomicMax(&s_bin[bin_of(qx, qy)], packed);
      }
    }
  }
  flush();
}

// For every bin: its winner W (if any) and the nearest winners L before and R
// after it (cyclically), as coordinates.  One block per set.
//
// Also a disk inside the winners' polygon (the winners in bin order).  When
// O is strictly left of every edge W -> R, each edge turns by less than 180
// degrees about O; the winners follow the bins' monotone pseudo-angle, so
// the turns add up to one full turn and the polygon is simple and
// star-shaped about O: the union of the triangles (O, W, R), inside the hull
// of the input.  Its centre C is the winners' mean truncated to integers; C
// is inside iff a ray from C crosses the polygon an odd number of times
// (exact tests), and then every point closer to C than each edge segment is
// strictly inside it.  h->refine_r2 gets the squared distance from C to the
// nearest segment in float32 (at most 2^-22 too large), shrunk by 2^-18 and
// rounded down, which also covers the float32 rounding of the per-point test
// (at most 2^-21); or -1 when a condition fails.  h->refine_cx/cy get C.
__global__ void __launch_bounds__(REFINE_BINS) k_refine_links(Sets S, const uint32_t* gstatus,
                                                               const unsigned long long* __restrict__ keys_base,
                                                               int4* __restrict__ tri_base) {
  __shared__ int s_x[REFINE_BINS], s_y[REFINE_BINS];
  __shared__ unsigned s_mask[REFINE_BINS / 32];
  const int set = blockIdx.x;
  WsHeader* h = S.h(set);
  const unsigned long long* keys = keys_base + S.off_at(set);
  int4* tri = tri_base + (size_t)set * 2 * REFINE_BINS;
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(gstatus) != 0;
  const int b = threadIdx.x;
  const unsigned long long w = dead ? 0ull : h->rbin[b];
  const bool has = w != 0;
  if (has) {
    const unsigned long long k = keys[(uint32_t)w];
    s_x[b] = key_x(k);
    s_y[b] = key_y(k);
  }
  // nearest bins with a winner before and after b (cyclically), from the
  // warps' ballots of "has a winner"
  constexpr int NWARP = REFINE_BINS / 32;
  const int lane = b & 31, wp = b >> 5;
  const unsigned bal = __ballot_sync(0xFFFFFFFFu, has);
  if (lane == 0) s_mask[wp] = bal;
  const int nw = __syncthreads_count(has);
  int l = -1, r = -1;
  if (nw > 0) {
    const unsigned below = bal & ((1u << lane) - 1u);
    if (below) {
      l = wp * 32 + 31 - __clz(below);
    } else {
      for (int d = 1; d <= NWARP; ++d) {
        const int w = (wp - d + NWARP) % NWARP;
        // last, the own warp's bins after b (reached after wrapping around)
        const unsigned mk = s_mask[w] & (d == NWARP ? (lane == 31 ? 0u : ~((2u << lane) - 1u)) : 0xFFFFFFFFu);
        if (mk) { l = w * 32 + 31 - __clz(mk); break; }
      }
    }
    const unsigned above = lane == 31 ? 0u : bal & ~((2u << lane) - 1u);
    if (above) {
      r = wp * 32 + __ffs(above) - 1;
    } else {
      for (int d = 1; d <= NWARP; ++d) {
        const int w = (wp + d) % NWARP;
        // last, the own warp's bins before b
        const unsigned mk = s_mask[w] & (d == NWARP ? ((1u << lane) - 1u) : 0xFFFFFFFFu);
        if (mk) { r = w * 32 + __ffs(mk) - 1; break; }
      }
    }
    // a lone winner is its own neighbour on both sides
    if (l < 0 && has) l = b;
    if (r < 0 && has) r = b;
  }
  int4 a = make_int4(0, 0, 0, 0), c = make_int4(0, 0, 0, 0);
  int flags = 0;
  const bool on = !dead && h->poly.refine_on;
  if (on && nw >= 2 && l >= 0 && r >= 0) {
    flags = 1 | (has ? 2 : 0);
    a = make_int4(s_x[l], s_y[l], has ? s_x[b] : 0, has ? s_y[b] : 0);
    c = make_int4(s_x[r], s_y[r], flags, 0);
  }
  tri[2 * b] = a;
  tri[2 * b + 1] = c;
  // the disk: the winners' mean, then every winner's edge to the next winner
  __shared__ long long s_sum[2][NWARP];
  __shared__ int s_c[2];
  __shared__ unsigned s_d2;  // float bits of the minimum (non-negative floats order as integers)
  __shared__ int s_bad;
  long long sx = has ? s_x[b] : 0, sy = has ? s_y[b] : 0;
  for (int off = 16; off; off >>= 1) {
    sx += __shfl_xor_sync(FULL, sx, off);
    sy += __shfl_xor_sync(FULL, sy, off);
  }
  if (lane == 0) { s_sum[0][wp] = sx; s_sum[1][wp] = sy; }
  __syncthreads();
  if (b == 0) {
    long long tx = 0, ty = 0;
    for (int w = 0; w < NWARP; ++w) { tx += s_sum[0][w]; ty += s_sum[1][w]; }
    s_c[0] = nw > 0 ? (int)(tx / nw) : 0;
    s_c[1] = nw > 0 ? (int)(ty / nw) : 0;
    s_d2 = 0x7F7FFFFFu;
    s_bad = (on && nw >= 3) ? 0 : 1;
  }
  __syncthreads();
  int cross = 0;
  if (has && on && nw >= 3) {
    const long long ox = h->poly.rox, oy = h->poly.roy, cx = s_c[0], cy = s_c[1];
    const long long wx = s_x[b], wy = s_y[b], rx = s_x[r], ry = s_y[r];
    const long long ex = rx - wx, ey = ry - wy, e2 = ex * ex + ey * ey;
    const long long oo = ex * (oy - wy) - ey * (ox - wx);  // orient(W, R, O)
    const long long oc = ex * (cy - wy) - ey * (cx - wx);  // orient(W, R, C)
    if (oo <= 0 || oc == 0 || e2 == 0) {
      atomicOr(&s_bad, 1);
    } else {
      // the ray from C towards +x crosses this edge (half-open in y)
      if ((wy > cy) != (ry > cy)) cross = (ry > wy) ? (oc > 0) : (oc < 0);
      // squared distance from C to the segment W R, in float32 (four
      // roundings to nearest at most: at most 2^-22 too large)
      const long long dot = (cx - wx) * ex + (cy - wy) * ey;
      float d2;
      if (dot <= 0) {
        d2 = __ll2float_rn((cx - wx) * (cx - wx) + (cy - wy) * (cy - wy));
      } else if (dot >= e2) {
        d2 = __ll2float_rn((cx - rx) * (cx - rx) + (cy - ry) * (cy - ry));
      } else {
        const float of = __ll2float_rn(oc);
        d2 = __fmul_rn(of, of) / __ll2float_rn(e2);
      }
      atomicMin(&s_d2, __float_as_uint(d2));
    }
  }
  // C is inside the (simple) polygon iff the ray crosses it an odd number of times
  const int ncross = __syncthreads_count(cross);
  if (b == 0 && !(ncross & 1)) s_bad = 1;
  __syncthreads();
  if (b == 0) {
    h->refine_r2 = (dead || s_bad) ? -1.0f : __fmul_rd(__uint_as_float(s_d2), 1.0f - 0x1p-18f);
    h->refine_cx = s_c[0];
    h->refine_cy = s_c[1];
  }
}

// Exact orientation of (a, b, p) for lattice points within +-2^24: every
// difference fits in 32 bits, every product is one widening multiply.
__device__ __forceinline__ long long orient_ll(int ax, int ay, int bx, int by, int px, int py) {
  return (long long)(bx - ax) * (py - ay) - (long long)(by - ay) * (px - ax);
}

// Pass 2: keep the survivors not strictly inside their bin's triangles;
// compacted to the set's (kout, vout) region, count in its n_surv2.  Few
// survive, so each warp appends its survivors with one atomic.
__global__ void __launch_bounds__(RBLOCK) k_refine_filter(Sets S, Tiles T, const uint32_t* gstatus,
                                                           const unsigned long long* __restrict__ kin_base,
                                                           const uint32_t* __restrict__ vin_base,
                                                           unsigned long long* __restrict__ kout_base,
                                                           uint32_t* __restrict__ vout_base,
                                                           const int4* __restrict__ tri_base) {
  __shared__ int4 s_tri[2 * REFINE_BINS];
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t nt = T.total(S, gstatus);
  int cur = -1;
  WsHeader* h = nullptr;
  int ox = 0, oy = 0;
  int cx = 0, cy = 0;
  float oxf = 0.0f, oyf = 0.0f, rr2 = -1.0f;
  int64_t m = 0;
  const unsigned long long* kin = nullptr;
  const uint32_t* vin = nullptr;
  unsigned long long* kout = nullptr;
  uint32_t* vout = nullptr;
  for (int64_t t = blockIdx.x; t < nt; t += gridDim.x) {
    const int s = T.set_of(t);
    if (s != cur) {
      __syncthreads();
      cur = s;
      const int4* tri = tri_base + (size_t)s * 2 * REFINE_BINS;
      for (int k = tid; k < 2 * REFINE_BINS; k += RBLOCK) s_tri[k] = tri[k];
      h = S.h(s);
      ox = h->poly.rox;
      oy = h->poly.roy;
      oxf = (float)ox;
      oyf = (float)oy;
      m = count_of(h, &h->n_surv);
      rr2 = *reinterpret_cast<const volatile float*>(&h->refine_r2);
      cx = *reinterpret_cast<const volatile int*>(&h->refine_cx);
      cy = *reinterpret_cast<const volatile int*>(&h->refine_cy);
      const int64_t o = S.off_at(s);
      kin = kin_base + o; vin = vin_base + o; kout = kout_base + o; vout = vout_base + o;
      __syncthreads();
    }
    const int64_t j0 = (t - T.first(s)) * RT;
    unsigned long long kv[RU];
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int64_t j = j0 + u * RBLOCK + tid;
      kv[u] = j < m ? kin[j] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < RU; ++u) {
      const int64_t j = j0 + u * RBLOCK + tid;
      bool keep = false;
      const unsigned long long key = kv[u];
      const int px = key_x(key), py = key_y(key);
      // inside the disk: strictly inside the winners' polygon
      const float fx = (float)(px - cx), fy = (float)(py - cy);
      if (j < m && !(fmaf(fx, fx, fy * fy) < rr2)) {
        // One triangle (O, A, B) per bin and side, chosen without branching:
        // with a winner W, (O, L, W) on the L side of the ray O->W and
        // (O, W, R) on the other; without one, (O, L, R).  p is dropped iff
        // it is strictly inside (all three orientations positive); a point
        // on the ray O->W has a zero orientation and stays.
        const int b = bin_of((float)px - oxf, (float)py - oyf);
        const int4 a = s_tri[2 * b], c = s_tri[2 * b + 1];
        const bool has_w = (c.z & 2) != 0;
        const bool l_side = has_w && orient_ll(ox, oy, a.z, a.w, px, py) < 0;
        const int ax_ = has_w && !l_side ? a.z : a.x, ay_ = has_w && !l_side ? a.w : a.y;
        const int bx_ = has_w && l_side ? a.z : c.x, by_ = has_w && l_side ? a.w : c.y;
        const bool inside = orient_ll(ox, oy, ax_, ay_, px, py) > 0 && orient_ll(ax_, ay_, bx_, by_, px, py) > 0 &&
                            orient_ll(bx_, by_, ox, oy, px, py) > 0;
        keep = !((c.z & 1) && inside);
      }
      const unsigned bal = __ballot_sync(FULL, keep);
      if (bal) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&h->n_surv2, (unsigned long long)__popc(bal));
        base = __shfl_sync(FULL, base, 0);
        if (keep) {
          const unsigned long long pos = base + __popc(bal & ((1u << lane) - 1u));
          kout[pos] = kv[u];
          vout[pos] = vin[j];
        }
      }
    }
  }
}

// Tile prefix over the sets' survivor counts (one block).
__global__ void __launch_bounds__(1024) k_tile_prefix(Sets S, const uint32_t* gstatus, int which, int rt,
                                                       int64_t* tp) {
  __shared__ int64_t s_w[32];
  __shared__ int64_t s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool dead = *reinterpret_cast<const volatile uint32_t*>(gstatus) != 0;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int s0 = 0; s0 < S.S; s0 += 1024) {
    const int s = s0 + threadIdx.x;
    int64_t v = 0;
    if (s < S.S && !dead) {
      const WsHeader* h = S.h(s);
      const int64_t m = count_of(h, which == 0 ? &h->n_surv : &h->n_surv2);
      v = (m + rt - 1) / rt;
    }
    int64_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
      const int64_t u = __shfl_up_sync(FULL, incl, off);
      if (lane >= off) incl += u;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    int64_t wpre = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
      const int64_t x = s_w[w];
      if (w < warp) wpre += x;
      tot += x;
    }
    const int64_t carry = s_carry;
    if (s < S.S) tp[s] = carry + wpre + incl - v;
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) tp[S.S] = s_carry;
}

}  // namespace

cudaError_t launch_refine(const Sets& S, const uint32_t* gstatus, int64_t* tp, const unsigned long long* keys_in,
                          const uint32_t* vals_in, unsigned long long* keys_out, uint32_t* vals_out, int4* tri,
                          int64_t cap, cudaStream_t st) {
  // one wave of resident blocks (the filter's triangle table limits it)
  const int sms = device_sm_count();
  static int occ_cache[64][2] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!occ_cache[dev][0]) {
    int a = 0, b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_refine_bins, RBLOCK, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_refine_filter, RBLOCK, 0);
    occ_cache[dev][0] = std::max(a, 1);
    occ_cache[dev][1] = std::max(b, 1);
  }
  const int64_t tiles = (cap + RT - 1) / RT;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * occ_cache[dev][0]));
  const unsigned gf = (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * occ_cache[dev][1]));
  Tiles T;
  T.S = S.S;
  T.tp = S.S > 1 ? tp : nullptr;
  int k = 3;
  if (T.tp) {
    k_tile_prefix<<<1, 1024, 0, st>>>(S, gstatus, 0, RT, tp);
    ++k;
  }
  k_refine_bins<<<g, RBLOCK, 0, st>>>(S, T, gstatus, keys_in);
  k_refine_links<<<(unsigned)S.S, REFINE_BINS, 0, st>>>(S, gstatus, keys_in, tri);
  k_refine_filter<<<gf, RBLOCK, 0, st>>>(S, T, gstatus, keys_in, vals_in, keys_out, vals_out, tri);
  count_launches(k);
  return cudaGetLastError();
}

}  // namespace cudapre
