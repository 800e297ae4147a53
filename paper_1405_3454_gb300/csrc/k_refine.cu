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

// Pass 1: per bin, the survivor farthest from O (packed squared distance and
// survivor position; ties go to the larger position, any choice is valid).
__global__ void __launch_bounds__(RBLOCK) k_refine_bins(const unsigned long long* __restrict__ keys,
                                                         WsHeader* h) {
  __shared__ unsigned long long s_bin[REFINE_BINS];
  for (int k = threadIdx.x; k < REFINE_BINS; k += RBLOCK) s_bin[k] = 0;
  __syncthreads();
  const int64_t m = count_of(h, &h->n_surv);
  const float ox = (float)h->poly.rox, oy = (float)h->poly.roy;
  if (h->poly.refine_on) {
    // 4 independent loads in flight per thread
    const int64_t stride = (int64_t)gridDim.x * RBLOCK;
    for (int64_t j0 = (int64_t)blockIdx.x * RBLOCK + threadIdx.x; j0 < m; j0 += 4 * stride) {
      unsigned long long kv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) kv[u] = j0 + u * stride < m ? keys[j0 + u * stride] : 0ull;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t j = j0 + u * stride;
        if (j < m) {
          const float qx = (float)key_x(kv[u]) - ox, qy = (float)key_y(kv[u]) - oy;
          const float r2 = fmaf(qx, qx, qy * qy);
          const unsigned long long packed = ((unsigned long long)__float_as_uint(r2) << 32) | (uint32_t)j;
          atomicMax(&s_bin[bin_of(qx, qy)], packed);
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < REFINE_BINS; k += RBLOCK)
    if (s_bin[k]) atomicMax(&h->rbin[k], s_bin[k]);
}

// For every bin: its winner W (if any) and the nearest winners L before and R
// after it (cyclically), as coordinates.
__global__ void __launch_bounds__(REFINE_BINS) k_refine_links(const unsigned long long* __restrict__ keys,
                                                               WsHeader* h, int4* __restrict__ tri) {
  __shared__ int s_x[REFINE_BINS], s_y[REFINE_BINS], s_has[REFINE_BINS];
  const int b = threadIdx.x;
  const unsigned long long w = h->rbin[b];
  const bool has = w != 0;
  s_has[b] = has;
  if (has) {
    const unsigned long long k = keys[(uint32_t)w];
    s_x[b] = key_x(k);
    s_y[b] = key_y(k);
  }
  __syncthreads();
  int l = -1, r = -1;
  for (int d = 1; d < REFINE_BINS; ++d) {
    if (l < 0 && s_has[(b - d + REFINE_BINS) % REFINE_BINS]) l = (b - d + REFINE_BINS) % REFINE_BINS;
    if (r < 0 && s_has[(b + d) % REFINE_BINS]) r = (b + d) % REFINE_BINS;
    if (l >= 0 && r >= 0) break;
  }
  const int nw = __syncthreads_count(has);
  int4 a = make_int4(0, 0, 0, 0), c = make_int4(0, 0, 0, 0);
  int flags = 0;
  if (h->poly.refine_on && nw >= 2 && l >= 0 && r >= 0) {
    flags = 1 | (has ? 2 : 0);
    a = make_int4(s_x[l], s_y[l], has ? s_x[b] : 0, has ? s_y[b] : 0);
    c = make_int4(s_x[r], s_y[r], flags, 0);
  }
  tri[2 * b] = a;
  tri[2 * b + 1] = c;
}

__device__ __forceinline__ long long orient_ll(long long ax, long long ay, long long bx, long long by,
                                               long long px, long long py) {
  return (bx - ax) * (py - ay) - (by - ay) * (px - ax);
}

// Pass 2: keep the survivors not strictly inside their bin's triangles;
// compacted to (kout, vout), count in h->n_surv2.  Few survive, so each warp
// appends its survivors with one atomic (no block barrier).
__global__ void __launch_bounds__(RBLOCK) k_refine_filter(const unsigned long long* __restrict__ kin,
                                                           const uint32_t* __restrict__ vin,
                                                           unsigned long long* __restrict__ kout,
                                                           uint32_t* __restrict__ vout, WsHeader* h,
                                                           const int4* __restrict__ tri) {
  __shared__ int4 s_tri[2 * REFINE_BINS];
  const int tid = threadIdx.x, lane = tid & 31;
  for (int k = tid; k < 2 * REFINE_BINS; k += RBLOCK) s_tri[k] = tri[k];
  __syncthreads();
  const int64_t m = count_of(h, &h->n_surv);
  const long long ox = h->poly.rox, oy = h->poly.roy;
  const float oxf = (float)ox, oyf = (float)oy;
  const int64_t stride = (int64_t)gridDim.x * RBLOCK;
  // 4 independent loads in flight per thread; a warp handles 4 x 32
  // consecutive survivors per round
  for (int64_t j0 = (int64_t)blockIdx.x * RBLOCK * 4; j0 < m; j0 += 4 * stride) {
    unsigned long long kv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = j0 + u * RBLOCK + tid;
      kv[u] = j < m ? kin[j] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int64_t j = j0 + u * RBLOCK + tid;
      bool keep = false;
      if (j < m) {
        const unsigned long long key = kv[u];
        const long long px = key_x(key), py = key_y(key);
        keep = true;
        const int b = bin_of((float)px - oxf, (float)py - oyf);
        const int4 a = s_tri[2 * b], c = s_tri[2 * b + 1];
        if (c.z & 1) {
          if (c.z & 2) {
            const long long ow = orient_ll(ox, oy, a.z, a.w, px, py);
            if (ow < 0) {  // the L side of ray O->W: triangle (O, L, W)
              keep = !(orient_ll(ox, oy, a.x, a.y, px, py) > 0 && orient_ll(a.x, a.y, a.z, a.w, px, py) > 0);
            } else if (ow > 0) {  // triangle (O, W, R)
              keep = !(orient_ll(a.z, a.w, c.x, c.y, px, py) > 0 && orient_ll(c.x, c.y, ox, oy, px, py) > 0);
            }
          } else {  // empty bin: triangle (O, L, R)
            keep = !(orient_ll(ox, oy, a.x, a.y, px, py) > 0 && orient_ll(a.x, a.y, c.x, c.y, px, py) > 0 &&
                     orient_ll(c.x, c.y, ox, oy, px, py) > 0);
          }
        }
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

}  // namespace

cudaError_t launch_refine(WsHeader* h, const unsigned long long* keys_in, const uint32_t* vals_in,
                          unsigned long long* keys_out, uint32_t* vals_out, int4* tri, int64_t cap,
                          cudaStream_t st) {
  const int sms = device_sm_count();
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cap + RBLOCK - 1) / RBLOCK, (int64_t)sms * 8));
  k_refine_bins<<<g, RBLOCK, 0, st>>>(keys_in, h);
  k_refine_links<<<1, REFINE_BINS, 0, st>>>(keys_in, h, tri);
  k_refine_filter<<<g, RBLOCK, 0, st>>>(keys_in, vals_in, keys_out, vals_out, h, tri);
  count_launches(3);
  return cudaGetLastError();
}

}  // namespace cudapre
