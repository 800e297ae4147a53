// proj.cuh -- the projections of Step 1 (section 2), shared by the 2D
// extreme search and the 3D extension's (section 5): the binary64
// definition of each rotated coordinate, the float32 values the streaming
// searches track (order-preserving multiples of the rotated coordinates)
// with their error bands, and an order-preserving key of a double.
#pragma once

#include <cfloat>

#include "internal.cuh"

namespace cudapre {
namespace {

template <int ANG>
struct Dirs {
  static constexpr int NV = ANG == 0 ? 6 : 8;  // projected values per point
  static constexpr int ND = 2 * NV;            // directions = extreme slots computed
};

// (cos, sin) of rotation group g.  Cumulative: 0, 30, 75, 120 degrees;
// absolute: 0, 30, 45, 60 degrees (section 2 Step 1, Figure 1).
__device__ __forceinline__ void rot_cs(int ang, int g, double& c, double& s) {
  if (g == 0) { c = 1.0; s = 0.0; return; }
  if (g == 1) { c = K_S3; s = 0.5; return; }
  if (ang == 0) {
    if (g == 2) { c = K_C75; s = K_S75; } else { c = -0.5; s = K_S3; }
  } else {
    if (g == 2) { c = K_H; s = K_H; } else { c = 0.5; s = K_S3; }
  }
}

// Binary64 definition of value v (group v/2, axis v%2):
//   axis 0: RN(RN(x*c) - RN(y*s)),  axis 1: RN(RN(x*s) + RN(y*c)).
__device__ __forceinline__ double value64(int ang, int v, float xf, float yf) {
  double c, s;
  rot_cs(ang, v >> 1, c, s);
  double x = (double)xf, y = (double)yf;
  if ((v & 1) == 0) return __dsub_rn(__dmul_rn(x, c), __dmul_rn(y, s));
  return __dadd_rn(__dmul_rn(x, s), __dmul_rn(y, c));
}

// Score of direction d = 2v + k: value for k = 1 (max), -value for k = 0.
__device__ __forceinline__ double score64(int ang, int d, float x, float y) {
  double v = value64(ang, d >> 1, x, y);
  return (d & 1) ? v : -v;
}

// Order-preserving unsigned key of a (non-NaN) double: integer comparisons
// of keys order the doubles (FP64 compares are slow on this part).  -0.0 and
// +0.0 are equal doubles, so they must get one key: adding +0.0 in
// round-to-nearest turns -0.0 into +0.0 and leaves every other value as it
// is; without it a -0.0 score would lose a tie it wins by index.
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(__dadd_rn(v, 0.0));
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// Float32 values of one point: order-preserving multiples of the rotated
// coordinates (see BAND_LO / BAND_HI for the scales and error bounds).
template <int ANG>
__device__ __forceinline__ void values32(float x, float y, float* v) {
  v[0] = x;
  v[1] = y;
  v[2] = fmaf(x, F_2S3, -y);  // 2 x'(30) = 2 s3 x - y
  v[3] = fmaf(y, F_2S3, x);   // 2 y'(30) = x + 2 s3 y
  if (ANG == 0) {
    v[4] = fmaf(y, -F_T75, x);  // x'(75) / c75 = x - tan75 y
    v[5] = fmaf(x, F_T75, y);   // y'(75) / c75 = tan75 x + y
  } else {
    v[4] = x - y;               // x'(45) / h
    v[5] = x + y;               // y'(45) / h
    v[6] = fmaf(-y, F_2S3, x);  // 2 x'(60) = x - 2 s3 y
    v[7] = fmaf(x, F_2S3, y);   // 2 y'(60) = 2 s3 x + y
  }
}

// Band of value v (exact group 0: no band).
template <int ANG>
__device__ __forceinline__ float band_of(int v) {
  return v < 2 ? 0.0f : ((ANG == 0 && v >= 4) ? BAND_HI : BAND_LO);
}

// Value v alone, the same arithmetic as values32 (v is warp-uniform: no
// indexed local array).
template <int ANG>
__device__ __forceinline__ float value32(int v, float x, float y) {
  switch (v) {
    case 0: return x;
    case 1: return y;
    case 2: return fmaf(x, F_2S3, -y);
    case 3: return fmaf(y, F_2S3, x);
    case 4: return ANG == 0 ? fmaf(y, -F_T75, x) : x - y;
    case 5: return ANG == 0 ? fmaf(x, F_T75, y) : x + y;
    case 6: return fmaf(-y, F_2S3, x);
    default: return fmaf(x, F_2S3, y);
  }
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}


}  // namespace
}  // namespace cudapre
