// FP32-pair ("double-float") arithmetic on the FP32 units: a value is the
// unevaluated sum hi + lo of two FP32 numbers (about 48 significant bits).
// Products of the high parts are exact by FMA; sums use TwoSum.  GB300's FP64
// units (1.25 TFLOP/s) are too slow for the O(rows x columns) passes of the
// pivoted QRs; these helpers carry those passes at FP32 speed.
#pragma once

#include <cuda_runtime.h>

namespace idsk {

// a * (bh + bl) added to the FP32 pair (hi, lo): exact product error by FMA,
// TwoSum for the running sum, small terms gathered in lo (about 48 bits).
__device__ __forceinline__ void df_acc(float& hi, float& lo, float a, float bh, float bl) {
  const float p = a * bh;
  const float pe = fmaf(a, bh, -p);
  const float q = fmaf(a, bl, pe);
  const float t = hi + p;
  const float bp = t - hi;
  const float err = (hi - (t - bp)) + (p - bp);
  hi = t;
  lo += err + q;
}

// (hi, lo) += (bh, bl) for FP32 pairs: TwoSum of the high parts, low parts
// gathered in lo.
__device__ __forceinline__ void df_add(float& hi, float& lo, float bh, float bl) {
  const float t = hi + bh;
  const float bp = t - hi;
  const float err = (hi - (t - bp)) + (bh - bp);
  hi = t;
  lo += err + bl;
}

// FP32-pair numbers (value h + l, |l| <= ulp(h) / 2 after normalisation):
// about 48 significant bits on the FP32 units.
__device__ __forceinline__ float2 df_of(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
__device__ __forceinline__ double df_val(float2 a) { return (double)a.x + (double)a.y; }
__device__ __forceinline__ float2 df_norm(float h, float l) {   // |h| >= |l|
  const float s = h + l;
  return make_float2(s, l - (s - h));
}
// a * b: exact product of the high parts (FMA), cross terms in FP32
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  return df_norm(p, e);
}

}  // namespace idsk
