// Double-float arithmetic: a value is a pair of FP32 numbers hi + lo
// (|lo| <= ulp(hi)/2, about 48 significant bits). Sums use Knuth's TwoSum,
// products Dekker's TwoProduct through a fused multiply-add; both are exact
// transformations, so the only errors are the final roundings of the lo
// parts (a few units of 2^-48 relative to the magnitudes involved). The code
// must be compiled without fast-math reassociation (the build does not use
// it).
#pragma once

namespace trm {

struct F2 {
  float h, l;
};

// s + e = a + b exactly (any magnitudes).
__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
// s + e = a + b exactly when |a| >= |b| or a == 0.
__device__ __forceinline__ F2 quick_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ F2 df_add(F2 a, F2 b) {
  F2 s = two_sum(a.h, b.h);
  s.l += a.l + b.l;
  return quick_two_sum(s.h, s.l);
}
__device__ __forceinline__ F2 df_mul(F2 a, F2 b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ F2 df_of(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double to_double(F2 a) {
  return (double)a.h + (double)a.l;
}

// Accumulator of products of pairs: a.b by a fused multiply-add TwoProduct
// of the high parts plus the cross terms, added by TwoSum into the high part
// and plainly into the low part; norm() renormalises (call it every few
// dozen products). About 2^-46 relative to the sum of |a||b|.
struct DfAcc {
  float h = 0.f, l = 0.f;
  __device__ __forceinline__ void fma(float ah, float al, float bh, float bl) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const F2 t = two_sum(h, p);
    h = t.h;
    l += t.l + e;
  }
  __device__ __forceinline__ void norm() {
    const F2 t = quick_two_sum(h, l);
    h = t.h;
    l = t.l;
  }
};

}  // namespace trm
