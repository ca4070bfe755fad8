// Double-float arithmetic: a value carried as an unevaluated sum hi + lo of
// two FP32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits.  Built
// from the error-free transformations TwoSum (Knuth), FastTwoSum and
// TwoProduct (Dekker; here with an FMA), as in Dekker's 1971 double-length
// arithmetic and Bailey's double-double library, written for FP32 parts.
// Used by the FP32_HILO storage precision, whose spectra and intermediates
// are all FP32 pairs.
#pragma once

#include <cuda_runtime.h>

namespace s2w {

struct dfl {
  float hi, lo;
};

// s + e == a + b exactly (any a, b).
__device__ __forceinline__ dfl two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

// s + e == a + b exactly when |a| >= |b| or a == 0.
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}

// p + e == a * b exactly (barring underflow).
__device__ __forceinline__ dfl two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }

// x + y with both pairs' parts combined by error-free sums (relative error
// a small multiple of 2^-48 of |x| + |y|).
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = two_sum(x.hi, y.hi);
  const dfl t = two_sum(x.lo, y.lo);
  s.lo += t.hi;
  s = fast_two_sum(s.hi, s.lo);
  s.lo += t.lo;
  return fast_two_sum(s.hi, s.lo);
}

// x * y (the lo * lo term, ~2^-48 relative, is dropped).
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  dfl p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  return fast_two_sum(p.hi, p.lo);
}

// Compensated sum of many pair products: the high parts are added by TwoSum
// into s, every rounding error and low-order part into c (plain FP32: c
// stays ~2^-24 of the terms, so its own rounding is ~2^-48 of them).
struct dacc {
  float s, c;
};

__device__ __forceinline__ void acc_add(dacc& a, dfl v) {
  const dfl t = two_sum(a.s, v.hi);
  a.s = t.hi;
  a.c += t.lo + v.lo;
}

// a += x * y
__device__ __forceinline__ void acc_mac(dacc& a, dfl x, dfl y) {
  const dfl p = two_prod(x.hi, y.hi);
  const float cross = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, p.lo));
  const dfl t = two_sum(a.s, p.hi);
  a.s = t.hi;
  a.c += t.lo + cross;
}

// a += x * y for an FP32 x (exact input samples)
__device__ __forceinline__ void acc_mac_f(dacc& a, float x, dfl y) {
  const dfl p = two_prod(x, y.hi);
  const float cross = fmaf(x, y.lo, p.lo);
  const dfl t = two_sum(a.s, p.hi);
  a.s = t.hi;
  a.c += t.lo + cross;
}

// a + b of two partial accumulators
__device__ __forceinline__ dacc acc_merge(dacc a, dacc b) {
  const dfl t = two_sum(a.s, b.s);
  return {t.hi, a.c + b.c + t.lo};
}

__device__ __forceinline__ dfl acc_get(dacc a) { return two_sum(a.s, a.c); }

}  // namespace s2w
