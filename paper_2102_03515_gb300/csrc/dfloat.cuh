// Double-float arithmetic: a value held as an unevaluated sum hi + lo of two FP32 numbers,
// for FP64-grade sums and products on the FP32 pipe (GB300 issues FP32 at about 60 times
// its FP64 rate).  The error-free transformations are the published ones: Knuth's TwoSum
// (The Art of Computer Programming, vol. 2, Sec. 4.2.2), Dekker's FastTwoSum (1971) and the
// exact product error by one fused multiply-add (Dekker's TwoProduct with an FMA).
//
// Splitting an FP64 value x into (hi, lo) uses integer operations on its bit pattern
// only (no FP64 instruction): hi is x rounded to 24 significant bits, lo the remainder
// rounded to 24 bits, so hi + lo carries the top 48 bits of x (relative error <= 2^-49).
// The split is defined for x = 0 and 2^-74 <= |x| < 2^101, where hi and lo are normal
// FP32 numbers; callers fall back to FP64 arithmetic outside that range.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fem {

// exponent bounds (biased FP64) of the split's range
constexpr int kDfMinExp = 949;    // 2^-74
constexpr int kDfMaxExp = 1123;   // 2^100 <= |x| < 2^101

// x = hi + lo + (|x| 2^-49 at most); xs = hi + lo exactly, as an FP64 value.  Returns
// false (outputs unset) outside the range.
__device__ __forceinline__ bool df_split(double x, float& hi, float& lo, double& xs) {
  const uint64_t u = (uint64_t)__double_as_longlong(x);
  const uint64_t sgn = u & 0x8000000000000000ull;
  const uint64_t a = u ^ sgn;
  if (a == 0) {
    hi = 0.0f;
    lo = 0.0f;
    xs = 0.0;
    return true;
  }
  const int e = (int)(a >> 52);
  if (e < kDfMinExp || e > kDfMaxExp) return false;
  // round the magnitude at bit 29 of the pattern (to 24 significant bits, ties away from
  // zero); a carry into the exponent field is the correct rounding of 1.11..1 x 2^k
  const uint64_t ar = (a + (1ull << 28)) & ~((1ull << 29) - 1ull);
  const uint32_t s32 = (uint32_t)(sgn >> 32);
  hi = __uint_as_float(s32 | ((uint32_t)((int)(ar >> 52) - 896) << 23) |
                       (uint32_t)((ar >> 29) & 0x7FFFFFull));
  // remainder in units of the last place of x: |R| <= 2^28, value R 2^(e - 1075)
  const int R = (int)((int64_t)a - (int64_t)ar);
  if (R == 0) {
    lo = 0.0f;
    xs = __longlong_as_double((long long)(sgn | ar));
    return true;
  }
  const float fr = __int2float_rn(R);            // R rounded to 24 bits (exact as an integer)
  const int Rr = __float2int_rz(fr);
  uint32_t fb = __float_as_uint(fr) + ((uint32_t)(e - 1075) << 23);   // times 2^(e - 1075)
  lo = __uint_as_float(fb ^ s32);
  xs = __longlong_as_double((long long)(sgn | (uint64_t)((int64_t)ar + Rr)));
  return true;
}

// FP32 value times 2^-s as an FP64 value (exact); subnormal inputs count as zero
__device__ __forceinline__ double df_to_double(float f, int s) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t ex = (b >> 23) & 0xFFu;
  if (ex == 0) return 0.0;
  const uint64_t bits = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(ex + 896 - s) << 52) |
                        ((uint64_t)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}

// s + h exactly as s' + err (Knuth's TwoSum); the running sum keeps s' and collects err and
// the low part l of the added value in c
__device__ __forceinline__ void df_acc(float& s, float& c, float h, float l) {
  const float t = s + h;
  const float bp = t - s;
  const float err = (s - (t - bp)) + (h - bp);
  s = t;
  c += err + l;
}

// (C1 + C2 + C3) (s + c) as p + pl: p = C1 s rounded, pl = its exact error (one FMA) plus the
// remaining terms
__device__ __forceinline__ void df_mul(float C1, float C2, float C3, float s, float c, float& p,
                                       float& pl) {
  p = C1 * s;
  float t = fmaf(C1, s, -p);
  t = fmaf(C3, s, t);
  t = fmaf(C2, s, t);
  pl = fmaf(C1, c, t);
}

}  // namespace fem
