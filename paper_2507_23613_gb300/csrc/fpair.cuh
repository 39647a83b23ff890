// Filter sums of the FP64 wave solve as unevaluated float pairs.
//
// The FP64 step kernels accumulate q_m += w_{n,m} W^n (eq. pDefQ) for N_f frequencies at every
// point and step.  On sm_103a the FP64 pipe runs at about 1/60 of the FP32 rate (1.2 against
// 70 TFLOP/s measured), and these N_f FMAs are most of a step's FP64 work.  So the sums are
// kept as pairs (hi, lo) of floats with q = hi + lo exactly, stored in the 8 bytes of a
// double, and updated on the FP32 pipe:
//   - the product w x of two pairs by the FMA-based exact product of the high parts
//     (Dekker's two-product) plus the two cross terms (the lo * lo term, below 2^-48 |w x|,
//     is dropped);
//   - the sum by Knuth's branch-free two-sum of the high parts, the low parts folded into its
//     error, and a final renormalisation (fast two-sum) so that |lo| <= ulp(hi) / 2.
// One update has a relative error of a few 2^-48 of |q| + |w x|, against 2^-53 for one FP64
// FMA; the wave levels W themselves stay FP64.  The pair holds magnitudes from about 1e-30
// (below that lo loses bits to float underflow) up to the float range (3.4e38).
#pragma once

#include <cuda_runtime.h>

namespace mfwh {

// Pair of a double: hi = round-to-nearest float of v, lo = the float nearest to v - hi.
__device__ __forceinline__ float2 fpair_from(double v) {
  const float hi = __double2float_rn(v);
  return make_float2(hi, __double2float_rn(v - (double)hi));
}

__device__ __forceinline__ double fpair_value(float2 q) { return (double)q.x + (double)q.y; }

// Exact float of an integer |i| < 2^22 on the integer and FP32 pipes: the bit pattern of
// 1.5 * 2^23 + i (the float's unit in the last place is 1 there) minus 1.5 * 2^23.
__device__ __forceinline__ float small_int_to_float(int i) {
  return __int_as_float(0x4B400000 + i) - 12582912.0f;
}

// The pair of a double formed with integer and FP32 operations only, so that the FP64 pipe
// (the step kernels' bottleneck on sm_103a, which also executes conversions between integers
// or doubles and floats) is not used: three FP64-pipe conversions and a subtraction become
// about twenty-five integer and FP32 instructions.
//   hi: v rounded to 24 significant bits (ties away from zero) on its bit pattern (adding half
//       a unit at bit 28 and clearing bits 0-28 rounds the magnitude; the sign bit is untouched
//       for finite v, so no absolute value is formed);
//   lo: the remainder v - hi, an integer d (|d| <= 2^28, sign relative to v) in units of
//       2^(e-1075), e the biased exponent of v (the bit patterns differ by exactly d, also when
//       rounding carries hi into the next binade), converted to float exactly up to one
//       rounding (d = 4096 d1 + d0, both parts exact, joined by one FMA) and scaled.
// hi + lo equals v to within 2^-48 |v|, as for fpair_from (which it matches except on exact
// ties), for |v| from about 2^-101 (below, lo is a subnormal float and the pair keeps 2^-150
// absolute) to 2^116.  |v| below 2^-126 gives (0, 0); |v| of 2^116 and more gives an infinite
// hi, and NaN a NaN hi (so that non-finite sums still show).  No branch and no FP64
// instruction, not even under a predicate.
__device__ __forceinline__ float2 fpair_split(double v) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const unsigned long long h = (bits + (1ull << 28)) & ~((1ull << 29) - 1ull);
  const int eh = (int)(h >> 52) & 0x7FF;
  const int ev = (int)(bits >> 52) & 0x7FF;
  const unsigned sgn = (unsigned)(bits >> 32) & 0x80000000u;
  // float bits of hi: the exponent rebiased 1023 -> 127 (mod 2^32: bits above 31 drop out)
  const unsigned hb = ((unsigned)(h >> 29) - (896u << 23)) | sgn;
  const int d = (int)((unsigned)bits - (unsigned)h);            // |d| <= 2^28
  const float fd = fmaf(small_int_to_float(d >> 12), 4096.0f, small_int_to_float(d & 0xFFF));
  // lo = fd 2^k, k = ev - 1075, as fd 2^kk (kk = k, or k + 64 when 2^k is not a normal float)
  // times 2^(k - kk): both factors are normal floats for 885 <= ev <= 1138 and fd 2^kk stays
  // below 2^91; only a subnormal lo rounds.  fd carries d's sign, which is relative to v.
  const int k = ev - 1075;
  const bool low = k < -126;
  const int kk = low ? k + 64 : k;
  const float mag = (fd * __uint_as_float((unsigned)(kk + 127) << 23)) * (low ? 0x1p-64f : 1.0f);
  const float lo = __uint_as_float(__float_as_uint(mag) ^ sgn);
  // |v| >= 2^116, infinity or NaN: hi = +-inf, or a NaN for NaN
  const bool nan = ev == 2047 && (bits & 0x000FFFFFFFFFFFFFull) != 0;
  const unsigned big = sgn | 0x7F800000u | (nan ? 0x00400000u : 0u);
  const float hi = __uint_as_float(eh > 1138 ? big : hb);
  const bool zero = eh < 897 || eh > 1138;
  return make_float2(eh < 897 ? 0.0f : hi, zero ? 0.0f : lo);
}

// q + (wh + wl)(xh + xl) as a renormalised pair.
__device__ __forceinline__ float2 fpair_fma(float wh, float wl, float xh, float xl, float2 q) {
  const float ph = wh * xh;
  float pe = fmaf(wh, xh, -ph);        // exact error of the high product
  pe = fmaf(wh, xl, pe);
  pe = fmaf(wl, xh, pe);
  const float s = q.x + ph;            // two-sum of the high parts
  const float bv = s - q.x;
  float e = (q.x - (s - bv)) + (ph - bv);
  e += q.y + pe;
  const float hi = s + e;              // renormalise
  return make_float2(hi, e - (hi - s));
}

}  // namespace mfwh
