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
