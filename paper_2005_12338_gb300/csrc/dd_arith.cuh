// Double-float (fp32 pair) arithmetic shared by the deterministic block's
// kernels.  An fp64 value x is carried as x = hi + lo with hi = fl32(x),
// lo = fl32(x - hi) (a 48-bit significand); a multiply-add is an error-free
// TwoProduct (one fma, plus the two cross terms of the low parts) and Knuth's
// TwoSum, the error terms gathered in a second float.
#pragma once

namespace rssri {

__device__ __forceinline__ void df_mac2(float &S, float &E, float2 d, float xh, float xl) {
  // TwoProduct of the high parts plus the cross terms, then TwoSum S + p
  const float p = __fmul_rn(d.x, xh);
  float e = __fmaf_rn(d.x, xh, -p);
  e = __fmaf_rn(d.x, xl, e);
  e = __fmaf_rn(d.y, xh, e);
  const float s = __fadd_rn(S, p);
  const float bp = __fsub_rn(s, S);
  const float err = __fadd_rn(__fsub_rn(S, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  S = s;
  E = __fadd_rn(E, __fadd_rn(err, e));
}

// The same with both operands as pairs.
__device__ __forceinline__ void df_mac(float &S, float &E, float2 a, float2 b) {
  df_mac2(S, E, a, b.x, b.y);
}

// (TH, TL) += (S, E): double-float addition of two normalised pairs (TwoSum of
// the high parts, low parts and error added, Fast2Sum).  All fp32: on this GPU
// a few fp64 operations per output would cost as much as the products.
__device__ __forceinline__ void df_acc(float &TH, float &TL, float S, float E) {
  const float s = __fadd_rn(TH, S);
  const float bp = __fsub_rn(s, TH);
  const float err = __fadd_rn(__fsub_rn(TH, __fsub_rn(s, bp)), __fsub_rn(S, bp));
  const float t = __fadd_rn(__fadd_rn(TL, E), err);
  TH = __fadd_rn(s, t);
  TL = __fsub_rn(t, __fsub_rn(TH, s));
}

}  // namespace rssri
