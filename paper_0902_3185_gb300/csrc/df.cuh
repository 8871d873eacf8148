// Double-float arithmetic on float32 pairs (hi + lo, about 48 significant
// bits) for the double-float product: float64 inputs split into pairs with
// integer instructions, Dekker's product with a fused multiply-add and
// Knuth's two-sum.  GB300 issues float64 at 1/64 of its float32 rate, so
// these run on the float32 pipes; the integer split (about 28 instructions)
// pays off only where a split value is reused, as in a product tile.
#pragma once

#include <cstdint>

#include "tc_kernel.cuh"

namespace dmrg {

// v = hi + lo with hi = RN24(v) and lo = RN24(v - hi).  For hi in the normal
// float range: v - hi = +-(rem - up 2^29) 2^(e - 1075) from the 29 mantissa
// bits below hi's (rem) and hi's rounding carry (up); lo is dropped when that
// scale is below the float range (|v| < 2^-74).  Other inputs: hi only.
__device__ __forceinline__ float2 df_split(double v) {
  const uint32_t h = (uint32_t)__double2hiint(v), l = (uint32_t)__double2loint(v);
  const uint32_t e = (h >> 20) & 0x7ffu;
  if (e - 897u < 254u) {
    const uint32_t sign = h & 0x80000000u;
    const uint32_t m = ((h & 0xfffffu) << 3) | (l >> 29);
    const uint32_t rem = l & 0x1fffffffu;
    const uint32_t up = ((uint32_t)(rem > 0x10000000u) | ((uint32_t)(rem == 0x10000000u) & m)) & 1u;
    const float hi = __uint_as_float(sign | (((e - 896u) << 23) + m + up));
    const int r = (int)rem - (int)(up << 29);
    const int se = (int)e - 948;  // biased float exponent of 2^(e - 1075)
    float lo = se >= 1 ? __fmul_rn(__int2float_rn(r), __int_as_float(se << 23)) : 0.0f;
    return make_float2(hi, sign ? -lo : lo);
  }
  return make_float2(tc::d2f_rn(v), 0.0f);
}

// a * b as an unevaluated pair (p, e): p = RN(a.hi b.hi), e = its exact error
// plus the cross terms
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  return make_float2(p, e);
}

// (s, c) += a * b: the product's leading part enters s through a two-sum
// whose exact error, with the product's error terms, goes to c
__device__ __forceinline__ void df_fma(float2 a, float2 b, float& s, float& c) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float t = __fadd_rn(s, p);
  const float bv = __fsub_rn(t, s);
  const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bv)), __fsub_rn(p, bv));
  c = __fadd_rn(c, __fadd_rn(err, e));
  s = t;
}

__device__ __forceinline__ double df_value(float s, float c) { return tc::f2d_exact(s) + tc::f2d_exact(c); }

// s + c as a pair (hi, lo) by Knuth's two-sum (no ordering of |s|, |c| assumed)
__device__ __forceinline__ float2 df_two_sum(float s, float c) {
  const float hi = __fadd_rn(s, c);
  const float bv = __fsub_rn(hi, s);
  return make_float2(hi, __fadd_rn(__fsub_rn(s, __fsub_rn(hi, bv)), __fsub_rn(c, bv)));
}

// a + b of two pairs: two-sum of the high parts, the low parts and its error
// added into the low part, then the two-sum again (renormalised)
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float2 h = df_two_sum(a.x, b.x);
  return df_two_sum(h.x, __fadd_rn(h.y, __fadd_rn(a.y, b.y)));
}

// (s, c) of df_fma as a renormalised pair
__device__ __forceinline__ float2 df_pair(float s, float c) { return df_two_sum(s, c); }

}  // namespace dmrg
