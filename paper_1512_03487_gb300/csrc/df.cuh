// Double-float arithmetic for the FP64-accurate hop on a GPU whose FP64 units
// are few (GB300: 2 FP64 FMA per SM per clock against 128 FP32).
//
// A real number is the unevaluated sum hi + lo of two FP32 numbers with
// |lo| <= ulp(hi), about 48 significant bits. The operations are built from
// the error-free transformations of Knuth (two_sum: a + b = s + e exactly) and
// of Dekker, with a fused multiply-add for the product's error (a b = p + e
// exactly with e = fma(a, b, -p)); the addition is the "sloppy" double-double
// addition of Hida, Li and Bailey (one two_sum on the high parts, the low parts
// added with one rounding), whose error is below 2^-46 of the larger operand.
// Every step uses the explicitly rounded intrinsics (__fadd_rn, __fmul_rn,
// __fmaf_rn): contracting an add with a multiply would break the error terms.
//
// FP64 fields are read and written as they are (the LQCD_F64 layout): a double
// is split into (hi, lo) with integer operations on its bits, so no FP64
// conversion instruction runs; the result goes back to FP64 with one FP64
// addition of the two converted halves.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lqcd {

using ::fma;

struct dfl {
  float hi, lo;
  dfl() = default;
  __host__ __device__ constexpr dfl(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ constexpr dfl(int v) : hi((float)v), lo(0.f) {}
  __device__ explicit dfl(double d);
};

// a + b = s + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// a + b = s + e exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s, e);
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// a b + c
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return fast_two_sum(s, t);
}

__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
__device__ __forceinline__ dfl operator+(dfl a, dfl b) { return df_add(a, b); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return df_add(a, -b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) { return df_mul(a, b); }
__device__ __forceinline__ dfl fma(dfl a, dfl b, dfl c) { return df_fma(a, b, c); }

// Split of a double into hi (its mantissa cut to 24 bits, exactly representable
// as a float) and lo (the remaining 29 mantissa bits, rounded to 24), from the
// bits: hi's exponent is rebased from the FP64 bias 1023 to the FP32 bias 127
// and its mantissa is the top 23 stored bits; lo = m29 2^-52 2^(e - 1023) with
// the sign of the double (both factors are normal floats over hi's range, so lo
// underflows only gradually, where |lo| < 2^-126). |d| below 2^-126 (FP32's
// normal range) splits to zero; |d| must stay below 2^128.
__device__ __forceinline__ dfl df_split(double d) {
  const unsigned int hw = (unsigned int)__double2hiint(d);
  const unsigned int lw = (unsigned int)__double2loint(d);
  const unsigned int e = (hw >> 20) & 0x7ffu;
  const unsigned int sign = hw & 0x80000000u;
  unsigned int hb = __funnelshift_l(lw, hw - (896u << 20), 3);
  hb = (hb & 0x7fffffffu) | sign;
  const float m = __fmul_rn((float)(lw & 0x1fffffffu), 0x1p-52f);
  const float scale = __int_as_float((int)((e - 896u) << 23));  // 2^(e - 1023), normal for 897 <= e <= 1150
  const float lo = __int_as_float(__float_as_int(__fmul_rn(m, scale)) | (int)sign);
  const bool normal = e >= 897u;
  return dfl(normal ? __int_as_float((int)hb) : 0.f, normal ? lo : 0.f);
}

__device__ __forceinline__ dfl::dfl(double d) {
  const dfl s = df_split(d);
  hi = s.hi;
  lo = s.lo;
}

// float -> double from the bits, exact: the exponent is rebased from 127 to
// 1023; a subnormal x is first scaled by 2^64 into the normal range and the
// rebasing takes the 64 back
__device__ __forceinline__ double float_to_double_bits(float x) {
  const bool sub = (__float_as_uint(x) & 0x7f800000u) == 0u;  // zero or subnormal
  const unsigned int b = __float_as_uint(sub ? __fmul_rn(x, 0x1p64f) : x);
  const unsigned int mag = b & 0x7fffffffu;
  const unsigned int rebias = sub ? (832u << 20) : (896u << 20);
  const unsigned int hw = mag ? ((mag >> 3) + rebias) | (b & 0x80000000u) : (b & 0x80000000u);
  return __hiloint2double((int)hw, (int)(b << 29));
}

// hi + lo rounded to a double: one FP64 addition of the exact halves
__device__ __forceinline__ double df_to_double(dfl a) {
  return __dadd_rn(float_to_double_bits(a.hi), float_to_double_bits(a.lo));
}

}  // namespace lqcd
