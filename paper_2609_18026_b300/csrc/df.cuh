// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers
// with |lo| <= ulp(hi) / 2 (hi is the FP32 rounding of the sum), about 48 significant
// bits.  On this GPU an FP64 instruction issues once per 64 cycles per SM
// sub-partition while FP32 instructions issue every cycle.  So coefficient-space work
// of the mixed-precision forms that needs more than FP32 accuracy but not full FP64
// runs on the FP32 pipe in this representation: the vortex fields (rounded to FP32 for
// the transforms afterwards) and the recurrences of the half-width-2 implicit solve
// (rounded back to the FP64 state, unit roundoff about 2^-47 per multiply-add).
//
// The error-free transformations are the classical ones: the sum of two floats with
// its rounding error (Knuth's branch-free two-sum, and the three-operation form when
// the larger operand is known), and a product with its rounding error from one fused
// multiply-add.  Every operation is spelled with the _rn intrinsics so that the
// compiler neither fuses nor reorders them.
#pragma once

#include <stdint.h>

struct dfl { float hi, lo; };
struct dfl2 { dfl re, im; };

__device__ __forceinline__ dfl df_make(float hi, float lo) { dfl r; r.hi = hi; r.lo = lo; return r; }

// s + e = a + b exactly, s = fl(a + b)
__device__ __forceinline__ dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df_make(s, e);
}
// the same when |a| >= |b| (or a = 0)
__device__ __forceinline__ dfl df_fast_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = df_two_sum(x.hi, y.hi);
  const dfl t = df_two_sum(x.lo, y.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = df_fast_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return df_fast_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfl df_neg(dfl x) { return df_make(-x.hi, -x.lo); }
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, e);
  e = __fmaf_rn(x.lo, y.hi, e);
  return df_fast_sum(p, e);
}
// a b + c
__device__ __forceinline__ dfl df_fma(dfl a, dfl b, dfl c) { return df_add(df_mul(a, b), c); }
// a b + c with a single error-free sum (Dekker's add2 after the product): about 15
// FP32 operations against about 27 for df_fma; the error is bounded by a small
// multiple of 2^-47 (|a b| + |c|) -- the backward-stable error model of one FP64
// fused multiply-add with a larger unit roundoff, which is what a triangular
// recurrence needs (its relative error can be large only where a b and c cancel).
__device__ __forceinline__ dfl df_madd(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const dfl s = df_two_sum(p, c.hi);
  const float t = __fadd_rn(__fadd_rn(e, c.lo), s.lo);
  return df_fast_sum(s.hi, t);
}
// c - a b
__device__ __forceinline__ dfl df_nmadd(dfl a, dfl b, dfl c) { return df_madd(df_neg(a), b, c); }

// The FP64 value x as hi + lo by 32-bit integer operations on its two words (no FP64
// instruction): hi is the FP32 rounding of x (to nearest even; |x| < 2^-126 gives a
// signed 0, |x| >= 2^128 and non-finite values give +-inf with lo = 0), lo the FP32
// rounding of x - hi.
__device__ __forceinline__ dfl df_from_double(double x) {
  const unsigned h = (unsigned)__double2hiint(x), l = (unsigned)__double2loint(x);
  const unsigned sign = h & 0x80000000u, ah = h & 0x7fffffffu;
  const int E = (int)(ah >> 20);                                        // biased FP64 exponent
  if (E < 897) return df_make(__uint_as_float(sign), 0.0f);
  if (E >= 1151) return df_make(__uint_as_float(sign | 0x7f800000u), 0.0f);
  // exponent and the top 23 fraction bits; the increment of the rounding carries into
  // the exponent when the fraction overflows (and into inf above FLT_MAX)
  unsigned f = ((ah - (896u << 20)) << 3) | (l >> 29);
  const unsigned rem = l & 0x1fffffffu;                                  // the 29 bits below hi
  const unsigned up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (f & 1u));
  f += up;
  const float hi = __uint_as_float(sign | f);
  // |x| - |hi| = rem - up 2^29 in units of 2^(E - 1075), |.| <= 2^28: its FP32 rounding,
  // scaled through the exponent field (exact); a scaled value below 2^-126 (|x| below
  // about 2^-102) becomes 0, so such x keep FP32 precision only
  const int R = (int)rem - (int)(up << 29);
  const float lr = __int2float_rn(R);
  const int el = (int)((__float_as_uint(lr) >> 23) & 0xffu) + E - 1075;  // biased exponent after scaling
  const unsigned lb = (R == 0 || el <= 0) ? 0u : __float_as_uint(lr) + ((unsigned)(E - 1075) << 23);
  return df_make(hi, __uint_as_float(lb ^ sign));
}

// An FP32 value as FP64 by integer operations (exact; FP32 subnormals become a signed
// zero, inf and NaN stay inf and NaN)
__device__ __forceinline__ double df_f32_to_f64(float v) {
  const unsigned u = __float_as_uint(v);
  const unsigned sg = u & 0x80000000u, e = (u >> 23) & 0xffu, mt = u & 0x7fffffu;
  const unsigned eo = (e == 0u) ? 0u : (e == 255u ? 2047u : e + 896u);
  const unsigned hw = sg | (eo << 20) | (e == 0u ? 0u : ((mt >> 3) | (e == 255u && mt ? 1u : 0u)));
  const unsigned lw = (e == 0u) ? 0u : (mt << 29);
  return __hiloint2double((int)hw, (int)lw);
}
// hi + lo rounded to FP64: one FP64 addition
__device__ __forceinline__ double df_to_double(dfl x) { return __dadd_rn(df_f32_to_f64(x.hi), df_f32_to_f64(x.lo)); }

// the FP32 rounding of hi + lo as the FP64 -> FP32 rounding used by the split writers
// would give it (values below 2^-126 flush to a signed zero)
__device__ __forceinline__ float df_round_f32(dfl x) {
  return (fabsf(x.hi) < 1.17549435082228751e-38f) ? __uint_as_float(__float_as_uint(x.hi) & 0x80000000u) : x.hi;
}

__device__ __forceinline__ dfl2 dfc_make(dfl re, dfl im) { dfl2 r; r.re = re; r.im = im; return r; }
__device__ __forceinline__ dfl2 dfc_from(double2 v) { return dfc_make(df_from_double(v.x), df_from_double(v.y)); }
__device__ __forceinline__ dfl2 dfc_add(dfl2 a, dfl2 b) { return dfc_make(df_add(a.re, b.re), df_add(a.im, b.im)); }
__device__ __forceinline__ dfl2 dfc_sub(dfl2 a, dfl2 b) { return dfc_make(df_sub(a.re, b.re), df_sub(a.im, b.im)); }
// real a times complex v
__device__ __forceinline__ dfl2 dfc_scale(dfl a, dfl2 v) { return dfc_make(df_mul(a, v.re), df_mul(a, v.im)); }
// i a v
__device__ __forceinline__ dfl2 dfc_iscale(dfl a, dfl2 v) { return dfc_make(df_neg(df_mul(a, v.im)), df_mul(a, v.re)); }
// a v + w
__device__ __forceinline__ dfl2 dfc_fma(dfl a, dfl2 v, dfl2 w) { return dfc_make(df_fma(a, v.re, w.re), df_fma(a, v.im, w.im)); }
