// Split of an operand value into three BF16 parts for the BF16x3 tensor-core
// contraction, shared by every kernel that writes the contraction's split planes
// (one definition, so that all writers produce the same bits):
//   x_hi = bf16(x), x_mid = bf16(x - x_hi), x_lo = bf16(x - x_hi - x_mid)
// and the FP64 -> FP32 rounding by integer operations that precedes it for FP64
// values (no FP64 instruction).
#pragma once
#include <cuda_bf16.h>

template <typename T>
__device__ __forceinline__ void split3(T x, __nv_bfloat16& h, __nv_bfloat16& m, __nv_bfloat16& l) {
  h = __float2bfloat16_rn((float)x);
  const T r1 = x - (T)__bfloat162float(h);
  m = __float2bfloat16_rn((float)r1);
  const T r2 = r1 - (T)__bfloat162float(m);
  l = __float2bfloat16_rn((float)r2);
}

// FP64 -> FP32 round to nearest even, by integer operations on the two words
// (h = high word, l = low word); results below 2^-126 flush to zero, above FLT_MAX
// (and inf / NaN) become inf.
__device__ __forceinline__ float f64w_to_f32(unsigned h, unsigned l) {
  const unsigned sign = h & 0x80000000u;
  const unsigned ah = h & 0x7fffffffu;
  unsigned f = ((ah - (896u << 20)) << 3) | (l >> 29);
  const unsigned rem = l & 0x1fffffffu;
  f += (rem > 0x10000000u) | ((rem == 0x10000000u) & (f & 1u));
  f = (ah < (897u << 20)) ? 0u : f;
  f = (ah >= (1151u << 20)) ? 0x7f800000u : f;
  return __uint_as_float(sign | f);
}

// the three BF16 parts (as raw shorts) of an FP64 value
__device__ __forceinline__ void split3_f64(double v, unsigned short& h, unsigned short& m, unsigned short& l) {
  __nv_bfloat16 bh, bm, bl;
  split3<float>(f64w_to_f32((unsigned)__double2hiint(v), (unsigned)__double2loint(v)), bh, bm, bl);
  h = __bfloat16_as_ushort(bh);
  m = __bfloat16_as_ushort(bm);
  l = __bfloat16_as_ushort(bl);
}
