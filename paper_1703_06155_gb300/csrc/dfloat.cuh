// Double-float arithmetic on the FP32 pipe.
//
// A value is h + l with |l| <= ulp(h) / 2 (about 48 significant bits).  The
// operations use only correctly rounded single-precision adds and
// multiplies (the __f*_rn intrinsics, never contracted into FMAs) and fused
// multiply-adds: TwoSum (Knuth) and the FMA product error are exact, so
// every operation below is accurate to a few units of 2^-48 of its operands.
// On this GPU the FP32 pipe runs 64 FMAs for every FP64 FMA, so a
// double-float product (7 operations) or multiply-add (15) still costs a
// fraction of its FP64 counterpart.
#pragma once

#include <cuda_runtime.h>

namespace h2k {
namespace dfl {

struct df {
  float h, l;
};

__device__ __forceinline__ df quick_two_sum(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ df dadd(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return quick_two_sum(s.h, __fadd_rn(__fadd_rn(a.l, b.l), s.l));
}
__device__ __forceinline__ df dneg(df a) { return {-a.h, -a.l}; }
__device__ __forceinline__ df dsub(df a, df b) { return dadd(a, dneg(b)); }
__device__ __forceinline__ df dmul(df a, df b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return quick_two_sum(p, e);
}
// a * b + c
__device__ __forceinline__ df dfma(df a, df b, df c) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  const df s = two_sum(p, c.h);
  return quick_two_sum(s.h, __fadd_rn(__fadd_rn(e, c.l), s.l));
}
__device__ __forceinline__ df dscale(df a, float f) {  // exact power-of-two factor
  return {__fmul_rn(a.h, f), __fmul_rn(a.l, f)};
}
// 1 / sqrt(x), x > 0: a single-precision estimate and two Newton steps
// y <- y + y (1 - x y^2) / 2 carried in double-float
__device__ __forceinline__ df drsqrt(df x) {
  df y = {rsqrtf(x.h), 0.0f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df h = dsub(df{1.0f, 0.0f}, dmul(x, dmul(y, y)));
    y = dfma(y, dscale(h, 0.5f), y);
  }
  return y;
}
// 1 / x, x != 0: a single-precision estimate and two Newton steps
// y <- y + y (1 - x y)
__device__ __forceinline__ df drcp(df x) {
  df y = {__frcp_rn(x.h), 0.0f};
#pragma unroll
  for (int it = 0; it < 2; ++it) {
    const df h = dsub(df{1.0f, 0.0f}, dmul(x, y));
    y = dfma(y, h, y);
  }
  return y;
}
__device__ __forceinline__ df dsqrt(df x) {  // x >= 0
  if (!(x.h > 0.0f)) return {0.0f, 0.0f};
  return dmul(x, drsqrt(x));
}
__device__ __forceinline__ df dsplit(double v) {
  const float h = __double2float_rn(v);
  return {h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double djoin(df a) { return (double)a.h + (double)a.l; }

// warp butterfly sum (every lane gets the same value)
__device__ __forceinline__ df wsum(df v) {
  for (int o = 16; o > 0; o >>= 1) {
    const df w = {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    v = dadd(v, w);
  }
  return v;
}

// complex double-float entry in memory: {re.h, re.l, im.h, im.l} (16 bytes,
// the size of a complex128)
__device__ __forceinline__ df re_of(const float4& v) { return {v.x, v.y}; }
__device__ __forceinline__ df im_of(const float4& v) { return {v.z, v.w}; }
__device__ __forceinline__ float4 pack(df re, df im) { return make_float4(re.h, re.l, im.h, im.l); }

}  // namespace dfl
}  // namespace h2k
