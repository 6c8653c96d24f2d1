// Double-float arithmetic: an unevaluated sum hi + lo of two FP32 values (48
// significand bits), for the places where FP64's rate on this GPU (a small
// fraction of FP32's) would bound a kernel.  Error-free sums (Knuth's
// TwoSum) and products (by FMA), with the rounding intrinsics so that no step
// is contracted or reordered.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace ara {

struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_of(double v) {
  const float hi = static_cast<float>(v);
  return DF{hi, static_cast<float>(v - static_cast<double>(hi))};
}
__device__ __forceinline__ double df_val(DF v) { return static_cast<double>(v.hi) + static_cast<double>(v.lo); }
__device__ __forceinline__ DF df_norm(float s, float e) {  // |s| >= |e|
  const float h = __fadd_rn(s, e);
  return DF{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const float s = __fadd_rn(x.hi, y.hi);
  const float bb = __fsub_rn(s, x.hi);
  const float err = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
  return df_norm(s, __fadd_rn(err, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF df_add_f(DF x, float y) {
  const float s = __fadd_rn(x.hi, y);
  const float bb = __fsub_rn(s, x.hi);
  const float err = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y, bb));
  return df_norm(s, __fadd_rn(err, x.lo));
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.hi, y.hi);
  float e = __fmaf_rn(x.hi, y.hi, -p);
  e = __fmaf_rn(x.hi, y.lo, __fmaf_rn(x.lo, y.hi, e));
  return df_norm(p, e);
}
__device__ __forceinline__ DF df_neg(DF x) { return DF{-x.hi, -x.lo}; }
// x 2^k for an exponent k with 2^k a normal float (exact)
__device__ __forceinline__ DF df_scale(DF x, int k) {
  const float f = __int_as_float((127 + k) << 23);
  return DF{__fmul_rn(x.hi, f), __fmul_rn(x.lo, f)};
}
__device__ __forceinline__ int f_exponent(float v) { return ((__float_as_int(v) >> 23) & 255) - 127; }

// v as a double without the FP64 unit (whose rate would bound a kernel that
// writes FP64 outputs): the FP32 fields moved into the FP64 ones, exact for
// every input.  Normal: exponent re-biased by 1023 - 127, significand shifted
// by 52 - 23; subnormal (m * 2^-149): the leading one of m shifted to bit 23
// and the exponent lowered by the shift; zero keeps its sign; infinities and
// NaN take the all-ones exponent with their significand bits (a NaN comes
// out quiet).  Integer operations only, so that no branch falls back to the
// conversion instruction.
__device__ __forceinline__ double f32_to_f64(float v) {
  const uint32_t u = __float_as_uint(v);
  const uint32_t e = (u >> 23) & 0xFFu;
  uint32_t m = u & 0x7FFFFFu;
  uint32_t de = e + 896u;
  if (e == 0xFFu) {
    de = 0x7FFu;
    if (m) m |= 0x400000u;  // a NaN comes out quiet, as from the conversion
  } else if (e == 0u) {
    const uint32_t sh = m ? static_cast<uint32_t>(__clz(m)) - 8u : 0u;  // m < 2^23: sh >= 1
    m = (m << sh) & 0x7FFFFFu;
    de = m || sh ? 897u - sh : 0u;
  }
  return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(u >> 31) << 63) |
                                                     (static_cast<unsigned long long>(de) << 52) |
                                                     (static_cast<unsigned long long>(m) << 29)));
}
// hi + lo as a double: both parts moved exactly, one FP64 add (rounded once).
__device__ __forceinline__ double df_val_fast(DF v) { return f32_to_f64(v.hi) + f32_to_f64(v.lo); }

}  // namespace ara
