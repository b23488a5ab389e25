// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// float32 numbers (|lo| <= ulp(hi) / 2), about 48 significant bits, computed
// with error-free float32 transformations (Knuth's TwoSum for a sum, the
// FMA-based product error of Dekker's method for a product) on the FP32
// pipes.  On GB300, whose FP64 units run at 1/64 of its FP32 rate, this carries
// the FP64 iterative refinement's residual f - K u (Sec. 3.5 solve; the
// refinement needs its residual far more accurately than the 1e-6 tolerance,
// not to the last FP64 bit).  Sums and products follow the common "sloppy"
// double-float formulas: each result is correct to a few units of 2^-44 of
// its operands' magnitudes.
#pragma once

#include <cuda_runtime.h>

namespace afd {

struct dfloat {
  float hi, lo;
  dfloat() = default;   // trivial, so that arrays of it may live in shared memory
  // from a double: hi the nearest float, lo the nearest float to the remainder
  __host__ __device__ explicit dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
  __host__ __device__ dfloat(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
  __host__ __device__ explicit operator float() const { return hi + lo; }
};

// Renormalise s + e with |e| small against s into (hi, lo).
__device__ __forceinline__ dfloat df_fast_two_sum(float s, float e) {
  const float h = __fadd_rn(s, e);
  return dfloat(h, __fsub_rn(e, __fsub_rn(h, s)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
  // TwoSum of the leading parts, then the trailing parts and the renormalisation
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return df_fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
  // product of the leading parts with its exact rounding error (FMA), plus the cross terms
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_fast_two_sum(p, e);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }
__device__ __forceinline__ bool operator!=(dfloat a, dfloat b) { return a.hi != b.hi || a.lo != b.lo; }

// double -> dfloat without the FP64 unit (GB300 runs conversions there at the
// FP64 rate).  For |d| in [2^-103, 2^128): hi takes the sign, the exponent and
// the leading 23 stored mantissa bits of d (d truncated to 24 bits); lo is the
// next 23 bits, read as the float 2^(E-23) (1.m) and made exact by subtracting
// 2^(E-23).  The 6 trailing bits are dropped: hi + lo = d to 2^-46 relative.
// Zero (and FP64 subnormals) give 0; other values take the FP64 conversion.
__device__ __forceinline__ dfloat df_from_double(double d) {
  const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
  const int ed = (int)((hw >> 20) & 0x7FFu);   // biased FP64 exponent
  if (ed >= 1023 - 103 && ed < 1023 + 128) {
    const unsigned sgn = hw & 0x80000000u;
    const unsigned ef = (unsigned)(ed - 1023 + 127);   // biased FP32 exponent, in [24, 254]
    const float hi = __uint_as_float(sgn | (ef << 23) | ((hw & 0xFFFFFu) << 3) | (lw >> 29));
    const unsigned base = sgn | ((ef - 23u) << 23);
    const float lo = __fsub_rn(__uint_as_float(base | ((lw >> 6) & 0x7FFFFFu)), __uint_as_float(base));
    return dfloat(hi, lo);
  }
  if (ed == 0) return dfloat(0.f, 0.f);
  return dfloat(d);
}

// float -> double by its bits (normal floats and zero; others convert on the FP64 unit)
__device__ __forceinline__ double df_widen(float x) {
  const unsigned b = __float_as_uint(x);
  const unsigned ef = (b >> 23) & 0xFFu;
  if (ef != 0u && ef != 0xFFu) {
    const unsigned hw = (b & 0x80000000u) | ((ef + (1023u - 127u)) << 20) | ((b & 0x7FFFFFu) >> 3);
    return __hiloint2double((int)hw, (int)(b << 29));
  }
  if ((b & 0x7FFFFFFFu) == 0u) return __hiloint2double((int)(b & 0x80000000u), 0);
  return (double)x;
}

// dfloat -> double with one FP64 add
__device__ __forceinline__ double df_to_double(dfloat v) { return df_widen(v.hi) + df_widen(v.lo); }

// Conversion of loaded values into the arithmetic type C (a cast, or the
// bitwise double -> dfloat split) and of results back to storage type T.
template <typename C, typename T>
struct Arith {
  static __device__ __forceinline__ C in(T v) { return (C)v; }
  static __device__ __forceinline__ T out(C v) { return (T)v; }
};
template <>
struct Arith<dfloat, double> {
  static __device__ __forceinline__ dfloat in(double v) { return df_from_double(v); }
  static __device__ __forceinline__ double out(dfloat v) { return df_to_double(v); }
};

}  // namespace afd

// fma and the warp shuffles are overloaded at global scope, beside CUDA's own
// float and double forms: an afd:: overload would hide those from the
// unqualified calls inside namespace afd.
__device__ __forceinline__ afd::dfloat fma(afd::dfloat a, afd::dfloat b, afd::dfloat c) { return a * b + c; }
__device__ __forceinline__ afd::dfloat __shfl_down_sync(unsigned mask, afd::dfloat v, unsigned d) {
  return afd::dfloat(__shfl_down_sync(mask, v.hi, d), __shfl_down_sync(mask, v.lo, d));
}
__device__ __forceinline__ afd::dfloat __shfl_up_sync(unsigned mask, afd::dfloat v, unsigned d) {
  return afd::dfloat(__shfl_up_sync(mask, v.hi, d), __shfl_up_sync(mask, v.lo, d));
}
__device__ __forceinline__ afd::dfloat __shfl_xor_sync(unsigned mask, afd::dfloat v, int d) {
  return afd::dfloat(__shfl_xor_sync(mask, v.hi, d), __shfl_xor_sync(mask, v.lo, d));
}
