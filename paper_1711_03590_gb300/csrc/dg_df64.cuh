// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// binary32 numbers (|lo| <= 2^-23 |hi|), about 48 significant bits.  GB300
// executes binary32 fused multiply-adds 64 times faster than binary64 ones,
// so an FP64-accurate operator can run on the FP32 pipe.
//
// The operations are the classical error-free transformations (Knuth's
// two-sum, Dekker's fast two-sum, the FMA-based exact product) combined in
// the "sloppy" double-float add/multiply: the error of each operation is a
// small multiple of 2^-48 (|a| + |b|), the same kind of bound as for IEEE
// binary64 sums and dot products with 2^-53.  Every binary32 step uses the
// _rn intrinsics so that the compiler never contracts or reorders them.
//
// Range: values keep full accuracy for magnitudes in about [1e-30, 1e38];
// smaller parts flush to zero.
#pragma once

#include <cuda_runtime.h>

namespace dg {
// The type and its operations live in their own namespace so that they are
// found only by argument-dependent lookup on double-float arguments and never
// hide the binary32/binary64 math functions.
namespace dfp {

struct __align__(8) df64 {
  float hi, lo;
  df64() = default;
  __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
  // integer and floating literals used by the kernels (exact in binary32)
  __host__ __device__ explicit constexpr df64(int v) : hi((float)v), lo(0.f) {}
  __host__ __device__ explicit constexpr df64(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
};

__device__ __forceinline__ df64 df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df64(s, e);
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df64 df_quick_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  const df64 s = df_two_sum(a.hi, b.hi);
  return df_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_quick_two_sum(p, e);
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

// a b + c with one renormalization
__device__ __forceinline__ df64 fma(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const df64 s = df_two_sum(p, c.hi);
  return df_quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

__device__ __forceinline__ df64 fabs(df64 a) { return a.hi < 0.f ? -a : a; }

// 1 / a: the binary32 reciprocal refined by one Newton-Raphson step
// r = r0 + r0 (1 - a r0) in double-float arithmetic (the step doubles the
// number of correct bits, about 44 of them here).
__device__ __forceinline__ df64 df_recip(df64 a) {
  const float r0 = 1.0f / a.hi;
  const df64 e = df64(1.f, 0.f) - a * df64(r0, 0.f);
  return df64(r0, 0.f) + df64(r0, 0.f) * e;
}

__device__ __forceinline__ double df_to_double(df64 a) { return (double)a.hi + (double)a.lo; }

// binary64 -> double-float without the FP64 pipe: hi keeps the leading 24
// significant bits (truncated), lo the next 29 bits rounded to 24.  Doubles
// outside the binary32 exponent range go through the (slow) conversion.
__device__ __forceinline__ df64 df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int e = (int)((hw >> 20) & 0x7ffu);
  if (e < 1023 - 74 || e > 1023 + 127) {
    if (e == 0) return df64(0.f, 0.f);
    const float h = __double2float_rz(x);
    return df64(h, __double2float_rn(x - (double)h));
  }
  const unsigned sign = hw & 0x80000000u;
  const unsigned mh = ((hw & 0xfffffu) << 3) | (lw >> 29);
  const float h = __uint_as_float(sign | ((unsigned)(e - 1023 + 127) << 23) | mh);
  // remainder: the low 29 mantissa bits times 2^(e - 1023 - 52)
  const unsigned rem = lw & 0x1fffffffu;
  const float scale = __uint_as_float((unsigned)(e - 1023 - 52 + 127) << 23);
  const float l = __fmul_rn(__uint2float_rn(rem), scale);
  return df64(h, sign ? -l : l);
}

// Dot-product accumulator: sum of products kept as (s, error) and
// renormalized once at the end (12 binary32 operations per product).
struct DfAcc {
  float s, e;
  __device__ __forceinline__ void init() { s = 0.f; e = 0.f; }
  __device__ __forceinline__ void init(df64 c) { s = c.hi; e = c.lo; }
  __device__ __forceinline__ void add(df64 a, df64 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, pe);
    pe = __fmaf_rn(a.lo, b.hi, pe);
    const df64 t = df_two_sum(s, p);
    s = t.hi;
    e = __fadd_rn(e, __fadd_rn(t.lo, pe));
  }
  __device__ __forceinline__ df64 get() const { return df_two_sum(s, e); }
};

}  // namespace dfp
using dfp::df64;
using dfp::DfAcc;
}  // namespace dg
