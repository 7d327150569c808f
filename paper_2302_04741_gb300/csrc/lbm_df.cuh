// lbm_df.cuh -- float-float ("double-float") arithmetic for the FP64 step.
//
// GB300 executes FP64 instructions at about 1/73 of the FP32 rate (measured:
// DFMA and DADD 0.53 T/s, FFMA 38.8 T/s), and its double <-> float
// conversion instructions run at the FP64 rate too.  The FP64 step (FP64
// storage, about 620 FP64 operations per site) is therefore bound by the
// FP64 units at about 1/13 of its HBM roofline.  A value held as an
// unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)) carries about 48
// significant bits, and its arithmetic -- Dekker's and Knuth's error-free
// transformations (two-sum, and two-product through the fused multiply-add)
// -- runs on the FP32 pipe.  Populations stay IEEE doubles in memory: a load
// splits the double into hi + lo with integer bit operations (no conversion
// instruction), and a store rebuilds both halves as doubles bit by bit and
// adds them with one DADD, which rounds the float-float value to the nearest
// double.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace lbm {

// the float and double fma overloads stay visible next to the float-float one
using ::fma;

struct DF {
  float hi, lo;
  __host__ __device__ constexpr DF() : hi(0.f), lo(0.f) {}
  __host__ __device__ constexpr DF(float h, float l) : hi(h), lo(l) {}
  // small integers are exact in float
  __host__ __device__ constexpr explicit DF(int v) : hi(float(v)), lo(0.f) {}
  // compile-time constants: the split is folded by the compiler; values
  // known only at run time should go through df_split (no FP64 instruction)
  __host__ __device__ constexpr explicit DF(double v)
      : hi(float(v)), lo(float(v - double(float(v)))) {}
};

// Every float operation below carries an explicit round-to-nearest
// (__fadd_rn, __fmul_rn): without one the compiler may fuse a product into a
// following sum (one rounding instead of two), which these error-free
// transformations cannot tolerate -- and whether it fuses depends on
// register allocation.

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void df_fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

// Sums are renormalised (hi carries the value, |lo| <= ulp(hi)): after a
// cancellation the unrenormalised lo could exceed hi, and a following
// product, which forms lo hi in float only, would keep just float
// precision.  Products are left unrenormalised: their lo is the rounding
// error of hi times hi plus the cross terms, a few ulp(hi) at most, which the
// next sum absorbs; skipping the renormalisation there shortens the code
// (whose size stalls the instruction fetch of this kernel).
__device__ __forceinline__ DF operator+(DF a, DF b) {
  float s, e;
  df_two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  DF r;
  df_fast_two_sum(s, e, r.hi, r.lo);
  return r;
}
__device__ __forceinline__ DF operator-(DF a) { return DF(-a.hi, -a.lo); }
__device__ __forceinline__ DF operator-(DF a, DF b) { return a + (-b); }
__device__ __forceinline__ DF operator*(DF a, DF b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return DF(p, e);
}
// a / b: a float quotient, one correction from the float-float residual
__device__ __forceinline__ DF operator/(DF a, DF b) {
  df_fast_two_sum(b.hi, b.lo, b.hi, b.lo);
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const DF r = a - b * DF(q1, 0.f);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  DF q;
  df_fast_two_sum(q1, q2, q.hi, q.lo);
  return q;
}
__device__ __forceinline__ DF& operator+=(DF& a, DF b) { return a = a + b; }
__device__ __forceinline__ DF& operator-=(DF& a, DF b) { return a = a - b; }
__device__ __forceinline__ DF& operator*=(DF& a, DF b) { return a = a * b; }
__device__ __forceinline__ bool operator>(DF a, DF b) {
  const DF d = a - b;
  return __fadd_rn(d.hi, d.lo) > 0.f;
}
__device__ __forceinline__ bool operator<(DF a, DF b) { return b > a; }

// a * b + c
__device__ __forceinline__ DF fma(DF a, DF b, DF c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float pe = fmaf(a.hi, b.hi, -p);
  pe = fmaf(a.hi, b.lo, pe);
  pe = fmaf(a.lo, b.hi, pe);
  float s, e;
  df_two_sum(p, c.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(pe, c.lo));
  DF r;
  df_fast_two_sum(s, e, r.hi, r.lo);
  return r;
}

// The IEEE double d as hi + lo: hi holds the leading 24 significant bits,
// lo the next 29 bits rounded to 24; built from the bit fields with integer
// operations.  |d| < 2^-126 gives 0; infinities and NaN go through the
// conversion instruction (so that an unstable state stays visible).
__device__ __forceinline__ DF df_split(double d) {
  const unsigned hi32 = (unsigned)__double2hiint(d), lo32 = (unsigned)__double2loint(d);
  const unsigned E = (hi32 >> 20) & 0x7ffu;  // biased exponent
  if (E <= 896u) return DF(0.f, 0.f);
  if (E >= 1139u) return DF((float)d, 0.f);  // |d| >= 2^116 (the lo scale would overflow), inf, NaN
  const unsigned sign = hi32 & 0x80000000u;
  const unsigned m23 = ((hi32 & 0xfffffu) << 3) | (lo32 >> 29);
  const float hi = __uint_as_float(sign | ((E - 896u) << 23) | m23);
  // remainder L 2^(E - 1075), L < 2^29, scaled in two exact steps
  const float L = (float)(lo32 & 0x1fffffffu);
  float lo = __fmul_rn(__fmul_rn(L, 0x1p-64f), __uint_as_float((E - 884u) << 23));
  lo = __uint_as_float(__float_as_uint(lo) | sign);
  DF r;
  df_fast_two_sum(hi, lo, r.hi, r.lo);
  return r;
}

// The float f as a double, built bit by bit (exact; zero and float
// subnormals give 0; inf and NaN through the conversion instruction).
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  if (e == 0u) return 0.0;
  if (e == 0xffu) return (double)f;
  const unsigned hi32 = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
  return __hiloint2double((int)hi32, (int)(u << 29));
}

// hi + lo rounded to the nearest double: one DADD of the exact halves.
__device__ __forceinline__ double df_to_double(DF a) { return f2d_bits(a.hi) + f2d_bits(a.lo); }

}  // namespace lbm
