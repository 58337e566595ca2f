// Double-float arithmetic for the FP64-accurate operator on the FP32 pipe.
//
// GB300 issues two FP64 fused multiply-adds per clock per SM against 128 FP32
// ones. A double-float value is the unevaluated sum hi + lo of two binary32
// numbers with |lo| <= ulp(hi) / 2, about 48 significant bits (unit roundoff
// u^2 = 2^-48 with u = 2^-24), so that the operator can run on the FP32 pipe
// and still agree with an FP64 evaluation far below 1e-12.
//
// Building blocks (error-free transformations, all with explicit _rn
// intrinsics so that the compiler never contracts or reorders them):
//  * TwoSum (Knuth, TAOCP vol. 2, Sec. 4.2.2): s + t = a + b exactly, 6 flops;
//  * Fast2Sum (Dekker 1971), for |a| >= |b|: 3 flops;
//  * TwoProd with a fused multiply-add: p + e = a * b exactly, 2 flops.
// On these sit the double-word sum, product and fused multiply-add of Dekker
// (1971) and of Joldes, Muller and Popescu, "Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic" (ACM TOMS 44, 2017):
// the "sloppy" sum (error below a few u^2 (|a| + |b|)), the product with
// three FMAs (error below 5 u^2 |ab|), and Newton corrections for the quotient
// and the square root. Exponentials and powers (Butler-Volmer faces only) are
// evaluated in FP64 and rounded back.
//
// Range: binary32 exponents. Magnitudes below 2^-126 are flushed to zero when a
// double is split; the operator's data (concentrations, potentials,
// coefficients, geometry) stays far inside the range.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace enp {

struct df {
  float hi, lo;
  df() = default;
  __host__ __device__ __forceinline__ constexpr df(float h, float l) : hi(h), lo(l) {}
  __host__ __device__ __forceinline__ constexpr df(float f) : hi(f), lo(0.f) {}
  __host__ __device__ __forceinline__ constexpr df(int i) : hi((float)i), lo(0.f) {}
  __host__ __device__ __forceinline__ df(double d);
};

// ---------------------------------------------------------------- primitives
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float ab = __fsub_rn(s, bb);
  t = __fadd_rn(__fsub_rn(a, ab), __fsub_rn(b, bb));
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return df(s, __fsub_rn(b, z));
}

// Split a double into a normalised double-float with integer operations only
// (no FP64 instruction): hi takes the leading 24 significant bits, lo the
// remaining 29 bits rounded to 24, and Fast2Sum renormalises the pair.
__device__ __forceinline__ df df_from_double_dev(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const int e = (int)((hw >> 20) & 0x7ff);
  const unsigned sgn = hw & 0x80000000u;
  if (e < 897) return df(__int_as_float((int)sgn), 0.f);         // zero or below 2^-126
  if (e > 1150) {                                                // beyond binary32 (or inf/NaN)
    const bool nan = e == 2047 && (((hw & 0xfffff) | lw) != 0);
    return df(nan ? __int_as_float(0x7fc00000) : __int_as_float((int)(sgn | 0x7f800000u)), 0.f);
  }
  const unsigned fb = sgn | ((unsigned)(e - 896) << 23) | ((hw & 0xfffff) << 3) | (lw >> 29);
  const float hi = __int_as_float((int)fb);
  // the remainder: mantissa bits 28..0 times 2^(e - 1023 - 52)
  const float r = __uint2float_rn(lw & 0x1fffffffu);
  const float s1 = __int_as_float((e - 1023 + 127) << 23);       // 2^(e - 1023), a normal float
  float lo = __fmul_rn(__fmul_rn(r, 2.220446049250313e-16f), s1);  // r 2^-52 2^(e-1023)
  lo = sgn ? -lo : lo;
  return fast_two_sum(hi, lo);
}

// Widen a binary32 to a double with integer operations (subnormals flushed).
__device__ __forceinline__ double f32_to_f64_bits(float f) {
  const unsigned fb = (unsigned)__float_as_int(f);
  const unsigned sgn = fb & 0x80000000u;
  const unsigned ef = (fb >> 23) & 0xff;
  if (ef == 0) return __longlong_as_double((long long)((unsigned long long)sgn << 32));
  const unsigned ed = ef == 255 ? 2047u : ef + 896u;
  const unsigned m = fb & 0x7fffffu;
  const unsigned hw = sgn | (ed << 20) | (m >> 3);
  const unsigned lw = (m & 7u) << 29;
  return __longlong_as_double((long long)(((unsigned long long)hw << 32) | lw));
}

__host__ __device__ __forceinline__ df::df(double d) {
#ifdef __CUDA_ARCH__
  *this = df_from_double_dev(d);
#else
  hi = (float)d;
  lo = (float)(d - (double)hi);
#endif
}

// The double nearest hi + lo (one FP64 addition).
__host__ __device__ __forceinline__ double to_double(df a) {
#ifdef __CUDA_ARCH__
  return f32_to_f64_bits(a.hi) + f32_to_f64_bits(a.lo);
#else
  return (double)a.hi + (double)a.lo;
#endif
}

// ---------------------------------------------------------------- arithmetic
// Sloppy double-word sum: TwoSum of the leading parts, the trailing parts added
// in binary32, Fast2Sum.
__device__ __forceinline__ df operator+(df a, df b) {
  float s, t;
  two_sum(a.hi, b.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s, t);
}
__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }
// Product with three fused multiply-adds.
__device__ __forceinline__ df operator*(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}
// a * b + c with one renormalisation.
__device__ __forceinline__ df df_fma(df a, df b, df c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  float s, t;
  two_sum(p, c.hi, s, t);
  t = __fadd_rn(t, __fadd_rn(e, c.lo));
  return fast_two_sum(s, t);
}
// Quotient: the binary32 quotient of the leading parts, one Newton correction
// on the double-word remainder a - q b (Dekker 1971).
__device__ __forceinline__ df operator/(df a, df b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const df r = a - b * df(q1);
  const float q2 = __fdiv_rn(r.hi, b.hi);
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ df& operator+=(df& a, df b) { a = a + b; return a; }
__device__ __forceinline__ df& operator-=(df& a, df b) { a = a - b; return a; }
__device__ __forceinline__ df& operator*=(df& a, df b) { a = a * b; return a; }

// Ordering of normalised pairs: by the leading part, then the trailing one.
__device__ __forceinline__ bool operator<(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df a, df b) { return b < a; }
__device__ __forceinline__ bool operator<=(df a, df b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df a, df b) { return !(a < b); }
__device__ __forceinline__ bool operator==(df a, df b) { return a.hi == b.hi && a.lo == b.lo; }
__device__ __forceinline__ bool operator!=(df a, df b) { return !(a == b); }

__device__ __forceinline__ df absv(df a) { return a.hi < 0.f ? -a : a; }
// Square root: the binary32 root s of the leading part and one Newton step
// s + (a - s^2) / (2 s) on the double-word remainder.
__device__ __forceinline__ df sqrtv(df a) {
  if (!(a.hi > 0.f)) return df(0.f, 0.f);
  const float s = __fsqrt_rn(a.hi);
  const float p = __fmul_rn(s, s);
  const float e = __fmaf_rn(s, s, -p);
  // a - (p + e), leading part only is needed for the correction
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
  const float c = __fdiv_rn(r, __fmul_rn(2.f, s));
  return fast_two_sum(s, c);
}
// Butler-Volmer exponentials and the reaction-order power: FP64, rounded back.
__device__ __forceinline__ df expv(df a) { return df(exp(to_double(a))); }
__device__ __forceinline__ df powv(df a, df g) { return df(pow(to_double(a), to_double(g))); }
__device__ __forceinline__ df mad(df a, df b, df c) { return df_fma(a, b, c); }

// The storage type a kernel of arithmetic type R reads and writes in global
// memory: the double-float operator takes and returns FP64 vectors.
template <class R> struct IoType { using type = R; };
template <> struct IoType<df> { using type = double; };
template <class R> using io_t = typename IoType<R>::type;

__device__ __forceinline__ double to_io(double x) { return x; }
__device__ __forceinline__ float to_io(float x) { return x; }
__device__ __forceinline__ double to_io(df x) { return to_double(x); }

}  // namespace enp
