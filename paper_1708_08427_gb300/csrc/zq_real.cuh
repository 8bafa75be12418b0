// zq_real.cuh -- arithmetic types for the node-transform build.
//
// The build is written once over a real type R:
//   double  native FP64;
//   dd      double-single: an unevaluated sum hi + lo of two floats,
//           |lo| <= ulp(hi)/2, about 48 significant bits.  Every operation
//           runs on the FP32 pipes with error-free transformations
//           (Knuth's two-sum, Dekker's product via FMA), so it keeps FP64
//           class accuracy (relative error ~1e-14) at a fraction of the
//           cost of this GPU's FP64 units, which run at 1/64 of FP32.
// Reciprocals and reciprocal square roots of dd start from the FP32
// hardware estimate and take one Newton step evaluated in dd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace zq {

struct dd {
  float hi, lo;
};

__device__ __forceinline__ dd dd_make(float h, float l) {
  dd r;
  r.hi = h;
  r.lo = l;
  return r;
}

// ---------------------------------------------- error-free transformations
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ float quick_two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
  return s;
}

__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
  return p;
}

// ------------------------------------------------------------- dd ops
__device__ __forceinline__ dd operator-(dd a) { return dd_make(-a.hi, -a.lo); }

__device__ __forceinline__ dd operator+(dd a, dd b) {
  float e1, e2, l;
  const float s = two_sum(a.hi, b.hi, e1);
  const float t = two_sum(a.lo, b.lo, e2);
  e1 = __fadd_rn(e1, t);
  float h = quick_two_sum(s, e1, e1);
  e1 = __fadd_rn(e1, e2);
  h = quick_two_sum(h, e1, l);
  return dd_make(h, l);
}

__device__ __forceinline__ dd operator-(dd a, dd b) { return a + (-b); }

__device__ __forceinline__ dd operator*(dd a, dd b) {
  float e, l;
  const float p = two_prod(a.hi, b.hi, e);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float h = quick_two_sum(p, e, l);
  return dd_make(h, l);
}

// a + b for a and b of one sign (or zero): one error-free sum of the high
// parts with the low parts added to its error (the "sloppy" double-single
// sum).  Without cancellation between the operands its relative error is
// that of the general sum above, at about half the instructions.
__device__ __forceinline__ dd add_same_sign(dd a, dd b) {
  float e, l;
  const float s = two_sum(a.hi, b.hi, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = quick_two_sum(s, e, l);
  return dd_make(h, l);
}

// a * a (the cross term 2 hi lo in one fused multiply-add)
__device__ __forceinline__ dd dd_sqr(dd a) {
  float e, l;
  const float p = two_prod(a.hi, a.hi, e);
  e = __fmaf_rn(2.0f * a.hi, a.lo, e);
  const float h = quick_two_sum(p, e, l);
  return dd_make(h, l);
}

// dd times a float
__device__ __forceinline__ dd mul_f(dd a, float b) {
  float e, l;
  const float p = two_prod(a.hi, b, e);
  e = __fmaf_rn(a.lo, b, e);
  const float h = quick_two_sum(p, e, l);
  return dd_make(h, l);
}

__device__ __forceinline__ dd& operator+=(dd& a, dd b) { return a = a + b; }
__device__ __forceinline__ dd& operator-=(dd& a, dd b) { return a = a - b; }
__device__ __forceinline__ dd& operator*=(dd& a, dd b) { return a = a * b; }

// 1 / b: q0 = correctly rounded float reciprocal, then
// q = q0 + q0 (1 - b q0) with the residual in dd.
__device__ __forceinline__ dd dd_rcp(dd b) {
  const float q0 = __frcp_rn(b.hi);
  const dd r = dd_make(1.0f, 0.0f) - mul_f(b, q0);
  float l;
  const float h = quick_two_sum(q0, __fmul_rn(q0, r.hi), l);
  return dd_make(h, l);
}

// 1 / sqrt(y): float estimate with one float Newton step, then
// r = r0 + r0 (1 - y r0^2) / 2 with the residual in dd.
__device__ __forceinline__ dd dd_rsqrt(dd y) {
  float r0 = rsqrtf(y.hi);
  r0 = __fmul_rn(r0, __fmaf_rn(-0.5f * y.hi, __fmul_rn(r0, r0), 1.5f));
  const dd t = mul_f(mul_f(y, r0), r0);
  const dd e = dd_make(1.0f, 0.0f) - t;
  float l;
  const float h = two_sum(r0, __fmul_rn(__fmul_rn(0.5f, r0), e.hi), l);
  return dd_make(h, l);
}

// Split a double into hi = RN_float(x), lo = RN_float(x - hi) with integer
// and FP32 instructions only (no FP64) for 2^-70 <= |x| < 2^121; other
// values (zero included) take the FP64 conversions.
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

__device__ __forceinline__ dd dd_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  if (e < -70 || e > 120) {  // outside the coordinate range: convert with FP64
    const float h = __double2float_rn(x);
    return dd_make(h, __double2float_rn(x - (double)h));
  }
  const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned int mh = (unsigned int)(m >> 29);
  const unsigned int rem = (unsigned int)(m & ((1u << 29) - 1));
  if (rem > (1u << 28) || (rem == (1u << 28) && (mh & 1u))) mh += 1u;
  const int r = (int)((long long)m - ((long long)mh << 29));
  float hi = __fmul_rn(__uint2float_rn(mh), pow2f(e - 23));
  float lo = __fmul_rn(__int2float_rn(r), pow2f(e - 52));
  if (b >> 63) {
    hi = -hi;
    lo = -lo;
  }
  return dd_make(hi, lo);
}

// ---------------------------------------------------------- real traits
template <class R>
struct Real;

template <>
struct Real<double> {
  static __device__ __forceinline__ double from_double(double x) { return x; }
  static __device__ __forceinline__ double from_int(int n) { return (double)n; }
  static __device__ __forceinline__ double from_float(float x) { return (double)x; }
  static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
  static __device__ __forceinline__ double rsqrt(double x) { return ::rsqrt(x); }
  static __device__ __forceinline__ double scale(double x, float s) { return x * (double)s; }
  static __device__ __forceinline__ double add_same(double a, double b) { return a + b; }
  static __device__ __forceinline__ double sqr(double a) { return a * a; }
  static __device__ __forceinline__ bool is_zero(double x) { return x == 0.0; }
  static __device__ __forceinline__ bool ge_zero(double x) { return x >= 0.0; }
  static __device__ __forceinline__ double abs(double x) { return fabs(x); }
  // binary exponent, biased by a constant (comparisons of differences only)
  static __device__ __forceinline__ int bexp(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }
  static __device__ __forceinline__ float to_float(double x) { return (float)x; }
  static __device__ __forceinline__ double to_double(double x) { return x; }
};

template <>
struct Real<dd> {
  static __device__ __forceinline__ dd from_double(double x) { return dd_from_double(x); }
  static __device__ __forceinline__ dd from_int(int n) {  // exact for 0 <= n < 2^31
    float l;
    const float h = two_sum(__uint2float_rn((unsigned)n & 0xFFFFFF00u), __uint2float_rn((unsigned)n & 0xFFu), l);
    return dd_make(h, l);
  }
  static __device__ __forceinline__ dd from_float(float x) { return dd_make(x, 0.0f); }
  static __device__ __forceinline__ dd rcp(dd x) { return dd_rcp(x); }
  static __device__ __forceinline__ dd rsqrt(dd x) { return dd_rsqrt(x); }
  static __device__ __forceinline__ dd scale(dd x, float s) { return mul_f(x, s); }
  static __device__ __forceinline__ dd add_same(dd a, dd b) { return add_same_sign(a, b); }
  static __device__ __forceinline__ dd sqr(dd a) { return dd_sqr(a); }
  static __device__ __forceinline__ bool is_zero(dd x) { return x.hi == 0.0f; }
  static __device__ __forceinline__ bool ge_zero(dd x) { return x.hi >= 0.0f; }
  static __device__ __forceinline__ dd abs(dd x) { return x.hi < 0.0f ? -x : x; }
  static __device__ __forceinline__ int bexp(dd x) { return (__float_as_int(x.hi) >> 23) & 0xff; }
  static __device__ __forceinline__ float to_float(dd x) { return x.hi; }
  static __device__ __forceinline__ double to_double(dd x) { return (double)x.hi + (double)x.lo; }
};

}  // namespace zq
