// df.cuh -- double-float ("double-word") arithmetic on the FP32 pipes.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  GB300 retires FP32 fused multiply-adds about 64
// times faster than FP64 ones, so a double-float operation of 6-20 FP32
// instructions still costs a fraction of one FP64 pipe slot.
//
// The building blocks are the error-free transformations Fast2Sum (Dekker
// 1971), TwoSum (Knuth, TAOCP vol. 2) and the FMA-based exact product, and the
// double-word algorithms of Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44(2), 2017: accurate DW + DW (relative error <= 3u^2), DW + FP, DW x FP
// and DW x DW with FMA (<= 5u^2), u = 2^-24.  The reciprocal is one Newton
// correction of the correctly rounded float reciprocal, and x^(-1/5) a
// third-order correction of a float seed; both stay within a few u^2.
//
// Every function is __host__ __device__ so that the arithmetic can be checked
// against double precision on the host.
#pragma once

#include <cmath>
#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace ens {
namespace df {

struct DF {
  float hi, lo;
};

__host__ __device__ __forceinline__ float fma_f(float a, float b, float c) {
#ifdef __CUDA_ARCH__
  return __fmaf_rn(a, b, c);
#else
  return std::fmaf(a, b, c);
#endif
}

// error-free transformations
__host__ __device__ __forceinline__ DF fast_two_sum(float a, float b) {  // requires |a| >= |b| (or a == 0)
  const float s = a + b;
  const float z = s - a;
  return {s, b - z};
}
__host__ __device__ __forceinline__ DF two_sum(float a, float b) {
  const float s = a + b;
  const float ap = s - b;
  const float bp = s - ap;
  return {s, (a - ap) + (b - bp)};
}
__host__ __device__ __forceinline__ DF two_prod(float a, float b) {
  const float p = a * b;
  return {p, fma_f(a, b, -p)};
}

__host__ __device__ __forceinline__ DF make(float x) { return {x, 0.0f}; }
__host__ __device__ __forceinline__ DF neg(DF x) { return {-x.hi, -x.lo}; }

// accurate DW + DW (20 flops)
__host__ __device__ __forceinline__ DF add(DF x, DF y) {
  const DF s = two_sum(x.hi, y.hi);
  const DF t = two_sum(x.lo, y.lo);
  const float c = s.lo + t.hi;
  const DF v = fast_two_sum(s.hi, c);
  const float w = t.lo + v.lo;
  return fast_two_sum(v.hi, w);
}
__host__ __device__ __forceinline__ DF sub(DF x, DF y) { return add(x, neg(y)); }

// DW + DW in Dekker's form: the exact sum of the high parts plus the rounded
// sum of the low parts and the rounding error, renormalised (11 flops).  Its
// error is bounded in the operands' magnitude, |error| <= 2 u^2 (|x| + |y|),
// not in the result's: enough for a sum of Runge-Kutta stage terms, whose
// own conditioning is relative to the terms' magnitude (as FP64 arithmetic
// rounds them), where the accurate add above keeps a relative bound of the
// result even under cancellation.
__host__ __device__ __forceinline__ DF add_terms(DF x, DF y) {
  const DF s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, s.lo + (x.lo + y.lo));
}
// DW + FP (10 flops)
__host__ __device__ __forceinline__ DF add(DF x, float y) {
  const DF s = two_sum(x.hi, y);
  const float v = x.lo + s.lo;
  return fast_two_sum(s.hi, v);
}

// DW x FP (6 flops)
__host__ __device__ __forceinline__ DF mul(DF x, float y) {
  const DF c = two_prod(x.hi, y);
  const float cl3 = fma_f(x.lo, y, c.lo);
  return fast_two_sum(c.hi, cl3);
}

// DW x DW (9 flops)
__host__ __device__ __forceinline__ DF mul(DF x, DF y) {
  const DF c = two_prod(x.hi, y.hi);
  const float tl0 = x.lo * y.lo;
  const float tl1 = fma_f(x.hi, y.lo, tl0);
  const float cl2 = fma_f(x.lo, y.hi, tl1);
  return fast_two_sum(c.hi, c.lo + cl2);
}

// a b + c
__host__ __device__ __forceinline__ DF fma(DF a, DF b, DF c) { return add(mul(a, b), c); }
// a b + c with the sum in Dekker's form (20 flops against 29)
__host__ __device__ __forceinline__ DF fma_terms(DF a, DF b, DF c) { return add_terms(mul(a, b), c); }

// 1 / y: r0 = the correctly rounded float reciprocal of y.hi, then
// r = r0 (1 + e + e^2) with the residual e = 1 - y r0 formed in double-word
// (e is about u, so its float rounding costs about u^2).
__host__ __device__ __forceinline__ DF rcp(DF y) {
#ifdef __CUDA_ARCH__
  const float r0 = __frcp_rn(y.hi);
#else
  const float r0 = 1.0f / y.hi;
#endif
  const DF p = mul(y, r0);                       // y r0 = 1 - e
  const float e = (1.0f - p.hi) - p.lo;          // 1 - p.hi is exact (Sterbenz)
  return fast_two_sum(r0, r0 * fma_f(e, e, e));  // r0 (1 + e + e^2): error about e^3
}

// x^(-1/5) for x > 0: float seed v (about 22 correct bits), residual
// r = 1 - x v^5 in double-word, then v (1 + r/5 + 3 r^2/25), the binomial
// series of (1 - r)^(-1/5) to second order; the neglected term is 11 r^3/125.
__host__ __device__ __forceinline__ DF inv_fifth_root(DF x) {
#ifdef __CUDA_ARCH__
  float l, v;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x.hi));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(-0.2f * l));
#else
  const float v = std::pow(x.hi, -0.2f);
#endif
  const DF v2 = two_prod(v, v);
  const DF v4 = mul(v2, v2);
  const DF v5 = mul(v4, v);
  const DF xv5 = mul(x, v5);
  const DF r = add(neg(xv5), 1.0f);                          // about 1e-6
  const DF c = add(DF{0.2f, -2.98023224e-09f}, 0.12f * r.hi);   // 1/5 (as a pair) + 3 r / 25
  return add(make(v), mul(mul(r, c), v));
}

// sqrt(x) for x >= 0 (0 for x <= 0 or NaN): the correctly rounded float
// square root s0 of x.hi, then one Newton step s0 + r / (2 s0) on the
// residual r = x - s0^2.  s0^2 = p.hi + p.lo exactly (two_prod) and x.hi -
// p.hi is exact (the two are within a factor 2, Sterbenz), so r carries a
// float's relative accuracy; Newton's quadratic convergence leaves about
// u^2 s of the error of s0 (which includes x.lo), plus the float rounding
// of the correction: within 4 u^2 relative (tests/test_df_host.py).
__host__ __device__ __forceinline__ DF sqrt(DF x) {
  if (!(x.hi > 0.0f)) return {0.0f, 0.0f};
#ifdef __CUDA_ARCH__
  const float s0 = __fsqrt_rn(x.hi);
  const float inv2 = 0.5f * __frcp_rn(s0);
#else
  const float s0 = std::sqrt(x.hi);
  const float inv2 = 0.5f / s0;
#endif
  const DF p = two_prod(s0, s0);
  const float r = ((x.hi - p.hi) - p.lo) + x.lo;
  return fast_two_sum(s0, r * inv2);
}

// double <-> double-word through the integer pipe (a conversion instruction
// costs about one FP64 pipe slot on this part).  trunc_f truncates the
// significand of a double to 24 bits with the exponent rebiased; |x| below
// 2^-100 becomes 0 (far below the scales the solver works with).
__host__ __device__ __forceinline__ float trunc_f(double x) {
#ifdef __CUDA_ARCH__
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
#else
  uint64_t b;
  __builtin_memcpy(&b, &x, 8);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
#endif
  const unsigned sign = hi & 0x80000000u, mag = hi & 0x7fffffffu;
  const bool tiny = mag < ((1023u - 100u) << 20);
  const unsigned bits = tiny ? 0u : ((((mag - ((1023u - 127u) << 20)) << 3) | (lo >> 29)) | sign);
#ifdef __CUDA_ARCH__
  return __uint_as_float(bits);
#else
  float f;
  __builtin_memcpy(&f, &bits, 4);
  return f;
#endif
}
// float -> double, exact for zero and normal floats
__host__ __device__ __forceinline__ double widen(float v) {
#ifdef __CUDA_ARCH__
  const unsigned b = __float_as_uint(v);
#else
  unsigned b;
  __builtin_memcpy(&b, &v, 4);
#endif
  const unsigned sign = b & 0x80000000u, mag = b & 0x7fffffffu;
  const unsigned hi = mag == 0u ? sign : (((mag >> 3) + ((1023u - 127u) << 20)) | sign);
  const unsigned lo = mag << 29;
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const uint64_t bb = ((uint64_t)hi << 32) | lo;
  double d;
  __builtin_memcpy(&d, &bb, 8);
  return d;
#endif
}
// double -> double-word on the integer pipe: hi = trunc_f(x), and lo the
// exact remainder x - hi, which is the 29 low significand bits of x, cut to
// their leading 24 bits as trunc_f cuts it (0 below 2^-100).  This is the
// pair that trunc_f(x - widen(hi)) gives, without that FP64 subtraction
// (tests/test_df_host.py compares the two bit for bit).
__host__ __device__ __forceinline__ DF from_double(double x) {
  const float h = trunc_f(x);
#ifdef __CUDA_ARCH__
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long u;
  __builtin_memcpy(&u, &x, 8);
#endif
  const int ef = (int)((u >> 52) & 0x7ff);
  const unsigned long long L = u & 0x1fffffffull;  // x - hi = L 2^(ef - 1075)
#ifdef __CUDA_ARCH__
  const int p = 63 - __clzll((long long)(L | 1ull));  // leading bit of L (0..28)
#else
  const int p = 63 - __builtin_clzll(L | 1ull);
#endif
  const int e_low = ef - 1075 + p;                     // exponent of the remainder
  const unsigned frac = (unsigned)(((L << (63 - p)) << 1) >> 41);  // its next 23 bits, truncated
  const unsigned sign = (unsigned)(u >> 32) & 0x80000000u;
  const unsigned lb = (L == 0 || e_low < -100) ? 0u : ((((unsigned)(e_low + 127) << 23) | frac) | sign);
#ifdef __CUDA_ARCH__
  const float l = __uint_as_float(lb);
#else
  float l;
  __builtin_memcpy(&l, &lb, 4);
#endif
  return fast_two_sum(h, l);
}
// the same pair through one FP64 subtraction (the reference for the test)
__host__ __device__ __forceinline__ DF from_double_sub(double x) {
  const float h = trunc_f(x);
  const float l = trunc_f(x - widen(h));
  return fast_two_sum(h, l);
}
// double-word -> double: one FP64 addition
__host__ __device__ __forceinline__ double to_double(DF x) { return widen(x.hi) + widen(x.lo); }

// ordering of normalised pairs
__host__ __device__ __forceinline__ bool gt(DF a, DF b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

}  // namespace df
}  // namespace ens
