// fifth_root_fx.cuh -- x^(-1/5) with its refinement on the integer pipe.
//
// The Keller-Miksis right-hand side needs y1^(-1/5) for the polytropic term
// (1/y1)^(21/5) = (1/y1)^4 y1^(-1/5) (Sec. 4.2, exponent 3 gamma = 21/5), and
// the step-size controller needs E^(-1/5).  Refining a float seed in FP64
// costs 7 FP64 instructions; on GB300, whose FP64 pipe retires 2 lanes per
// clock per SM against the integer pipe's 64, this routine does the
// refinement in 64-bit fixed point:
//
//   1. x = m 2^e with m in [1, 2); e = 5 q + k with k in 0..4, so
//      x^(-1/5) = u^(-1/5) 2^(-q) with u = m 2^k in [1, 32) and
//      z = u^(-1/5) in (1/2, 1];
//   2. a float seed v of z (hardware base-2 logarithm and exponential, about
//      22 correct bits; the host takes the float power);
//   3. one step of the binomial series of (1 - r)^(-1/5) with the residual
//      r = 1 - u v^5:  z = v (1 + r/5 + 3 r^2/25 + 11 r^3/125), in fixed point
//      (values x 2^62, 64 x 64 -> high-64 products); the neglected term
//      44 r^4 / 625 is below 2^-66 for seeds within 2^-19 of z (the hardware
//      seed is within about 2^-21);
//   4. z rounded to the nearest double by integer normalisation, 2^(-q)
//      applied through the exponent field.
//
// Relative error below 2^-56 before the final rounding
// (tests/test_fifth_root_fx_host.py checks it against 50-digit arithmetic and
// with seeds off by up to 2^-19), so the result is the correctly rounded
// double except near rounding boundaries.  Valid for positive normal x; NaN
// for x <= 0, NaN and infinity (pow() gives NaN for the negative bases it
// replaces); subnormal x gives an unspecified finite value.  Branch-free.
#pragma once

#include <cmath>

#include "fixed64.cuh"

namespace ens {
namespace fx {

// x = m 2^e (normal, positive) -> (q, k, the float u = m 2^k truncated to 24 bits)
__host__ __device__ __forceinline__ void fifth_root_split(uint64_t b, int* q, int* k, float* uf) {
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  // floor(e / 5) for e in [-1022, 1023]: e + 1025 in [3, 2048] and
  // (x 52429) >> 18 is floor(x / 5) there (52429 / 2^18 - 1/5 < 7e-7)
  const int qq = (int)(((unsigned)(e + 1025) * 52429u) >> 18) - 205;
  *q = qq;
  *k = e - 5 * qq;
  const unsigned fb = ((unsigned)(127 + *k) << 23) | (unsigned)((b >> 29) & 0x7fffffu);
#ifdef __CUDA_ARCH__
  *uf = __uint_as_float(fb);
#else
  __builtin_memcpy(uf, &fb, 4);
#endif
}

// the refinement of the seed vf of z = u^(-1/5), u = m 2^k: z x 2^62 in
// (2^61, 2^62]
__host__ __device__ __forceinline__ uint64_t fifth_root_fixed(uint64_t b, int k, float vf) {
#ifdef __CUDA_ARCH__
  const unsigned vb = __float_as_uint(vf);
#else
  unsigned vb;
  __builtin_memcpy(&vb, &vf, 4);
#endif
  // v x 2^62 from the float's bits (exact): (2^23 + f) 2^(ev - 23) 2^62
  const int ev = (int)((vb >> 23) & 0xffu) - 127;
  const uint64_t V = (uint64_t)((vb & 0x7fffffu) | 0x800000u) << ((39 + ev) & 63);
  const uint64_t V2 = mulhi(V, V) << 2;     // v^2 x 2^62
  const uint64_t V4 = mulhi(V2, V2) << 2;   // v^4
  const uint64_t V5 = mulhi(V4, V) << 2;    // v^5 in [1/32, 1]
  const uint64_t M = ((b & 0x000fffffffffffffull) | 0x0010000000000000ull) << 11;  // m x 2^63
  const uint64_t P = mulhi(V5, M) << (1 + k);  // u v^5 x 2^62, close to 2^62
  const int64_t R = (int64_t)((1ull << 62) - P);   // r x 2^62, |r| about 2^-22
  const uint64_t Ra = R < 0 ? (uint64_t)0 - (uint64_t)R : (uint64_t)R;
  const uint64_t R2 = mulhi(Ra, Ra) << 2;                         // r^2 x 2^62
  const int64_t R3 = (int64_t)((uint64_t)smulhi(R, (int64_t)R2) << 2);  // r^3 x 2^62
  const int64_t T = smulhi(R, 0x3333333333333333ll)              // r / 5
                  + (int64_t)mulhi(R2, 0x1eb851eb851eb852ull)    // + 3 r^2 / 25
                  + smulhi(R3, 0x16872b020c49ba5ell);            // + 11 r^3 / 125
  return V + ((uint64_t)smulhi((int64_t)V, T) << 2);
}

// X 2^-62 2^s rounded to the nearest double (ties to even), X != 0; 0 below
// the normal range, infinity above it
__host__ __device__ __forceinline__ double fixed62_to_double(uint64_t X, int s) {
  const int lz = clz64(X);
  const uint64_t nrm = X << lz;
  uint64_t m53 = nrm >> 11;
  const unsigned rest = (unsigned)(nrm & 0x7ffu);
  m53 += (rest > 0x400u || (rest == 0x400u && (m53 & 1u))) ? 1u : 0u;
  // value = (nrm / 2^63) 2^(1 - lz + s): biased exponent 1024 - lz + s
  const int E = 1024 - lz + s;
  const uint64_t bits = ((uint64_t)(E - 1) << 52) + m53;
  return from_bits(E <= 0 ? 0ull : E >= 2047 ? 0x7ff0000000000000ull : bits);
}

// the seed of z = u^(-1/5) for the float u
__host__ __device__ __forceinline__ float fifth_root_seed(float uf) {
#ifdef __CUDA_ARCH__
  float l, vf;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(uf));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(vf) : "f"(-0.2f * l));
  return vf;
#else
  return std::pow(uf, -0.2f);
#endif
}

__host__ __device__ __forceinline__ bool positive_normal(uint64_t b) {
  const unsigned ef = (unsigned)((b >> 52) & 0x7ff);
  return (b >> 63) == 0 && ef != 0 && ef != 0x7ff;
}

}  // namespace fx

// x^(-1/5) for positive normal x (see above)
__host__ __device__ __forceinline__ double inv_fifth_root_fx(double x) {
  using namespace fx;
  const uint64_t b = dbits(x);
  int q, k;
  float uf;
  fifth_root_split(b, &q, &k, &uf);
  const double z = fixed62_to_double(fifth_root_fixed(b, k, fifth_root_seed(uf)), -q);
  return positive_normal(b) ? z : from_bits(0x7ff8000000000000ull);
}

// x^(-21/5) = z^21 2^(-21 q) for positive normal x, the polytropic power of
// the Keller-Miksis right-hand side with gamma = 7/5, from the same z: z^5 =
// 1/u in [1/32, 1] is renormalised to [1/2, 1] (its exponent n5 kept apart),
// then squared twice and multiplied by z.  The error is about 21 times that
// of z plus six truncations: within 1.5 ulp of x^(-21/5) (host test; the FP64
// form (1/y1)^4 y1^(-1/5) it replaces rounds five times after an approximate
// reciprocal); 0 or infinity where the result leaves the normal range.
__host__ __device__ __forceinline__ double pow_m21_5_fx(double x) {
  using namespace fx;
  const uint64_t b = dbits(x);
  int q, k;
  float uf;
  fifth_root_split(b, &q, &k, &uf);
  const uint64_t Z = fifth_root_fixed(b, k, fifth_root_seed(uf));
  const uint64_t Z2 = mulhi(Z, Z) << 2;
  const uint64_t Z4 = mulhi(Z2, Z2) << 2;
  const uint64_t Z5 = mulhi(Z4, Z) << 2;        // 1/u x 2^62 in [2^57, 2^62]
  const int c5 = clz64(Z5);                     // 1 (z^5 = 1) .. 7
  const int n5 = c5 > 2 ? c5 - 2 : 0;           // 0..5
  const uint64_t Z5n = Z5 << n5;                // z^5 2^n5 in [1/2, 1]: no square overflows
  const uint64_t Z10 = mulhi(Z5n, Z5n) << 2;
  const uint64_t Z20 = mulhi(Z10, Z10) << 2;
  const uint64_t Z21 = mulhi(Z20, Z) << 2;      // z^21 2^(4 n5), >= 2^57
  const double g = fixed62_to_double(Z21, -4 * n5 - 21 * q);
  return positive_normal(b) ? g : from_bits(0x7ff8000000000000ull);
}

}  // namespace ens
