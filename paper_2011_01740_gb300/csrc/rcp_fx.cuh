// rcp_fx.cuh -- 1/d with its refinement on the integer pipe.
//
// The step-size controller's error norm takes one reciprocal per component
// (the Cash-Karp kernels of Sec. 4.2 and 4.3).  An FP64
// refinement of the hardware seed (rcp.approx.f64 and a cubic Newton step)
// costs 3 FP64 instructions after the seed; this one refines a float seed in
// 64-bit fixed point, off the FP64 pipe:
//
//   1. |d| = m 2^e with m in [1, 2), so 1/|d| = (1/m) 2^(-e), 1/m in (1/2, 1];
//   2. v = the float reciprocal of m (hardware rcp.approx, about 23 correct
//      bits; the host divides);
//   3. one cubic Newton-Raphson step v (1 + s + s^2), s = 1 - m v, in fixed
//      point (values x 2^62, 64 x 64 -> high-64 products); the neglected
//      term s^3 is below 2^-66 for seeds within 2^-22 of 1/m;
//   4. rounding to the nearest double by integer normalisation, 2^(-e) and
//      the sign of d applied to the bits.
//
// Relative error below 2^-57 before the final rounding
// (tests/test_rcp_fx_host.py checks it against exact rationals and with seeds
// off by up to 2^-22).  Valid for normal d of either sign whose reciprocal is
// normal (|d| < 2^1022); zero, subnormal, infinite and NaN d give NaN.
// Branch-free.
#pragma once

#include "fixed64.cuh"

namespace ens {
namespace fx {

// the float m (24-bit truncation) of |d| = m 2^e
__host__ __device__ __forceinline__ float rcp_split(uint64_t b) {
  const unsigned fb = (127u << 23) | (unsigned)((b >> 29) & 0x7fffffu);
#ifdef __CUDA_ARCH__
  return __uint_as_float(fb);
#else
  float f;
  __builtin_memcpy(&f, &fb, 4);
  return f;
#endif
}

// the refinement of the seed vf of 1/m for the 53-bit significand mn of m
// (implicit bit set): 1/m x 2^62 in (2^61, 2^62]
__host__ __device__ __forceinline__ uint64_t rcp_fixed(uint64_t mn, float vf) {
#ifdef __CUDA_ARCH__
  const unsigned vb = __float_as_uint(vf);
#else
  unsigned vb;
  __builtin_memcpy(&vb, &vf, 4);
#endif
  // v x 2^62 from the float's bits (exact)
  const int ev = (int)((vb >> 23) & 0xffu) - 127;
  const uint64_t V = (uint64_t)((vb & 0x7fffffu) | 0x800000u) << ((39 + ev) & 63);
  const uint64_t M = mn << 10;                                        // m x 2^62
  const int64_t S = (int64_t)((1ull << 62) - (mulhi(M, V) << 2));    // s = 1 - m v, x 2^62
  const int64_t S2 = (int64_t)((uint64_t)smulhi(S, S) << 2);          // s^2 x 2^62
  return V + ((uint64_t)smulhi((int64_t)V, S + S2) << 2);
}

// the float seed of 1/m
__host__ __device__ __forceinline__ float rcp_seed(float mf) {
#ifdef __CUDA_ARCH__
  float vf;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(vf) : "f"(mf));
  return vf;
#else
  return 1.0f / mf;
#endif
}

// the refinement of the seed vf of 1/m and the result (1/m) 2^(-e) with the
// sign of d, as a double
__host__ __device__ __forceinline__ double rcp_refine(uint64_t b, float vf) {
  const int e = (int)((b >> 52) & 0x7ff) - 1023;
  const uint64_t W = rcp_fixed((b & 0x000fffffffffffffull) | 0x0010000000000000ull, vf);
  const int lz = clz64(W);
  const uint64_t nrm = W << lz;
  uint64_t m53 = nrm >> 11;
  const unsigned rest = (unsigned)(nrm & 0x7ffu);
  m53 += (rest > 0x400u || (rest == 0x400u && (m53 & 1u))) ? 1u : 0u;
  // value = (nrm / 2^63) 2^(1 - lz - e): biased exponent 1024 - lz - e
  return from_bits((((uint64_t)(1023 - lz - e) << 52) + m53) | (b & 0x8000000000000000ull));
}

}  // namespace fx

// 1/d (see above)
__host__ __device__ __forceinline__ double rcp_fx(double d) {
  using namespace fx;
  const uint64_t b = dbits(d);
  const double r = rcp_refine(b, rcp_seed(rcp_split(b)));
  const unsigned ef = (unsigned)((b >> 52) & 0x7ff);
  const bool ok = ef != 0 && ef < 0x7fd;  // normal, and 1/d normal (|d| < 2^1022)
  return ok ? r : from_bits(0x7ff8000000000000ull);
}

}  // namespace ens
