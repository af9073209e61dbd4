// sqrt_fx.cuh -- sqrt(x) with its refinement on the integer pipe.
//
// The pressure-relief-valve right-hand side takes sqrt(y3) in every
// evaluation (Sec. 4.3, y3' = beta (q - y1 sqrt(y3))).  An FP64 refinement of
// the hardware reciprocal-square-root seed costs 6 FP64 instructions; this
// one does the refinement in 64-bit fixed point, off the FP64 pipe:
//
//   1. x = m 2^e with m in [1, 2) (subnormal x normalised first); e = 2 q + k
//      with k in {0, 1}, so sqrt(x) = sqrt(u) 2^q with u = m 2^k in [1, 4);
//   2. a float seed v of z = u^(-1/2) in (1/2, 1] (hardware rsqrt.approx,
//      about 23 correct bits; the host takes the float root);
//   3. one step of the binomial series of (1 - r)^(-1/2) with the residual
//      r = 1 - u v^2:  z = v (1 + r/2 + 3 r^2/8 + 5 r^3/16), in fixed point
//      (values x 2^62, 64 x 64 -> high-64 products); the neglected term
//      35 r^4 / 128 is below 2^-70 for seeds within 2^-19 of z;
//   4. sqrt(u) = u z, rounded to the nearest double by integer
//      normalisation, 2^q applied through the exponent field.
//
// The result is within half an ulp plus 2^-58 relative of sqrt(x), exact
// for perfect squares (tests/test_sqrt_fx_host.py checks it against 60-digit
// values, exact squares, subnormal x, and seeds off by up to 2^-19).  +0 and -0
// give themselves, negative x and NaN give NaN, +infinity gives +infinity.
// Branch-free.
#pragma once

#include <cmath>

#include "fixed64.cuh"

namespace ens {
namespace fx {

// the refinement of the seed vf of u^(-1/2), u = m 2^k with m given as the
// 53-bit integer mn (implicit bit set), and sqrt(u) x 2^61 in [2^61, 2^62)
__host__ __device__ __forceinline__ uint64_t sqrt_fixed(uint64_t mn, int k, float vf) {
#ifdef __CUDA_ARCH__
  const unsigned vb = __float_as_uint(vf);
#else
  unsigned vb;
  __builtin_memcpy(&vb, &vf, 4);
#endif
  const int ev = (int)((vb >> 23) & 0xffu) - 127;
  const uint64_t V = (uint64_t)((vb & 0x7fffffu) | 0x800000u) << ((39 + ev) & 63);  // v x 2^62
  const uint64_t M = mn << 11;                  // m x 2^63
  const uint64_t V2 = mulhi(V, V) << 2;         // v^2 x 2^62
  const uint64_t P = mulhi(V2, M) << (1 + k);   // u v^2 x 2^62, close to 2^62
  const int64_t R = (int64_t)((1ull << 62) - P);  // r x 2^62
  const uint64_t Ra = R < 0 ? (uint64_t)0 - (uint64_t)R : (uint64_t)R;
  const uint64_t R2 = mulhi(Ra, Ra) << 2;                               // r^2 x 2^62
  const int64_t R3 = (int64_t)((uint64_t)smulhi(R, (int64_t)R2) << 2);  // r^3 x 2^62
  const int64_t T = (R >> 1) + (int64_t)((R2 >> 2) + (R2 >> 3))         // r/2 + 3 r^2/8
                  + ((R3 >> 2) + (R3 >> 4));                            // + 5 r^3/16
  const uint64_t Z = V + ((uint64_t)smulhi((int64_t)V, T) << 2);        // u^(-1/2) x 2^62
  return mulhi(Z, M) << k;                                              // u^(1/2) x 2^61
}

// X 2^-61 2^s rounded to the nearest double (ties to even), X in
// [2^61, 2^63): the exponent comes from s and the one leading-zero test
__host__ __device__ __forceinline__ double fixed61_to_double(uint64_t X, int s) {
  const int lz = clz64(X);  // 1 or 2
  const uint64_t nrm = X << lz;
  uint64_t m53 = nrm >> 11;
  const unsigned rest = (unsigned)(nrm & 0x7ffu);
  m53 += (rest > 0x400u || (rest == 0x400u && (m53 & 1u))) ? 1u : 0u;
  // value = (nrm / 2^63) 2^(2 - lz + s): biased exponent 1025 - lz + s
  return from_bits(((uint64_t)(1024 - lz + s) << 52) + m53);
}

__host__ __device__ __forceinline__ float rsqrt_seed(float uf) {
#ifdef __CUDA_ARCH__
  float v;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(v) : "f"(uf));
  return v;
#else
  return 1.0f / std::sqrt(uf);
#endif
}

}  // namespace fx

// sqrt(x) (see above)
__host__ __device__ __forceinline__ double sqrt_fx(double x) {
  using namespace fx;
  const uint64_t b = dbits(x);
  const int ef = (int)((b >> 52) & 0x7ff);
  const uint64_t frac = b & 0x000fffffffffffffull;
  // normal: m = 2^52 + frac, e = ef - 1023; subnormal: frac shifted up to bit 52
  const int sh = ef == 0 ? (frac == 0 ? 0 : clz64(frac) - 11) : 0;
  const uint64_t mn = ef == 0 ? (frac << sh) : (frac | 0x0010000000000000ull);
  const int e = ef == 0 ? -1022 - sh : ef - 1023;
  const int k = e & 1;
  const int q = (e - k) / 2;  // exact: e - k is even
  const unsigned fb = ((unsigned)(127 + k) << 23) | (unsigned)((mn >> 29) & 0x7fffffu);
#ifdef __CUDA_ARCH__
  const float uf = __uint_as_float(fb);
#else
  float uf;
  __builtin_memcpy(&uf, &fb, 4);
#endif
  const double r = fixed61_to_double(sqrt_fixed(mn, k, rsqrt_seed(uf)), q);
  const bool zero = (b << 1) == 0;
  const bool neg = (b >> 63) != 0;
  const bool inf_or_nan = ef == 0x7ff;
  return zero ? x
       : (neg || (inf_or_nan && frac != 0)) ? from_bits(0x7ff8000000000000ull)
       : inf_or_nan ? x
       : r;
}

}  // namespace ens
