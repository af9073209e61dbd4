// sincos_fx.cuh -- sine and cosine of 2 pi x on the integer pipe.
//
// The Keller-Miksis forcing (Sec. 4.2) needs sin and cos of 2 pi tau at five
// stage times of every trial.  On GB300 the FP64 pipe retires 2 lanes per
// clock per SM while the integer pipe retires 64, so this evaluation works in
// 64-bit fixed point and leaves the FP64 pipe to the rest of the step:
//
//   1. x in turns: F = round(x 2^64) mod 2^64 from the significand and
//      exponent bits of x (exact up to the final rounding, at any |x|);
//   2. q = the nearest quarter turn, r = x - q/4 with |r| <= 1/8 turn, held
//      as w = 4 r in [-1/2, 1/2) (value x 2^64);
//   3. the Taylor series of sin(pi w / 2) and cos(pi w / 2) by Horner's rule
//      in v = w^2 on unsigned 64-bit values with 64 x 64 -> high-64
//      products; coefficients and their bounds from gen_sincos_fx.py;
//   4. the quarter-turn identities (sin, cos)(q pi/2 + a) = (s, c), (c, -s),
//      (-s, -c), (-c, s), and the fixed-point magnitudes rounded to the
//      nearest double by integer normalisation.
//
// Absolute error of both results below 1e-18 before the final rounding
// (tests/test_sincos_fx_host.py checks it against 50-digit arithmetic), so the
// doubles are the correctly rounded values except within 1e-18 of a rounding
// boundary.  The bound is absolute: a sine of magnitude 1e-6 keeps about 12
// significant digits, which is what a forcing term added to terms of order
// one needs.  NaN and infinite x give NaN.
//
// The code has selects, not branches, so that a trial's right-hand sides and
// forcing evaluations stay one basic block the compiler can interleave (the
// integer work then fills the FP64 pipe's gaps).  Every function is
// __host__ __device__ so that the host can test it.
#pragma once

#include "fixed64.cuh"

namespace ens {
namespace fx {

// round(x 2^64) mod 2^64 (ties up) for finite x: x = m 2^(e-52) with the
// 53-bit integer m, so x 2^64 = m 2^s, s = e + 12; bits at or above 2^64 are
// whole turns and drop out.  |x| below 2^-76 and subnormals give 0.
__host__ __device__ __forceinline__ uint64_t turns(uint64_t b) {
  const int ef = (int)((b >> 52) & 0x7ff);
  const uint64_t m = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
  const int s = ef - 1011;
  const int rs = (-s) & 63;  // right shift, 1..63 where used
  const uint64_t left = m << (s & 63);
  const uint64_t right = (m >> rs) + ((m >> ((rs - 1) & 63)) & 1u);
  uint64_t F = s >= 0 ? left : right;
  F = (ef == 0 || s >= 64 || s <= -64) ? 0ull : F;
  return (b >> 63) ? (uint64_t)0 - F : F;
}

// X 2^-64 rounded to the nearest double (ties to even), X != 0.  With
// nrm = X 2^lz in [2^63, 2^64) the value is (nrm / 2^63) 2^(-1-lz), biased
// exponent 1022 - lz; adding the 53-bit m (implicit bit included) to the
// exponent field minus one lets a rounding carry step the exponent.
__host__ __device__ __forceinline__ double fixed_to_double(uint64_t X) {
  const int lz = clz64(X);
  const uint64_t nrm = X << lz;
  uint64_t m = nrm >> 11;
  const unsigned rest = (unsigned)(nrm & 0x7ffu);
  m += (rest > 0x400u || (rest == 0x400u && (m & 1u))) ? 1u : 0u;
  return from_bits(((uint64_t)(1021 - lz) << 52) + m);
}

// Taylor coefficients S_k, Q_k, value x 2^64 (gen_sincos_fx.py)
__host__ __device__ __forceinline__ constexpr uint64_t kS(int k) {
  return k == 0 ? 0xc90fdaa22168c235ull : k == 1 ? 0x52aef39896f94afbull : k == 2 ? 0x0a335e33bad570e9ull
       : k == 3 ? 0x009969667315ec2eull : k == 4 ? 0x000541e0d21fb9e0ull : k == 5 ? 0x00001e3074fde887ull
       : k == 6 ? 0x0000007a3d0d3406ull : k == 7 ? 0x000000016fadb9f1ull : k == 8 ? 0x000000000355d865ull
       : 0x0000000000062901ull;
}
__host__ __device__ __forceinline__ constexpr uint64_t kQ(int k) {
  return k == 0 ? 0x9de9e64df22ef2d2ull : k == 1 ? 0x20783e1036b58767ull : k == 2 ? 0x02aba78fc797ff40ull
       : k == 3 ? 0x001e1f506891babbull : k == 4 ? 0x0000d368f9510254ull : k == 5 ? 0x000003f3a7146ec8ull
       : k == 6 ? 0x0000000db7127a26ull : k == 7 ? 0x000000002418c586ull : 0x00000000004a8316ull;
}

}  // namespace fx

// sn = sin(2 pi x), cs = cos(2 pi x)
__host__ __device__ __forceinline__ void sincos2pi_fx(double x, double* sn, double* cs) {
  using namespace fx;
  const uint64_t b = dbits(x);
  const bool finite = ((b >> 52) & 0x7ff) != 0x7ff;
  const uint64_t F = turns(b) + (1ull << 61);  // + 1/8 turn
  const unsigned q = (unsigned)(F >> 62);      // nearest quarter turn
  const uint64_t W = ((F & 0x3fffffffffffffffull) - (1ull << 61)) << 2;  // w 2^64, two's complement
  const bool neg = (W >> 63) != 0;
  const uint64_t A = neg ? (uint64_t)0 - W : W;  // |w| 2^64 <= 2^63
  const uint64_t V = mulhi(A, A);                // w^2 2^64 <= 2^62
  uint64_t p = kS(9);
#pragma unroll
  for (int k = 8; k >= 0; --k) p = kS(k) - mulhi(V, p);
  const uint64_t sa = mulhi(A, p) << 1;  // |sin(pi w / 2)| 2^64 <= 0.7072 2^64
  uint64_t r = kQ(8);
#pragma unroll
  for (int k = 7; k >= 0; --k) r = kQ(k) - mulhi(V, r);
  const uint64_t cx = mulhi(V, r) << 1;  // (1 - cos(pi w / 2)) 2^64
  const uint64_t sgn = neg ? 0x8000000000000000ull : 0ull;
  const uint64_t sbits = sa == 0 ? sgn : (dbits(fixed_to_double(sa)) | sgn);
  const uint64_t cbits = cx == 0 ? 0x3ff0000000000000ull : dbits(fixed_to_double((uint64_t)0 - cx));
  // quarter turns: (sin, cos)(q pi/2 + a) = (s, c), (c, -s), (-s, -c), (-c, s)
  const uint64_t ab = (q & 1u) ? cbits : sbits;
  const uint64_t bb = (q & 1u) ? sbits : cbits;
  const uint64_t fa = (uint64_t)(q & 2u) << 62, fb = (uint64_t)((q + 1u) & 2u) << 62;
  *sn = from_bits(finite ? (ab ^ fa) : 0x7ff8000000000000ull);  // NaN for NaN or infinite x
  *cs = from_bits(finite ? (bb ^ fb) : 0x7ff8000000000000ull);
}

}  // namespace ens
