// Host build of the integer-pipe square root of csrc/sqrt_fx.cuh for
// tests/test_sqrt_fx_host.py.
#include <cmath>
#include <cstdint>

#include "sqrt_fx.cuh"

extern "C" void sqrt_fx_n(int64_t n, const double* x, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = ens::sqrt_fx(x[i]);
}

// the refinement of a seed off by (1 + seed_rel), positive normal x only
extern "C" void sqrt_fx_seed(int64_t n, const double* x, double seed_rel, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t b = ens::fx::dbits(x[i]);
    const int e = (int)((b >> 52) & 0x7ff) - 1023;
    const uint64_t mn = (b & 0x000fffffffffffffull) | 0x0010000000000000ull;
    const int k = e & 1, q = (e - k) / 2;
    const double u = std::ldexp((double)mn, k - 52);
    const float vf = (float)((1.0 / std::sqrt(u)) * (1.0 + seed_rel));
    out[i] = ens::fx::fixed61_to_double(ens::fx::sqrt_fixed(mn, k, vf), q);
  }
}
