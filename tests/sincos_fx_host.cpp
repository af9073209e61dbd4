// Host build of the integer-pipe sine / cosine of csrc/sincos_fx.cuh for
// tests/test_sincos_fx_host.py.
#include <cstdint>

#include "sincos_fx.cuh"

extern "C" void sincos_fx(int64_t n, const double* x, double* s, double* c) {
  for (int64_t i = 0; i < n; ++i) ens::sincos2pi_fx(x[i], &s[i], &c[i]);
}

extern "C" uint64_t turns_fx(double x) { return ens::fx::turns(ens::fx::dbits(x)); }

extern "C" double fixed_to_double_fx(uint64_t X) { return ens::fx::fixed_to_double(X); }
