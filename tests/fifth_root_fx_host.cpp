// Host build of the integer-pipe x^(-1/5) of csrc/fifth_root_fx.cuh for
// tests/test_fifth_root_fx_host.py.
#include <cmath>
#include <cstdint>

#include "fifth_root_fx.cuh"

extern "C" void fifth_root_fx(int64_t n, const double* x, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = ens::inv_fifth_root_fx(x[i]);
}

// the refinement from the float power seed scaled by (1 + seed_rel)
extern "C" void fifth_root_fx_seed(int64_t n, const double* x, double seed_rel, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t b = ens::fx::dbits(x[i]);
    int q, k;
    float uf;
    ens::fx::fifth_root_split(b, &q, &k, &uf);
    const float vf = (float)(std::pow((double)uf, -0.2) * (1.0 + seed_rel));
    out[i] = ens::fx::fixed62_to_double(ens::fx::fifth_root_fixed(b, k, vf), -q);
  }
}

extern "C" void pow_m21_5_fx_n(int64_t n, const double* x, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = ens::pow_m21_5_fx(x[i]);
}
