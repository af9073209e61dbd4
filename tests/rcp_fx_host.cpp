// Host build of the integer-pipe reciprocal of csrc/rcp_fx.cuh for
// tests/test_rcp_fx_host.py.
#include <cstdint>

#include "rcp_fx.cuh"

extern "C" void rcp_fx_n(int64_t n, const double* d, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = ens::rcp_fx(d[i]);
}

// the refinement from the correctly rounded float seed scaled by (1 + seed_rel)
extern "C" void rcp_fx_seed(int64_t n, const double* d, double seed_rel, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    const uint64_t b = ens::fx::dbits(d[i]);
    const float mf = ens::fx::rcp_split(b);
    const float vf = (float)((1.0 / (double)mf) * (1.0 + seed_rel));
    out[i] = ens::fx::rcp_refine(b, vf);
  }
}
