// df_host.cpp -- host build of the double-float arithmetic (df.cuh) and of
// the double-float Keller-Miksis right-hand side (km_df.cuh) for the CPU
// tests (test_df_host.py); compiled with g++ -ffp-contract=off.
#include <cmath>
#include <cstdint>
#include "km_df.cuh"
#include "valve_df.cuh"
using namespace ens::df;
extern "C" {
// C: [13][n] SoA like the library; fs, fc: forcing values; out: y2'
void accel_df(int n, const double* C, const double* fs, const double* fc, const double* y1, const double* y2, double* out) {
  for (int i = 0; i < n; ++i) {
    KmDFCoef k;
    k.load(C, n, i);
    DF a = k.accel(from_double(fs[i]), from_double(fc[i]), from_double(y1[i]), from_double(y2[i]));
    out[i] = to_double(a);
  }
}
// params [5][n] like the library (q, kappa, delta, beta, r); y [3][n]; dy [3][n]
void valve_df(int n, const double* P, const double* y, double* dy) {
  for (int i = 0; i < n; ++i) {
    ValveDF v;
    v.load(P, n, i);
    DF yy[3] = {from_double(y[i]), from_double(y[n + i]), from_double(y[2 * n + i])}, d[3];
    v.f(yy, d);
    for (int c = 0; c < 3; ++c) dy[c * n + i] = to_double(d[c]);
  }
}
void add_terms_df(int n, const double* a, const double* b, double* out) {
  for (int i = 0; i < n; ++i) out[i] = to_double(add_terms(from_double(a[i]), from_double(b[i])));
}
void sqrt_df(int n, const double* a, double* out) {
  for (int i = 0; i < n; ++i) out[i] = to_double(ens::df::sqrt(from_double(a[i])));
}
void prims(int n, const double* a, const double* b, double* out) {
  // out[6][n]: add, mul, rcp(a), inv5(a), from/to round trip of a, a - b
  for (int i = 0; i < n; ++i) {
    DF x = from_double(a[i]), y = from_double(b[i]);
    out[i] = to_double(add(x, y));
    out[n + i] = to_double(mul(x, y));
    out[2 * n + i] = to_double(rcp(x));
    out[3 * n + i] = to_double(inv_fifth_root(x));
    out[4 * n + i] = to_double(x);
    out[5 * n + i] = to_double(sub(x, y));
  }
}
// the integer double -> pair split against the FP64-subtraction form: hi and lo
// floats of both (out [4][n]: hi, lo, hi_ref, lo_ref)
void split_df(int n, const double* x, float* out) {
  for (int i = 0; i < n; ++i) {
    const DF a = from_double(x[i]), b = from_double_sub(x[i]);
    out[i] = a.hi;
    out[n + i] = a.lo;
    out[2 * n + i] = b.hi;
    out[3 * n + i] = b.lo;
  }
}
}
