// km_df.cuh -- the dimensionless Keller-Miksis right-hand side (Sec. 4.2,
// Eqs. dimensionless_system1-2, numerator, denominator) in double-float
// arithmetic (df.cuh), for the double-float Cash-Karp kernel (df64.cu).
//
// The formula and its operation order are those of KellerMiksis::accel in
// rhs.cuh with the exponent C10 = 21/5 (one reciprocal w = 1/(y1 D) for both
// 1/y1 = D w and 1/D; (1/y1)^(21/5) = (1/y1)^4 y1^(-1/5)); only the arithmetic
// differs.  The forcing sums depend on tau alone and stay in FP64 (the
// sincos2pi_poly of rhs.cuh), split into pairs once per stage.
#pragma once

#include "df.cuh"

namespace ens {
namespace df {

struct KmDFCoef {
  DF C0, C1, C2, C3, C4, C9, C4C9, C9h;
  __host__ __device__ __forceinline__ void load(const double* P, int64_t n, int64_t i) {
    C0 = from_double(P[i]);
    C1 = from_double(P[n + i]);
    C2 = from_double(P[2 * n + i]);
    C3 = from_double(P[3 * n + i]);
    C4 = from_double(P[4 * n + i]);
    C9 = from_double(P[9 * n + i]);
    C4C9 = from_double(P[4 * n + i] * P[9 * n + i]);
    C9h = from_double(-0.5 * P[9 * n + i]);
  }
  // y2' = N_KM / D_KM with the forcing terms fs = C5 sin + C6 sin(...) and
  // fc = C7 cos + C8 cos(...) given as pairs
  __host__ __device__ __forceinline__ DF accel(DF fs, DF fc, DF y1, DF y2) const {
    const DF c9y2 = mul(C9, y2);
    const DF D = add(mul(y1, add(neg(c9y2), 1.0f)), C4C9);    // y1 (1 - C9 y2) + C4 C9
    const DF w = rcp(mul(y1, D));
    const DF rx = mul(D, w);                                  // 1 / y1
    const DF rx2 = mul(rx, rx);
    const DF g = mul(mul(rx2, rx2), inv_fifth_root(y1));      // (1/y1)^(21/5)
    const DF one_c9y2 = add(c9y2, 1.0f);
    DF N = mul(add(mul(C1, y2), C0), g);
    N = sub(N, mul(C2, one_c9y2));
    N = sub(N, mul(add(mul(C4, y2), C3), rx));
    N = sub(N, mul(add(mul(C9h, y2), 1.5f), mul(y2, y2)));   // (1 - C9 y2 / 3) (3/2) y2^2
    N = sub(N, mul(fs, one_c9y2));
    N = sub(N, mul(y1, fc));
    return mul(N, mul(y1, w));                                // N / D
  }
};

}  // namespace df
}  // namespace ens
