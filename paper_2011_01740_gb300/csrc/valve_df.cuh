// valve_df.cuh -- the pressure relief valve right-hand side (Sec. 4.3, Eqs.
// pressure_relief_valve_1-3) in double-float arithmetic (df.cuh):
//   y1' = y2,  y2' = -kappa y2 - (y1 + delta) + y3,  y3' = beta (q - y1 sqrt(y3)),
// with sqrt of max(y3, 0) (y3 >= 0 for q > 0; the clamp keeps a rounding
// excursion below zero from producing a NaN).  __host__ __device__, so the
// CPU tests check it against the float64 oracle.
#pragma once

#include "df.cuh"

namespace ens {
namespace df {

struct ValveDF {
  DF q, mkappa, delta, beta;  // mkappa = -kappa
  double qd, deltad, betad, r;
  __host__ __device__ __forceinline__ void load(const double* P, int64_t n, int64_t i) {
    qd = P[i];
    mkappa = from_double(-P[n + i]);
    deltad = P[2 * n + i];
    betad = P[3 * n + i];
    r = P[4 * n + i];
    q = from_double(qd);
    delta = from_double(deltad);
    beta = from_double(betad);
  }
  __host__ __device__ __forceinline__ void f(const DF* y, DF* dy) const {
    dy[0] = y[1];
    dy[1] = add(sub(y[2], add(y[0], delta)), mul(mkappa, y[1]));
    dy[2] = mul(sub(q, mul(y[0], sqrt(y[2]))), beta);
  }
};

}  // namespace df
}  // namespace ens
