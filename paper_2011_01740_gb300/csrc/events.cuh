// events.cuh -- location of the falling event functions of event mode
// (Sec. 4.3): the root estimate that shortens an overshooting trial.
#pragma once

#include "common.cuh"

namespace ens {

// Root estimate of a falling event function over a trial of length h, as a
// fraction of h: g0 > 0 with slope d0 at the start (from k1), g1 < 0 at the
// end.  The quadratic g0 + B x + A x^2 (B = d0 h, A = g1 - g0 - B) changes
// sign once on (0, 1), at x = 2 g0 / (-B + sqrt(B^2 - 4 A g0)) for either sign
// of A.  It is exact for a constant second derivative, so retries converge at
// grazing impacts, where a chord from the fixed start of the retried step
// closes in only linearly.  The chord g0 / (g0 - g1) stands in if rounding
// takes the root out of (0, 1).
__device__ __forceinline__ double event_frac(double g0, double d0, double g1, double h) {
  const double B = d0 * h;
  const double A = g1 - g0 - B;
  const double D = fma(B, B, -4.0 * A * g0);
  const double chord = g0 / (g0 - g1);
  if (!(D >= 0.0)) return chord;
  const double den = sqrt(D) - B;
  const double x = 2.0 * g0 / den;
  return (den > 0.0 && x > 0.0 && x < 1.0) ? x : chord;
}

}  // namespace ens
