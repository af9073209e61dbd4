// rhs.cuh -- right-hand sides of the built-in systems as inlined device code.
//
// Each system is a struct with the state dimension, a parameter loader (from
// the SoA parameter array into registers) and the RHS evaluation.  Two
// arithmetic flavours exist for the fixed-step systems:
//   - fast   : fused multiply-add wherever it shortens the FP64 pipe work;
//   - strict : IEEE double with no contraction, operations in the order the
//              paper writes the equation (bit-reproducible against a plain
//              C evaluation of the same formula).
#pragma once

#include "common.cuh"
#include "fifth_root_fx.cuh"
#include "sincos_fx.cuh"
#include "sqrt_fx.cuh"

namespace ens {

// Double operations that the compiler may not fuse (strict flavour).
__device__ __forceinline__ double sadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double ssub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double smul(double a, double b) { return __dmul_rn(a, b); }

// ---------------------------------------------------------------------------
// x' = x^2 - p   (Sec. 3, Eq. exemplary_system)
// ---------------------------------------------------------------------------
struct X2P {
  static constexpr int kDim = 1;
  static constexpr int kPar = 1;
  static constexpr int kPhaseRows = 0;  // no per-phase hook
  double p;
  __device__ __forceinline__ void load(const double* P, int64_t n, int64_t i) { p = P[i]; }
  template <bool STRICT>
  __device__ __forceinline__ void f(double t, const double* y, double* dy) const {
    (void)t;
    if (STRICT) dy[0] = ssub(smul(y[0], y[0]), p);
    else dy[0] = fma(y[0], y[0], -p);
  }
};

// ---------------------------------------------------------------------------
// Lorenz (Sec. 4.1, Eqs. Lorenz1-3): x1' = sigma (x2 - x1),
// x2' = rho x1 - x2 - x1 x3, x3' = x1 x2 - b x3.
// ---------------------------------------------------------------------------
struct Lorenz {
  static constexpr int kDim = 3;
  static constexpr int kPar = 3;
  static constexpr int kPhaseRows = 0;
  double rho, sigma, b;
  __device__ __forceinline__ void load(const double* P, int64_t n, int64_t i) {
    rho = P[i];
    sigma = P[n + i];
    b = P[2 * n + i];
  }
  template <bool STRICT>
  __device__ __forceinline__ void f(double t, const double* y, double* dy) const {
    (void)t;
    if (STRICT) {
      dy[0] = smul(sigma, ssub(y[1], y[0]));
      dy[1] = ssub(ssub(smul(rho, y[0]), y[1]), smul(y[0], y[2]));
      dy[2] = ssub(smul(y[0], y[1]), smul(b, y[2]));
    } else {
      dy[0] = sigma * (y[1] - y[0]);
      dy[1] = fma(-y[0], y[2], fma(rho, y[0], -y[1]));
      dy[2] = fma(y[0], y[1], -b * y[2]);
    }
  }
};

// 1/d to about 1 ulp: the hardware reciprocal approximation (PTX
// rcp.approx.ftz.f64, on the leading bits of d) refined by one cubic
// Newton-Raphson step, v (1 + e + e^2) with e = 1 - d v, which cubes the
// seed's relative error.  Not correctly rounded; 3 FP64 instructions after
// the seed.  Zero, infinite and subnormal d give NaN or garbage: callers use it
// on values bounded away from those.  The right-hand side keeps this FP64 form
// although rcp_fx (rcp_fx.cuh) moves the step to the integer pipe: the
// reciprocal sits on the chain of every stage, and there the fixed-point
// step's latency cost the tail-bound 362 x 362 sweep 6 % (2.48 s against
// 2.34 s) for 4 % on the throughput-bound 1024 x 1024 grid.  The error norm,
// off that chain, takes rcp_fx.
__device__ __forceinline__ double rcp_nr(double d) {
  double v;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(v) : "d"(d));
  const double e = fma(-d, v, 1.0);
  return fma(fma(e, e, e), v, v);
}


// sin(2 pi x) and cos(2 pi x) together for |x| < 2^49, in FP64 arithmetic.
// The argument is split exactly as x = k/4 + r with k the nearest integer to
// 4x (the 1.5 * 2^52 shift) and |r| <= 1/8 (x - k/4 is exact);
// sin(2 pi r) = r P(r^2) and cos(2 pi r) = 1 + r^2 Q(r^2) with P, Q of degree
// 6 from a weighted minimax fit (Remez exchange) on r^2 in [0, 1/64]:
// relative error of P below 5e-17 and absolute error of 1 + r^2 Q below 2e-17
// after rounding the coefficients to double (`gen_sincos2pi.py` next to this
// file recomputes them).  The k mod 4 quarter turns then select and negate
// (the sign flips are integer XORs on the high word).  18 FP64 instructions.
// The double-float kernels use it: their FP32 and integer pipes carry the
// step, so the FP64 pipe is their spare one.  The FP64 kernels take the
// integer-pipe sincos2pi_fx (sincos_fx.cuh) instead.
__device__ __forceinline__ void sincos2pi_poly(double x, double* sn, double* cs) {
  const double shift = 6755399441055744.0;  // 1.5 * 2^52
  const double t = fma(x, 4.0, shift);
  const int q = __double2loint(t);
  const double k = t - shift;
  const double r = fma(k, -0.25, x);
  const double u = r * r;
  double p = 0x1.e3eed5d16d705p+1;
  p = fma(p, u, -0x1.e30063a031f57p+3);
  p = fma(p, u, 0x1.50782fca38c0ep+5);
  p = fma(p, u, -0x1.32d2cce2d5361p+6);
  p = fma(p, u, 0x1.466bc67758700p+6);
  p = fma(p, u, -0x1.4abbce625be41p+5);
  p = fma(p, u, 0x1.921fb54442d18p+2);
  const double s = r * p;
  double c = -0x1.b26fe85b71b00p+0;
  c = fma(c, u, 0x1.f9cc6acfc67d7p+2);
  c = fma(c, u, -0x1.a6d1ecb740183p+4);
  c = fma(c, u, 0x1.e1f50683b42cap+5);
  c = fma(c, u, -0x1.55d3c7e3c95bcp+6);
  c = fma(c, u, 0x1.03c1f081b5ab0p+6);
  c = fma(c, u, -0x1.3bd3cc9be45dep+4);
  c = fma(c, u, 1.0);
  // quarter turns: (sin, cos) of q pi/2 + a = (s, c), (c, -s), (-s, -c), (-c, s)
  const double a = (q & 1) ? c : s;
  const double b = (q & 1) ? s : c;
  const unsigned fa = (unsigned)(q & 2) << 30, fb = (unsigned)((q + 1) & 2) << 30;
  *sn = __hiloint2double((int)((unsigned)__double2hiint(a) ^ fa), __double2loint(a));
  *cs = __hiloint2double((int)((unsigned)__double2hiint(b) ^ fb), __double2loint(b));
}

// (1/y1)^(21/5) for the Keller-Miksis polytropic term with gamma = 7/5: in
// fixed point on the integer pipe from y1 alone (fifth_root_fx.cuh).  rx =
// 1/y1 is not needed here; the tangent system's dual-number overload
// (dual.cuh) takes its derivative from it.
__device__ __forceinline__ double polytropic_215(double y1, double rx) {
  (void)rx;
  return pow_m21_5_fx(y1);
}

// Right-hand sides used by the adaptive kernels expose their time-only part
// separately: drive(t) evaluates it, fd(d, t, y, dy) the rest.  A Cash-Karp
// trial ends at t + h, where the next trial's first stage starts, so the
// kernels carry that stage's drive over instead of evaluating it twice.
// Autonomous systems use NoDrive.
struct NoDrive {};

// ---------------------------------------------------------------------------
// Dimensionless Keller-Miksis (Sec. 4.2, Eqs. dimensionless_system1-2,
// numerator, denominator):
//   y1' = y2,   y2' = N_KM / D_KM,
//   N_KM = (C0 + C1 y2) (1/y1)^C10 - C2 (1 + C9 y2) - C3/y1 - C4 y2/y1
//          - (1 - C9 y2 / 3) (3/2) y2^2
//          - (C5 sin 2 pi tau + C6 sin(2 pi C11 tau + C12)) (1 + C9 y2)
//          - y1 (C7 cos 2 pi tau + C8 cos(2 pi C11 tau + C12)),
//   D_KM = y1 - C9 y1 y2 + C4 C9.
// Following the paper's cost notes (Sec. 3.3): one reciprocal (rcp_nr)
// yields both 1/y1 (shared by the three 1/y1 terms) and 1/D_KM, sine and
// cosine of one angle come from one evaluation
// (sincos2pi_fx, on the integer pipe), and the rational power is not sent
// through pow(): with EXP215 the exponent C10 = 3 gamma = 4.2 = 21/5
// (gamma = 1.4) is applied as y1^(-21/5) = (y1^(-1/5))^21 in fixed point
// (polytropic_215; the host selects this form when every system's C10 lies
// within 4 ulp of 21/5; otherwise pow() is used).
// The two forcing sums depend on tau alone and form the Drive.
// DUAL selects the second driving frequency (C6, C8 != 0).
// ---------------------------------------------------------------------------
template <bool DUAL, bool EXP215 = false>
struct KellerMiksis {
  static constexpr int kDim = 2;
  static constexpr int kPar = 13;
  static constexpr int kPhaseRows = 0;
  double C0, C1, C2, C3, C4, C5, C6, C7, C8, C9, C10, C11, C12f, C4C9, C9h;
  struct Drive {
    double fs, fc;  // C5 sin 2 pi tau + C6 sin(...), C7 cos 2 pi tau + C8 cos(...)
  };
  __device__ __forceinline__ void load(const double* P, int64_t n, int64_t i) {
    C0 = P[i];
    C1 = P[n + i];
    C2 = P[2 * n + i];
    C3 = P[3 * n + i];
    C4 = P[4 * n + i];
    C5 = P[5 * n + i];
    C6 = P[6 * n + i];
    C7 = P[7 * n + i];
    C8 = P[8 * n + i];
    C9 = P[9 * n + i];
    C10 = P[10 * n + i];
    C11 = P[11 * n + i];
    C12f = P[12 * n + i] * (0.5 / 3.141592653589793238462643383279502884);  // C12 in turns
    C4C9 = C4 * C9;
    C9h = -0.5 * C9;
  }
  __device__ __forceinline__ Drive drive(double tau) const {
    double s1, c1;
    sincos2pi_fx(tau, &s1, &c1);
    Drive d{C5 * s1, C7 * c1};
    if (DUAL) {
      double s2, c2;
      sincos2pi_fx(fma(C11, tau, C12f), &s2, &c2);
      d.fs = fma(C6, s2, d.fs);
      d.fc = fma(C8, c2, d.fc);
    }
    return d;
  }
  // y2' = N_KM / D_KM for a scalar type T: double, or the Dual of dual.cuh
  // (the same operations then also carry a directional derivative).
  template <class T>
  __device__ __forceinline__ T accel(const Drive& d, T y1, T y2) const {
    // one reciprocal serves both 1/y1 and 1/D: w = 1 / (y1 D), 1/y1 = D w, N/D = N y1 w;
    // D = y1 (1 - C9 y2) + C4 C9
    const T D = fma(y1, fma(-C9, y2, 1.0), C4C9);
    const T w = rcp_nr(y1 * D);
    const T rx = D * w;
    T g;
    if (EXP215) {
      g = polytropic_215(y1, rx);
    } else {
      g = pow(rx, C10);
    }
    const T one_c9y2 = fma(C9, y2, 1.0);
    T N = fma(C1, y2, C0) * g;
    N = fma(-C2, one_c9y2, N);
    N = fma(-fma(C4, y2, C3), rx, N);
    // - (1 - C9 y2 / 3) * 1.5 * y2^2 = - (1.5 - 0.5 C9 y2) y2^2
    N = fma(-fma(C9h, y2, 1.5), y2 * y2, N);
    N = fma(-d.fs, one_c9y2, N);
    N = fma(-y1, d.fc, N);
    return N * (y1 * w);
  }
  __device__ __forceinline__ void fd(const Drive& d, double tau, const double* y, double* dy) const {
    (void)tau;
    dy[0] = y[1];
    dy[1] = accel<double>(d, y[0], y[1]);
  }
  __device__ __forceinline__ void f(double tau, const double* y, double* dy) const {
    fd(drive(tau), tau, y, dy);
  }
};

// ---------------------------------------------------------------------------
// Pressure relief valve (Sec. 4.3, Eqs. pressure_relief_valve_1-3):
//   y1' = y2, y2' = -kappa y2 - (y1 + delta) + y3, y3' = beta (q - y1 sqrt(y3)).
// sqrt is taken of max(y3, 0): y3 >= 0 for q > 0, the clamp only keeps a
// rounding excursion from producing a NaN; it is sqrt_fx (refined in fixed
// point on the integer pipe, within half an ulp plus 2^-58).  The
// clamp tests the sign bit on the integer pipe (negative values and -0 give
// +0), which spares the FP64 pipe a min / max per evaluation.
// ---------------------------------------------------------------------------
struct ReliefValve {
  static constexpr int kDim = 3;
  static constexpr int kPar = 5;
  static constexpr int kPhaseRows = 0;
  double q, kappa, delta, beta, r;
  __device__ __forceinline__ void load(const double* P, int64_t n, int64_t i) {
    q = P[i];
    kappa = P[n + i];
    delta = P[2 * n + i];
    beta = P[3 * n + i];
    r = P[4 * n + i];
  }
  __device__ __forceinline__ void f(double t, const double* y, double* dy) const {
    (void)t;
    dy[0] = y[1];
    dy[1] = fma(-kappa, y[1], y[2] - (y[0] + delta));
    const double y3 = __double2hiint(y[2]) < 0 ? 0.0 : y[2];
    dy[2] = beta * fma(-y[0], sqrt_fx(y3), q);
  }
  using Drive = NoDrive;
  __device__ __forceinline__ Drive drive(double) const { return {}; }
  __device__ __forceinline__ void fd(const Drive&, double t, const double* y, double* dy) const { f(t, y, dy); }
};

}  // namespace ens
