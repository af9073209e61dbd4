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

// x^(-1/5) for a positive double inside the float range.  Float seed from the
// hardware base-2 logarithm and exponential (PTX lg2.approx / ex2.approx,
// about 22 correct bits), then one third-order step of the binomial series
// of (1 - r)^(-1/5) with the residual r = 1 - x v^5:
//   v <- v (1 + r / 5 + 3 r^2 / 25).
// The neglected r^3 term is below 2^-60 for the seed's accuracy, so the result
// is within about 2 ulp of x^(-1/5).  Cost: 7 FP64 instructions and two
// conversions, against roughly a hundred FP64 instructions for pow().
__device__ __forceinline__ double inv_fifth_root(double x) {
  const float xf = __double2float_rn(x);
  float l, vf;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(xf));
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(vf) : "f"(-0.2f * l));
  const double v = (double)vf;
  const double v2 = v * v;
  const double r = fma(-x, (v2 * v2) * v, 1.0);
  return fma(v * fma(0.12, r, 0.2), r, v);
}

// sin(pi x) and cos(pi x) together for |x| < 2^50.  The argument is split
// exactly as x = k/2 + r with k = nearest integer to 2x and |r| <= 1/4 (the
// rounding to an integer uses the 1.5 * 2^52 shift, which also leaves k in
// the low bits); sin(pi r) and cos(pi r) come from their Maclaurin series
// (coefficients (-1)^j pi^n / n!, n = 2j+1 and 2j) truncated where the next
// term is below 1e-17 on |r| <= 1/4; k mod 4 quarter turns then select and
// negate.  22 FP64 instructions, against about 32 for sincospi().
__device__ __forceinline__ void sincospi_poly(double x, double* sn, double* cs) {
  const double shift = 6755399441055744.0;  // 1.5 * 2^52
  const double t = fma(x, 2.0, shift);
  const int q = __double2loint(t) & 3;
  const double k = t - shift;
  const double r = fma(k, -0.5, x);
  const double r2 = r * r;
  double ps = 0x1.aaec32af93359p-21;
  ps = fma(ps, r2, -0x1.6fadb9f155744p-16);
  ps = fma(ps, r2, 0x1.e8f434d018d63p-12);
  ps = fma(ps, r2, -0x1.e3074fde8871fp-8);
  ps = fma(ps, r2, 0x1.50783487ee782p-4);
  ps = fma(ps, r2, -0x1.32d2cce62bd86p-1);
  ps = fma(ps, r2, 0x1.466bc6775aae2p+1);
  ps = fma(ps, r2, -0x1.4abbce625be53p+2);
  ps = fma(ps, r2, 0x1.921fb54442d18p+1);
  const double s = r * ps;
  double pc = 0x1.20c62c2f2d7f5p-18;
  pc = fma(pc, r2, -0x1.b6e24f44b128fp-14);
  pc = fma(pc, r2, 0x1.f9d38a3763cc3p-10);
  pc = fma(pc, r2, -0x1.a6d1f2a204a8cp-6);
  pc = fma(pc, r2, 0x1.e1f506891babbp-3);
  pc = fma(pc, r2, -0x1.55d3c7e3cbffap+0);
  pc = fma(pc, r2, 0x1.03c1f081b5ac4p+2);
  pc = fma(pc, r2, -0x1.3bd3cc9be45dep+2);
  const double c = fma(pc, r2, 1.0);
  // rotate by q quarter turns
  const double a = (q & 1) ? c : s;
  const double b = (q & 1) ? s : c;
  *sn = (q & 2) ? -a : a;
  *cs = ((q + 1) & 2) ? -b : b;
}

// ---------------------------------------------------------------------------
// Dimensionless Keller-Miksis (Sec. 4.2, Eqs. dimensionless_system1-2,
// numerator, denominator):
//   y1' = y2,   y2' = N_KM / D_KM,
//   N_KM = (C0 + C1 y2) (1/y1)^C10 - C2 (1 + C9 y2) - C3/y1 - C4 y2/y1
//          - (1 - C9 y2 / 3) (3/2) y2^2
//          - (C5 sin 2 pi tau + C6 sin(2 pi C11 tau + C12)) (1 + C9 y2)
//          - y1 (C7 cos 2 pi tau + C8 cos(2 pi C11 tau + C12)),
//   D_KM = y1 - C9 y1 y2 + C4 C9.
// Following the paper's cost notes (Sec. 3.3): one division yields both
// 1/y1 (shared by the three 1/y1 terms) and 1/D_KM, sine and cosine of one
// angle come from one evaluation (sincospi_poly, with the angle 2 pi tau
// passed as 2 tau in units of pi), and the rational power is not sent
// through pow(): with EXP215 the exponent
// C10 = 3 gamma = 4.2 = 21/5 (gamma = 1.4) is applied as
//   (1/y1)^(21/5) = (1/y1)^4 * y1^(-1/5)
// with y1^(-1/5) from inv_fifth_root (the host selects this form when every
// system's C10 lies within 4 ulp of 21/5; otherwise pow() is used).
// DUAL selects the second driving frequency (C6, C8 != 0).
// ---------------------------------------------------------------------------
template <bool DUAL, bool EXP215 = false>
struct KellerMiksis {
  static constexpr int kDim = 2;
  static constexpr int kPar = 13;
  double C0, C1, C2, C3, C4, C5, C6, C7, C8, C9, C10, C11, C12pi, C4C9;
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
    C12pi = P[12 * n + i] * (1.0 / 3.141592653589793238462643383279502884);
    C4C9 = C4 * C9;
  }
  __device__ __forceinline__ void f(double tau, const double* y, double* dy) const {
    const double y1 = y[0], y2 = y[1];
    // one division serves both 1/y1 and 1/D: w = 1 / (y1 D), 1/y1 = D w, N/D = N y1 w
    const double D = fma(-C9 * y1, y2, y1) + C4C9;
    const double w = 1.0 / (y1 * D);
    const double rx = D * w;
    double g;
    if (EXP215) {
      const double rx2 = rx * rx;
      g = (rx2 * rx2) * inv_fifth_root(y1);
    } else {
      g = pow(rx, C10);
    }
    double s1, c1;
    sincospi_poly(2.0 * tau, &s1, &c1);
    const double one_c9y2 = fma(C9, y2, 1.0);
    double forc_s = C5 * s1;
    double forc_c = C7 * c1;
    if (DUAL) {
      double s2, c2;
      sincospi_poly(fma(2.0 * C11, tau, C12pi), &s2, &c2);
      forc_s = fma(C6, s2, forc_s);
      forc_c = fma(C8, c2, forc_c);
    }
    // (1 - C9 y2 / 3) * 1.5 * y2^2 = (1.5 - 0.5 C9 y2) y2^2
    const double kin = fma(-0.5 * C9, y2, 1.5) * (y2 * y2);
    double N = fma(C1, y2, C0) * g;
    N = fma(-C2, one_c9y2, N);
    N = fma(-fma(C4, y2, C3), rx, N);
    N -= kin;
    N = fma(-forc_s, one_c9y2, N);
    N = fma(-y1, forc_c, N);
    dy[0] = y2;
    dy[1] = N * (y1 * w);
  }
};

// ---------------------------------------------------------------------------
// Pressure relief valve (Sec. 4.3, Eqs. pressure_relief_valve_1-3):
//   y1' = y2, y2' = -kappa y2 - (y1 + delta) + y3, y3' = beta (q - y1 sqrt(y3)).
// sqrt is taken of max(y3, 0): y3 >= 0 for q > 0, the clamp only keeps a
// rounding excursion from producing a NaN.
// ---------------------------------------------------------------------------
struct ReliefValve {
  static constexpr int kDim = 3;
  static constexpr int kPar = 5;
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
    dy[2] = beta * fma(-y[0], sqrt(fmax(y[2], 0.0)), q);
  }
};

}  // namespace ens
