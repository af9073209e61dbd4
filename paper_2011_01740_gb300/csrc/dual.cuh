// dual.cuh -- forward-mode dual numbers for Jacobian-vector products.
//
// A Dual carries a value and a directional derivative, v + d e with e^2 = 0.
// Evaluating a right-hand side on Duals seeded with (y, v) returns f(y) and
// J(y) v in one pass: the tangent (variational) equation without a
// hand-written Jacobian.  Only the operations the right-hand sides use are
// defined; each derivative rule is the textbook one and is stated beside it.
#pragma once

#include "rhs.cuh"

namespace ens {

// the overloads below must not hide the double versions inside namespace ens
using ::fma;
using ::pow;

struct Dual {
  double v, d;
};

__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) {
  a = a - b;
  return a;
}
// (a b)' = a' b + a b'
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, fma(a.d, b.v, a.v * b.d)}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }

// fma(a, b, c) = a b + c: derivative a' b + a b' + c'
__device__ __forceinline__ Dual fma(Dual a, Dual b, Dual c) {
  return {fma(a.v, b.v, c.v), fma(a.d, b.v, fma(a.v, b.d, c.d))};
}
__device__ __forceinline__ Dual fma(double a, Dual b, Dual c) { return {fma(a, b.v, c.v), fma(a, b.d, c.d)}; }
__device__ __forceinline__ Dual fma(double a, Dual b, double c) { return {fma(a, b.v, c), a * b.d}; }
__device__ __forceinline__ Dual fma(Dual a, double b, Dual c) { return {fma(a.v, b, c.v), fma(a.d, b, c.d)}; }
__device__ __forceinline__ Dual fma(Dual a, Dual b, double c) {
  return {fma(a.v, b.v, c), fma(a.d, b.v, a.v * b.d)};
}

// (1/x)' = -x' / x^2 = -r^2 x'
__device__ __forceinline__ Dual rcp_nr(Dual x) {
  const double r = rcp_nr(x.v);
  return {r, -(r * r) * x.d};
}
// g = y1^(-21/5): the value from the same fixed-point evaluation as the
// plain right-hand side (so the tangent system's state part stays bitwise
// that of KellerMiksis), g' = -(21/5) g y1' / y1 with rx = 1/y1
__device__ __forceinline__ Dual polytropic_215(Dual y1, Dual rx) {
  const double g = pow_m21_5_fx(y1.v);
  return {g, (-4.2 * g) * (rx.v * y1.d)};
}
// (x^p)' = p x^p x' / x
__device__ __forceinline__ Dual pow(Dual x, double p) {
  const double r = pow(x.v, p);
  return {r, p * r * x.d / x.v};
}

// ---------------------------------------------------------------------------
// Keller-Miksis with its tangent (variational) equation, for the largest
// Lyapunov exponent: y = (y1, y2, v1, v2), (y1, y2)' as KellerMiksis and
// v' = J(y) v from one Dual evaluation of the acceleration seeded with
// (y1 + v1 e, y2 + v2 e).  In phase mode the tangent vector is scaled to unit
// length at the start and at every phase end, and the log of its length there
// is recorded (renormalisation between phases, the trajectory manipulation
// between phases of Sec. 1; Benettin's method for Lyapunov exponents).
// ---------------------------------------------------------------------------
template <bool DUAL, bool EXP215 = false>
struct KellerMiksisTangent : KellerMiksis<DUAL, EXP215> {
  using Base = KellerMiksis<DUAL, EXP215>;
  using Drive = typename Base::Drive;
  static constexpr int kDim = 4;
  static constexpr int kPhaseRows = 1;  // ln |v| at each phase end
  __device__ __forceinline__ void fd(const Drive& d, double tau, const double* y, double* dy) const {
    (void)tau;
    const Dual a = this->template accel<Dual>(d, Dual{y[0], y[2]}, Dual{y[1], y[3]});
    dy[0] = y[1];
    dy[1] = a.v;
    dy[2] = y[3];
    dy[3] = a.d;
  }
  __device__ __forceinline__ void f(double tau, const double* y, double* dy) const {
    fd(this->drive(tau), tau, y, dy);
  }
  // Scale the tangent vector to unit length; returns the log of its length.
  __device__ __forceinline__ double phase_hook(double* y) const {
    const double nv = hypot(y[2], y[3]);
    y[2] /= nv;
    y[3] /= nv;
    return log(nv);
  }
};

}  // namespace ens
