// df64.cu -- Keller-Miksis Cash-Karp kernel in double-float arithmetic.
//
// The state, the stage states and slopes, the right-hand side (km_df.cuh),
// the fifth-order update, the error estimate and the step controller are
// double-float pairs on the FP32 pipes (df.cuh, about 48 significant bits).
// The FP64 pipe keeps the phase-local time tau, the step h and the forcing
// sin / cos (sincos2pi_poly of rhs.cuh, split into pairs): about 110 FP64
// instructions per trial against 384 for the FP64 kernel.
//
// The algorithm is that of ck_phased_kernel with KellerMiksis (rhs.cuh,
// rkck45.cu) in every step: the same tableau (weights as float pairs), the
// same stage-5 forcing carried to the next k1, the same controller
// (E = max_i |err_i| / (atol + rtol max(|y_i|, |y5_i|)), accept iff E <= 1,
// fac = clamp(0.9 E^(-1/5), 0.2, 5) on E clamped to [1e-4, 2000], NaN gives
// 0.2 and a rejection), the same phase, transient and accessory handling.
// Only the rounding differs: relative errors of a few 1e-15 per operation
// instead of 1e-16, so results agree with the FP64 kernel to the sensitivity
// of each system to such perturbations.
#include "common.cuh"
#include "events.cuh"
#include "fcmp.cuh"
#include "km_df.cuh"
#include "rhs.cuh"
#include "valve_df.cuh"

namespace ens {

namespace {

using df::DF;

__host__ __device__ constexpr DF pair_of(double x) { return DF{(float)x, (float)(x - (double)(float)x)}; }

// Cash-Karp weights as pairs
constexpr DF A21 = pair_of(ck::a21);
constexpr DF A31 = pair_of(ck::a31), A32 = pair_of(ck::a32);
constexpr DF A41 = pair_of(ck::a41), A42 = pair_of(ck::a42), A43 = pair_of(ck::a43);
constexpr DF A51 = pair_of(ck::a51), A52 = pair_of(ck::a52), A53 = pair_of(ck::a53), A54 = pair_of(ck::a54);
constexpr DF A61 = pair_of(ck::a61), A62 = pair_of(ck::a62), A63 = pair_of(ck::a63), A64 = pair_of(ck::a64),
             A65 = pair_of(ck::a65);
constexpr DF B1 = pair_of(ck::b1), B3 = pair_of(ck::b3), B4 = pair_of(ck::b4), B6 = pair_of(ck::b6);
constexpr DF D1 = pair_of(ck::d1), D3 = pair_of(ck::d3), D4 = pair_of(ck::d4), D5 = pair_of(ck::d5),
             D6 = pair_of(ck::d6);
constexpr DF kSafety = pair_of(0.9);

// forcing of the dual-frequency Keller-Miksis (KellerMiksis::drive): sin and
// cos of the phase angles in FP64 (sincos2pi_poly), split into pairs, the
// amplitude products and the sum of the two components in double-word.  The
// FP64 polynomial, not the integer-pipe sincos2pi_fx of the FP64 kernels:
// here the FP32 and integer pipes carry the step and the FP64 pipe is the
// spare one (1024 x 1024 grid, 8 periods: 1.30 s against 1.64 s with
// sincos2pi_fx).
template <bool DUAL>
struct KmForcing {
  DF C5, C6, C7, C8;
  double C11, C12f;
  __device__ __forceinline__ void load(const double* P, int64_t n, int64_t i) {
    C5 = df::from_double(P[5 * n + i]);
    C6 = df::from_double(P[6 * n + i]);
    C7 = df::from_double(P[7 * n + i]);
    C8 = df::from_double(P[8 * n + i]);
    C11 = P[11 * n + i];
    C12f = P[12 * n + i] * (0.5 / 3.141592653589793238462643383279502884);  // C12 in turns
  }
  __device__ __forceinline__ void eval(double tau, DF& fs, DF& fc) const {
    double s1, c1;
    sincos2pi_poly(tau, &s1, &c1);
    fs = df::mul(C5, df::from_double(s1));
    fc = df::mul(C7, df::from_double(c1));
    if (DUAL) {
      double s2, c2;
      sincos2pi_poly(fma(C11, tau, C12f), &s2, &c2);
      fs = df::add(df::mul(C6, df::from_double(s2)), fs);
      fc = df::add(df::mul(C8, df::from_double(c2)), fc);
    }
  }
};

__device__ __forceinline__ DF dabs(DF x) { return x.hi < 0.0f ? df::neg(x) : x; }
__device__ __forceinline__ DF dmax(DF a, DF b) { return df::gt(a, b) ? a : b; }

}  // namespace

template <bool DUAL>
__global__ void __launch_bounds__(256) ck_phased_df_kernel(AdaptArgs a) {
  using namespace df;
  const double tau_end = a.t0 + a.phase_len;
  const uint64_t deadline = global_ns() + a.timeout_ns;
  int64_t i = -1;
  if (a.persistent) {
    const unsigned long long k = atomicAdd(&a.scratch->next, 1ULL);
    if (k < (unsigned long long)a.n) i = a.order ? (int64_t)a.order[k] : (int64_t)k;
  } else {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < a.n) i = g;
  }
  bool timed_out = false;
  KmDFCoef s;
  KmForcing<DUAL> frc;
  const DF rtol = from_double(a.rtol), atol = from_double(a.atol);
  DF y1, y2;                  // state
  DF k1x, k1v;                // slopes at the trial start
  DF f0s, f0c, fks, fkc;      // forcing at the phase start and at the current tau
  DF ymax, ymin;
  double tau = a.t0, dt = a.dt0;
  int32_t ph = 0, st = 0;
  uint32_t trials = 0, nacc = 0, nrej = 0, nrhs = 0, iter = 0;
  bool k1valid = false;

  auto start_system = [&](int64_t sys) {
    s.load(a.params, a.n, sys);
    frc.load(a.params, a.n, sys);
    y1 = from_double(a.y0[sys]);
    y2 = from_double(a.y0[a.n + sys]);
    tau = a.t0;
    dt = a.dt0;
    ph = 0;
    st = timed_out ? kStTimeout : 0;
    trials = nacc = nrej = nrhs = 0;
    k1valid = false;
    ymax = ymin = y1;
    frc.eval(a.t0, f0s, f0c);
    fks = f0s;
    fkc = f0c;
  };
  auto finish_system = [&](int64_t sys) {
    for (int p = max(ph, a.n_transient); p < a.n_phases; ++p) {
      a.acc[(int64_t)(2 * (p - a.n_transient)) * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
      a.acc[(int64_t)(2 * (p - a.n_transient) + 1) * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
    }
    a.y[sys] = to_double(y1);
    a.y[a.n + sys] = to_double(y2);
    a.t_out[sys] = tau;
    a.dt_out[sys] = dt;
    a.status[sys] = st;
    a.nacc[sys] = nacc;
    a.nrej[sys] = nrej;
    a.nrhs[sys] = nrhs;
    if (st) atomicOr(&a.scratch->any_status, (unsigned)st);
  };
  auto claim_next = [&]() -> int64_t {
    if (!a.persistent) return -1;
    const unsigned long long k = atomicAdd(&a.scratch->next, 1ULL);
    if (k >= (unsigned long long)a.n) return -1;
    return a.order ? (int64_t)a.order[k] : (int64_t)k;
  };
  auto record = [&](int64_t sys) {
    if (ph >= a.n_transient) {
      a.acc[(int64_t)(2 * (ph - a.n_transient)) * a.n + sys] = to_double(ymax);
      a.acc[(int64_t)(2 * (ph - a.n_transient) + 1) * a.n + sys] = to_double(ymin);
    }
  };

  if (i >= 0) start_system(i);
  while (i >= 0) {
    bool sys_done = false;
    if (st == 0) {
      if ((++iter & 127u) == 0 && global_ns() > deadline) timed_out = true;
      if (timed_out) st |= kStTimeout;
      else if (trials >= (uint64_t)a.max_steps) st |= kStMaxSteps;
    }
    if (st != 0) {
      if (ph < a.n_phases) {
        record(i);
        ++ph;
      }
      sys_done = true;
    } else {
      double h = dt;
      bool clamped = false;
      if (h >= tau_end - tau) {
        h = tau_end - tau;
        clamped = true;
      }
      const DF hd = from_double(h);
      if (!k1valid) {
        k1x = y2;
        k1v = s.accel(fks, fkc, y1, y2);
        ++nrhs;
        k1valid = true;
      }
      DF fs, fc;
      // stage 2
      DF sx = mul(A21, k1x), sv = mul(A21, k1v);
      DF x = add(y1, mul(sx, hd)), v = add(y2, mul(sv, hd));
      frc.eval(::fma(ck::c2, h, tau), fs, fc);
      const DF k2x = v, k2v = s.accel(fs, fc, x, v);
      // stage 3
      sx = df::fma(A32, k2x, mul(A31, k1x));
      sv = df::fma(A32, k2v, mul(A31, k1v));
      x = add(y1, mul(sx, hd));
      v = add(y2, mul(sv, hd));
      frc.eval(::fma(ck::c3, h, tau), fs, fc);
      const DF k3x = v, k3v = s.accel(fs, fc, x, v);
      // stage 4
      sx = df::fma(A43, k3x, df::fma(A42, k2x, mul(A41, k1x)));
      sv = df::fma(A43, k3v, df::fma(A42, k2v, mul(A41, k1v)));
      x = add(y1, mul(sx, hd));
      v = add(y2, mul(sv, hd));
      frc.eval(::fma(ck::c4, h, tau), fs, fc);
      const DF k4x = v, k4v = s.accel(fs, fc, x, v);
      // stage 5 (c5 = 1): its forcing is the next trial's k1 forcing
      sx = df::fma(A54, k4x, df::fma(A53, k3x, df::fma(A52, k2x, mul(A51, k1x))));
      sv = df::fma(A54, k4v, df::fma(A53, k3v, df::fma(A52, k2v, mul(A51, k1v))));
      x = add(y1, mul(sx, hd));
      v = add(y2, mul(sv, hd));
      DF f5s, f5c;
      frc.eval(tau + h, f5s, f5c);
      const DF k5x = v, k5v = s.accel(f5s, f5c, x, v);
      // stage 6
      sx = df::fma(A65, k5x, df::fma(A64, k4x, df::fma(A63, k3x, df::fma(A62, k2x, mul(A61, k1x)))));
      sv = df::fma(A65, k5v, df::fma(A64, k4v, df::fma(A63, k3v, df::fma(A62, k2v, mul(A61, k1v)))));
      x = add(y1, mul(sx, hd));
      v = add(y2, mul(sv, hd));
      frc.eval(::fma(ck::c6, h, tau), fs, fc);
      const DF k6x = v, k6v = s.accel(fs, fc, x, v);
      nrhs += 5;
      ++trials;
      // fifth-order solution and error estimate
      const DF bx = df::fma(B6, k6x, df::fma(B4, k4x, df::fma(B3, k3x, mul(B1, k1x))));
      const DF bv = df::fma(B6, k6v, df::fma(B4, k4v, df::fma(B3, k3v, mul(B1, k1v))));
      const DF n1 = add(y1, mul(bx, hd)), n2 = add(y2, mul(bv, hd));
      const DF ex = mul(df::fma(D6, k6x, df::fma(D5, k5x, df::fma(D4, k4x, df::fma(D3, k3x, mul(D1, k1x))))), hd);
      const DF ev = mul(df::fma(D6, k6v, df::fma(D5, k5v, df::fma(D4, k4v, df::fma(D3, k3v, mul(D1, k1v))))), hd);
      // controller
      const DF sc1 = df::fma(rtol, dmax(dabs(y1), dabs(n1)), atol);
      const DF sc2 = df::fma(rtol, dmax(dabs(y2), dabs(n2)), atol);
      const DF r1 = mul(dabs(ex), rcp(sc1)), r2 = mul(dabs(ev), rcp(sc2));
      const bool nan = isnan(r1.hi) || isnan(r2.hi);
      const DF E = dmax(r1, r2);
      DF fac;
      if (nan) {
        fac = make(0.2f);
      } else {
        const DF Ec = E.hi < 1e-4f ? pair_of(1e-4) : (E.hi > 2000.0f ? make(2000.0f) : E);
        fac = mul(kSafety, inv_fifth_root(Ec));
        fac = fac.hi < 0.2f ? make(0.2f) : fac;
        fac = fac.hi > 5.0f ? make(5.0f) : fac;
      }
      const bool accept = !nan && !gt(E, make(1.0f));
      const double facd = to_double(fac);
      if (accept) {
        tau = clamped ? tau_end : tau + h;
        y1 = n1;
        y2 = n2;
        fks = f5s;  // forcing at tau + h; a phase end below resets it
        fkc = f5c;
        k1valid = false;
        ++nacc;
        if (gt(y1, ymax)) ymax = y1;
        if (gt(ymin, y1)) ymin = y1;
        if (!clamped) {
          dt = h * facd;
          dt = dt > a.dt_max ? a.dt_max : dt;
          dt = dt < a.dt_min ? a.dt_min : dt;
        }
        if (!(tau < tau_end)) {
          record(i);
          ++ph;
          if (ph >= a.n_phases) {
            sys_done = true;
          } else {
            tau = a.t0;
            fks = f0s;
            fkc = f0c;
            ymax = ymin = y1;
          }
        }
      } else {
        ++nrej;
        dt = h * facd;
        if (dt < a.dt_min) st |= kStDtUnderflow;
      }
    }
    if (sys_done) {
      finish_system(i);
      i = claim_next();
      if (i >= 0) start_system(i);
    }
  }
}

// ---------------------------------------------------------------------------
// Relief valve (event mode, Sec. 4.3) in double-float arithmetic.  The state,
// the stage states and slopes, the right-hand side (valve_df.cuh, with a
// double-word square root), the fifth-order update, the error estimate and
// the controller are pairs on the FP32 pipes.  FP64 keeps the time t, the
// step h, the event tests and root estimates (event_frac), the impact law
// y2 <- -r y2 and the closed-form sticking interval: the steps whose result
// decides where an event lies.  The valve's right-hand side does not depend
// on t, so a trial needs no FP64 work besides the conversions of the state
// that the event tests read.  Every rule is that of ck_events_kernel
// (rkck45.cu): overshoot beyond the band |g| <= event_tol discards the trial
// and retries with the step cut to the earliest estimated root (one half when
// the impact starts inside the band, at most 40 retries); otherwise the step
// is accepted and events are located at its end; a rebound whose apex stays
// inside the band leaves the valve on the seat until y3 = delta.  The sums of
// stage terms and the error scale atol + rtol max(|y|, |y5|) take the
// double-word addition in Dekker's form (error bounded in the terms'
// magnitude, as FP64 rounding bounds them; the scale's terms are positive);
// the state update y + h S takes the accurate form.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ck_events_df_kernel(AdaptArgs a) {
  using namespace df;
  constexpr int D = 3;
  const uint64_t deadline = global_ns() + a.timeout_ns;
  const double etol = a.event_tol;
  const long long kt = okey(etol), knt = okey(-etol);
  int64_t i = -1;
  if (a.persistent) {
    const unsigned long long k = atomicAdd(&a.scratch->next, 1ULL);
    if (k < (unsigned long long)a.n) i = a.order ? (int64_t)a.order[k] : (int64_t)k;
  } else {
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < a.n) i = g;
  }
  bool timed_out = false;
  ValveDF s;
  const DF rtol = from_double(a.rtol), atol = from_double(a.atol);
  DF y[D], k1[D];
  double t = a.t0, dt = a.dt0, h_ev = 0.0, ymin = 0.0;
  int32_t st = 0, ev_retries = 0;
  uint32_t trials = 0, nacc = 0, nrej = 0, nrhs = 0, nmax = 0, nimp = 0, iter = 0;
  bool k1v = false, stuck = false;

  auto start_system = [&](int64_t sys) {
    s.load(a.params, a.n, sys);
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = from_double(a.y0[c * a.n + sys]);
    t = a.t0;
    dt = a.dt0;
    h_ev = 0.0;
    st = timed_out ? kStTimeout : 0;
    ev_retries = 0;
    trials = nacc = nrej = nrhs = nmax = nimp = 0;
    k1v = false;
    stuck = false;
    ymin = (t >= a.acc_t_start) ? a.y0[sys] : __longlong_as_double(0x7ff0000000000000LL);
    for (int r = 0; r < kRing; ++r)
      a.acc[(int64_t)r * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
  };
  auto finish_system = [&](int64_t sys) {
#pragma unroll
    for (int c = 0; c < D; ++c) a.y[c * a.n + sys] = to_double(y[c]);
    a.acc[(int64_t)kRing * a.n + sys] = ymin;
    a.acc[(int64_t)(kRing + 1) * a.n + sys] = (double)nmax;
    a.acc[(int64_t)(kRing + 2) * a.n + sys] = (double)nimp;
    a.t_out[sys] = t;
    a.dt_out[sys] = dt;
    a.status[sys] = st;
    a.nacc[sys] = nacc;
    a.nrej[sys] = nrej;
    a.nrhs[sys] = nrhs;
    if (st) atomicOr(&a.scratch->any_status, (unsigned)st);
  };
  auto claim_next = [&]() -> int64_t {
    if (!a.persistent) return -1;
    const unsigned long long k = atomicAdd(&a.scratch->next, 1ULL);
    if (k >= (unsigned long long)a.n) return -1;
    return a.order ? (int64_t)a.order[k] : (int64_t)k;
  };

  if (i >= 0) start_system(i);
  while (i >= 0) {
    bool sys_done = false;
    if (st == 0) {
      if ((++iter & 127u) == 0 && global_ns() > deadline) timed_out = true;
      if (timed_out) st |= kStTimeout;
      else if (!stuck && trials >= (uint64_t)a.max_steps) st |= kStMaxSteps;
    }
    if (st != 0) {
      sys_done = true;
    } else if (stuck) {
      // closed-form interval on the seat: y1 = y2 = 0, y3' = beta q
      const double y3 = to_double(y[2]);
      const double t_lift = t + (s.deltad - y3) / (s.betad * s.qd);
      if (t_lift >= a.t1) {
        y[2] = from_double(y3 + s.betad * s.qd * (a.t1 - t));
        t = a.t1;
      } else {
        y[2] = s.delta;
        t = t_lift;
        stuck = false;
      }
      k1v = false;
      if (okey(t) >= okey(a.acc_t_start) && okey(0.0) < okey(ymin)) ymin = 0.0;
      if (okey(t) >= okey(a.t1)) sys_done = true;
    } else {
      double h = dt;
      int limited = 0;
      const double rest = a.t1 - t;  // > 0 before the end
      if (nnbits(h) >= nnbits(rest)) {
        h = rest;
        limited = 1;
      }
      if (nnbits(h_ev) > 0 && nnbits(h_ev) < nnbits(h)) {  // h_ev >= 0
        h = h_ev;
        limited = 2;
      }
      if (!k1v) {
        s.f(y, k1);
        ++nrhs;
        k1v = true;
      }
      const DF hd = from_double(h);
      DF k2[D], k3[D], k4[D], k5[D], k6[D], x[D];
#pragma unroll
      for (int c = 0; c < D; ++c) x[c] = add(y[c], mul(mul(A21, k1[c]), hd));
      s.f(x, k2);
#pragma unroll
      for (int c = 0; c < D; ++c) x[c] = add(y[c], mul(fma_terms(A32, k2[c], mul(A31, k1[c])), hd));
      s.f(x, k3);
#pragma unroll
      for (int c = 0; c < D; ++c)
        x[c] = add(y[c], mul(fma_terms(A43, k3[c], fma_terms(A42, k2[c], mul(A41, k1[c]))), hd));
      s.f(x, k4);
#pragma unroll
      for (int c = 0; c < D; ++c)
        x[c] = add(y[c],
                   mul(fma_terms(A54, k4[c], fma_terms(A53, k3[c], fma_terms(A52, k2[c], mul(A51, k1[c])))), hd));
      s.f(x, k5);
#pragma unroll
      for (int c = 0; c < D; ++c)
        x[c] = add(y[c], mul(fma_terms(A65, k5[c],
                                     fma_terms(A64, k4[c], fma_terms(A63, k3[c], fma_terms(A62, k2[c], mul(A61, k1[c]))))),
                             hd));
      s.f(x, k6);
      nrhs += 5;
      ++trials;
      // fifth-order solution, error estimate and error norm
      DF n[D], E = make(0.0f);
      bool nan = false;
#pragma unroll
      for (int c = 0; c < D; ++c) {
        n[c] = add(y[c], mul(fma_terms(B6, k6[c], fma_terms(B4, k4[c], fma_terms(B3, k3[c], mul(B1, k1[c])))), hd));
        const DF e = mul(fma_terms(D6, k6[c], fma_terms(D5, k5[c], fma_terms(D4, k4[c], fma_terms(D3, k3[c], mul(D1, k1[c]))))),
                         hd);
        const DF sc = fma_terms(rtol, dmax(dabs(y[c]), dabs(n[c])), atol);
        const DF r = mul(dabs(e), rcp(sc));
        nan |= isnan(r.hi) || isnan(n[c].hi);
        E = dmax(E, r);
      }
      DF fac;
      if (nan) {
        fac = make(0.2f);
      } else {
        const DF Ec = E.hi < 1e-4f ? pair_of(1e-4) : (E.hi > 2000.0f ? make(2000.0f) : E);
        fac = mul(kSafety, inv_fifth_root(Ec));
        fac = fac.hi < 0.2f ? make(0.2f) : fac;
        fac = fac.hi > 5.0f ? make(5.0f) : fac;
      }
      const double facd = to_double(fac);
      if (nan || gt(E, make(1.0f))) {
        ++nrej;
        dt = h * facd;
        h_ev = 0.0;
        if (nnbits(dt) < nnbits(a.dt_min)) st |= kStDtUnderflow;
      } else {
        // events: decided in FP64 on the state at both ends of the trial
        const double y0d = to_double(y[0]), y1d = to_double(y[1]);
        const double n0d = to_double(n[0]), n1d = to_double(n[1]);
        double best = 2.0;
        bool overshoot = false;
        if (okey(n0d) < knt) {  // impact beyond the band
          const double frac = (okey(y0d) > kt) ? event_frac(y0d, to_double(k1[0]), n0d, h) : 0.5;
          best = nnmin(frac, best);
          overshoot = true;
        }
        if (okey(y1d) > kt && okey(n1d) < knt) {  // maximum beyond the band
          const double frac = event_frac(y1d, to_double(k1[1]), n1d, h);
          best = nnmin(frac, best);
          overshoot = true;
        }
        if (overshoot) {
          if (++ev_retries > kEventRetries) st |= kStEventNoConverge;
          else h_ev = h * best;
        } else {
#pragma unroll
          for (int c = 0; c < D; ++c) y[c] = n[c];
          t = (limited == 1) ? a.t1 : t + h;
          k1v = false;
          ++nacc;
          ev_retries = 0;
          h_ev = 0.0;
          if (!limited) dt = bounded_step(h, facd, a.dt_min, a.dt_max);
          double cur0 = n0d;
          if (okey(y1d) > kt && nnbits(absd(n1d)) <= nnbits(etol)) {  // Poincare point
            a.acc[(int64_t)(nmax % kRing) * a.n + i] = n0d;
            ++nmax;
          }
          // impact law (Eqs. impact_law_1-3) in FP64: y1 <- 0, y2 <- -r y2
          if (nnbits(absd(n0d)) <= nnbits(etol) && okey(n1d) < -1LL) {
            const double v = -s.r * n1d;
            y[0] = make(0.0f);
            y[1] = from_double(v);
            cur0 = 0.0;
            ++nimp;
            const double push = s.deltad - to_double(y[2]);
            if (push > 0.0 && v * v <= 2.0 * push * etol) {
              y[1] = make(0.0f);
              stuck = true;
            }
          }
          if (okey(t) >= okey(a.acc_t_start) && okey(cur0) < okey(ymin)) ymin = cur0;
          if (okey(t) >= okey(a.t1)) sys_done = true;
        }
      }
    }
    if (sys_done) {
      finish_system(i);
      i = claim_next();
      if (i >= 0) start_system(i);
    }
  }
}

cudaError_t launch_ck45_df_events(const AdaptArgs& a, AdaptLaunch L, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (a.n_phases != 0 || a.pair != kCashKarp) return cudaErrorInvalidValue;
  if (L.grid <= 0 || L.grid > 0x7fffffffLL || L.block <= 0) return cudaErrorInvalidConfiguration;
  ck_events_df_kernel<<<dim3((unsigned)L.grid), dim3((unsigned)L.block), 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ck45_df(unsigned flags, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (a.n_phases <= 0) return cudaErrorInvalidValue;
  if (L.grid <= 0 || L.grid > 0x7fffffffLL || L.block <= 0) return cudaErrorInvalidConfiguration;
  const dim3 g((unsigned)L.grid), b((unsigned)L.block);
  if (flags & kKmDual) ck_phased_df_kernel<true><<<g, b, 0, s>>>(a);
  else ck_phased_df_kernel<false><<<g, b, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ens
