// rkck45.cu -- adaptive Cash-Karp 4(5) ensemble kernels.
//
// One lane integrates one system at a time with state, the six stage
// derivatives and the parameters in registers.  Every loop iteration of a lane
// is exactly one trial step, so all lanes of a warp run the same instruction
// stream (the six right-hand-side evaluations) whatever their system's time,
// step size or phase; only the short accept / reject / event / phase-end
// branches diverge (Sec. 3.2.1 on divergence; Sec. 4.2 on asynchronous time
// stepping).
//
// Two launch modes:
//   plain       : system = global thread index; the lane retires when its
//                 system is done.
//   persistent  : a fixed grid of lanes; a lane that finishes its system
//                 claims the next one with atomicAdd on a device counter
//                 (work stealing), so uneven step counts do not leave warps
//                 idle.  An optional claim order lets the host schedule the
//                 longest systems first.
//
// Step-size control (the paper gives only the tolerances, Sec. 4.2.1):
//   sc_i = atol + rtol max(|y_i|, |y5_i|),  E = max_i |err_i| / sc_i,
//   accept iff E <= 1, fac = clamp(0.9 E^(-1/5), 0.2, 5) (5 if E = 0, 0.2 if
//   E is not a number), new step h fac bounded by [dt_min, dt_max]; a step
//   shortened to land on a phase end or an event keeps the previous proposal.
// Loops are bounded: max_steps trials per system, 40 event retries in a row,
// and a wall-clock budget read from %globaltimer; there are no spin-waits.
#include "common.cuh"
#include "dual.cuh"
#include "events.cuh"
#include "fcmp.cuh"
#include "rcp_fx.cuh"
#include "rhs.cuh"

namespace ens {

// ---------------------------------------------------------------------------
// one Cash-Karp trial: stages 2..6 from k1, fifth-order solution and error.
// d5 receives the drive (time-only part of the RHS) at t + h, the time of
// the next trial's first stage after an accepted step.
// ---------------------------------------------------------------------------
template <class Sys>
__device__ __forceinline__ void ck_trial(const Sys& s, double t, double h, const double* y,
                                         const double* k1, double* y5, double* err,
                                         typename Sys::Drive& d5) {
  constexpr int D = Sys::kDim;
  double k2[D], k3[D], k4[D], k5[D], k6[D], ys[D];
  double ts;
#pragma unroll
  for (int c = 0; c < D; ++c) ys[c] = fma(h, ck::a21 * k1[c], y[c]);
  ts = fma(ck::c2, h, t);
  s.fd(s.drive(ts), ts, ys, k2);
#pragma unroll
  for (int c = 0; c < D; ++c) ys[c] = fma(h, fma(ck::a32, k2[c], ck::a31 * k1[c]), y[c]);
  ts = fma(ck::c3, h, t);
  s.fd(s.drive(ts), ts, ys, k3);
#pragma unroll
  for (int c = 0; c < D; ++c)
    ys[c] = fma(h, fma(ck::a43, k3[c], fma(ck::a42, k2[c], ck::a41 * k1[c])), y[c]);
  ts = fma(ck::c4, h, t);
  s.fd(s.drive(ts), ts, ys, k4);
#pragma unroll
  for (int c = 0; c < D; ++c)
    ys[c] = fma(h, fma(ck::a54, k4[c], fma(ck::a53, k3[c], fma(ck::a52, k2[c], ck::a51 * k1[c]))),
                y[c]);
  ts = t + h;  // c5 = 1
  d5 = s.drive(ts);
  s.fd(d5, ts, ys, k5);
#pragma unroll
  for (int c = 0; c < D; ++c)
    ys[c] = fma(h,
                fma(ck::a65, k5[c],
                    fma(ck::a64, k4[c], fma(ck::a63, k3[c], fma(ck::a62, k2[c], ck::a61 * k1[c])))),
                y[c]);
  ts = fma(ck::c6, h, t);
  s.fd(s.drive(ts), ts, ys, k6);
#pragma unroll
  for (int c = 0; c < D; ++c) {
    y5[c] = fma(h, fma(ck::b6, k6[c], fma(ck::b4, k4[c], fma(ck::b3, k3[c], ck::b1 * k1[c]))), y[c]);
    err[c] = h * fma(ck::d6, k6[c],
                     fma(ck::d5, k5[c], fma(ck::d4, k4[c], fma(ck::d3, k3[c], ck::d1 * k1[c]))));
  }
}

// ---------------------------------------------------------------------------
// one Dormand-Prince trial: stages 2..7 from k1.  The seventh stage's state is
// y5 and k7 = f(t + h, y5) is returned for reuse as the next k1; stages 6
// and 7 share the drive at t + h (returned in d7).
// ---------------------------------------------------------------------------
template <class Sys>
__device__ __forceinline__ void dp_trial(const Sys& s, double t, double h, const double* y,
                                         const double* k1, double* y5, double* err, double* k7,
                                         typename Sys::Drive& d7) {
  constexpr int D = Sys::kDim;
  double k2[D], k3[D], k4[D], k5[D], k6[D], ys[D];
  double ts;
#pragma unroll
  for (int c = 0; c < D; ++c) ys[c] = fma(h, dp::a21 * k1[c], y[c]);
  ts = fma(dp::c2, h, t);
  s.fd(s.drive(ts), ts, ys, k2);
#pragma unroll
  for (int c = 0; c < D; ++c) ys[c] = fma(h, fma(dp::a32, k2[c], dp::a31 * k1[c]), y[c]);
  ts = fma(dp::c3, h, t);
  s.fd(s.drive(ts), ts, ys, k3);
#pragma unroll
  for (int c = 0; c < D; ++c)
    ys[c] = fma(h, fma(dp::a43, k3[c], fma(dp::a42, k2[c], dp::a41 * k1[c])), y[c]);
  ts = fma(dp::c4, h, t);
  s.fd(s.drive(ts), ts, ys, k4);
#pragma unroll
  for (int c = 0; c < D; ++c)
    ys[c] = fma(h, fma(dp::a54, k4[c], fma(dp::a53, k3[c], fma(dp::a52, k2[c], dp::a51 * k1[c]))),
                y[c]);
  ts = fma(dp::c5, h, t);
  s.fd(s.drive(ts), ts, ys, k5);
#pragma unroll
  for (int c = 0; c < D; ++c)
    ys[c] = fma(h,
                fma(dp::a65, k5[c],
                    fma(dp::a64, k4[c], fma(dp::a63, k3[c], fma(dp::a62, k2[c], dp::a61 * k1[c])))),
                y[c]);
  ts = t + h;  // c6 = c7 = 1
  d7 = s.drive(ts);
  s.fd(d7, ts, ys, k6);
#pragma unroll
  for (int c = 0; c < D; ++c)
    y5[c] = fma(h,
                fma(dp::b6, k6[c],
                    fma(dp::b5, k5[c], fma(dp::b4, k4[c], fma(dp::b3, k3[c], dp::b1 * k1[c])))),
                y[c]);
  s.fd(d7, ts, y5, k7);
#pragma unroll
  for (int c = 0; c < D; ++c)
    err[c] = h * fma(dp::e7, k7[c],
                     fma(dp::e6, k6[c],
                         fma(dp::e5, k5[c], fma(dp::e4, k4[c], fma(dp::e3, k3[c], dp::e1 * k1[c])))));
}

// One trial of the selected pair.  dn receives the drive at t + h; for
// Dormand-Prince kn receives k7 = f(t + h, y5), the next k1 after acceptance.
template <int PAIR, class Sys>
__device__ __forceinline__ void pair_trial(const Sys& s, double t, double h, const double* y,
                                           const double* k1, double* y5, double* err, double* kn,
                                           typename Sys::Drive& dn) {
  if (PAIR == kDormandPrince) dp_trial(s, t, h, y, k1, y5, err, kn, dn);
  else ck_trial(s, t, h, y, k1, y5, err, dn);
}
// right-hand-side evaluations of one trial besides k1
constexpr uint32_t pair_rhs(int PAIR) { return PAIR == kDormandPrince ? 6u : 5u; }

// E = max_c |err_c| / (atol + rtol max(|y_c|, |y5_c|)), >= 0, or NaN (sign
// clear) when a trial blew up.  rcp_fx (integer pipe) is within half an ulp
// plus 2^-57 of 1/sc for the normal sc below 2^1022 of a solve; a zero,
// subnormal, infinite or NaN sc gives NaN, and a NaN stays the maximum.
template <int D>
__device__ __forceinline__ double err_norm(const double* y, const double* y5, const double* err,
                                           double rtol, double atol) {
  double E = 0.0;
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const double sc = fma(rtol, nnmax(absd(y[c]), absd(y5[c])), atol);
    const double r = absd(absd(err[c]) * rcp_fx(sc));
    E = nnmax(E, r);
  }
  return E;
}
// accept iff E <= 1 (false for NaN)
__device__ __forceinline__ bool accept(double E) { return nnbits(E) <= nnbits(1.0); }

// fac = clamp(0.9 E^(-1/5), 0.2, 5).  0.9 E^(-1/5) leaves [0.2, 5] for
// E > 4.5^5 = 1845.3 and E < 0.18^5 = 1.9e-4, so E is clamped to [1e-4, 2000]
// first (same result, and keeps the float seed of inv_fifth_root_fx in range).
// E >= 0 or NaN as err_norm returns it.
__device__ __forceinline__ double step_factor(double E) {
  if (nnbits(E) > nnbits(__longlong_as_double(0x7ff0000000000000LL))) return 0.2;  // NaN
  const double Ec = nnmin(nnmax(E, 1e-4), 2000.0);
  const double fac = 0.9 * inv_fifth_root_fx(Ec);
  return nnmin(nnmax(fac, 0.2), 5.0);
}

// Claim the next system of a persistent lane (or the lane's own system in
// plain mode).  Returns -1 when no work is left.
__device__ __forceinline__ int64_t claim(const AdaptArgs& a, bool first) {
  if (!a.persistent) {
    if (!first) return -1;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    return i < a.n ? i : -1;
  }
  const unsigned long long k = atomicAdd(&a.scratch->next, 1ULL);
  if (k >= (unsigned long long)a.n) return -1;
  return a.order ? (int64_t)a.order[k] : (int64_t)k;
}

// First claim of a lane in a persistent, longest-first launch with one block
// per SM, deterministic and aware of the sub-partitions: warp w of a block
// runs on sub-partition w mod 4, and a warp that shares its sub-partition
// gets about half of that sub-partition's FP64 pipe.  The lanes of warps that
// own their sub-partition take the first ranks of the claim order (the
// longest systems), the others the next ones; later claims continue from rank
// gridDim.x * blockDim.x in order (claim_next_after_ranked).  The claim order
// never changes what a system computes.
__device__ __forceinline__ int64_t claim_first_by_subpartition(const AdaptArgs& a) {
  const int W = (int)(blockDim.x >> 5), w = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  int u_total = 0, u_before = 0;
  for (int x = 0; x < W; ++x) {
    const bool own = ((W - (x & 3) + 3) >> 2) == 1;  // the only warp of block x's sub-partition
    u_total += own;
    u_before += own && x < w;
  }
  const bool own = ((W - (w & 3) + 3) >> 2) == 1;
  const int64_t U = (int64_t)gridDim.x * u_total * 32;
  const int64_t rank = own ? ((int64_t)blockIdx.x * u_total + u_before) * 32 + lane
                           : U + ((int64_t)blockIdx.x * (W - u_total) + (w - u_before)) * 32 + lane;
  return rank < a.n ? (int64_t)a.order[rank] : -1;
}
__device__ __forceinline__ int64_t claim_next_after_ranked(const AdaptArgs& a) {
  const unsigned long long k = (unsigned long long)gridDim.x * blockDim.x + atomicAdd(&a.scratch->next, 1ULL);
  return k < (unsigned long long)a.n ? (int64_t)a.order[k] : -1;
}

// ---------------------------------------------------------------------------
// Phase mode (Keller-Miksis, Sec. 4.2): n_phases integrations over
// tau in [t0, t0 + phase_len] with tau reset at each phase start; running max
// and min of y1 over the accepted step points and the phase start.  Systems
// with kPhaseRows (the tangent system) also run their phase_hook at the start
// and at every phase end, recording its value in a row after the max / min.
// ---------------------------------------------------------------------------
template <class Sys, int PAIR>
__global__ void __launch_bounds__(256) ck_phased_kernel(AdaptArgs a) {
  constexpr int D = Sys::kDim;
  const double tau_end = a.t0 + a.phase_len;
  const uint64_t deadline = global_ns() + a.timeout_ns;
  int64_t i = a.first_by_subpartition ? claim_first_by_subpartition(a) : claim(a, true);
  bool timed_out = false;
  Sys s;
  // drive at the phase start (tau = t0), at the current tau, and at tau + h
  typename Sys::Drive d0, dk, d5;
  double y[D], k1[D], y5[D], err[D], kn[D];
  double tau = a.t0, dt = a.dt0, ymax = 0.0, ymin = 0.0;
  int32_t ph = 0, st = 0;
  uint32_t trials = 0, nacc = 0, nrej = 0, nrhs = 0, iter = 0;
  bool k1v = false;

  auto start_system = [&](int64_t sys) {
    s.load(a.params, a.n, sys);
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = a.y0[c * a.n + sys];
    tau = a.t0;
    dt = a.dt0;
    ph = 0;
    st = timed_out ? kStTimeout : 0;
    trials = nacc = nrej = nrhs = 0;
    k1v = false;
    ymax = ymin = y[0];
    d0 = s.drive(a.t0);
    dk = d0;
    if constexpr (Sys::kPhaseRows > 0) s.phase_hook(y);   // tangent vector to unit length
  };
  // per-phase hook row of recorded phase p (after the 2 acc_phases max / min rows)
  auto hook_row = [&](int p) { return (int64_t)(2 * a.acc_phases + p - a.n_transient) * a.n; };
  auto finish_system = [&](int64_t sys) {
    // recorded phases that were not completed are marked NaN
    for (int p = max(ph, a.n_transient); p < a.n_phases; ++p) {
      a.acc[(int64_t)(2 * (p - a.n_transient)) * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
      a.acc[(int64_t)(2 * (p - a.n_transient) + 1) * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
      if constexpr (Sys::kPhaseRows > 0) a.acc[hook_row(p) + sys] = __longlong_as_double(0x7ff8000000000000LL);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) a.y[c * a.n + sys] = y[c];
    a.t_out[sys] = tau;
    a.dt_out[sys] = dt;
    a.status[sys] = st;
    a.nacc[sys] = nacc;
    a.nrej[sys] = nrej;
    a.nrhs[sys] = nrhs;
    if (st) atomicOr(&a.scratch->any_status, (unsigned)st);
  };

  if (i >= 0) start_system(i);
  while (i >= 0) {
    bool sys_done = false;
    if (st == 0) {
      if ((++iter & 127u) == 0 && global_ns() > deadline) timed_out = true;
      if (timed_out) {
        st |= kStTimeout;
      } else if (trials >= (uint64_t)a.max_steps) {
        st |= kStMaxSteps;
      }
    }
    if (st != 0) {
      // close the current phase with what it has, then retire the system
      if (ph < a.n_phases) {
        if (ph >= a.n_transient) {
          a.acc[(int64_t)(2 * (ph - a.n_transient)) * a.n + i] = ymax;
          a.acc[(int64_t)(2 * (ph - a.n_transient) + 1) * a.n + i] = ymin;
          if constexpr (Sys::kPhaseRows > 0) a.acc[hook_row(ph) + i] = __longlong_as_double(0x7ff8000000000000LL);
        }
        ++ph;
      }
      sys_done = true;
    } else {
      double h = dt;
      bool clamped = false;
      const double rest = tau_end - tau;  // > 0 inside a phase
      if (nnbits(h) >= nnbits(rest)) {
        h = rest;
        clamped = true;
      }
      if (!k1v) {
        s.fd(dk, tau, y, k1);
        ++nrhs;
        k1v = true;
      }
      pair_trial<PAIR>(s, tau, h, y, k1, y5, err, kn, d5);
      nrhs += pair_rhs(PAIR);
      ++trials;
      const double E = err_norm<D>(y, y5, err, a.rtol, a.atol);
      const double fac = step_factor(E);
      if (accept(E)) {
        tau = clamped ? tau_end : tau + h;
        dk = d5;  // drive at tau + h; a phase end below resets it
#pragma unroll
        for (int c = 0; c < D; ++c) {
          y[c] = y5[c];
          if (PAIR == kDormandPrince) k1[c] = kn[c];
        }
        k1v = PAIR == kDormandPrince;  // k7 = f(tau + h, y5); a phase end below clears it
        ++nacc;
        ymax = omax(ymax, y[0]);
        ymin = omin(ymin, y[0]);
        if (!clamped) dt = bounded_step(h, fac, a.dt_min, a.dt_max);
        if (okey(tau) >= okey(tau_end)) {  // !(tau < tau_end): tau + h may round onto the end
          if (ph >= a.n_transient) {
            a.acc[(int64_t)(2 * (ph - a.n_transient)) * a.n + i] = ymax;
            a.acc[(int64_t)(2 * (ph - a.n_transient) + 1) * a.n + i] = ymin;
          }
          if constexpr (Sys::kPhaseRows > 0) {
            // renormalise the tangent vector between phases and record its growth
            const double gr = s.phase_hook(y);
            if (ph >= a.n_transient) a.acc[hook_row(ph) + i] = gr;
          }
          ++ph;
          if (ph >= a.n_phases) {
            sys_done = true;
          } else {
            tau = a.t0;
            dk = d0;
            k1v = false;
            ymax = ymin = y[0];
          }
        }
      } else {
        ++nrej;
        dt = h * fac;
        if (nnbits(dt) < nnbits(a.dt_min)) st |= kStDtUnderflow;  // retired at the next iteration
      }
    }
    if (sys_done) {
      finish_system(i);
      i = a.first_by_subpartition ? claim_next_after_ranked(a) : claim(a, false);
      if (i >= 0) start_system(i);
    }
  }
}

// ---------------------------------------------------------------------------
// Phase mode with two systems per thread (persistent launch, Cash-Karp): each
// lane holds two slots, each claiming systems like a lane of
// ck_phased_kernel.  Per iteration both slots' first stage and trial are
// computed in one straight-line block, independent chains that the compiler
// interleaves for the FP64 pipe; then each slot's accept / reject / phase-end
// logic runs.  Persistent launches only: the slots claim from the counter.  The first stage is evaluated in every iteration, also after a
// rejection, where its inputs are those of the last evaluation, so every
// value equals that of one system per thread bit for bit (the right-hand-side
// count counts only the evaluations that were needed).  A slot without work
// computes on its last values and stores nothing.
// ---------------------------------------------------------------------------
template <class Sys>
struct PhaseSlot {
  Sys s;
  typename Sys::Drive d0, dk, d5;  // drive at the phase start, at tau, at tau + h
  double y[Sys::kDim], k1[Sys::kDim], y5[Sys::kDim], err[Sys::kDim];
  double tau, dt, ymax, ymin, h, E, fac;
  int64_t i;
  int32_t ph, st;
  uint32_t trials, nacc, nrej, nrhs;
  bool k1v, clamped;
};

template <class Sys>
__global__ void __launch_bounds__(128) ck_phased2_kernel(AdaptArgs a) {
  static_assert(Sys::kPhaseRows == 0, "two systems per thread: systems without a phase hook");
  constexpr int D = Sys::kDim;
  constexpr int SPT = 2;
  const double tau_end = a.t0 + a.phase_len;
  const uint64_t deadline = global_ns() + a.timeout_ns;
  bool timed_out = false;
  uint32_t iter = 0;
  PhaseSlot<Sys> S[SPT];

  auto start_system = [&](PhaseSlot<Sys>& L) {
    L.s.load(a.params, a.n, L.i);
#pragma unroll
    for (int c = 0; c < D; ++c) L.y[c] = a.y0[c * a.n + L.i];
    L.tau = a.t0;
    L.dt = a.dt0;
    L.ph = 0;
    L.st = timed_out ? kStTimeout : 0;
    L.trials = L.nacc = L.nrej = L.nrhs = 0;
    L.k1v = false;
    L.ymax = L.ymin = L.y[0];
    L.d0 = L.s.drive(a.t0);
    L.dk = L.d0;
  };
  auto finish_system = [&](PhaseSlot<Sys>& L) {
    const int64_t sys = L.i;
    for (int p = max(L.ph, a.n_transient); p < a.n_phases; ++p) {
      a.acc[(int64_t)(2 * (p - a.n_transient)) * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
      a.acc[(int64_t)(2 * (p - a.n_transient) + 1) * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
    }
#pragma unroll
    for (int c = 0; c < D; ++c) a.y[c * a.n + sys] = L.y[c];
    a.t_out[sys] = L.tau;
    a.dt_out[sys] = L.dt;
    a.status[sys] = L.st;
    a.nacc[sys] = L.nacc;
    a.nrej[sys] = L.nrej;
    a.nrhs[sys] = L.nrhs;
    if (L.st) atomicOr(&a.scratch->any_status, (unsigned)L.st);
  };

  // a slot without a first system computes on a copy of system 0 (n > 0)
#pragma unroll
  for (int q = 0; q < SPT; ++q) {
    const int64_t k = claim(a, true);
    S[q].i = k >= 0 ? k : 0;
    start_system(S[q]);
    S[q].i = k;
  }
  while (S[0].i >= 0 || S[1].i >= 0) {
    if ((++iter & 127u) == 0 && global_ns() > deadline) timed_out = true;
    // per slot: budgets and the step of this iteration
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
      PhaseSlot<Sys>& L = S[q];
      if (L.i >= 0 && L.st == 0) {
        if (timed_out) L.st |= kStTimeout;
        else if (L.trials >= (uint64_t)a.max_steps) L.st |= kStMaxSteps;
      }
      L.h = L.dt;
      L.clamped = false;
      const double rest = tau_end - L.tau;
      if (nnbits(L.h) >= nnbits(rest)) {
        L.h = rest;
        L.clamped = true;
      }
    }
    // both slots' first stage and trial: independent straight-line chains
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
      PhaseSlot<Sys>& L = S[q];
      L.s.fd(L.dk, L.tau, L.y, L.k1);
      ck_trial(L.s, L.tau, L.h, L.y, L.k1, L.y5, L.err, L.d5);
      L.E = err_norm<D>(L.y, L.y5, L.err, a.rtol, a.atol);
      L.fac = step_factor(L.E);
    }
    // per slot: the outcome
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
      PhaseSlot<Sys>& L = S[q];
      if (L.i < 0) continue;
      bool sys_done = false;
      if (L.st != 0) {
        // close the current phase with what it has, then retire the system
        if (L.ph < a.n_phases) {
          if (L.ph >= a.n_transient) {
            a.acc[(int64_t)(2 * (L.ph - a.n_transient)) * a.n + L.i] = L.ymax;
            a.acc[(int64_t)(2 * (L.ph - a.n_transient) + 1) * a.n + L.i] = L.ymin;
          }
          ++L.ph;
        }
        sys_done = true;
      } else {
        if (!L.k1v) {
          ++L.nrhs;
          L.k1v = true;
        }
        L.nrhs += pair_rhs(kCashKarp);
        ++L.trials;
        if (accept(L.E)) {
          L.tau = L.clamped ? tau_end : L.tau + L.h;
          L.dk = L.d5;
#pragma unroll
          for (int c = 0; c < D; ++c) L.y[c] = L.y5[c];
          L.k1v = false;
          ++L.nacc;
          L.ymax = omax(L.ymax, L.y[0]);
          L.ymin = omin(L.ymin, L.y[0]);
          if (!L.clamped) L.dt = bounded_step(L.h, L.fac, a.dt_min, a.dt_max);
          if (okey(L.tau) >= okey(tau_end)) {
            if (L.ph >= a.n_transient) {
              a.acc[(int64_t)(2 * (L.ph - a.n_transient)) * a.n + L.i] = L.ymax;
              a.acc[(int64_t)(2 * (L.ph - a.n_transient) + 1) * a.n + L.i] = L.ymin;
            }
            ++L.ph;
            if (L.ph >= a.n_phases) {
              sys_done = true;
            } else {
              L.tau = a.t0;
              L.dk = L.d0;
              L.k1v = false;
              L.ymax = L.ymin = L.y[0];
            }
          }
        } else {
          ++L.nrej;
          L.dt = L.h * L.fac;
          if (nnbits(L.dt) < nnbits(a.dt_min)) L.st |= kStDtUnderflow;
        }
      }
      if (sys_done) {
        finish_system(L);
        L.i = claim(a, false);
        if (L.i >= 0) start_system(L);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Event mode (pressure relief valve, Sec. 4.3).  Events g1 = y1 (impact,
// body reaching the seat while moving towards it) and g2 = y2 (local maximum
// of y1, the Poincare section), both falling, absolute tolerance event_tol:
//   - after a trial that passes the error test, the impact overshoots when
//     y1(t+h) < -tol, the maximum when y2(t) > tol and y2(t+h) < -tol; the
//     trial is redone with the step cut to the earliest overshooting event's
//     estimated root, event_frac (one half when the impact starts inside the
//     band |y1| <= tol);
//   - otherwise the step is accepted; at its end the maximum is located when
//     y2(t) > tol and |y2| <= tol (y1 goes to the ring of Poincare points), the
//     impact when |y1| <= tol and y2 < 0 (y1 <- 0, y2 <- -r y2, Eqs.
//     impact_law_1-3);
//   - a bounce whose apex would stay inside the band (v^2 <= 2 a tol with
//     a = delta - y3 > 0 pressing the body onto the seat) leaves the body on
//     the seat: y1 = y2 = 0 while y3 rises as beta q until y3 = delta, an
//     interval advanced in closed form.
// ---------------------------------------------------------------------------
template <int PAIR>
__global__ void __launch_bounds__(256) ck_events_kernel(AdaptArgs a) {
  using Sys = ReliefValve;
  constexpr int D = Sys::kDim;
  const uint64_t deadline = global_ns() + a.timeout_ns;
  const double etol = a.event_tol;
  int64_t i = claim(a, true);
  bool timed_out = false;
  Sys s;
  Sys::Drive d5;  // autonomous: empty
  double y[D], k1[D], y5[D], err[D], kn[D];
  double t = a.t0, dt = a.dt0, h_ev = 0.0, ymin = 0.0;
  int32_t st = 0, ev_retries = 0;
  uint32_t trials = 0, nacc = 0, nrej = 0, nrhs = 0, nmax = 0, nimp = 0, iter = 0;
  bool k1v = false, stuck = false;

  auto start_system = [&](int64_t sys) {
    s.load(a.params, a.n, sys);
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = a.y0[c * a.n + sys];
    t = a.t0;
    dt = a.dt0;
    h_ev = 0.0;
    st = timed_out ? kStTimeout : 0;
    ev_retries = 0;
    trials = nacc = nrej = nrhs = nmax = nimp = 0;
    k1v = false;
    stuck = false;
    ymin = (t >= a.acc_t_start) ? y[0] : __longlong_as_double(0x7ff0000000000000LL);
    for (int r = 0; r < kRing; ++r)
      a.acc[(int64_t)r * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
  };
  auto finish_system = [&](int64_t sys) {
#pragma unroll
    for (int c = 0; c < D; ++c) a.y[c * a.n + sys] = y[c];
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
      const double t_lift = t + (s.delta - y[2]) / (s.beta * s.q);
      if (t_lift >= a.t1) {
        y[2] = y[2] + s.beta * s.q * (a.t1 - t);
        t = a.t1;
      } else {
        y[2] = s.delta;
        t = t_lift;
        stuck = false;
      }
      k1v = false;
      if (okey(t) >= okey(a.acc_t_start) && okey(y[0]) < okey(ymin)) ymin = y[0];
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
        s.f(t, y, k1);
        ++nrhs;
        k1v = true;
      }
      pair_trial<PAIR>(s, t, h, y, k1, y5, err, kn, d5);
      nrhs += pair_rhs(PAIR);
      ++trials;
      const double E = err_norm<D>(y, y5, err, a.rtol, a.atol);
      const double fac = step_factor(E);
      if (!accept(E)) {
        ++nrej;
        dt = h * fac;
        h_ev = 0.0;
        if (nnbits(dt) < nnbits(a.dt_min)) st |= kStDtUnderflow;
      } else {
        // y and y5 are finite here (a non-finite trial has E = NaN and is rejected)
        const long long kt = okey(etol), knt = okey(-etol);
        double best = 2.0;
        bool overshoot = false;
        if (okey(y5[0]) < knt) {  // impact beyond the band
          const double frac = (okey(y[0]) > kt) ? event_frac(y[0], k1[0], y5[0], h) : 0.5;
          best = nnmin(frac, best);
          overshoot = true;
        }
        if (okey(y[1]) > kt && okey(y5[1]) < knt) {  // maximum beyond the band
          const double frac = event_frac(y[1], k1[1], y5[1], h);
          best = nnmin(frac, best);
          overshoot = true;
        }
        if (overshoot) {
          if (++ev_retries > kEventRetries) st |= kStEventNoConverge;
          else h_ev = h * best;
        } else {
          const double y1_old = y[1];
#pragma unroll
          for (int c = 0; c < D; ++c) {
            y[c] = y5[c];
            if (PAIR == kDormandPrince) k1[c] = kn[c];
          }
          t = (limited == 1) ? a.t1 : t + h;
          k1v = PAIR == kDormandPrince;  // k7 = f(t + h, y5); the impact law clears it
          ++nacc;
          ev_retries = 0;
          h_ev = 0.0;
          if (!limited) dt = bounded_step(h, fac, a.dt_min, a.dt_max);
          if (okey(y1_old) > kt && nnbits(absd(y[1])) <= nnbits(etol)) {  // Poincare point
            a.acc[(int64_t)(nmax % kRing) * a.n + i] = y[0];
            ++nmax;
          }
          // impact law when |y1| <= tol and y2 < 0 (okey(-0.0) = -1: -0 is not below zero)
          if (nnbits(absd(y[0])) <= nnbits(etol) && okey(y[1]) < -1LL) {
            y[0] = 0.0;
            y[1] = -s.r * y[1];
            k1v = false;
            ++nimp;
            const double push = s.delta - y[2];
            if (push > 0.0 && y[1] * y[1] <= 2.0 * push * etol) {
              y[1] = 0.0;
              stuck = true;
            }
          }
          if (okey(t) >= okey(a.acc_t_start) && okey(y[0]) < okey(ymin)) ymin = y[0];
          if (okey(t) >= okey(a.t1)) sys_done = true;
        }
      }
    }
    if (sys_done) {
      finish_system(i);
      i = claim(a, false);
      if (i >= 0) start_system(i);
    }
  }
}

// ---------------------------------------------------------------------------
// plain adaptive integration over [t0, t1] (no phases, no events)
// ---------------------------------------------------------------------------
template <class Sys, int PAIR>
__global__ void __launch_bounds__(256) ck_plain_kernel(AdaptArgs a) {
  constexpr int D = Sys::kDim;
  const uint64_t deadline = global_ns() + a.timeout_ns;
  int64_t i = claim(a, true);
  bool timed_out = false;
  Sys s;
  typename Sys::Drive dk, d5;  // drive at t and at t + h
  double y[D], k1[D], y5[D], err[D], kn[D];
  double t = a.t0, dt = a.dt0;
  int32_t st = 0;
  uint32_t trials = 0, nacc = 0, nrej = 0, nrhs = 0, iter = 0;
  bool k1v = false;
  auto start_system = [&](int64_t sys) {
    s.load(a.params, a.n, sys);
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = a.y0[c * a.n + sys];
    t = a.t0;
    dt = a.dt0;
    st = timed_out ? kStTimeout : 0;
    trials = nacc = nrej = nrhs = 0;
    k1v = false;
    dk = s.drive(a.t0);
  };
  auto finish_system = [&](int64_t sys) {
#pragma unroll
    for (int c = 0; c < D; ++c) a.y[c * a.n + sys] = y[c];
    a.t_out[sys] = t;
    a.dt_out[sys] = dt;
    a.status[sys] = st;
    a.nacc[sys] = nacc;
    a.nrej[sys] = nrej;
    a.nrhs[sys] = nrhs;
    if (st) atomicOr(&a.scratch->any_status, (unsigned)st);
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
      sys_done = true;
    } else {
      double h = dt;
      bool clamped = false;
      const double rest = a.t1 - t;  // > 0 before the end
      if (nnbits(h) >= nnbits(rest)) {
        h = rest;
        clamped = true;
      }
      if (!k1v) {
        s.fd(dk, t, y, k1);
        ++nrhs;
        k1v = true;
      }
      pair_trial<PAIR>(s, t, h, y, k1, y5, err, kn, d5);
      nrhs += pair_rhs(PAIR);
      ++trials;
      const double E = err_norm<D>(y, y5, err, a.rtol, a.atol);
      const double fac = step_factor(E);
      if (accept(E)) {
        t = clamped ? a.t1 : t + h;
        dk = d5;  // t + h; a clamped step ends the system
#pragma unroll
        for (int c = 0; c < D; ++c) {
          y[c] = y5[c];
          if (PAIR == kDormandPrince) k1[c] = kn[c];
        }
        k1v = PAIR == kDormandPrince;
        ++nacc;
        if (!clamped) dt = bounded_step(h, fac, a.dt_min, a.dt_max);
        if (okey(t) >= okey(a.t1)) sys_done = true;
      } else {
        ++nrej;
        dt = h * fac;
        if (nnbits(dt) < nnbits(a.dt_min)) st |= kStDtUnderflow;
      }
    }
    if (sys_done) {
      finish_system(i);
      i = claim(a, false);
      if (i >= 0) start_system(i);
    }
  }
}

// Adapter so that fixed-step systems can run through the adaptive kernels.
template <class Fixed>
struct AdaptFixed : Fixed {
  using Drive = NoDrive;
  __device__ __forceinline__ void f(double t, const double* y, double* dy) const {
    Fixed::template f<false>(t, y, dy);
  }
  __device__ __forceinline__ Drive drive(double) const { return {}; }
  __device__ __forceinline__ void fd(const Drive&, double t, const double* y, double* dy) const {
    f(t, y, dy);
  }
};

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int PAIR>
cudaError_t launch_pair(int sys, unsigned flags, const AdaptArgs& a, dim3 g, dim3 b, cudaStream_t s) {
  const bool dual = flags & kKmDual;
  const bool exp215 = !(flags & kKmGeneralExponent);
  if (a.n_phases > 0) {
    switch (sys) {
      case ENS_SYS_KELLER_MIKSIS:
        if (dual) {
          if (exp215) ck_phased_kernel<KellerMiksis<true, true>, PAIR><<<g, b, 0, s>>>(a);
          else ck_phased_kernel<KellerMiksis<true, false>, PAIR><<<g, b, 0, s>>>(a);
        } else {
          if (exp215) ck_phased_kernel<KellerMiksis<false, true>, PAIR><<<g, b, 0, s>>>(a);
          else ck_phased_kernel<KellerMiksis<false, false>, PAIR><<<g, b, 0, s>>>(a);
        }
        break;
      case ENS_SYS_KELLER_MIKSIS_TANGENT:
        if (dual) {
          if (exp215) ck_phased_kernel<KellerMiksisTangent<true, true>, PAIR><<<g, b, 0, s>>>(a);
          else ck_phased_kernel<KellerMiksisTangent<true, false>, PAIR><<<g, b, 0, s>>>(a);
        } else {
          if (exp215) ck_phased_kernel<KellerMiksisTangent<false, true>, PAIR><<<g, b, 0, s>>>(a);
          else ck_phased_kernel<KellerMiksisTangent<false, false>, PAIR><<<g, b, 0, s>>>(a);
        }
        break;
      case ENS_SYS_LORENZ: ck_phased_kernel<AdaptFixed<Lorenz>, PAIR><<<g, b, 0, s>>>(a); break;
      case ENS_SYS_TOY_X2P: ck_phased_kernel<AdaptFixed<X2P>, PAIR><<<g, b, 0, s>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
  } else if (sys == ENS_SYS_RELIEF_VALVE) {
    ck_events_kernel<PAIR><<<g, b, 0, s>>>(a);
  } else {
    switch (sys) {
      case ENS_SYS_KELLER_MIKSIS:
        if (dual) {
          if (exp215) ck_plain_kernel<KellerMiksis<true, true>, PAIR><<<g, b, 0, s>>>(a);
          else ck_plain_kernel<KellerMiksis<true, false>, PAIR><<<g, b, 0, s>>>(a);
        } else {
          if (exp215) ck_plain_kernel<KellerMiksis<false, true>, PAIR><<<g, b, 0, s>>>(a);
          else ck_plain_kernel<KellerMiksis<false, false>, PAIR><<<g, b, 0, s>>>(a);
        }
        break;
      case ENS_SYS_LORENZ: ck_plain_kernel<AdaptFixed<Lorenz>, PAIR><<<g, b, 0, s>>>(a); break;
      case ENS_SYS_TOY_X2P: ck_plain_kernel<AdaptFixed<X2P>, PAIR><<<g, b, 0, s>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaGetLastError();
}

// Two systems per thread: the Keller-Miksis phase mode with Cash-Karp, one
// driving frequency and the exponent 21/5, persistent lanes.
cudaError_t launch_ck45_spt2(int sys, unsigned flags, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (sys != ENS_SYS_KELLER_MIKSIS || a.n_phases <= 0 || a.pair != kCashKarp || !a.persistent ||
      (flags & (kKmDual | kKmGeneralExponent)))
    return cudaErrorNotSupported;
  if (L.grid <= 0 || L.grid > 0x7fffffffLL || L.block <= 0 || L.block > 128) return cudaErrorInvalidConfiguration;
  ck_phased2_kernel<KellerMiksis<false, true>><<<dim3((unsigned)L.grid), dim3((unsigned)L.block), 0, s>>>(a);
  return cudaGetLastError();
}

// Adaptive launch with the pair a.pair selects (Cash-Karp or Dormand-Prince).
cudaError_t launch_ck45(int sys, unsigned flags, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (L.grid <= 0 || L.grid > 0x7fffffffLL || L.block <= 0) return cudaErrorInvalidConfiguration;
  const dim3 g((unsigned)L.grid), b((unsigned)L.block);
  if (a.pair == kDormandPrince) return launch_pair<kDormandPrince>(sys, flags, a, g, b, s);
  if (a.pair != kCashKarp) return cudaErrorInvalidValue;
  return launch_pair<kCashKarp>(sys, flags, a, g, b, s);
}

}  // namespace ens

namespace ens {

// One right-hand-side evaluation per system with the same device code the
// solvers inline (test and inspection hook): dy = f(t, y; p).
template <class Sys>
__global__ void rhs_eval_kernel(int64_t n, const double* P, const double* t, const double* y, double* dy) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    Sys s;
    s.load(P, n, i);
    double yy[Sys::kDim], d[Sys::kDim];
#pragma unroll
    for (int c = 0; c < Sys::kDim; ++c) yy[c] = y[c * n + i];
    s.f(t[i], yy, d);
#pragma unroll
    for (int c = 0; c < Sys::kDim; ++c) dy[c * n + i] = d[c];
  }
}

cudaError_t launch_rhs_eval(int sys, unsigned flags, int64_t n, const double* P, const double* t,
                            const double* y, double* dy, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  blocks = blocks > 8192 ? 8192 : blocks;
  const bool dual = flags & kKmDual, exp215 = !(flags & kKmGeneralExponent);
  switch (sys) {
    case ENS_SYS_TOY_X2P: rhs_eval_kernel<AdaptFixed<X2P>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy); break;
    case ENS_SYS_LORENZ: rhs_eval_kernel<AdaptFixed<Lorenz>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy); break;
    case ENS_SYS_RELIEF_VALVE: rhs_eval_kernel<ReliefValve><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy); break;
    case ENS_SYS_KELLER_MIKSIS_TANGENT:
      if (dual) {
        if (exp215) rhs_eval_kernel<KellerMiksisTangent<true, true>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy);
        else rhs_eval_kernel<KellerMiksisTangent<true, false>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy);
      } else {
        if (exp215) rhs_eval_kernel<KellerMiksisTangent<false, true>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy);
        else rhs_eval_kernel<KellerMiksisTangent<false, false>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy);
      }
      break;
    case ENS_SYS_KELLER_MIKSIS:
      if (dual) {
        if (exp215) rhs_eval_kernel<KellerMiksis<true, true>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy);
        else rhs_eval_kernel<KellerMiksis<true, false>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy);
      } else {
        if (exp215) rhs_eval_kernel<KellerMiksis<false, true>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy);
        else rhs_eval_kernel<KellerMiksis<false, false>><<<(unsigned)blocks, 256, 0, s>>>(n, P, t, y, dy);
      }
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ens
