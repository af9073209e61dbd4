// fp32c.cu -- Keller-Miksis Cash-Karp kernel in split precision.
//
// GB300 executes FP32 fused multiply-adds about 60 times faster than FP64
// ones, so this variant moves the bulk of a trial step to FP32 and keeps in
// FP64 only what the step-size control and the clock need:
//   FP32   right-hand side, stage sums, error estimate components;
//   FP32 x2 the state (hi + lo pair, renormalised after every update) and the
//          increments added to it, so rounding does not accumulate over the
//          ~10^5 steps of a run;
//   FP64   the phase-local time tau, the step h and its proposal, the
//          acceptance test |err_i| <= atol + rtol max(|y_i|, |y5_i|)
//          (err_i and the scale come from float quantities; the comparison
//          and the tolerances are double).
// The step factor s E^(-1/5) only scales the next proposal and is formed in
// FP32, with the safety factor s = 0.8 (the FP64 kernels use 0.9).  This
// variant runs at loose tolerances (1e-7, 1e-8), where the Keller-Miksis
// collapses make the step proposal overshoot often: on the 1024 x 1024 sweep
// at 1e-8, 26 % of the trials were rejected with 0.9 and 7.9 % with 0.8,
// which ran 7 % faster with slightly smaller errors (0.7: 2.8 %, but 12 %
// slower again).
//
// Stage sums use a compensated dot product (Ogita, Rump & Oishi, "Accurate
// sum and dot product", SIAM J. Sci. Comput. 26, 2005: TwoProduct via fma and
// TwoSum, Algorithm Dot2), with each tableau weight split into a float pair,
// so the strongly cancelling Cash-Karp rows (e.g. -11/54, 5/2, -70/27, 35/27)
// are summed to float accuracy of the result rather than of the terms.
//
// The right-hand side is rearranged for float: with the identity
// C0 = C2 + C3 of the coefficient definitions (Eq. coefficients) the
// near-cancelling terms of N_KM become
//   C0 g - C2 - C3 / y1 = R0 g + C2 (g - 1) + C3 (1/y1) ((1/y1)^(C10-1) - 1)
// with R0 = C0 - C2 - C3 (formed in double on load, zero up to rounding), and
// g - 1 = expm1(-C10 log1p(y1 - 1)) evaluated from the deviation y1 - 1, which
// the float pair holds exactly.  Near equilibrium the float error then scales
// with |y1 - 1| instead of with C0.
#include "common.cuh"
#include "fcmp.cuh"
#include "rhs.cuh"

namespace ens {

namespace {

constexpr float kSafety = 0.8f;  // step-factor safety (see the header)

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ ff fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return {s, b - (s - a)};
}

// tableau weight as a float pair
struct w2 {
  float hi, lo;
};

__device__ __forceinline__ constexpr w2 split(double x) { return {(float)x, (float)(x - (double)(float)x)}; }

// Compensated dot product accumulator (Dot2).
struct dot2 {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(w2 w, float k) {
    const float p = w.hi * k;
    const float ep = fmaf(w.hi, k, -p) + w.lo * k;  // exact product error + low weight part
    const ff t = two_sum(s, p);
    s = t.hi;
    c += t.lo + ep;
  }
  __device__ __forceinline__ float value() const { return s + c; }
};

__device__ __forceinline__ float expm1_f(float x) { return expm1f(x); }

// Keller-Miksis in float (see the file comment for the rearrangement).
template <bool DUAL>
struct KmF32 {
  float R0, C1, C2, C3, C4, C5, C6, C7, C8, C9, C10, C11, C12pi, C4C9, C9C2;
  __device__ __forceinline__ void load(const double* P, int64_t n, int64_t i) {
    const double c0 = P[i], c2 = P[2 * n + i], c3 = P[3 * n + i];
    R0 = (float)(c0 - c2 - c3);
    C1 = (float)P[n + i];
    C2 = (float)c2;
    C3 = (float)c3;
    C4 = (float)P[4 * n + i];
    C5 = (float)P[5 * n + i];
    C6 = (float)P[6 * n + i];
    C7 = (float)P[7 * n + i];
    C8 = (float)P[8 * n + i];
    C9 = (float)P[9 * n + i];
    C10 = (float)P[10 * n + i];
    C11 = (float)P[11 * n + i];
    C12pi = (float)(P[12 * n + i] * (1.0 / 3.141592653589793238462643383279502884));
    C4C9 = (float)(P[4 * n + i] * P[9 * n + i]);
    C9C2 = (float)(P[9 * n + i] * c2);
  }
  // x = y1 - 1 (deviation), v = y2, tau2 = 2 tau (units of pi)
  __device__ __forceinline__ float f(float x, float v, float tau2) const {
    const float y1 = 1.0f + x;
    const float rx = __frcp_rn(y1);
    const float L = log1pf(x);
    const float em = expm1_f(-C10 * L);            // (1/y1)^C10 - 1
    const float em1 = expm1_f((1.0f - C10) * L);   // (1/y1)^(C10-1) - 1
    const float g = 1.0f + em;
    float s1, c1;
    sincospif(tau2, &s1, &c1);
    float fs = C5 * s1, fc = C7 * c1;
    if (DUAL) {
      float s2, c2;
      sincospif(fmaf(C11, tau2, C12pi), &s2, &c2);
      fs = fmaf(C6, s2, fs);
      fc = fmaf(C8, c2, fc);
    }
    const float one_c9v = fmaf(C9, v, 1.0f);
    float N = fmaf(C2, em, R0 * g);
    N = fmaf(C3 * rx, em1, N);
    N = fmaf(v, fmaf(C1, g, -fmaf(C4, rx, C9C2)), N);
    N = fmaf(-fmaf(-0.5f * C9, v, 1.5f), v * v, N);
    N = fmaf(-fs, one_c9v, N);
    N = fmaf(-y1, fc, N);
    const float D = fmaf(-C9 * y1, v, y1) + C4C9;
    return __fdiv_rn(N, D);
  }
};

// Cash-Karp weights as float pairs
constexpr w2 A21 = split(ck::a21);
constexpr w2 A31 = split(ck::a31), A32 = split(ck::a32);
constexpr w2 A41 = split(ck::a41), A42 = split(ck::a42), A43 = split(ck::a43);
constexpr w2 A51 = split(ck::a51), A52 = split(ck::a52), A53 = split(ck::a53), A54 = split(ck::a54);
constexpr w2 A61 = split(ck::a61), A62 = split(ck::a62), A63 = split(ck::a63), A64 = split(ck::a64),
             A65 = split(ck::a65);
constexpr w2 B1 = split(ck::b1), B3 = split(ck::b3), B4 = split(ck::b4), B6 = split(ck::b6);
constexpr w2 D1 = split(ck::d1), D3 = split(ck::d3), D4 = split(ck::d4), D5 = split(ck::d5),
             D6 = split(ck::d6);

// ff comparison (renormalised pairs)
__device__ __forceinline__ bool ff_gt(ff a, ff b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }

__device__ __forceinline__ double ff_to_d(ff a) { return (double)a.hi + (double)a.lo; }

// Exact conversions between double and float on the integer pipe: a
// conversion instruction costs an FP64 pipe slot on this part.
//   to_d:   float -> double, exact for zero and normal floats (a subnormal
//           float becomes a double of about the same, tiny size; the
//           acceptance test below compares such values against atol);
//   rn_f32: double -> float rounded to nearest, ties to even, as the
//           conversion instruction rounds, for zero and |x| in
//           [2^-126, 2^128) (the step, its low part and the time here).
__device__ __forceinline__ double to_d(float v) {
  const unsigned b = __float_as_uint(v);
  const unsigned sign = b & 0x80000000u, mag = b & 0x7fffffffu;
  const unsigned hi = mag == 0 ? sign : (((mag >> 3) + ((1023u - 127u) << 20)) | sign);
  return __hiloint2double((int)hi, (int)(mag << 29));
}
__device__ __forceinline__ float rn_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const unsigned long long mag = b & 0x7fffffffffffffffull;
  const unsigned long long r = mag - ((unsigned long long)(1023 - 127) << 52);  // exponent rebiased
  const unsigned q = (unsigned)(r >> 29);                                     // exponent and 23 bits
  const unsigned rest = (unsigned)(r & 0x1fffffffu);
  const unsigned up = (rest > 0x10000000u || (rest == 0x10000000u && (q & 1u))) ? 1u : 0u;
  return __uint_as_float(mag == 0 ? sign : ((q + up) | sign));  // a carry steps the exponent
}

// y + h * sum  with y a float pair, h = hh + hl a float pair, sum = s + c
__device__ __forceinline__ ff ff_axpy(ff y, float hh, float hl, float s, float c) {
  const float p = hh * s;
  const float ep = fmaf(hh, s, -p) + fmaf(hh, c, hl * s);
  const ff t = two_sum(y.hi, p);
  return fast_two_sum(t.hi, t.lo + (y.lo + ep));
}

}  // namespace

template <bool DUAL>
__global__ void __launch_bounds__(256) ck_phased_fp32c_kernel(AdaptArgs a) {
  const double tau_end = a.t0 + a.phase_len;
  const uint64_t deadline = global_ns() + a.timeout_ns;
  int64_t i = (a.persistent) ? -1 : blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (a.persistent) {
    const unsigned long long k = atomicAdd(&a.scratch->next, 1ULL);
    i = k < (unsigned long long)a.n ? (a.order ? (int64_t)a.order[k] : (int64_t)k) : -1;
  } else if (i >= a.n) {
    i = -1;
  }
  bool timed_out = false;
  KmF32<DUAL> s;
  ff y0v, y1v;               // state: x-deviation form is formed on the fly
  float k1x = 0.f, k1v = 0.f;
  bool k1valid = false;
  double tau = a.t0, dt = a.dt0;
  ff ymax{0.f, 0.f}, ymin{0.f, 0.f};
  int32_t ph = 0, st = 0;
  uint32_t trials = 0, nacc = 0, nrej = 0, nrhs = 0, iter = 0;
  const float rtol_f = (float)a.rtol, atol_f = (float)a.atol;

  auto start_system = [&](int64_t sys) {
    s.load(a.params, a.n, sys);
    const double u = a.y0[sys], v = a.y0[a.n + sys];
    y0v = {(float)u, (float)(u - (double)(float)u)};
    y1v = {(float)v, (float)(v - (double)(float)v)};
    tau = a.t0;
    dt = a.dt0;
    ph = 0;
    st = timed_out ? kStTimeout : 0;
    trials = nacc = nrej = nrhs = 0;
    k1valid = false;
    ymax = ymin = y0v;
  };
  auto finish_system = [&](int64_t sys) {
    for (int p = max(ph, a.n_transient); p < a.n_phases; ++p) {
      a.acc[(int64_t)(2 * (p - a.n_transient)) * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
      a.acc[(int64_t)(2 * (p - a.n_transient) + 1) * a.n + sys] = __longlong_as_double(0x7ff8000000000000LL);
    }
    a.y[sys] = ff_to_d(y0v);
    a.y[a.n + sys] = ff_to_d(y1v);
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
        if (ph >= a.n_transient) {
          a.acc[(int64_t)(2 * (ph - a.n_transient)) * a.n + i] = ff_to_d(ymax);
          a.acc[(int64_t)(2 * (ph - a.n_transient) + 1) * a.n + i] = ff_to_d(ymin);
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
      const float hh = rn_f32(h), hl = rn_f32(h - to_d(hh));
      // deviation of the stage base: x0 = (y1 - 1) exactly as a float sum
      const float xb = (y0v.hi - 1.0f) + y0v.lo;
      const float vb = y1v.hi + y1v.lo;
      const float t2 = 2.0f * rn_f32(tau), h2 = 2.0f * hh;  // 2 RN(tau) = RN(2 tau)
      if (!k1valid) {
        k1x = vb;
        k1v = s.f(xb, vb, t2);
        ++nrhs;
        k1valid = true;
      }
      // stage 2
      dot2 sx, sv;
      sx.add(A21, k1x); sv.add(A21, k1v);
      float x2 = fmaf(hh, sx.value(), xb), v2 = fmaf(hh, sv.value(), vb);
      const float k2x = v2, k2v = s.f(x2, v2, fmaf((float)ck::c2, h2, t2));
      // stage 3
      dot2 s3x, s3v;
      s3x.add(A31, k1x); s3x.add(A32, k2x);
      s3v.add(A31, k1v); s3v.add(A32, k2v);
      const float x3 = fmaf(hh, s3x.value(), xb), v3 = fmaf(hh, s3v.value(), vb);
      const float k3x = v3, k3v = s.f(x3, v3, fmaf((float)ck::c3, h2, t2));
      // stage 4
      dot2 s4x, s4v;
      s4x.add(A41, k1x); s4x.add(A42, k2x); s4x.add(A43, k3x);
      s4v.add(A41, k1v); s4v.add(A42, k2v); s4v.add(A43, k3v);
      const float x4 = fmaf(hh, s4x.value(), xb), v4 = fmaf(hh, s4v.value(), vb);
      const float k4x = v4, k4v = s.f(x4, v4, fmaf((float)ck::c4, h2, t2));
      // stage 5
      dot2 s5x, s5v;
      s5x.add(A51, k1x); s5x.add(A52, k2x); s5x.add(A53, k3x); s5x.add(A54, k4x);
      s5v.add(A51, k1v); s5v.add(A52, k2v); s5v.add(A53, k3v); s5v.add(A54, k4v);
      const float x5 = fmaf(hh, s5x.value(), xb), v5 = fmaf(hh, s5v.value(), vb);
      const float k5x = v5, k5v = s.f(x5, v5, t2 + h2);
      // stage 6
      dot2 s6x, s6v;
      s6x.add(A61, k1x); s6x.add(A62, k2x); s6x.add(A63, k3x); s6x.add(A64, k4x); s6x.add(A65, k5x);
      s6v.add(A61, k1v); s6v.add(A62, k2v); s6v.add(A63, k3v); s6v.add(A64, k4v); s6v.add(A65, k5v);
      const float x6 = fmaf(hh, s6x.value(), xb), v6 = fmaf(hh, s6v.value(), vb);
      const float k6x = v6, k6v = s.f(x6, v6, fmaf((float)ck::c6, h2, t2));
      nrhs += 5;
      ++trials;
      // fifth-order solution into the float pairs; error estimate
      dot2 bx, bv, ex, ev;
      bx.add(B1, k1x); bx.add(B3, k3x); bx.add(B4, k4x); bx.add(B6, k6x);
      bv.add(B1, k1v); bv.add(B3, k3v); bv.add(B4, k4v); bv.add(B6, k6v);
      ex.add(D1, k1x); ex.add(D3, k3x); ex.add(D4, k4x); ex.add(D5, k5x); ex.add(D6, k6x);
      ev.add(D1, k1v); ev.add(D3, k3v); ev.add(D4, k4v); ev.add(D5, k5v); ev.add(D6, k6v);
      const ff n0 = ff_axpy(y0v, hh, hl, bx.s, bx.c);
      const ff n1 = ff_axpy(y1v, hh, hl, bv.s, bv.c);
      // acceptance in FP64: |err_i| <= atol + rtol max(|y_i|, |y5_i|).  err_i
      // is a float quantity and the scale needs only the leading (hi) parts of
      // the states, so ten FP64 instructions decide the step.
      const float exv = ex.value(), evv = ev.value();
      const float m0 = fmaxf(fabsf(y0v.hi), fabsf(n0.hi)), m1 = fmaxf(fabsf(y1v.hi), fabsf(n1.hi));
      const double e0 = absd(h * to_d(exv)), e1 = absd(h * to_d(evv));
      const double sc0 = fma(a.rtol, to_d(m0), a.atol), sc1 = fma(a.rtol, to_d(m1), a.atol);
      // e <= sc on the bit patterns (e >= +0 or NaN, sc > 0): false for NaN
      const bool accept = nnbits(e0) <= nnbits(sc0) && nnbits(e1) <= nnbits(sc1);
      // step factor from the float ratio E = max_i |err_i| / sc_i
      const float E = fmaxf(__fdividef(fabsf(hh * exv), fmaf(rtol_f, m0, atol_f)),
                            __fdividef(fabsf(hh * evv), fmaf(rtol_f, m1, atol_f)));
      float fac;
      if (isnan(E)) {
        fac = 0.2f;
      } else {
        const float Ec = fminf(fmaxf(E, 1e-4f), 2000.f);
        float l, r;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(Ec));
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(-0.2f * l));
        fac = fminf(fmaxf(kSafety * r, 0.2f), 5.0f);
      }
      if (accept) {
        tau = clamped ? tau_end : tau + h;
        y0v = n0;
        y1v = n1;
        k1valid = false;
        ++nacc;
        if (ff_gt(y0v, ymax)) ymax = y0v;
        if (ff_gt(ymin, y0v)) ymin = y0v;
        if (!clamped) dt = bounded_step(h, to_d(fac), a.dt_min, a.dt_max);
        if (okey(tau) >= okey(tau_end)) {  // !(tau < tau_end)
          if (ph >= a.n_transient) {
            a.acc[(int64_t)(2 * (ph - a.n_transient)) * a.n + i] = ff_to_d(ymax);
            a.acc[(int64_t)(2 * (ph - a.n_transient) + 1) * a.n + i] = ff_to_d(ymin);
          }
          ++ph;
          if (ph >= a.n_phases) {
            sys_done = true;
          } else {
            tau = a.t0;
            ymax = ymin = y0v;
          }
        }
      } else {
        ++nrej;
        dt = h * to_d(fac);
        if (nnbits(dt) < nnbits(a.dt_min)) st |= kStDtUnderflow;
      }
    }
    if (sys_done) {
      finish_system(i);
      i = claim_next();
      if (i >= 0) start_system(i);
    }
  }
}

cudaError_t launch_ck45_fp32c(unsigned flags, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (a.n_phases <= 0) return cudaErrorInvalidValue;
  if (L.grid <= 0 || L.grid > 0x7fffffffLL || L.block <= 0) return cudaErrorInvalidConfiguration;
  const dim3 g((unsigned)L.grid), b((unsigned)L.block);
  if (flags & kKmDual) ck_phased_fp32c_kernel<true><<<g, b, 0, s>>>(a);
  else ck_phased_fp32c_kernel<false><<<g, b, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ens
