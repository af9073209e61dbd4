// fcmp.cuh -- compares, max / min and clamps of doubles on the integer pipe.
#pragma once

#include "common.cuh"

namespace ens {

// Compares, max / min and clamps of doubles on the integer pipe.  On this
// part the FP64 pipe carries every flop of the solver and is the bottleneck; a
// compare or a min / max costs it a full FP64 issue slot, the same as an FMA.
// For x >= +0 (with +inf, and NaN with its sign bit clear, above every finite
// value) the IEEE bit pattern read as a signed 64-bit integer orders exactly
// as the value does, so these need no FP64 instruction.  For doubles of
// either sign, okey() flips the magnitude bits of negatives, which orders all
// finite values (with -0 just below +0).
__device__ __forceinline__ long long nnbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double absd(double x) {
  return __hiloint2double(__double2hiint(x) & 0x7fffffff, __double2loint(x));
}
// a, b >= +0 or NaN (sign clear): NaN dominates max
__device__ __forceinline__ double nnmax(double a, double b) { return nnbits(a) >= nnbits(b) ? a : b; }
__device__ __forceinline__ double nnmin(double a, double b) { return nnbits(a) <= nnbits(b) ? a : b; }
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
// the larger / smaller of two finite doubles, keeping `a` on ties (as
// `if (b > a) a = b` does)
__device__ __forceinline__ double omax(double a, double b) { return okey(b) > okey(a) ? b : a; }
__device__ __forceinline__ double omin(double a, double b) { return okey(b) < okey(a) ? b : a; }

// the next step proposal after an accepted trial, within [dt_min, dt_max]
__device__ __forceinline__ double bounded_step(double h, double fac, double dt_min, double dt_max) {
  return nnmax(nnmin(h * fac, dt_max), dt_min);
}

}  // namespace ens
