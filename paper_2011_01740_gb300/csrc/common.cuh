// common.cuh -- types and helpers shared by the solver kernels and the C ABI.
//
// Layout convention (all kernels): structure-of-arrays, element k of system i
// at [k * n + i], so that one warp touching 32 consecutive systems issues one
// coalesced 256-byte access per element.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ens.h"

namespace ens {

constexpr int kMaxDim = 3;
constexpr int kMaxPar = 13;
constexpr int kRing = 32;             // relief valve: Poincare maxima kept
constexpr int kPrvAccRows = kRing + 3;
constexpr int kEventRetries = 40;     // consecutive event-location retries allowed

// Keller-Miksis kernel selection flags (set by the host from the parameters).
constexpr unsigned kKmDual = 1u;             // some system has C6 or C8 != 0
constexpr unsigned kKmGeneralExponent = 2u;  // some system's C10 is not 21/5

// Per-system status bits (mirror ENS_SYS_* of ens.h).
constexpr int32_t kStDtUnderflow = ENS_SYS_DT_UNDERFLOW;
constexpr int32_t kStMaxSteps = ENS_SYS_MAX_STEPS;
constexpr int32_t kStNonFinite = ENS_SYS_NONFINITE;
constexpr int32_t kStEventNoConverge = ENS_SYS_EVENT_NO_CONVERGE;
constexpr int32_t kStTimeout = ENS_SYS_TIMEOUT;

inline int sys_dim(int sys) {
  switch (sys) {
    case ENS_SYS_TOY_X2P: return 1;
    case ENS_SYS_LORENZ: return 3;
    case ENS_SYS_KELLER_MIKSIS: return 2;
    case ENS_SYS_RELIEF_VALVE: return 3;
    case ENS_SYS_KELLER_MIKSIS_TANGENT: return 4;
    default: return 0;
  }
}

// Systems whose parameters are the Keller-Miksis coefficients C0..C12.
inline bool is_km(int sys) { return sys == ENS_SYS_KELLER_MIKSIS || sys == ENS_SYS_KELLER_MIKSIS_TANGENT; }

inline int sys_npar(int sys) {
  switch (sys) {
    case ENS_SYS_TOY_X2P: return 1;
    case ENS_SYS_LORENZ: return 3;
    case ENS_SYS_KELLER_MIKSIS: return 13;
    case ENS_SYS_RELIEF_VALVE: return 5;
    case ENS_SYS_KELLER_MIKSIS_TANGENT: return 13;
    default: return 0;
  }
}

// Device scratch of one context: the work-stealing claim counter and the OR
// of all per-system status words.  Reset to zero before every solve.
struct Scratch {
  unsigned long long next;   // next unclaimed position in the claim order
  unsigned int any_status;   // OR of status words of finished systems
  unsigned int pad;
};

// Arguments of the fixed-step kernels.
struct Rk4Args {
  int64_t n;
  const double* params;  // [npar][n]
  const double* y0;      // [dim][n]
  double* y;             // [dim][n]
  double* t_out;         // [n]
  double* dt_out;        // [n]
  int32_t* status;       // [n]
  int64_t* nacc;         // [n]
  int64_t* nrej;         // [n]
  int64_t* nrhs;         // [n]
  Scratch* scratch;
  double t0, dt;
  int64_t nsteps;
};

// Arguments of the adaptive kernels.
struct AdaptArgs {
  int64_t n;
  const double* params;  // [npar][n]
  const double* y0;      // [dim][n]
  double* y;             // [dim][n]
  double* t_out;         // [n]
  double* dt_out;        // [n]
  double* acc;           // [rows][n]
  int32_t* status;       // [n]
  int64_t* nacc;         // [n]
  int64_t* nrej;         // [n]
  int64_t* nrhs;         // [n]
  const int32_t* order;  // claim order (persistent mode), may be null
  Scratch* scratch;
  double rtol, atol, dt0, dt_min, dt_max, event_tol;
  double t0, t1, phase_len, acc_t_start;
  int64_t max_steps;
  int32_t n_phases;
  int32_t n_transient;   // phases before this one are not recorded
  int32_t acc_phases;    // recorded phases of the accessory layout (rows of per-phase hooks follow
                         // the 2 acc_phases max / min rows)
  int32_t persistent;
  int32_t pair;          // kCashKarp or kDormandPrince
  uint64_t timeout_ns;
  // phase mode, persistent, longest-first, one block per SM: the first claims
  // go to the lanes of warps that own their sub-partition first (see
  // claim_first_by_subpartition); 0 elsewhere
  int32_t first_by_subpartition;
};

// Grid of an adaptive launch.
struct AdaptLaunch {
  int64_t grid;
  int block;
  int spt = 1;  // systems per thread (2: the persistent Keller-Miksis phase-mode kernel)
};

// Nanosecond wall clock of the GPU (PTX %globaltimer).
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Cash & Karp (ACM TOMS 16(3), 1990) embedded 4(5) pair, written as exact
// rationals; kB* are the fifth-order weights that advance the solution, kD*
// the differences b - b* of the error estimate (b2 = b*2 = 0, b5 = 0).
namespace ck {
constexpr double c2 = 1.0 / 5.0, c3 = 3.0 / 10.0, c4 = 3.0 / 5.0, c5 = 1.0, c6 = 7.0 / 8.0;
constexpr double a21 = 1.0 / 5.0;
constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
constexpr double a41 = 3.0 / 10.0, a42 = -9.0 / 10.0, a43 = 6.0 / 5.0;
constexpr double a51 = -11.0 / 54.0, a52 = 5.0 / 2.0, a53 = -70.0 / 27.0, a54 = 35.0 / 27.0;
constexpr double a61 = 1631.0 / 55296.0, a62 = 175.0 / 512.0, a63 = 575.0 / 13824.0,
                 a64 = 44275.0 / 110592.0, a65 = 253.0 / 4096.0;
constexpr double b1 = 37.0 / 378.0, b3 = 250.0 / 621.0, b4 = 125.0 / 594.0, b6 = 512.0 / 1771.0;
constexpr double bs1 = 2825.0 / 27648.0, bs3 = 18575.0 / 48384.0, bs4 = 13525.0 / 55296.0,
                 bs5 = 277.0 / 14336.0, bs6 = 1.0 / 4.0;
constexpr double d1 = b1 - bs1, d3 = b3 - bs3, d4 = b4 - bs4, d5 = -bs5, d6 = b6 - bs6;
}  // namespace ck

// Dormand & Prince (1980) 5(4) pair.  The seventh stage (c7 = 1) has the
// fifth-order weights as its coupling row, so its state is the new solution
// and k7 = f(t + h, y5) serves as the next step's k1 (first same as last).
// e_i = b_i - bs_i are the weights of the embedded error estimate.
namespace dp {
constexpr double c2 = 1.0 / 5.0, c3 = 3.0 / 10.0, c4 = 4.0 / 5.0, c5 = 8.0 / 9.0;
constexpr double a21 = 1.0 / 5.0;
constexpr double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
constexpr double a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
constexpr double a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0, a53 = 64448.0 / 6561.0,
                 a54 = -212.0 / 729.0;
constexpr double a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0, a64 = 49.0 / 176.0,
                 a65 = -5103.0 / 18656.0;
constexpr double b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0, b5 = -2187.0 / 6784.0,
                 b6 = 11.0 / 84.0;
constexpr double e1 = b1 - 5179.0 / 57600.0, e3 = b3 - 7571.0 / 16695.0, e4 = b4 - 393.0 / 640.0,
                 e5 = b5 + 92097.0 / 339200.0, e6 = b6 - 187.0 / 2100.0, e7 = -1.0 / 40.0;
}  // namespace dp

// Embedded Runge-Kutta pair of the adaptive kernels.
enum Pair : int { kCashKarp = 0, kDormandPrince = 1 };

// Loosest tolerance of the claim-order pilot.  The pilot only ranks systems by
// their step counts, so it runs at max(tol, 1e-7): a quarter of the steps of a
// 1e-10 pilot, and the claim order never changes what a system computes.
constexpr double kPilotTol = 1e-7;

// Host helpers of abi.cu shared with the other entry points.
// Validates the solver settings of an adaptive or fixed-step solve; on failure
// writes the message to ctx (or, for ctx == nullptr, to ens_last_error(NULL)).
ens_status check_tol(ens_ctx* ctx, ens_solver solver, ens_system sys, const ens_tol& t);
// ORs the Keller-Miksis kernel-selection flags (kKmDual, kKmGeneralExponent)
// of n systems' coefficients C [13][n] into *flags (device memory), on s.
cudaError_t launch_km_flags(const double* C, int64_t n, unsigned* flags, cudaStream_t s);

}  // namespace ens
