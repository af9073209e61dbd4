// abi.cu -- the C ABI of include/ens.h: contexts, host planner, launch
// selection, CUDA-graph replay and the autotuner.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace ens {
cudaError_t launch_rk4(int sys, bool strict, const Rk4Args& a, int block, cudaStream_t s);
cudaError_t launch_ck45(int sys, unsigned flags, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s);
cudaError_t launch_ck45_fp32c(unsigned flags, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s);
cudaError_t launch_ck45_df(unsigned flags, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s);
cudaError_t launch_order(const int64_t* steps, int64_t n, int32_t* order, unsigned* hist,
                         cudaStream_t s);
cudaError_t launch_rhs_eval(int sys, unsigned flags, int64_t n, const double* P, const double* t,
                            const double* y, double* dy, cudaStream_t s);
}  // namespace ens

using namespace ens;

struct ens_ctx {
  int device = 0;
  int sm_count = 0;
  ens_system sys = ENS_SYS_TOY_X2P;
  ens_solver solver = ENS_RK4;
  ens_tol tol{};
  int64_t n = 0;
  int dim = 0, npar = 0;
  int64_t acc_rows = 0;
  double t0 = 0.0, t1 = 0.0;
  unsigned km_flags = 0;  // Keller-Miksis kernel selection (kKmDual, kKmGeneralExponent)
  // device buffers
  double* params = nullptr;
  double* y0 = nullptr;
  double* y = nullptr;
  double* t_out = nullptr;
  double* dt_out = nullptr;
  double* acc = nullptr;
  int32_t* status = nullptr;
  int64_t* nacc = nullptr;
  int64_t* nrej = nullptr;
  int64_t* nrhs = nullptr;
  int32_t* order = nullptr;     // claim order (cost_order)
  unsigned* hist = nullptr;     // histogram scratch of the claim-order sort
  Scratch* scratch = nullptr;
  ens_launch launch{};
  // CUDA graph of one solve
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t graph_stream = nullptr;
  bool graph_valid = false;
  cudaStream_t last_stream = nullptr;
  // events around the main solve kernel of the last solve (ens_kernel_ms)
  cudaEvent_t kev[2] = {nullptr, nullptr};
  bool kev_recorded = false;
  char err[512] = {0};
};

namespace {

thread_local char g_create_err[512] = {0};

void set_err(ens_ctx* c, const char* fmt, ...) {
  char* buf = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
}

ens_status cuda_fail(ens_ctx* c, cudaError_t e, const char* what) {
  set_err(c, "%s: %s", what, cudaGetErrorString(e));
  return ENS_ECUDA;
}

#define ENS_CUDA(ctx, call)                                          \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);       \
  } while (0)

ens_launch default_launch(const ens_ctx* c) {
  ens_launch L{};
  if (c->solver == ENS_RK4) {
    L.mode = ENS_LAUNCH_PLAIN;
    L.block = 32;
    L.blocks_per_sm = 0;
  } else {
    // about one warp per SM sub-partition saturates the FP64 pipe.  More warps
    // share the pipe and lengthen the critical path of the longest system
    // (each warp then advances more slowly); fewer leave the pipe idle on
    // dependent-instruction latency.  Five warps per SM measured fastest on
    // the 362 x 362 Keller-Miksis sweep, with longest-first claiming.
    L.mode = ENS_LAUNCH_PERSISTENT;
    L.block = 160;
    L.blocks_per_sm = 1;
    L.cost_order = 1;
  }
  L.use_graph = 0;
  return L;
}

bool valid_launch(const ens_launch& L) {
  if (L.mode != ENS_LAUNCH_PLAIN && L.mode != ENS_LAUNCH_PERSISTENT) return false;
  if (L.block < 32 || L.block > 256 || (L.block % 32) != 0) return false;
  if (L.mode == ENS_LAUNCH_PERSISTENT && (L.blocks_per_sm < 1 || L.blocks_per_sm > 32)) return false;
  return true;
}

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void**)p, count * sizeof(T));
}

void free_buffers(ens_ctx* c) {
  cudaFree(c->params);
  cudaFree(c->y0);
  cudaFree(c->y);
  cudaFree(c->t_out);
  cudaFree(c->dt_out);
  cudaFree(c->acc);
  cudaFree(c->status);
  cudaFree(c->nacc);
  cudaFree(c->nrej);
  cudaFree(c->nrhs);
  cudaFree(c->order);
  cudaFree(c->hist);
  cudaFree(c->scratch);
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  for (cudaEvent_t& e : c->kev) {
    if (e) cudaEventDestroy(e);
    e = nullptr;
  }
}

// Record one of the main-kernel timing events on s.  Inside a stream capture
// the record becomes an event node of the graph (external record), so every
// replay of the graph records it again.
cudaError_t record_kernel_event(ens_ctx* c, int which, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  return cs == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(c->kev[which], s, cudaEventRecordExternal)
                                             : cudaEventRecord(c->kev[which], s);
}

ens_status detect_flags(ens_ctx* c) {
  c->km_flags = 0;
  if (!is_km(c->sys) || c->n == 0) return ENS_OK;
  ENS_CUDA(c, cudaMemset(&c->scratch->any_status, 0, sizeof(unsigned)));
  ENS_CUDA(c, launch_km_flags(c->params, c->n, &c->scratch->any_status, 0));
  unsigned flag = 0;
  ENS_CUDA(c, cudaMemcpy(&flag, &c->scratch->any_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  c->km_flags = flag;
  return ENS_OK;
}

uint64_t timeout_ns(const ens_tol& t) {
  const double s = t.timeout_s > 0.0 ? t.timeout_s : 600.0;
  return (uint64_t)(s * 1e9);
}

// the adaptive kernel of the context's precision
cudaError_t launch_adaptive(const ens_ctx* c, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s) {
  if (c->tol.prec == ENS_FP32_COMP) return launch_ck45_fp32c(c->km_flags, a, L, s);
  if (c->tol.prec == ENS_FP32X2) return launch_ck45_df(c->km_flags, a, L, s);
  return launch_ck45(c->sys, c->km_flags, a, L, s);
}

AdaptArgs adapt_args(ens_ctx* c) {
  AdaptArgs a{};
  a.n = c->n;
  a.params = c->params;
  a.y0 = c->y0;
  a.y = c->y;
  a.t_out = c->t_out;
  a.dt_out = c->dt_out;
  a.acc = c->acc;
  a.status = c->status;
  a.nacc = c->nacc;
  a.nrej = c->nrej;
  a.nrhs = c->nrhs;
  a.order = nullptr;
  a.scratch = c->scratch;
  a.rtol = c->tol.rtol;
  a.atol = c->tol.atol;
  a.dt0 = c->tol.dt0;
  a.dt_min = c->tol.dt_min;
  a.dt_max = c->tol.dt_max;
  a.event_tol = c->tol.event_tol;
  a.t0 = c->t0;
  a.t1 = c->t1;
  a.phase_len = c->tol.phase_len;
  a.acc_t_start = c->tol.acc_t_start;
  a.max_steps = c->tol.max_steps;
  a.n_phases = c->tol.n_phases;
  a.n_transient = c->tol.n_transient;
  a.acc_phases = c->tol.n_phases - c->tol.n_transient;
  a.persistent = 0;
  a.pair = c->solver == ENS_DOPRI5 ? kDormandPrince : kCashKarp;
  a.timeout_ns = timeout_ns(c->tol);
  return a;
}

AdaptLaunch adapt_launch(const ens_ctx* c, const ens_launch& L) {
  AdaptLaunch out;
  out.block = L.block;
  if (L.mode == ENS_LAUNCH_PERSISTENT) {
    out.grid = (int64_t)c->sm_count * L.blocks_per_sm;
    const int64_t need = (c->n + L.block - 1) / L.block;  // never more lanes than systems
    if (out.grid > need) out.grid = need;
    if (out.grid < 1) out.grid = 1;
  } else {
    out.grid = (c->n + L.block - 1) / L.block;
  }
  return out;
}

// Enqueue one solve (no graph).  `L` is the launch to use; `shorten` > 0 runs
// a reduced problem for tuning and planning (phases / horizon / steps cut).

ens_status enqueue_solve(ens_ctx* c, const ens_launch& L, cudaStream_t s, int shorten) {
  ENS_CUDA(c, cudaMemsetAsync(c->scratch, 0, sizeof(Scratch), s));
  if (c->solver == ENS_RK4) {
    Rk4Args a{};
    a.n = c->n;
    a.params = c->params;
    a.y0 = c->y0;
    a.y = c->y;
    a.t_out = c->t_out;
    a.dt_out = c->dt_out;
    a.status = c->status;
    a.nacc = c->nacc;
    a.nrej = c->nrej;
    a.nrhs = c->nrhs;
    a.scratch = c->scratch;
    a.t0 = c->t0;
    a.dt = c->tol.dt0;
    a.nsteps = shorten > 0 ? std::min<int64_t>(c->tol.n_steps, shorten) : c->tol.n_steps;
    ENS_CUDA(c, record_kernel_event(c, 0, s));
    cudaError_t e = launch_rk4(c->sys, c->tol.prec == ENS_FP64_STRICT, a, L.block, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "rk4 launch");
    ENS_CUDA(c, record_kernel_event(c, 1, s));
    c->kev_recorded = true;
    return ENS_OK;
  }
  if (c->tol.prec == ENS_FP32X2 && (c->km_flags & kKmGeneralExponent)) {
    set_err(c, "ENS_FP32X2 needs C10 = 21/5 (polytropic exponent 1.4) in every system");
    return ENS_ENOTSUP;
  }
  AdaptArgs a = adapt_args(c);
  if (shorten > 0) {
    if (a.n_phases > 0) a.n_phases = std::min<int32_t>(a.n_phases, shorten);
    else a.t1 = a.t0 + (a.t1 - a.t0) / 16.0;
  }
  a.persistent = L.mode == ENS_LAUNCH_PERSISTENT;
  if (a.persistent && L.cost_order && shorten == 0) {
    // pilot: one phase (or 1/16 of the horizon) of every system in plain
    // mode, then order systems by decreasing pilot step count.  The pilot
    // only ranks the systems, so it runs at a tolerance of at least 1e-7: a
    // quarter of the steps of a 1e-10 pilot, and on the 362 x 362
    // Keller-Miksis sweep a whole solve 1.4 % faster with the same results
    // (the claim order never changes what a system computes).
    AdaptArgs p = a;
    p.persistent = 0;
    if (p.n_phases > 0) p.n_phases = 1;
    else p.t1 = p.t0 + (p.t1 - p.t0) / 16.0;
    p.rtol = p.rtol > kPilotTol ? p.rtol : kPilotTol;
    p.atol = p.atol > kPilotTol ? p.atol : kPilotTol;
    AdaptLaunch PL{(c->n + 127) / 128, 128};
    cudaError_t e = launch_adaptive(c, p, PL, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "pilot launch");
    e = launch_order(c->nacc, c->n, c->order, c->hist, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "order launch");
    ENS_CUDA(c, cudaMemsetAsync(c->scratch, 0, sizeof(Scratch), s));
    a.order = c->order;
  }
  AdaptLaunch AL = adapt_launch(c, L);
  ENS_CUDA(c, record_kernel_event(c, 0, s));
  cudaError_t e = launch_adaptive(c, a, AL, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "adaptive launch");
  ENS_CUDA(c, record_kernel_event(c, 1, s));
  c->kev_recorded = true;
  return ENS_OK;
}

std::mutex g_tune_mu;

}  // namespace

namespace ens {
// Message of a failed call that has no context, returned by ens_last_error(NULL).
void set_call_error(const char* msg) { set_err(nullptr, "%s", msg); }

// Keller-Miksis kernel selection: bit kKmDual if any system drives with a
// second frequency (C6 or C8 != 0), bit kKmGeneralExponent if any C10 is not
// within 4 ulp of 21/5 (then pow() is used instead of the fifth-root form).
__global__ void km_flags_kernel(const double* C, int64_t n, unsigned* flags) {
  const double lo = 4.2 - 4 * 8.881784197001252e-16, hi = 4.2 + 4 * 8.881784197001252e-16;
  unsigned f = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (C[6 * n + i] != 0.0 || C[8 * n + i] != 0.0) f |= kKmDual;
    const double e = C[10 * n + i];
    if (!(e >= lo && e <= hi)) f |= kKmGeneralExponent;
  }
  if (f) atomicOr(flags, f);
}

cudaError_t launch_km_flags(const double* C, int64_t n, unsigned* flags, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  km_flags_kernel<<<(unsigned)blocks, 256, 0, s>>>(C, n, flags);
  return cudaGetLastError();
}

ens_status check_tol(ens_ctx* c, ens_solver solver, ens_system sys, const ens_tol& t) {
  if (solver == ENS_RK4) {
    if (!(t.dt0 > 0.0) || t.n_steps < 0) {
      set_err(c, "RK4 needs dt0 > 0 and n_steps >= 0");
      return ENS_EINVAL;
    }
    if (sys != ENS_SYS_TOY_X2P && sys != ENS_SYS_LORENZ) {
      set_err(c, "RK4 runs the smooth systems (x2p, Lorenz); the relief valve needs event "
                 "handling and Keller-Miksis needs step control");
      return ENS_ENOTSUP;
    }
    if (t.prec != ENS_FP64 && t.prec != ENS_FP64_STRICT) {
      set_err(c, "RK4 supports ENS_FP64 and ENS_FP64_STRICT");
      return ENS_ENOTSUP;
    }
    return ENS_OK;
  }
  if (!(t.rtol >= 0.0) || !(t.atol >= 0.0) || !(t.rtol > 0.0 || t.atol > 0.0) || !(t.dt0 > 0.0) ||
      !(t.dt_min > 0.0) || !(t.dt_max >= t.dt_min) || t.max_steps <= 0 || t.n_phases < 0) {
    set_err(c, "adaptive solve needs rtol, atol >= 0 (not both 0), 0 < dt_min <= dt_max, dt0 > 0, "
               "max_steps > 0, n_phases >= 0");
    return ENS_EINVAL;
  }
  if (t.n_phases > 0 && !(t.phase_len > 0.0)) {
    set_err(c, "phase mode needs phase_len > 0");
    return ENS_EINVAL;
  }
  if (t.n_transient < 0 || (t.n_phases > 0 ? t.n_transient >= t.n_phases : t.n_transient != 0)) {
    set_err(c, "n_transient must satisfy 0 <= n_transient < n_phases (0 outside phase mode)");
    return ENS_EINVAL;
  }
  if (sys == ENS_SYS_RELIEF_VALVE && !(t.event_tol > 0.0)) {
    set_err(c, "the relief valve needs event_tol > 0");
    return ENS_EINVAL;
  }
  if (sys == ENS_SYS_KELLER_MIKSIS_TANGENT && !(t.n_phases > 0 && t.prec == ENS_FP64)) {
    set_err(c, "the tangent system runs in phase mode (n_phases > 0) in FP64");
    return ENS_ENOTSUP;
  }
  if (sys == ENS_SYS_RELIEF_VALVE && t.n_phases > 0) {
    set_err(c, "the relief valve runs in event mode (n_phases must be 0)");
    return ENS_ENOTSUP;
  }
  if ((t.prec == ENS_FP32_COMP || t.prec == ENS_FP32X2) &&
      !(sys == ENS_SYS_KELLER_MIKSIS && t.n_phases > 0 && solver == ENS_RKCK45)) {
    set_err(c, "ENS_FP32_COMP and ENS_FP32X2 are implemented for the Keller-Miksis phase mode with Cash-Karp");
    return ENS_ENOTSUP;
  }
  if (t.prec != ENS_FP64 && t.prec != ENS_FP32_COMP && t.prec != ENS_FP32X2) {
    set_err(c, "adaptive solves support ENS_FP64, ENS_FP32_COMP and ENS_FP32X2");
    return ENS_ENOTSUP;
  }
  return ENS_OK;
}

}  // namespace ens

namespace {

std::map<std::tuple<int, int, int, int64_t, int, int>, ens_launch> g_tune_cache;

}  // namespace

extern "C" {

const char* ens_version(void) { return "ens 0.1 (sm_103a)"; }

ens_status ens_create(ens_ctx** out, ens_system sys, int64_t n, const double* params,
                      const double* y0, const double t_span[2], ens_solver solver,
                      const ens_tol* tol) {
  if (!out) {
    set_err(nullptr, "out is NULL");
    return ENS_EINVAL;
  }
  *out = nullptr;
  if (n < 0 || !tol || !t_span || (n > 0 && (!params || !y0))) {
    set_err(nullptr, "bad arguments: n < 0 or a NULL tol / t_span / params / y0");
    return ENS_EINVAL;
  }
  if (sys_dim(sys) == 0) {
    set_err(nullptr, "unknown system %d", (int)sys);
    return ENS_EINVAL;
  }
  if (solver != ENS_RK4 && solver != ENS_RKCK45 && solver != ENS_DOPRI5) {
    set_err(nullptr, "unknown solver %d", (int)solver);
    return ENS_EINVAL;
  }
  ens_status st = check_tol(nullptr, solver, sys, *tol);
  if (st != ENS_OK) return st;
  if (solver != ENS_RK4 && tol->n_phases == 0 && !(t_span[1] > t_span[0])) {
    set_err(nullptr, "t_span[1] must exceed t_span[0]");
    return ENS_EINVAL;
  }
  ens_ctx* c = new (std::nothrow) ens_ctx();
  if (!c) {
    set_err(nullptr, "host allocation failed");
    return ENS_ENOMEM;
  }
  c->sys = sys;
  c->solver = solver;
  c->tol = *tol;
  c->n = n;
  c->dim = sys_dim(sys);
  c->npar = sys_npar(sys);
  c->t0 = t_span[0];
  c->t1 = t_span[1];
  if (solver != ENS_RK4) {
    if (tol->n_phases > 0)
      c->acc_rows = (sys == ENS_SYS_KELLER_MIKSIS_TANGENT ? 3 : 2) * (int64_t)(tol->n_phases - tol->n_transient);
    else if (sys == ENS_SYS_RELIEF_VALVE) c->acc_rows = kPrvAccRows;
  }
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
  const size_t nn = (size_t)n;
  if (e == cudaSuccess) e = dalloc(&c->params, nn * c->npar);
  if (e == cudaSuccess) e = dalloc(&c->y0, nn * c->dim);
  if (e == cudaSuccess) e = dalloc(&c->y, nn * c->dim);
  if (e == cudaSuccess) e = dalloc(&c->t_out, nn);
  if (e == cudaSuccess) e = dalloc(&c->dt_out, nn);
  if (e == cudaSuccess) e = dalloc(&c->acc, nn * (size_t)std::max<int64_t>(c->acc_rows, 1));
  if (e == cudaSuccess) e = dalloc(&c->status, nn);
  if (e == cudaSuccess) e = dalloc(&c->nacc, nn);
  if (e == cudaSuccess) e = dalloc(&c->nrej, nn);
  if (e == cudaSuccess) e = dalloc(&c->nrhs, nn);
  if (e == cudaSuccess) e = dalloc(&c->order, nn);
  if (e == cudaSuccess) e = dalloc(&c->hist, 512);
  if (e == cudaSuccess) e = dalloc(&c->scratch, 1);
  if (e == cudaSuccess) e = cudaEventCreate(&c->kev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&c->kev[1]);
  if (e != cudaSuccess) {
    set_err(nullptr, "device allocation: %s", cudaGetErrorString(e));
    free_buffers(c);
    delete c;
    return e == cudaErrorMemoryAllocation ? ENS_ENOMEM : ENS_ECUDA;
  }
  // zero the outputs so that reads before a solve are defined
  const size_t zero_sizes[] = {nn * c->dim * sizeof(double), nn * sizeof(double), nn * sizeof(double),
                               nn * (size_t)std::max<int64_t>(c->acc_rows, 1) * sizeof(double),
                               nn * sizeof(int32_t), nn * sizeof(int64_t), nn * sizeof(int64_t),
                               nn * sizeof(int64_t)};
  void* zero_ptrs[] = {c->y, c->t_out, c->dt_out, c->acc, c->status, c->nacc, c->nrej, c->nrhs};
  for (int k = 0; k < 8 && e == cudaSuccess; ++k)
    if (zero_sizes[k]) e = cudaMemset(zero_ptrs[k], 0, zero_sizes[k]);
  if (e == cudaSuccess && n > 0)
    e = cudaMemcpy(c->params, params, nn * c->npar * sizeof(double), cudaMemcpyDefault);
  if (e == cudaSuccess && n > 0) e = cudaMemcpy(c->y0, y0, nn * c->dim * sizeof(double), cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemset(c->scratch, 0, sizeof(Scratch));
  if (e != cudaSuccess) {
    set_err(nullptr, "input copy: %s", cudaGetErrorString(e));
    free_buffers(c);
    delete c;
    return ENS_ECUDA;
  }
  c->launch = default_launch(c);
  st = detect_flags(c);
  if (st != ENS_OK) {
    set_err(nullptr, "%s", c->err);
    free_buffers(c);
    delete c;
    return st;
  }
  *out = c;
  return ENS_OK;
}

ens_status ens_set_inputs(ens_ctx* c, const double* params, const double* y0, void* stream) {
  if (!c) return ENS_EINVAL;
  if (c->n == 0) return ENS_OK;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn = (size_t)c->n;
  if (params)
    ENS_CUDA(c, cudaMemcpyAsync(c->params, params, nn * c->npar * sizeof(double), cudaMemcpyDefault, s));
  if (y0) ENS_CUDA(c, cudaMemcpyAsync(c->y0, y0, nn * c->dim * sizeof(double), cudaMemcpyDefault, s));
  c->last_stream = s;
  if (params && is_km(c->sys)) {
    ENS_CUDA(c, cudaStreamSynchronize(s));
    const unsigned was = c->km_flags;
    ens_status st = detect_flags(c);
    if (st != ENS_OK) return st;
    if (was != c->km_flags) c->graph_valid = false;
  }
  return ENS_OK;
}

ens_status ens_set_launch(ens_ctx* c, const ens_launch* cfg) {
  if (!c) return ENS_EINVAL;
  ens_launch L = cfg ? *cfg : default_launch(c);
  if (!valid_launch(L)) {
    set_err(c, "invalid launch: mode %d block %d blocks_per_sm %d", L.mode, L.block, L.blocks_per_sm);
    return ENS_EINVAL;
  }
  if (c->solver == ENS_RK4 && L.mode != ENS_LAUNCH_PLAIN) {
    set_err(c, "RK4 runs one system per thread (plain launch)");
    return ENS_ENOTSUP;
  }
  c->launch = L;
  c->graph_valid = false;
  return ENS_OK;
}

ens_status ens_get_launch(const ens_ctx* c, ens_launch* cfg) {
  if (!c || !cfg) return ENS_EINVAL;
  *cfg = c->launch;
  return ENS_OK;
}

ens_status ens_solve(ens_ctx* c, void* stream) {
  if (!c) return ENS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  if (c->n == 0) return ENS_OK;
  if (!c->launch.use_graph) return enqueue_solve(c, c->launch, s, 0);
  if (!c->graph_valid || c->graph_stream != s) {
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->gexec = nullptr;
    cudaGraph_t g = nullptr;
    // a private capture stream keeps the caller's stream free of capture state
    cudaStream_t cap = nullptr;
    ENS_CUDA(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      cudaStreamDestroy(cap);
      return cuda_fail(c, e, "cudaStreamBeginCapture");
    }
    ens_status st = enqueue_solve(c, c->launch, cap, 0);
    e = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (st != ENS_OK) {
      if (g) cudaGraphDestroy(g);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&c->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    c->graph_valid = true;
    c->graph_stream = s;
  }
  ENS_CUDA(c, cudaGraphLaunch(c->gexec, s));
  return ENS_OK;
}

ens_status ens_sync(ens_ctx* c) {
  if (!c) return ENS_EINVAL;
  ENS_CUDA(c, cudaStreamSynchronize(c->last_stream));
  if (c->n == 0) return ENS_OK;
  unsigned any = 0;
  ENS_CUDA(c, cudaMemcpy(&any, &c->scratch->any_status, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (any & kStTimeout) {
    set_err(c, "solve stopped at its wall-clock budget (%.1f s)", c->tol.timeout_s);
    return ENS_ETIMEOUT;
  }
  if (any) {
    set_err(c, "some systems finished with status bits 0x%x", any);
    return ENS_ESYSTEM;
  }
  return ENS_OK;
}

ens_status ens_kernel_ms(ens_ctx* c, double* ms) {
  if (!c || !ms) return ENS_EINVAL;
  *ms = 0.0;
  if (!c->kev_recorded) {
    set_err(c, "no solve kernel has been enqueued on this context");
    return ENS_EINVAL;
  }
  float f = 0.0f;
  ENS_CUDA(c, cudaEventElapsedTime(&f, c->kev[0], c->kev[1]));
  *ms = (double)f;
  return ENS_OK;
}

ens_status ens_read(ens_ctx* c, int which, void* dst, size_t dst_bytes) {
  if (!c) return ENS_EINVAL;
  const size_t nn = (size_t)c->n;
  const void* src = nullptr;
  size_t bytes = 0;
  switch (which) {
    case ENS_STATE: src = c->y; bytes = nn * c->dim * sizeof(double); break;
    case ENS_ACC: src = c->acc; bytes = nn * (size_t)c->acc_rows * sizeof(double); break;
    case ENS_STATUS: src = c->status; bytes = nn * sizeof(int32_t); break;
    case ENS_NSTEPS: src = c->nacc; bytes = nn * sizeof(int64_t); break;
    case ENS_NREJ: src = c->nrej; bytes = nn * sizeof(int64_t); break;
    case ENS_NRHS: src = c->nrhs; bytes = nn * sizeof(int64_t); break;
    case ENS_TIME: src = c->t_out; bytes = nn * sizeof(double); break;
    case ENS_DT: src = c->dt_out; bytes = nn * sizeof(double); break;
    default: set_err(c, "unknown selector %d", which); return ENS_EINVAL;
  }
  if (bytes == 0) return ENS_OK;
  if (!dst || dst_bytes < bytes) {
    set_err(c, "destination holds %zu bytes, selector %d needs %zu", dst_bytes, which, bytes);
    return ENS_EINVAL;
  }
  ENS_CUDA(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, c->last_stream));
  ENS_CUDA(c, cudaStreamSynchronize(c->last_stream));
  return ENS_OK;
}

int64_t ens_acc_rows(const ens_ctx* c) { return c ? c->acc_rows : 0; }
int64_t ens_size(const ens_ctx* c) { return c ? c->n : 0; }
int32_t ens_dim(const ens_ctx* c) { return c ? c->dim : 0; }
int32_t ens_npar(const ens_ctx* c) { return c ? c->npar : 0; }

ens_status ens_autotune(ens_ctx* c, void* stream, ens_launch* best) {
  if (!c) return ENS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (c->n == 0) {
    if (best) *best = c->launch;
    return ENS_OK;
  }
  const auto key = std::make_tuple((int)c->sys, (int)c->solver, (int)c->tol.prec, c->n,
                                   (int)c->tol.n_phases, c->device);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      c->launch = it->second;
      c->graph_valid = false;
      if (best) *best = c->launch;
      return ENS_OK;
    }
  }
  std::vector<ens_launch> cands;
  if (c->solver == ENS_RK4) {
    for (int b : {32, 64, 128, 256}) {
      ens_launch L{};
      L.mode = ENS_LAUNCH_PLAIN;
      L.block = b;
      cands.push_back(L);
    }
  } else {
    for (int b : {64, 128}) {
      ens_launch L{};
      L.mode = ENS_LAUNCH_PLAIN;
      L.block = b;
      cands.push_back(L);
    }
    const int shapes[][2] = {{32, 4}, {64, 2}, {128, 1}, {96, 1}, {160, 1}, {192, 1}, {128, 2}, {256, 1}};
    for (const auto& sh : shapes) {
      ens_launch L{};
      L.mode = ENS_LAUNCH_PERSISTENT;
      L.block = sh[0];
      L.blocks_per_sm = sh[1];
      cands.push_back(L);
    }
  }
  const int shorten = c->solver == ENS_RK4 ? 200 : 2;
  cudaEvent_t e0, e1;
  ENS_CUDA(c, cudaEventCreate(&e0));
  ENS_CUDA(c, cudaEventCreate(&e1));
  float best_ms = 1e30f;
  ens_launch best_L = c->launch;
  for (const ens_launch& L : cands) {
    ens_status st = enqueue_solve(c, L, s, shorten);  // warm-up
    if (st != ENS_OK) break;
    ENS_CUDA(c, cudaEventRecord(e0, s));
    st = enqueue_solve(c, L, s, shorten);
    if (st != ENS_OK) break;
    ENS_CUDA(c, cudaEventRecord(e1, s));
    ENS_CUDA(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    ENS_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best_L = L;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  best_L.use_graph = c->launch.use_graph;
  best_L.cost_order = c->launch.cost_order;
  c->launch = best_L;
  c->graph_valid = false;
  c->last_stream = s;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best_L;
  }
  if (best) *best = best_L;
  return ENS_OK;
}

ens_status ens_eval_rhs(ens_system sys, int64_t n, const double* params, const double* t, const double* y,
                        double* dy, void* stream) {
  if (n < 0 || sys_dim(sys) == 0) return ENS_EINVAL;
  if (n == 0) return ENS_OK;
  if (!params || !t || !y || !dy) return ENS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned flags = 0;
  if (is_km(sys)) {
    unsigned* f = nullptr;
    if (cudaMalloc(&f, sizeof(unsigned)) != cudaSuccess) return ENS_ENOMEM;
    cudaMemsetAsync(f, 0, sizeof(unsigned), s);
    cudaError_t e = launch_km_flags(params, n, f, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, f, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(f);
    if (e != cudaSuccess) return ENS_ECUDA;
  }
  return launch_rhs_eval(sys, flags, n, params, t, y, dy, s) == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

const char* ens_last_error(const ens_ctx* c) { return c ? c->err : g_create_err; }

void ens_destroy(ens_ctx* c) {
  if (!c) return;
  free_buffers(c);
  delete c;
}

}  // extern "C"
