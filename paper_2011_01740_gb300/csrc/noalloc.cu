// noalloc.cu -- ens_solve_noalloc: the adaptive Cash-Karp solve for callers
// that cannot allocate device memory.
//
// The regular entry points allocate their own device buffers (ens_create
// cudaMallocs the context's state, outputs and scratch).  Some callers cannot
// do that: a host process whose device memory is owned by another allocator
// (a framework's caching pool, a preallocated arena in a real-time or embedded
// deployment) that must not be fragmented or bypassed, or a plugin that is
// only handed device buffers by its host.  This entry point takes every input
// and output as a caller-owned device buffer and never allocates: the only
// memory it needs besides the caller's buffers -- the work-stealing claim
// counter, the OR of the status words and the longest-first claim order -- is
// a fixed array declared in this file.
#include <mutex>

#include "common.cuh"

namespace ens {
cudaError_t launch_ck45(int sys, unsigned flags, const AdaptArgs& a, AdaptLaunch L, cudaStream_t s);
cudaError_t launch_order(const int64_t* steps, int64_t n, int32_t* order, unsigned* hist, cudaStream_t s);
void set_call_error(const char* msg);  // text returned by ens_last_error(NULL)
}  // namespace ens

using namespace ens;

namespace {

// Largest ensemble this entry point accepts: the claim order needs one int32
// per system.
constexpr int64_t kNoAllocMaxSystems = 1 << 20;
constexpr size_t kOffHist = 256;                           // after the Scratch words
constexpr size_t kOffFlags = kOffHist + 2 * 256 * sizeof(unsigned);
constexpr size_t kOffOrder = kOffFlags + 256;
constexpr size_t kScratchBytes = kOffOrder + (size_t)kNoAllocMaxSystems * sizeof(int32_t);  // ~4.2 MB

// The scratch.  Every GPU that loads the library holds one copy until the
// process exits.  In host code its name only stands in for the symbol; the
// device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {nullptr};
int g_sm_count[kMaxDevices] = {0};

// Device address of the scratch on the current device (looked up once per
// device, with that device current).
cudaError_t scratch_for_device(int dev, unsigned char** ptr, int* sms) {
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    g_sm_count[dev] = n;
  }
  *ptr = g_scratch_addr[dev];
  *sms = g_sm_count[dev];
  return cudaSuccess;
}

ens_status fail(ens_status st, const char* msg) {
  set_call_error(msg);
  return st;
}

// Whether p is memory that a kernel on device `dev` may address directly:
// device memory of that device, or managed memory.  Device memory of another
// GPU is refused: the kernel would reach it as a peer address, which faults
// unless peer access is enabled.  cudaGetLastError clears only the error a
// failed attribute query of this call left, not one of the caller's.
bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeDevice && at.device == dev;
}

}  // namespace

extern "C" ens_status ens_solve_noalloc(ens_system sys, int64_t n, const double* params, const double* y0,
                                        const double t_span[2], const ens_tol* tol, double* y, double* t_out,
                                        double* dt_out, double* acc, int32_t* status, int64_t* nacc,
                                        int64_t* nrej, int64_t* nrhs, int32_t cost_order, void* stream) {
  if (!tol || !t_span || n < 0) return fail(ENS_EINVAL, "ens_solve_noalloc: NULL tol / t_span or n < 0");
  if (n > kNoAllocMaxSystems)
    return fail(ENS_EINVAL, "ens_solve_noalloc: n exceeds the fixed scratch (at most 1048576 systems)");
  if (sys != ENS_SYS_KELLER_MIKSIS && sys != ENS_SYS_RELIEF_VALVE)
    return fail(ENS_ENOTSUP, "ens_solve_noalloc: Keller-Miksis (phase mode) or relief valve (events) only");
  if (tol->prec != ENS_FP64) return fail(ENS_ENOTSUP, "ens_solve_noalloc: FP64 only");
  if ((sys == ENS_SYS_KELLER_MIKSIS) != (tol->n_phases > 0))
    return fail(ENS_EINVAL, "ens_solve_noalloc: Keller-Miksis needs n_phases > 0, the relief valve n_phases = 0");
  // the same validation as ens_create (tolerances, steps, phases, event band)
  const ens_status tst = check_tol(nullptr, ENS_RKCK45, sys, *tol);
  if (tst != ENS_OK) return tst;
  if (sys == ENS_SYS_RELIEF_VALVE && !(t_span[1] > t_span[0]))
    return fail(ENS_EINVAL, "ens_solve_noalloc: t_span[1] must exceed t_span[0]");
  if (n == 0) return ENS_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(ENS_ECUDA, "ens_solve_noalloc: no current device");
  }
  const void* arrays[] = {params, y0, y, t_out, dt_out, acc, status, nacc, nrej, nrhs};
  for (const void* p : arrays)
    if (!on_device(p, dev))
      return fail(ENS_EINVAL, "ens_solve_noalloc: every array must be device (or managed) memory of the current device");
  unsigned char* base = nullptr;
  int sms = 0;
  if (scratch_for_device(dev, &base, &sms) != cudaSuccess)
    return fail(ENS_ECUDA, "ens_solve_noalloc: cudaGetSymbolAddress of the scratch failed");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch* scr = reinterpret_cast<Scratch*>(base);
  unsigned* hist = reinterpret_cast<unsigned*>(base + kOffHist);
  unsigned* flags_d = reinterpret_cast<unsigned*>(base + kOffFlags);
  int32_t* order = reinterpret_cast<int32_t*>(base + kOffOrder);

  unsigned flags = 0;
  if (sys == ENS_SYS_KELLER_MIKSIS) {
    if (cudaMemsetAsync(flags_d, 0, sizeof(unsigned), s) != cudaSuccess)
      return fail(ENS_ECUDA, "ens_solve_noalloc: clearing the scratch failed");
    if (launch_km_flags(params, n, flags_d, s) != cudaSuccess ||
        cudaMemcpyAsync(&flags, flags_d, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return fail(ENS_ECUDA, "ens_solve_noalloc: kernel selection failed");
  }

  AdaptArgs a{};
  a.n = n;
  a.params = params;
  a.y0 = y0;
  a.y = y;
  a.t_out = t_out;
  a.dt_out = dt_out;
  a.acc = acc;
  a.status = status;
  a.nacc = nacc;
  a.nrej = nrej;
  a.nrhs = nrhs;
  a.scratch = scr;
  a.rtol = tol->rtol;
  a.atol = tol->atol;
  a.dt0 = tol->dt0;
  a.dt_min = tol->dt_min;
  a.dt_max = tol->dt_max;
  a.event_tol = tol->event_tol;
  a.t0 = t_span[0];
  a.t1 = t_span[1];
  a.phase_len = tol->phase_len;
  a.acc_t_start = tol->acc_t_start;
  a.max_steps = tol->max_steps;
  a.n_phases = tol->n_phases;
  a.n_transient = tol->n_transient;
  a.timeout_ns = (uint64_t)((tol->timeout_s > 0.0 ? tol->timeout_s : 600.0) * 1e9);

  // the claim counter and the status OR must start at zero on every call
  if (cudaMemsetAsync(scr, 0, sizeof(Scratch), s) != cudaSuccess)
    return fail(ENS_ECUDA, "ens_solve_noalloc: clearing the scratch failed");
  if (cost_order) {
    AdaptArgs p = a;
    p.persistent = 0;
    if (p.n_phases > 0) p.n_phases = 1;
    else p.t1 = p.t0 + (p.t1 - p.t0) / 16.0;
    p.rtol = p.rtol > kPilotTol ? p.rtol : kPilotTol;
    p.atol = p.atol > kPilotTol ? p.atol : kPilotTol;
    if (launch_ck45(sys, flags, p, AdaptLaunch{(n + 127) / 128, 128}, s) != cudaSuccess ||
        launch_order(nacc, n, order, hist, s) != cudaSuccess ||
        cudaMemsetAsync(scr, 0, sizeof(Scratch), s) != cudaSuccess)
      return fail(ENS_ECUDA, "ens_solve_noalloc: claim-order pass failed");
    a.order = order;
  }
  a.persistent = 1;
  int64_t grid = sms;  // one block of 128 lanes per SM
  const int64_t need = (n + 127) / 128;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  if (launch_ck45(sys, flags, a, AdaptLaunch{grid, 128}, s) != cudaSuccess)
    return fail(ENS_ECUDA, "ens_solve_noalloc: launch failed");
  return ENS_OK;
}
