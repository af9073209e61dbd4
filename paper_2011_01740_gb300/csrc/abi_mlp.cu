// abi_mlp.cu -- C ABI of the surrogate network (include/ens.h, "Surrogate"):
// model state, training driver, screening, and the device helpers of the
// screening pipeline (features, labels, compaction, merge).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "mlp.cuh"

using namespace ens;

struct ens_mlp {
  int members = 0;
  float* master = nullptr;        // [members][kP]
  __nv_bfloat16* wbf = nullptr;   // [members][kPS]
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grad = nullptr;
  int64_t adam_t = 0;
  // batch scratch
  int64_t cap = 0;
  float* xb = nullptr;
  float* yb = nullptr;
  float* z = nullptr;
  float* gp = nullptr;            // gelu'(z) of the tcgen05 forward, [members][B][4][128]
  float* dz = nullptr;
  float* out = nullptr;
  float* dout = nullptr;
  float* loss = nullptr;          // [members]
  float* gpart = nullptr;         // [kMaxSplits][members][kP] partial gradients of the batch slices
  // training products: 1 tcgen05 kernels (mlp_tc05_train.cu), 0 mma.sync kernels (mlp.cu)
  int train_impl = 1;
  unsigned* train_err = nullptr;  // set by a tcgen05 training kernel whose wait expired
  __nv_bfloat16* wbfT = nullptr;  // [members][3][128][128] transposed hidden weights (tcgen05 backward)
  // screening on the tcgen05 tensor cores
  int screen_impl = 1;            // 1: tcgen05 kernel, 0: mma.sync fused kernel
  float* screen_out = nullptr;    // [members][screen_cap][2]
  int64_t screen_cap = 0;
  unsigned* screen_err = nullptr;
  int sms = 0;
  char err[512] = {0};
};

namespace {

thread_local char g_mlp_err[512] = {0};

void merr(ens_mlp* m, const char* fmt, ...) {
  char* buf = m ? m->err : g_mlp_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
}

#define MLP_CUDA(m, call)                                                   \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      merr((m), "%s: %s", #call, cudaGetErrorString(e_));                   \
      return ENS_ECUDA;                                                     \
    }                                                                       \
  } while (0)

bool is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at{};
  const bool ok = cudaPointerGetAttributes(&at, p) == cudaSuccess;
  cudaGetLastError();
  return ok && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
}

unsigned grid_for(int64_t n, int block = 256, int64_t cap = 8192) {
  int64_t g = (n + block - 1) / block;
  if (g < 1) g = 1;
  return (unsigned)std::min<int64_t>(g, cap);
}

ens_status ensure_batch(ens_mlp* m, int64_t B) {
  if (B <= m->cap) return ENS_OK;
  cudaFree(m->xb);
  cudaFree(m->yb);
  cudaFree(m->z);
  cudaFree(m->gp);
  cudaFree(m->dz);
  cudaFree(m->out);
  cudaFree(m->dout);
  m->xb = m->yb = m->z = m->gp = m->dz = m->out = m->dout = nullptr;
  m->cap = 0;
  const size_t M = (size_t)m->members;
  cudaError_t e = cudaMalloc(&m->xb, B * 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->yb, B * 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->z, M * B * 4 * mlp::H * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->gp, M * B * 4 * mlp::H * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->dz, M * 4 * B * mlp::H * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->out, M * B * 2 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->dout, M * B * 2 * sizeof(float));
  if (e == cudaSuccess && !m->gpart)
    e = cudaMalloc(&m->gpart, (size_t)mlp::kMaxSplits * M * mlp::kP * sizeof(float));
  if (e == cudaSuccess && !m->wbfT) e = cudaMalloc(&m->wbfT, M * 3 * mlp::H * mlp::H * sizeof(__nv_bfloat16));
  if (e == cudaSuccess && !m->train_err) {
    e = cudaMalloc(&m->train_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(m->train_err, 0, sizeof(unsigned));
  }
  if (e != cudaSuccess) {
    merr(m, "batch scratch: %s", cudaGetErrorString(e));
    return ENS_ENOMEM;
  }
  m->cap = B;
  return ENS_OK;
}

// arguments of the tcgen05 training kernels over the batch scratch
mlp::TrainTcArgs tc_args(ens_mlp* m, int64_t B, const float* x, float* out, float* loss, int64_t rows) {
  mlp::TrainTcArgs t{};
  t.n = B;
  t.members = m->members;
  t.x = x;
  t.y = m->yb;
  t.master = m->master;
  t.wbf = m->wbf;
  t.wbfT = m->wbfT;
  t.z = m->z;
  t.gp = m->gp;
  t.out = out;
  t.dout = m->dout;
  t.dz = m->dz;
  t.loss = loss;
  t.grad = m->gpart;
  t.rows = rows;
  t.error = m->train_err;
  return t;
}

// forward (training form) + backward + weight gradients of one batch already
// in m->xb / m->yb; loss[members] accumulates the per-sample loss sum.  The
// gradient is left as slice partials in m->gpart, their number in *splits;
// with splits == nullptr they are summed into m->grad.
ens_status batch_grad(ens_mlp* m, int64_t B, float* loss, cudaStream_t s, int* splits_out) {
  const int splits = mlp::grad_splits(B);
  const int64_t rows = ((B + splits - 1) / splits + mlp::kChunk - 1) / mlp::kChunk * mlp::kChunk;
  if (m->train_impl == 1) {
    // tcgen05: forward, input gradients, weight gradients (the 2-wide layers
    // 1 and 5 in FP32 by blocks of the same launch)
    const mlp::TrainTcArgs t = tc_args(m, B, m->xb, m->out, loss, rows);
    MLP_CUDA(m, mlp::launch_train_tc05(0, t, splits, s));
    MLP_CUDA(m, mlp::launch_train_tc05(1, t, splits, s));
    MLP_CUDA(m, mlp::launch_train_tc05(2, t, splits, s));
  } else {
    mlp::FwdArgs f{};
    f.n = B;
    f.members = m->members;
    f.x = m->xb;
    f.master = m->master;
    f.wbf = m->wbf;
    f.z = m->z;
    f.out = m->out;
    MLP_CUDA(m, mlp::launch_forward_train(f, s));
    mlp::BwdArgs b{};
    b.n = B;
    b.y = m->yb;
    b.master = m->master;
    b.wbf = m->wbf;
    b.z = m->z;
    b.out = m->out;
    b.dout = m->dout;
    b.dz = m->dz;
    b.loss = loss;
    MLP_CUDA(m, mlp::launch_backward(b, m->members, s));
    mlp::GradArgs g{};
    g.n = B;
    g.x = m->xb;
    g.z = m->z;
    g.dz = m->dz;
    g.dout = m->dout;
    g.grad = m->gpart;
    g.rows = rows;
    MLP_CUDA(m, mlp::launch_wgrad(g, m->members, splits, s));
  }
  if (splits_out)
    *splits_out = splits;
  else
    MLP_CUDA(m, mlp::launch_grad_reduce(m->members, splits, m->gpart, m->grad, s));
  return ENS_OK;
}

// after a synchronous call: a tcgen05 training kernel that gave up waiting
// for its tensor cores leaves invalid results
ens_status check_train_err(ens_mlp* m) {
  if (m->train_impl != 1 || !m->train_err) return ENS_OK;
  unsigned e = 0;
  MLP_CUDA(m, cudaMemcpy(&e, m->train_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (e) {
    merr(m, "tcgen05 training kernel: wait for the tensor cores expired");
    return ENS_ECUDA;
  }
  return ENS_OK;
}

ens_status set_smem_attrs(ens_mlp* m) {
  // once per process (thread-safe static initialisation)
  static const cudaError_t attr = mlp::set_smem_limits();
  MLP_CUDA(m, attr);
  return ENS_OK;
}

// ---------------------------------------------------------------------------
// screening-pipeline helpers
// ---------------------------------------------------------------------------

__global__ void km_features_kernel(int64_t n, const double* pA, const double* f, double la0, double la1,
                                   double lf0, double lf1, float* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[2 * i] = (float)(2.0 * (log(pA[i]) - la0) / (la1 - la0) - 1.0);
    x[2 * i + 1] = (float)(2.0 * (log(f[i]) - lf0) / (lf1 - lf0) - 1.0);
  }
}

// Targets from per-phase accessories acc[2 n_phases][n]: y0 = ln(max of the
// per-phase maxima over phases [first, n_phases)), y1 = 1 if those maxima
// spread by less than spread_tol relative (period-1 response), else 0.
__global__ void km_labels_kernel(int64_t n, const double* acc, int n_phases, int first, double spread_tol,
                                 float* y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double mx = -INFINITY, mn = INFINITY;
    for (int p = first; p < n_phases; ++p) {
      const double v = acc[(int64_t)(2 * p) * n + i];
      mx = fmax(mx, v);
      mn = fmin(mn, v);
    }
    y[2 * i] = (float)log(mx);
    y[2 * i + 1] = ((mx - mn) / mx < spread_tol) ? 1.0f : 0.0f;
  }
}

// Deterministic stream compaction of {i : v[i] > thr} in increasing order.
constexpr int kSelBlock = 1024;

// i is selected when v[i] > thr, or, with a second array w, when w[i] > thr_w
__device__ __forceinline__ bool gate(int64_t i, int64_t n, const float* v, float thr, const float* w, float thr_w) {
  return i < n && (v[i] > thr || (w != nullptr && w[i] > thr_w));
}

__global__ void select_count_kernel(int64_t n, const float* v, float thr, const float* w, float thr_w,
                                    unsigned* counts) {
  const int64_t i = blockIdx.x * (int64_t)kSelBlock + threadIdx.x;
  const int c = __syncthreads_count(gate(i, n, v, thr, w, thr_w));
  if (threadIdx.x == 0) counts[blockIdx.x] = (unsigned)c;
}

__global__ void select_scan_kernel(unsigned* counts, int64_t nblocks, long long* total) {
  // one block of 1024 threads; each thread scans a contiguous segment
  __shared__ unsigned long long part[1024];
  const int t = threadIdx.x;
  const int64_t per = (nblocks + 1023) / 1024;
  const int64_t lo = t * per, hi = std::min<int64_t>(nblocks, lo + per);
  unsigned long long s = 0;
  for (int64_t b = lo; b < hi; ++b) s += counts[b];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    unsigned long long run = 0;
    for (int k = 0; k < 1024; ++k) {
      const unsigned long long c = part[k];
      part[k] = run;
      run += c;
    }
    *total = (long long)run;
  }
  __syncthreads();
  unsigned long long run = part[t];
  for (int64_t b = lo; b < hi; ++b) {
    const unsigned c = counts[b];
    counts[b] = (unsigned)run;
    run += c;
  }
}

__global__ void select_scatter_kernel(int64_t n, const float* v, float thr, const float* w, float thr_w,
                                      const unsigned* offs, int32_t* idx) {
  __shared__ unsigned warp_base[kSelBlock / 32];
  const int64_t i = blockIdx.x * (int64_t)kSelBlock + threadIdx.x;
  const bool flag = gate(i, n, v, thr, w, thr_w);
  const unsigned ballot = __ballot_sync(0xffffffffu, flag);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) warp_base[warp] = __popc(ballot);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int w = 0; w < kSelBlock / 32; ++w) {
      const unsigned c = warp_base[w];
      warp_base[w] = run;
      run += c;
    }
  }
  __syncthreads();
  if (flag) {
    const unsigned rank = __popc(ballot & ((1u << lane) - 1u));
    idx[offs[blockIdx.x] + warp_base[warp] + rank] = (int32_t)i;
  }
}

__global__ void gather_f64_kernel(int64_t k, const int32_t* idx, const double* src, double* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[idx[i]];
}

__global__ void scatter_f32_kernel(int64_t k, const int32_t* idx, const float* src, float* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    dst[idx[i]] = src[2 * i];
}

// Steepness of a map v on a rows x cols grid (row-major, columns fastest):
// the largest |v(neighbour) - v| / distance over the up to four neighbours
// `stride` points away (inv_dr, inv_dc: inverse distances at that stride).
__global__ void grid_gradient_kernel(int64_t rows, int64_t cols, int64_t stride, const float* v, float inv_dr,
                                     float inv_dc, float* g) {
  const int64_t n = rows * cols;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / cols, c = i - r * cols;
    const float v0 = v[i];
    float m = 0.f;
    if (r >= stride) m = fmaxf(m, fabsf(v[i - stride * cols] - v0) * inv_dr);
    if (r + stride < rows) m = fmaxf(m, fabsf(v[i + stride * cols] - v0) * inv_dr);
    if (c >= stride) m = fmaxf(m, fabsf(v[i - stride] - v0) * inv_dc);
    if (c + stride < cols) m = fmaxf(m, fabsf(v[i + stride] - v0) * inv_dc);
    g[i] = m;
  }
}

// Five feature points per input point: x, x +- d0 along feature 0, x +- d1
// along feature 1; out [5][n][2].
__global__ void feature_stencil_kernel(int64_t n, const float* x, float d0, float d1, float* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = x[2 * i], b = x[2 * i + 1];
    const float pa[5] = {a, a + d0, a - d0, a, a};
    const float pb[5] = {b, b, b, b + d1, b - d1};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      out[2 * (k * n + i)] = pa[k];
      out[2 * (k * n + i) + 1] = pb[k];
    }
  }
}

// Steepness at stencil centres from the map's values v [5][n] at the points
// of feature_stencil_kernel: the grid gradient's definition on a stencil.
__global__ void stencil_gradient_kernel(int64_t n, const float* v, float inv_d0, float inv_d1, float* g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v0 = v[i];
    float m = fmaxf(fabsf(v[n + i] - v0), fabsf(v[2 * n + i] - v0)) * inv_d0;
    m = fmaxf(m, fmaxf(fabsf(v[3 * n + i] - v0), fabsf(v[4 * n + i] - v0)) * inv_d1);
    g[i] = m;
  }
}

}  // namespace

extern "C" {

ens_status ens_mlp_create(ens_mlp** out, int32_t members, uint64_t seed) {
  if (!out || members < 1 || members > mlp::kMaxMembers) {
    merr(nullptr, "ens_mlp_create: need out != NULL and 1 <= members <= %d", mlp::kMaxMembers);
    return ENS_EINVAL;
  }
  *out = nullptr;
  ens_mlp* m = new (std::nothrow) ens_mlp();
  if (!m) return ENS_ENOMEM;
  m->members = members;
  const size_t tot = (size_t)members * mlp::kP;
  cudaError_t e = cudaMalloc(&m->master, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->wbf, (size_t)members * mlp::kPS * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemset(m->wbf, 0, (size_t)members * mlp::kPS * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc(&m->m1, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->m2, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->grad, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&m->loss, (size_t)members * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->m1, 0, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->m2, 0, tot * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->grad, 0, tot * sizeof(float));
  if (e == cudaSuccess) {
    e = mlp::launch_init(members, seed, m->master, nullptr);
    if (e == cudaSuccess) e = mlp::launch_to_bf16((int64_t)tot, m->master, m->wbf, nullptr);
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  ens_status st = e == cudaSuccess ? set_smem_attrs(m) : ENS_ECUDA;
  if (e != cudaSuccess || st != ENS_OK) {
    merr(nullptr, "ens_mlp_create: %s", e != cudaSuccess ? cudaGetErrorString(e) : m->err);
    cudaFree(m->master);
    cudaFree(m->wbf);
    cudaFree(m->m1);
    cudaFree(m->m2);
    cudaFree(m->grad);
    cudaFree(m->loss);
    delete m;
    return e == cudaErrorMemoryAllocation ? ENS_ENOMEM : ENS_ECUDA;
  }
  *out = m;
  return ENS_OK;
}

int64_t ens_mlp_param_count(void) { return mlp::kP; }

ens_status ens_mlp_set_params(ens_mlp* m, const float* params, size_t bytes) {
  if (!m || !params) return ENS_EINVAL;
  const size_t tot = (size_t)m->members * mlp::kP;
  if (bytes < tot * sizeof(float)) {
    merr(m, "params hold %zu bytes, need %zu", bytes, tot * sizeof(float));
    return ENS_EINVAL;
  }
  MLP_CUDA(m, cudaMemcpy(m->master, params, tot * sizeof(float), cudaMemcpyDefault));
  MLP_CUDA(m, mlp::launch_to_bf16((int64_t)tot, m->master, m->wbf, nullptr));
  MLP_CUDA(m, cudaMemset(m->m1, 0, tot * sizeof(float)));
  MLP_CUDA(m, cudaMemset(m->m2, 0, tot * sizeof(float)));
  MLP_CUDA(m, cudaDeviceSynchronize());
  m->adam_t = 0;
  return ENS_OK;
}

ens_status ens_mlp_get_params(ens_mlp* m, float* params, size_t bytes) {
  if (!m || !params) return ENS_EINVAL;
  const size_t tot = (size_t)m->members * mlp::kP;
  if (bytes < tot * sizeof(float)) {
    merr(m, "params hold %zu bytes, need %zu", bytes, tot * sizeof(float));
    return ENS_EINVAL;
  }
  MLP_CUDA(m, cudaDeviceSynchronize());
  MLP_CUDA(m, cudaMemcpy(params, m->master, tot * sizeof(float), cudaMemcpyDefault));
  return ENS_OK;
}

ens_status ens_mlp_forward(ens_mlp* m, int64_t n, const float* x, float* out, void* stream) {
  if (!m || n < 0) return ENS_EINVAL;
  if (n == 0) return ENS_OK;
  if (!is_device(x) || !is_device(out)) {
    merr(m, "ens_mlp_forward: x and out must be device memory");
    return ENS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ens_status st = ensure_batch(m, n);
  if (st != ENS_OK) return st;
  if (m->train_impl == 1) {
    MLP_CUDA(m, mlp::launch_train_tc05(0, tc_args(m, n, x, out, m->loss, n), 1, s));
    return ENS_OK;
  }
  mlp::FwdArgs f{};
  f.n = n;
  f.members = m->members;
  f.x = x;
  f.master = m->master;
  f.wbf = m->wbf;
  f.z = m->z;
  f.out = out;
  MLP_CUDA(m, mlp::launch_forward_train(f, s));
  return ENS_OK;
}

ens_status ens_mlp_loss_grad(ens_mlp* m, int64_t n, const float* x, const float* y, float* loss, float* grad,
                             void* stream) {
  if (!m || n <= 0 || !loss || !grad) return ENS_EINVAL;
  if (!is_device(x) || !is_device(y)) {
    merr(m, "ens_mlp_loss_grad: x and y must be device memory");
    return ENS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  ens_status st = ensure_batch(m, n);
  if (st != ENS_OK) return st;
  MLP_CUDA(m, cudaMemcpyAsync(m->xb, x, n * 2 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  MLP_CUDA(m, cudaMemcpyAsync(m->yb, y, n * 2 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  MLP_CUDA(m, cudaMemsetAsync(m->loss, 0, m->members * sizeof(float), s));
  MLP_CUDA(m, cudaMemsetAsync(m->train_err, 0, sizeof(unsigned), s));
  st = batch_grad(m, n, m->loss, s, nullptr);
  if (st != ENS_OK) return st;
  std::vector<float> l(m->members);
  MLP_CUDA(m, cudaMemcpyAsync(l.data(), m->loss, m->members * sizeof(float), cudaMemcpyDeviceToHost, s));
  MLP_CUDA(m, cudaMemcpyAsync(grad, m->grad, (size_t)m->members * mlp::kP * sizeof(float), cudaMemcpyDefault, s));
  MLP_CUDA(m, cudaStreamSynchronize(s));
  st = check_train_err(m);
  if (st != ENS_OK) return st;
  for (int k = 0; k < m->members; ++k) loss[k] = l[k] / (float)n;
  return ENS_OK;
}

ens_status ens_mlp_train(ens_mlp* m, int64_t n, const float* x, const float* y, const ens_train_cfg* cfg,
                         float* loss_hist, void* stream) {
  if (!m || n <= 0 || !cfg || cfg->epochs < 0 || cfg->batch <= 0 || !(cfg->lr > 0.f) || !(cfg->lr_final >= 0.f))
    return ENS_EINVAL;
  if (n > 0x7fffffffLL) return ENS_EINVAL;
  if (!is_device(x) || !is_device(y)) {
    merr(m, "ens_mlp_train: x and y must be device memory");
    return ENS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t B = std::min<int64_t>(cfg->batch, n);
  ens_status st = ensure_batch(m, B);
  if (st != ENS_OK) return st;
  int32_t* perm_d = nullptr;
  float* hist_d = nullptr;
  MLP_CUDA(m, cudaMalloc(&perm_d, n * sizeof(int32_t)));
  cudaError_t e = cudaMalloc(&hist_d, (size_t)std::max(1, cfg->epochs) * m->members * sizeof(float));
  if (e != cudaSuccess) {
    cudaFree(perm_d);
    merr(m, "train scratch: %s", cudaGetErrorString(e));
    return ENS_ENOMEM;
  }
  e = cudaMemsetAsync(hist_d, 0, (size_t)std::max(1, cfg->epochs) * m->members * sizeof(float), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->train_err, 0, sizeof(unsigned), s);
  std::vector<int32_t> perm(n);
  const int64_t tot = (int64_t)m->members * mlp::kP;
  const int64_t steps_total = (int64_t)cfg->epochs * ((n + B - 1) / B);
  int64_t step = 0;
  for (int ep = 0; ep < cfg->epochs && e == cudaSuccess; ++ep) {
    // Fisher-Yates with splitmix64 draws (stream seed + epoch)
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    uint64_t ctr = (cfg->seed + 0x51ed2701ULL * (uint64_t)(ep + 1)) << 20;
    for (int64_t i = n - 1; i > 0; --i) {
      const uint64_t r = mlp::splitmix64(ctr++);
      const int64_t j = (int64_t)(r % (uint64_t)(i + 1));
      std::swap(perm[i], perm[j]);
    }
    e = cudaMemcpyAsync(perm_d, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s);
    for (int64_t b0 = 0; b0 < n && e == cudaSuccess; b0 += B) {
      const int64_t nb = std::min<int64_t>(B, n - b0);
      e = mlp::launch_gather(nb, perm_d + b0, x, y, m->xb, m->yb, s);
      if (e != cudaSuccess) break;
      int splits = 1;
      st = batch_grad(m, nb, hist_d + (size_t)ep * m->members, s, &splits);
      if (st != ENS_OK) break;
      m->adam_t += 1;
      const float c1 = 1.0f - powf(cfg->beta1, (float)m->adam_t);
      const float c2 = 1.0f - powf(cfg->beta2, (float)m->adam_t);
      // cosine schedule: lr at the first step, lr_final at the last
      float lr = cfg->lr;
      if (cfg->lr_final > 0.f && steps_total > 1) {
        const double x = (double)step / (double)(steps_total - 1);
        lr = (float)(cfg->lr_final + 0.5 * (cfg->lr - cfg->lr_final) * (1.0 + cos(3.14159265358979323846 * x)));
      }
      ++step;
      e = mlp::launch_adam(tot, m->master, m->wbf, m->gpart, splits, m->m1, m->m2, lr, cfg->beta1, cfg->beta2,
                           cfg->eps, c1, c2, s);
    }
    if (st != ENS_OK) break;
    // the loss accumulates per-sample sums over batches whose gradient was
    // averaged per batch; the epoch value reported is the mean per sample
  }
  if (e == cudaSuccess && st == ENS_OK && loss_hist && cfg->epochs > 0) {
    std::vector<float> h((size_t)cfg->epochs * m->members);
    e = cudaMemcpyAsync(h.data(), hist_d, h.size() * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (size_t k = 0; k < h.size(); ++k) loss_hist[k] = h[k] / (float)n;
  } else if (e == cudaSuccess) {
    e = cudaStreamSynchronize(s);
  }
  cudaFree(perm_d);
  cudaFree(hist_d);
  if (st != ENS_OK) return st;
  if (e != cudaSuccess) {
    merr(m, "training: %s", cudaGetErrorString(e));
    return ENS_ECUDA;
  }
  return check_train_err(m);
}

ens_status ens_mlp_screen(ens_mlp* m, int64_t n, const float* x, float* mean, float* stdv, float* p1,
                          void* stream) {
  if (!m || n < 0) return ENS_EINVAL;
  if (n == 0) return ENS_OK;
  if (!is_device(x) || !is_device(mean) || !is_device(stdv) || !is_device(p1)) {
    merr(m, "ens_mlp_screen: arrays must be device memory");
    return ENS_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (m->screen_impl == 1) {
    if (n > m->screen_cap) {
      cudaFree(m->screen_out);
      m->screen_out = nullptr;
      m->screen_cap = 0;
      MLP_CUDA(m, cudaMalloc(&m->screen_out, (size_t)m->members * n * 2 * sizeof(float)));
      m->screen_cap = n;
    }
    if (!m->screen_err) MLP_CUDA(m, cudaMalloc(&m->screen_err, sizeof(unsigned)));
    if (!m->sms) {
      int dev = 0;
      MLP_CUDA(m, cudaGetDevice(&dev));
      MLP_CUDA(m, cudaDeviceGetAttribute(&m->sms, cudaDevAttrMultiProcessorCount, dev));
    }
    MLP_CUDA(m, cudaMemsetAsync(m->screen_err, 0, sizeof(unsigned), s));
    MLP_CUDA(m, mlp::launch_screen_tc05(n, m->members, x, m->master, m->wbf, m->screen_out, m->screen_err, mean,
                                        stdv, p1, m->sms, s));
    return ENS_OK;
  }
  mlp::FwdArgs f{};
  f.n = n;
  f.members = m->members;
  f.x = x;
  f.master = m->master;
  f.wbf = m->wbf;
  f.mean = mean;
  f.stdv = stdv;
  f.p1 = p1;
  MLP_CUDA(m, mlp::launch_forward_screen(f, s));
  return ENS_OK;
}

ens_status ens_mlp_set_screen_impl(ens_mlp* m, int32_t impl, int32_t* wait_expired) {
  if (!m || (impl != 0 && impl != 1)) return ENS_EINVAL;
  if (wait_expired) {
    unsigned e = 0;
    if (m->screen_err) MLP_CUDA(m, cudaMemcpy(&e, m->screen_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    *wait_expired = (int32_t)e;
  }
  m->screen_impl = impl;
  return ENS_OK;
}

ens_status ens_mlp_set_train_impl(ens_mlp* m, int32_t impl, int32_t* wait_expired) {
  if (!m || (impl != 0 && impl != 1)) return ENS_EINVAL;
  if (wait_expired) {
    unsigned e = 0;
    if (m->train_err) MLP_CUDA(m, cudaMemcpy(&e, m->train_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    *wait_expired = (int32_t)e;
  }
  m->train_impl = impl;
  return ENS_OK;
}

const char* ens_mlp_last_error(const ens_mlp* m) { return m ? m->err : g_mlp_err; }

void ens_mlp_destroy(ens_mlp* m) {
  if (!m) return;
  cudaFree(m->master);
  cudaFree(m->wbf);
  cudaFree(m->m1);
  cudaFree(m->m2);
  cudaFree(m->grad);
  cudaFree(m->loss);
  cudaFree(m->gpart);
  cudaFree(m->xb);
  cudaFree(m->yb);
  cudaFree(m->z);
  cudaFree(m->gp);
  cudaFree(m->dz);
  cudaFree(m->out);
  cudaFree(m->dout);
  cudaFree(m->screen_out);
  cudaFree(m->screen_err);
  cudaFree(m->train_err);
  cudaFree(m->wbfT);
  delete m;
}

ens_status ens_km_features(int64_t n, const double* pA, const double* f, const double range[4], float* x,
                           void* stream) {
  if (n < 0 || !range) return ENS_EINVAL;
  if (n == 0) return ENS_OK;
  if (!is_device(pA) || !is_device(f) || !is_device(x)) return ENS_EINVAL;
  if (!(range[0] > 0 && range[1] > range[0] && range[2] > 0 && range[3] > range[2])) return ENS_EINVAL;
  km_features_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, pA, f, log(range[0]), log(range[1]),
                                                                    log(range[2]), log(range[3]), x);
  return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

ens_status ens_km_labels(int64_t n, const double* acc, int32_t n_phases, int32_t first_phase, double spread_tol,
                         float* y, void* stream) {
  if (n < 0 || first_phase < 0 || first_phase >= n_phases) return ENS_EINVAL;
  if (n == 0) return ENS_OK;
  if (!is_device(acc) || !is_device(y)) return ENS_EINVAL;
  km_labels_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, acc, n_phases, first_phase, spread_tol, y);
  return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

ens_status ens_select_gate(int64_t n, const float* v, float thr, const float* w, float thr_w, int32_t* idx,
                           int64_t* count, void* stream) {
  if (n < 0 || !count) return ENS_EINVAL;
  if (n == 0) {
    *count = 0;
    return ENS_OK;
  }
  if (n > 0x7fffffffLL || !is_device(v) || !is_device(idx) || (w && !is_device(w))) return ENS_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nb = (n + kSelBlock - 1) / kSelBlock;
  unsigned* counts = nullptr;
  long long* total = nullptr;
  if (cudaMalloc(&counts, nb * sizeof(unsigned)) != cudaSuccess) return ENS_ENOMEM;
  if (cudaMalloc(&total, sizeof(long long)) != cudaSuccess) {
    cudaFree(counts);
    return ENS_ENOMEM;
  }
  select_count_kernel<<<(unsigned)nb, kSelBlock, 0, s>>>(n, v, thr, w, thr_w, counts);
  select_scan_kernel<<<1, 1024, 0, s>>>(counts, nb, total);
  select_scatter_kernel<<<(unsigned)nb, kSelBlock, 0, s>>>(n, v, thr, w, thr_w, counts, idx);
  long long t = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&t, total, sizeof(long long), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(counts);
  cudaFree(total);
  if (e != cudaSuccess) return ENS_ECUDA;
  *count = t;
  return ENS_OK;
}

ens_status ens_select_above(int64_t n, const float* v, float thr, int32_t* idx, int64_t* count, void* stream) {
  return ens_select_gate(n, v, thr, nullptr, 0.f, idx, count, stream);
}

ens_status ens_grid_gradient(int64_t rows, int64_t cols, int64_t stride, const float* v, float d_row, float d_col,
                             float* g, void* stream) {
  if (rows < 0 || cols < 0 || stride < 1 || !(d_row > 0.f) || !(d_col > 0.f)) return ENS_EINVAL;
  if (rows == 0 || cols == 0) return ENS_OK;
  if (!is_device(v) || !is_device(g)) return ENS_EINVAL;
  grid_gradient_kernel<<<grid_for(rows * cols), 256, 0, (cudaStream_t)stream>>>(
      rows, cols, stride, v, 1.f / (d_row * stride), 1.f / (d_col * stride), g);
  return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

ens_status ens_feature_stencil(int64_t n, const float* x, float d0, float d1, float* out, void* stream) {
  if (n < 0 || !(d0 > 0.f) || !(d1 > 0.f)) return ENS_EINVAL;
  if (n == 0) return ENS_OK;
  if (!is_device(x) || !is_device(out)) return ENS_EINVAL;
  feature_stencil_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, x, d0, d1, out);
  return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

ens_status ens_stencil_gradient(int64_t n, const float* v, float d0, float d1, float* g, void* stream) {
  if (n < 0 || !(d0 > 0.f) || !(d1 > 0.f)) return ENS_EINVAL;
  if (n == 0) return ENS_OK;
  if (!is_device(v) || !is_device(g)) return ENS_EINVAL;
  stencil_gradient_kernel<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(n, v, 1.f / d0, 1.f / d1, g);
  return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

ens_status ens_gather_f64(int64_t k, const int32_t* idx, const double* src, double* dst, void* stream) {
  if (k < 0) return ENS_EINVAL;
  if (k == 0) return ENS_OK;
  if (!is_device(idx) || !is_device(src) || !is_device(dst)) return ENS_EINVAL;
  gather_f64_kernel<<<grid_for(k), 256, 0, (cudaStream_t)stream>>>(k, idx, src, dst);
  return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

ens_status ens_scatter_labels(int64_t k, const int32_t* idx, const float* y, float* dst, void* stream) {
  if (k < 0) return ENS_EINVAL;
  if (k == 0) return ENS_OK;
  if (!is_device(idx) || !is_device(y) || !is_device(dst)) return ENS_EINVAL;
  scatter_f32_kernel<<<grid_for(k), 256, 0, (cudaStream_t)stream>>>(k, idx, y, dst);
  return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
}

}  // extern "C"
