// planner.cu -- host planner pieces: Keller-Miksis coefficients (Sec. 4.2,
// Eq. coefficients) and the longest-first claim order of the persistent
// adaptive kernels.
#include <cmath>
#include <cstdio>

#include "common.cuh"

namespace ens {

// C0..C12 of one system from SI parameters.  s = 2 pi / (R_E w1) is the
// velocity scale of the dimensionless time tau = w1 t / (2 pi).
__host__ __device__ inline void km_coeffs_one(double pA1, double f1, double pA2, double f2,
                                              double theta, double RE, const ens_liquid& L,
                                              double* C) {
  const double two_pi = 6.283185307179586476925286766559;
  const double w1 = two_pi * f1;
  const double w2 = two_pi * f2;
  const double s = two_pi / (RE * w1);
  const double s2 = s * s;
  const double pg0 = L.pinf - L.pv + 2.0 * L.sigma / RE;  // gas pressure at equilibrium
  C[0] = pg0 / L.rho * s2;
  C[1] = (1.0 - 3.0 * L.gamma) / (L.rho * L.c) * pg0 * s;
  C[2] = (L.pinf - L.pv) / L.rho * s2;
  C[3] = 2.0 * L.sigma / (L.rho * RE) * s2;
  C[4] = 4.0 * L.mu / (L.rho * RE * RE) * (two_pi / w1);
  C[5] = pA1 / L.rho * s2;
  C[6] = pA2 / L.rho * s2;
  C[7] = RE * w1 * pA1 / (L.rho * L.c) * s2;
  C[8] = RE * w2 * pA2 / (L.rho * L.c) * s2;  // omega2: derivative of the second term
  C[9] = RE * w1 / (two_pi * L.c);
  C[10] = 3.0 * L.gamma;
  C[11] = w2 / w1;
  C[12] = theta;
}

__global__ void km_coeff_kernel(int64_t n, const double* pA1, const double* f1, const double* pA2,
                                const double* f2, const double* theta, const double* RE,
                                ens_liquid L, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double C[13];
    km_coeffs_one(pA1[i], f1[i], pA2[i], f2[i], theta[i], RE[i], L, C);
#pragma unroll
    for (int k = 0; k < 13; ++k) out[k * n + i] = C[k];
  }
}

// ---------------------------------------------------------------------------
// Longest-first claim order: counting sort of the systems by a quarter-octave
// bucket of their pilot step count, largest bucket first.
// ---------------------------------------------------------------------------
constexpr int kBuckets = 256;

__device__ __forceinline__ int step_bucket(int64_t steps) {
  const double l = log2((double)(steps < 0 ? 0 : steps) + 1.0) * 4.0;
  int b = (int)l;
  return b < 0 ? 0 : (b >= kBuckets ? kBuckets - 1 : b);
}

__global__ void order_hist_kernel(const int64_t* steps, int64_t n, unsigned* hist) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[step_bucket(steps[i])], 1u);
}

// one block of kBuckets threads: offsets[b] = number of systems in buckets > b
__global__ void order_scan_kernel(unsigned* hist) {
  __shared__ unsigned cnt[kBuckets];
  const int b = threadIdx.x;
  cnt[b] = hist[b];
  __syncthreads();
  if (b == 0) {
    unsigned run = 0;
    for (int k = kBuckets - 1; k >= 0; --k) {
      const unsigned c = cnt[k];
      cnt[k] = run;
      run += c;
    }
  }
  __syncthreads();
  hist[kBuckets + b] = cnt[b];
}

__global__ void order_scatter_kernel(const int64_t* steps, int64_t n, unsigned* hist, int32_t* order) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned pos = atomicAdd(&hist[kBuckets + step_bucket(steps[i])], 1u);
    order[pos] = (int32_t)i;
  }
}

cudaError_t launch_order(const int64_t* steps, int64_t n, int32_t* order, unsigned* hist,
                         cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (n > 0x7fffffffLL) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(hist, 0, 2 * kBuckets * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  const unsigned blocks = (unsigned)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  order_hist_kernel<<<blocks, 256, 0, s>>>(steps, n, hist);
  order_scan_kernel<<<1, kBuckets, 0, s>>>(hist);
  order_scatter_kernel<<<blocks, 256, 0, s>>>(steps, n, hist, order);
  return cudaGetLastError();
}

}  // namespace ens

using namespace ens;

extern "C" ens_status ens_km_coefficients(int64_t n, const double* pA1, const double* f1,
                                          const double* pA2, const double* f2, const double* theta,
                                          const double* RE, const ens_liquid* liquid, double* out,
                                          void* stream) {
  if (n < 0 || !liquid) return ENS_EINVAL;
  if (n == 0) return ENS_OK;
  if (!pA1 || !f1 || !pA2 || !f2 || !theta || !RE || !out) return ENS_EINVAL;
  cudaPointerAttributes at{};
  bool device = false;
  if (cudaPointerGetAttributes(&at, out) == cudaSuccess)
    device = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
  cudaGetLastError();  // clear a possible error from an unregistered host pointer
  if (device) {
    const int64_t blocks = (n + 255) / 256 < 8192 ? (n + 255) / 256 : 8192;
    km_coeff_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(n, pA1, f1, pA2, f2, theta,
                                                                         RE, *liquid, out);
    return cudaGetLastError() == cudaSuccess ? ENS_OK : ENS_ECUDA;
  }
  for (int64_t i = 0; i < n; ++i) {
    double C[13];
    km_coeffs_one(pA1[i], f1[i], pA2[i], f2[i], theta[i], RE[i], *liquid, C);
    for (int k = 0; k < 13; ++k) out[k * n + i] = C[k];
  }
  return ENS_OK;
}
