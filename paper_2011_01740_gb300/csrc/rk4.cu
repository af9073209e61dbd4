// rk4.cu -- fixed-step classic RK4 ensemble kernels (Sec. 3; Sec. 4.1).
//
// One thread integrates one system for nsteps steps with state, stage
// derivatives and parameters in registers; global memory is touched once to
// load and once to store (the "per-thread approach", Sec. 3.2.1).  The fast
// flavour accumulates k1 + 2 k2 + 2 k3 + k4 as it goes and uses fused
// multiply-adds; the strict flavour evaluates
//   y_new = y + h/6 (k1 + 2 k2 + 2 k3 + k4)
// literally, without contraction.
#include "common.cuh"
#include "rhs.cuh"

namespace ens {

template <class Sys, bool STRICT>
__global__ void __launch_bounds__(256) rk4_kernel(Rk4Args a) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  constexpr int D = Sys::kDim;
  Sys sys;
  sys.load(a.params, a.n, i);
  double y[D];
#pragma unroll
  for (int k = 0; k < D; ++k) y[k] = a.y0[k * a.n + i];
  const double h = a.dt;
  if (STRICT) {
    const double h2 = __ddiv_rn(h, 2.0);
    const double h6 = __ddiv_rn(h, 6.0);
    for (int64_t j = 0; j < a.nsteps; ++j) {
      const double t = sadd(a.t0, smul((double)j, h));
      double k1[D], k2[D], k3[D], k4[D], ys[D];
      sys.template f<true>(t, y, k1);
#pragma unroll
      for (int k = 0; k < D; ++k) ys[k] = sadd(y[k], smul(h2, k1[k]));
      sys.template f<true>(sadd(t, h2), ys, k2);
#pragma unroll
      for (int k = 0; k < D; ++k) ys[k] = sadd(y[k], smul(h2, k2[k]));
      sys.template f<true>(sadd(t, h2), ys, k3);
#pragma unroll
      for (int k = 0; k < D; ++k) ys[k] = sadd(y[k], smul(h, k3[k]));
      sys.template f<true>(sadd(t, h), ys, k4);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const double s = sadd(sadd(sadd(k1[k], smul(2.0, k2[k])), smul(2.0, k3[k])), k4[k]);
        y[k] = sadd(y[k], smul(h6, s));
      }
    }
  } else {
    const double h2 = 0.5 * h;
    const double h6 = h * (1.0 / 6.0);
    for (int64_t j = 0; j < a.nsteps; ++j) {
      const double t = fma((double)j, h, a.t0);
      double k[D], ks[D], ys[D];
      sys.template f<false>(t, y, k);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        ks[c] = k[c];
        ys[c] = fma(h2, k[c], y[c]);
      }
      sys.template f<false>(t + h2, ys, k);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        ks[c] = fma(2.0, k[c], ks[c]);
        ys[c] = fma(h2, k[c], y[c]);
      }
      sys.template f<false>(t + h2, ys, k);
#pragma unroll
      for (int c = 0; c < D; ++c) {
        ks[c] = fma(2.0, k[c], ks[c]);
        ys[c] = fma(h, k[c], y[c]);
      }
      sys.template f<false>(t + h, ys, k);
#pragma unroll
      for (int c = 0; c < D; ++c) y[c] = fma(h6, ks[c] + k[c], y[c]);
    }
  }
  int32_t st = 0;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    a.y[k * a.n + i] = y[k];
    if (!isfinite(y[k])) st = kStNonFinite;
  }
  a.t_out[i] = fma((double)a.nsteps, h, a.t0);
  a.dt_out[i] = h;
  a.status[i] = st;
  a.nacc[i] = a.nsteps;
  a.nrej[i] = 0;
  a.nrhs[i] = 4 * a.nsteps;
  if (st) atomicOr(&a.scratch->any_status, (unsigned)st);
}

// Launcher: returns the CUDA error of the launch.
cudaError_t launch_rk4(int sys, bool strict, const Rk4Args& a, int block, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (block <= 0) block = 64;
  const int64_t grid = (a.n + block - 1) / block;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const dim3 g((unsigned)grid), b((unsigned)block);
  switch (sys) {
    case ENS_SYS_TOY_X2P:
      if (strict) rk4_kernel<X2P, true><<<g, b, 0, s>>>(a);
      else rk4_kernel<X2P, false><<<g, b, 0, s>>>(a);
      break;
    case ENS_SYS_LORENZ:
      if (strict) rk4_kernel<Lorenz, true><<<g, b, 0, s>>>(a);
      else rk4_kernel<Lorenz, false><<<g, b, 0, s>>>(a);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace ens
