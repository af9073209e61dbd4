// rk4.cu -- fixed-step classic RK4 ensemble kernels (Sec. 3; Sec. 4.1).
//
// One thread integrates one system (or SPT of them, interleaved) for nsteps
// steps with state, stage derivatives and parameters in registers; global
// memory is touched once to load and once to store (the "per-thread
// approach", Sec. 3.2.1).  The fast
// flavour accumulates k1 + 2 k2 + 2 k3 + k4 as it goes and uses fused
// multiply-adds; the strict flavour evaluates
//   y_new = y + h/6 (k1 + 2 k2 + 2 k3 + k4)
// literally, without contraction.
#include "common.cuh"
#include "rhs.cuh"

namespace ens {

// SPT systems per thread: thread t of block b integrates systems
// b * blockDim * SPT + s * blockDim + t for s < SPT (each slot's systems are
// consecutive across the block, so loads and stores stay coalesced).  The
// slots' steps are independent chains in one instruction stream, which the
// compiler interleaves; each slot's arithmetic is exactly that of SPT = 1.
template <class Sys, bool STRICT, int SPT>
__global__ void __launch_bounds__(256) rk4_kernel(Rk4Args a) {
  constexpr int D = Sys::kDim;
  const int64_t base = blockIdx.x * (int64_t)blockDim.x * SPT + threadIdx.x;
  int64_t idx[SPT];
  bool live[SPT];
  Sys sys[SPT];
  double y[SPT][D];
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    idx[s] = base + (int64_t)s * blockDim.x;
    live[s] = idx[s] < a.n;
    // a slot past the end integrates a copy of system 0 and stores nothing
    const int64_t i = live[s] ? idx[s] : 0;
    sys[s].load(a.params, a.n, i);
#pragma unroll
    for (int k = 0; k < D; ++k) y[s][k] = a.y0[k * a.n + i];
  }
  if (!live[0]) return;
  const double h = a.dt;
  if (STRICT) {
    const double h2 = __ddiv_rn(h, 2.0);
    const double h6 = __ddiv_rn(h, 6.0);
    for (int64_t j = 0; j < a.nsteps; ++j) {
      const double t = sadd(a.t0, smul((double)j, h));
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        double k1[D], k2[D], k3[D], k4[D], ys[D];
        sys[s].template f<true>(t, y[s], k1);
#pragma unroll
        for (int k = 0; k < D; ++k) ys[k] = sadd(y[s][k], smul(h2, k1[k]));
        sys[s].template f<true>(sadd(t, h2), ys, k2);
#pragma unroll
        for (int k = 0; k < D; ++k) ys[k] = sadd(y[s][k], smul(h2, k2[k]));
        sys[s].template f<true>(sadd(t, h2), ys, k3);
#pragma unroll
        for (int k = 0; k < D; ++k) ys[k] = sadd(y[s][k], smul(h, k3[k]));
        sys[s].template f<true>(sadd(t, h), ys, k4);
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const double sum = sadd(sadd(sadd(k1[k], smul(2.0, k2[k])), smul(2.0, k3[k])), k4[k]);
          y[s][k] = sadd(y[s][k], smul(h6, sum));
        }
      }
    }
  } else {
    const double h2 = 0.5 * h;
    const double h6 = h * (1.0 / 6.0);
    for (int64_t j = 0; j < a.nsteps; ++j) {
      const double t = fma((double)j, h, a.t0);
      double k[SPT][D], ks[SPT][D], ys[SPT][D];
      // stage by stage across the slots, so that independent work sits side by side
#pragma unroll
      for (int s = 0; s < SPT; ++s) sys[s].template f<false>(t, y[s], k[s]);
#pragma unroll
      for (int s = 0; s < SPT; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          ks[s][c] = k[s][c];
          ys[s][c] = fma(h2, k[s][c], y[s][c]);
        }
#pragma unroll
      for (int s = 0; s < SPT; ++s) sys[s].template f<false>(t + h2, ys[s], k[s]);
#pragma unroll
      for (int s = 0; s < SPT; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          ks[s][c] = fma(2.0, k[s][c], ks[s][c]);
          ys[s][c] = fma(h2, k[s][c], y[s][c]);
        }
#pragma unroll
      for (int s = 0; s < SPT; ++s) sys[s].template f<false>(t + h2, ys[s], k[s]);
#pragma unroll
      for (int s = 0; s < SPT; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c) {
          ks[s][c] = fma(2.0, k[s][c], ks[s][c]);
          ys[s][c] = fma(h, k[s][c], y[s][c]);
        }
#pragma unroll
      for (int s = 0; s < SPT; ++s) sys[s].template f<false>(t + h, ys[s], k[s]);
#pragma unroll
      for (int s = 0; s < SPT; ++s)
#pragma unroll
        for (int c = 0; c < D; ++c) y[s][c] = fma(h6, ks[s][c] + k[s][c], y[s][c]);
    }
  }
  unsigned any = 0;
#pragma unroll
  for (int s = 0; s < SPT; ++s) {
    if (!live[s]) continue;
    const int64_t i = idx[s];
    int32_t st = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      a.y[k * a.n + i] = y[s][k];
      if (!isfinite(y[s][k])) st = kStNonFinite;
    }
    a.t_out[i] = fma((double)a.nsteps, h, a.t0);
    a.dt_out[i] = h;
    a.status[i] = st;
    a.nacc[i] = a.nsteps;
    a.nrej[i] = 0;
    a.nrhs[i] = 4 * a.nsteps;
    any |= (unsigned)st;
  }
  if (any) atomicOr(&a.scratch->any_status, any);
}

// Launcher: returns the CUDA error of the launch.  spt: systems per thread
// (1, 2 or 4).
template <class Sys, bool STRICT>
cudaError_t launch_rk4_spt(int spt, const Rk4Args& a, dim3 b, cudaStream_t s) {
  const int64_t per_block = (int64_t)b.x * spt;
  const int64_t grid = (a.n + per_block - 1) / per_block;
  if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
  const dim3 g((unsigned)grid);
  switch (spt) {
    case 1: rk4_kernel<Sys, STRICT, 1><<<g, b, 0, s>>>(a); break;
    case 2: rk4_kernel<Sys, STRICT, 2><<<g, b, 0, s>>>(a); break;
    case 4: rk4_kernel<Sys, STRICT, 4><<<g, b, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_rk4(int sys, bool strict, const Rk4Args& a, int block, int spt, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (block <= 0) block = 64;
  if (spt <= 0) spt = 1;
  const dim3 b((unsigned)block);
  switch (sys) {
    case ENS_SYS_TOY_X2P:
      return strict ? launch_rk4_spt<X2P, true>(spt, a, b, s) : launch_rk4_spt<X2P, false>(spt, a, b, s);
    case ENS_SYS_LORENZ:
      return strict ? launch_rk4_spt<Lorenz, true>(spt, a, b, s) : launch_rk4_spt<Lorenz, false>(spt, a, b, s);
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace ens
