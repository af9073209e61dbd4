// mlp.cu -- surrogate network of the Keller-Miksis response: training and
// screening kernels on the BF16 tensor cores.
//
// Network (per ensemble member): 2 -> 128 -> 128 -> 128 -> 128 -> 2, GELU
// (erf form) after the first four layers.  Weights are stored [out][in]; the
// parameter vector of one member is
//   W1[128][2] b1[128] W2[128][128] b2[128] W3[128][128] b3[128]
//   W4[128][128] b4[128] W5[2][128] b5[2]                    (50,178 floats).
// FP32 master weights, BF16 copies of the weights for the forward pass; the
// three 128x128 layers (forward, input gradients and weight gradients) run as
// BF16 x BF16 -> FP32 tensor-core products (mma.sync m16n8k16), the 2-wide
// first and last layers as FP32 FMAs.  One block holds a 128-sample tile: 8
// warps, each owning 16 samples x 128 features in mma accumulators.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "mlp.cuh"

namespace ens {
namespace mlp {

__host__ __device__ constexpr int64_t w_off(int l) { return l == 1 ? oW1 : l == 2 ? oW2 : l == 3 ? oW3 : l == 4 ? oW4 : oW5; }
__host__ __device__ constexpr int64_t b_off(int l) { return l == 1 ? ob1 : l == 2 ? ob2 : l == 3 ? ob3 : l == 4 ? ob4 : ob5; }

// D += A * B for one m16n8k16 tile (BF16 inputs, FP32 accumulate).
__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp: acc[16 n-tiles][4] += A[16 rows][K] * B, with A row-major (stride
// lda) and B given as Bs[n][k] (stride ldb), N = 128, K a multiple of 16.
__device__ __forceinline__ void warp_strip(const __nv_bfloat16* A, int lda, const __nv_bfloat16* Bs,
                                           int ldb, int K, float (*acc)[4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(&A[g * lda + k0 + 2 * t]);
    a[1] = *reinterpret_cast<const uint32_t*>(&A[(g + 8) * lda + k0 + 2 * t]);
    a[2] = *reinterpret_cast<const uint32_t*>(&A[g * lda + k0 + 8 + 2 * t]);
    a[3] = *reinterpret_cast<const uint32_t*>(&A[(g + 8) * lda + k0 + 8 + 2 * t]);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      uint32_t b[2];
      b[0] = *reinterpret_cast<const uint32_t*>(&Bs[(nt * 8 + g) * ldb + k0 + 2 * t]);
      b[1] = *reinterpret_cast<const uint32_t*>(&Bs[(nt * 8 + g) * ldb + k0 + 8 + 2 * t]);
      mma16816(acc[nt], a, b);
    }
  }
}

// Copy W_l (bf16, [out][in] row-major) into Ws[n][k] for the forward product
// (B[k = in][n = out] = W[out][in]).
__device__ __forceinline__ void stage_w_forward(const __nv_bfloat16* W, __nv_bfloat16* Ws) {
  for (int idx = threadIdx.x; idx < H * (H / 8); idx += blockDim.x) {
    const int row = idx / (H / 8), c8 = idx % (H / 8);
    *reinterpret_cast<uint4*>(&Ws[row * LDA + c8 * 8]) = *reinterpret_cast<const uint4*>(&W[row * H + c8 * 8]);
  }
}

// Copy W_l transposed into Ws[n][k] for the input-gradient product
// (B[k = out][n = in] = W[out][in], so Ws[n = in][k = out] = W[k][n]).
__device__ __forceinline__ void stage_w_backward(const __nv_bfloat16* W, __nv_bfloat16* Ws) {
  for (int idx = threadIdx.x; idx < H * H; idx += blockDim.x) {
    const int k = idx / H, n = idx % H;
    Ws[n * LDA + k] = W[idx];
  }
}


// Forward of one member on the block's tile; the last hidden activations are
// left in act (bf16) and the outputs in outs[row][2] (shared).
__device__ void tile_forward(const FwdArgs& a, int m, int64_t row0, int rows, __nv_bfloat16* act0,
                             __nv_bfloat16* act1, __nv_bfloat16* Ws, float* outs, bool train) {
  const float* P = a.master + (int64_t)m * kP;
  const __nv_bfloat16* Pb = a.wbf + (int64_t)m * kPS;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  // layer 1 (2 -> 128) in FP32: thread = (row, half of the features)
  {
    const int r = tid >> 1, f0 = (tid & 1) * 64;
    const bool live = r < rows;
    const float x0 = live ? a.x[2 * (row0 + r)] : 0.f, x1 = live ? a.x[2 * (row0 + r) + 1] : 0.f;
    for (int f = f0; f < f0 + 64; ++f) {
      const float w0 = __bfloat162float(Pb[oW1 + 2 * f]), w1 = __bfloat162float(Pb[oW1 + 2 * f + 1]);
      const float z = fmaf(w1, x1, fmaf(w0, x0, P[ob1 + f]));
      act0[r * LDA + f] = __float2bfloat16(gelu(z));
      if (train && live) a.z[(((int64_t)m * a.n + row0 + r) * 4 + 0) * H + f] = z;
    }
  }
  __nv_bfloat16* in = act0;
  __nv_bfloat16* outa = act1;
  // layers 2..4 on the tensor cores
  for (int l = 2; l <= 4; ++l) {
    __syncthreads();
    stage_w_forward(Pb + w_off(l), Ws);
    __syncthreads();
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    warp_strip(in + warp * 16 * LDA, LDA, Ws, LDA, H, acc);
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int col = nt * 8 + 2 * t;
      const float b0 = P[b_off(l) + col], b1 = P[b_off(l) + col + 1];
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int r = warp * 16 + g + 8 * half;
        const float z0 = acc[nt][2 * half] + b0, z1 = acc[nt][2 * half + 1] + b1;
        __nv_bfloat162 hv;
        hv.x = __float2bfloat16(gelu(z0));
        hv.y = __float2bfloat16(gelu(z1));
        *reinterpret_cast<__nv_bfloat162*>(&outa[r * LDA + col]) = hv;
        if (train && r < rows) {
          float2 zz = make_float2(z0, z1);
          *reinterpret_cast<float2*>(&a.z[(((int64_t)m * a.n + row0 + r) * 4 + (l - 1)) * H + col]) = zz;
        }
      }
    }
    __nv_bfloat16* tmp = in;
    in = outa;
    outa = tmp;
  }
  __syncthreads();
  // layer 5 (128 -> 2) in FP32: thread = (row, output)
  {
    const int r = tid >> 1, j = tid & 1;
    float o = P[ob5 + j];
    for (int f = 0; f < H; ++f) o = fmaf(__bfloat162float(in[r * LDA + f]), __bfloat162float(Pb[oW5 + j * H + f]), o);
    outs[r * 2 + j] = o;
    if (train && r < rows) a.out[((int64_t)m * a.n + row0 + r) * 2 + j] = o;
  }
  __syncthreads();
}


// grid.x = tiles, grid.y = member (training) or 1 (screening: all members).
template <bool TRAIN>
__global__ void __launch_bounds__(kThreads) mlp_forward_kernel(FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* act0 = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* act1 = act0 + H * LDA;
  __nv_bfloat16* Ws = act1 + H * LDA;
  float* outs = reinterpret_cast<float*>(Ws + H * LDA);  // [members][kTile][2]
  const int64_t row0 = (int64_t)blockIdx.x * kTile;
  const int rows = (int)((a.n - row0) < kTile ? (a.n - row0) : kTile);
  if constexpr (TRAIN) {
    tile_forward(a, blockIdx.y, row0, rows, act0, act1, Ws, outs, true);
  } else {
    for (int m = 0; m < a.members; ++m) tile_forward(a, m, row0, rows, act0, act1, Ws, outs + m * kTile * 2, false);
    const int r = threadIdx.x;
    if (r < rows) {
      float s = 0.f, s2 = 0.f, p = 0.f;
      for (int m = 0; m < a.members; ++m) {
        const float o = outs[m * kTile * 2 + r * 2];
        s += o;
        p += 1.0f / (1.0f + __expf(-outs[m * kTile * 2 + r * 2 + 1]));
      }
      const float mu = s / a.members;
      for (int m = 0; m < a.members; ++m) {
        const float d = outs[m * kTile * 2 + r * 2] - mu;
        s2 += d * d;
      }
      a.mean[row0 + r] = mu;
      a.stdv[row0 + r] = sqrtf(s2 / a.members);
      a.p1[row0 + r] = p / a.members;
    }
  }
}


// Output gradients and input gradients of all layers for one tile of one member.
__global__ void __launch_bounds__(kThreads) mlp_backward_kernel(BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* act = reinterpret_cast<__nv_bfloat16*>(smem);   // dz_l as A operand
  __nv_bfloat16* Ws = act + H * LDA;
  float* dsh = reinterpret_cast<float*>(Ws + H * LDA);           // [kTile][2] dout
  __shared__ float red[kThreads / 32];
  const int m = blockIdx.y;
  const __nv_bfloat16* Pb = a.wbf + (int64_t)m * kPS;
  const int64_t row0 = (int64_t)blockIdx.x * kTile;
  const int rows = (int)((a.n - row0) < kTile ? (a.n - row0) : kTile);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  const float inv_n = 1.0f / (float)a.n;
  // loss and output gradient: thread = (row, output)
  float lsum = 0.f;
  {
    const int r = tid >> 1, j = tid & 1;
    float d = 0.f;
    if (r < rows) {
      const float o = a.out[((int64_t)m * a.n + row0 + r) * 2 + j];
      const float yv = a.y[(row0 + r) * 2 + j];
      if (j == 0) {
        d = 2.0f * (o - yv) * inv_n;
        lsum = (o - yv) * (o - yv);
      } else {
        d = (1.0f / (1.0f + __expf(-o)) - yv) * inv_n;
        lsum = fmaxf(o, 0.f) - o * yv + log1pf(__expf(-fabsf(o)));
      }
      a.dout[((int64_t)m * a.n + row0 + r) * 2 + j] = d;
    }
    dsh[r * 2 + j] = d;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if (lane == 0) red[warp] = lsum;
  __syncthreads();
  if (tid == 0) {
    float s = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    atomicAdd(&a.loss[m], s);
  }
  // dz4 = (dout W5) * gelu'(z4): thread = (row, half of the features)
  {
    const int r = tid >> 1, f0 = (tid & 1) * 64;
    for (int f = f0; f < f0 + 64; ++f) {
      float dzv = 0.f;
      if (r < rows) {
        const float dh = dsh[r * 2] * __bfloat162float(Pb[oW5 + f]) + dsh[r * 2 + 1] * __bfloat162float(Pb[oW5 + H + f]);
        dzv = dh * gelu_grad(a.z[(((int64_t)m * a.n + row0 + r) * 4 + 3) * H + f]);
        a.dz[(((int64_t)m * 4 + 3) * a.n + row0 + r) * H + f] = dzv;
      }
      act[r * LDA + f] = __float2bfloat16(dzv);
    }
  }
  // dh_{l-1} = dz_l W_l, dz_{l-1} = dh_{l-1} * gelu'(z_{l-1}) for l = 4, 3, 2
  for (int l = 4; l >= 2; --l) {
    __syncthreads();
    stage_w_backward(Pb + w_off(l), Ws);
    __syncthreads();
    float acc[16][4];
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
    warp_strip(act + warp * 16 * LDA, LDA, Ws, LDA, H, acc);
    __syncthreads();  // every warp has read act before it is overwritten
#pragma unroll
    for (int nt = 0; nt < 16; ++nt) {
      const int col = nt * 8 + 2 * t;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int r = warp * 16 + g + 8 * half;
        float d0 = 0.f, d1 = 0.f;
        if (r < rows) {
          const float* zr = &a.z[(((int64_t)m * a.n + row0 + r) * 4 + (l - 2)) * H + col];
          d0 = acc[nt][2 * half] * gelu_grad(zr[0]);
          d1 = acc[nt][2 * half + 1] * gelu_grad(zr[1]);
          *reinterpret_cast<float2*>(&a.dz[(((int64_t)m * 4 + (l - 2)) * a.n + row0 + r) * H + col]) =
              make_float2(d0, d1);
        }
        __nv_bfloat162 hv;
        hv.x = __float2bfloat16(d0);
        hv.y = __float2bfloat16(d1);
        *reinterpret_cast<__nv_bfloat162*>(&act[r * LDA + col]) = hv;
      }
    }
  }
}



// Weight and bias gradients.  grid = (members, 5, slices): y = layer - 1,
// z = batch slice of a.rows samples; each block writes the slice's partial
// gradient (the slices are summed in order by mlp_grad_reduce).  Layers 2..4
// on the tensor cores (dW[out][in] = sum_b dz[b][out] h[b][in], K = batch),
// layers 1 and 5 in FP32.
__global__ void __launch_bounds__(kThreads) mlp_wgrad_kernel(GradArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int m = blockIdx.x, l = blockIdx.y + 1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t = lane & 3;
  float* G = a.grad + ((int64_t)blockIdx.z * gridDim.x + m) * kP;
  float* part = reinterpret_cast<float*>(smem);  // reduction scratch
  const int64_t r0 = (int64_t)blockIdx.z * a.rows;
  const int64_t r1 = r0 + a.rows < a.n ? r0 + a.rows : a.n;
  if (l == 1 || l == 5) {
    wgrad_fp32_layer(l, m, a.n, r0, r1, a.x, a.z, a.dz, a.dout, G, part);
    return;
  }
  // tensor-core layers: As[out][k] = dz_l[b][out], Bs[in][k] = gelu(z_{l-1}[b][in])
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(smem);
  __nv_bfloat16* Bs = As + H * LDC;
  float* bpart = reinterpret_cast<float*>(Bs + H * LDC);  // [kThreads]
  float acc[16][4];
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
  float bsum = 0.f;  // bias gradient partial of feature tid % 128
  for (int64_t c0 = r0; c0 < r1; c0 += kChunk) {
    __syncthreads();
    for (int idx = tid; idx < kChunk * H; idx += kThreads) {
      const int bk = idx / H, f = idx % H;
      const int64_t b = c0 + bk;
      float d = 0.f, h = 0.f;
      if (b < r1) {
        d = a.dz[(((int64_t)m * 4 + (l - 1)) * a.n + b) * H + f];
        h = gelu(a.z[(((int64_t)m * a.n + b) * 4 + (l - 2)) * H + f]);
      }
      bsum += d;
      As[f * LDC + bk] = __float2bfloat16(d);
      Bs[f * LDC + bk] = __float2bfloat16(h);
    }
    __syncthreads();
    warp_strip(As + warp * 16 * LDC, LDC, Bs, LDC, kChunk, acc);
  }
  bpart[tid] = bsum;
  __syncthreads();
  if (tid < H) G[b_off(l) + tid] = bpart[tid] + bpart[tid + H];
#pragma unroll
  for (int nt = 0; nt < 16; ++nt) {
    const int col = nt * 8 + 2 * t;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int r = warp * 16 + g + 8 * half;
      G[w_off(l) + r * H + col] = acc[nt][2 * half];
      G[w_off(l) + r * H + col + 1] = acc[nt][2 * half + 1];
    }
  }
}


// Adam (Kingma & Ba 2015) on the FP32 master weights; refreshes the BF16 copy.
// Adam step; the gradient is the sum of the slice partials part[k][i], k in
// order (the same sums as mlp_grad_reduce_kernel)
__global__ void adam_kernel(int64_t total, float* w, __nv_bfloat16* wb, const float* part, int splits, float* m1,
                            float* m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    float gi = part[i];
    for (int k = 1; k < splits; ++k) gi += part[(int64_t)k * total + i];
    const float a = fmaf(b1, m1[i], (1.0f - b1) * gi);
    const float v = fmaf(b2, m2[i], (1.0f - b2) * gi * gi);
    m1[i] = a;
    m2[i] = v;
    const float upd = lr * (a / c1) / (sqrtf(v / c2) + eps);
    w[i] -= upd;
    wb[(i / kP) * kPS + i % kP] = __float2bfloat16(w[i]);
  }
}

__global__ void to_bf16_kernel(int64_t total, const float* w, __nv_bfloat16* wb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x)
    wb[(i / kP) * kPS + i % kP] = __float2bfloat16(w[i]);
}


// Weights uniform in [-1/sqrt(fan_in), 1/sqrt(fan_in)], biases 0; member k
// draws from the stream seed + k.
__global__ void init_kernel(int members, uint64_t seed, float* w) {
  const int64_t total = (int64_t)members * kP;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int m = (int)(i / kP);
    const int64_t j = i % kP;
    float fan = 0.f;
    if (j < ob1) fan = 2.f;
    else if ((j >= oW2 && j < ob2) || (j >= oW3 && j < ob3) || (j >= oW4 && j < ob4) || (j >= oW5 && j < ob5)) fan = (float)H;
    if (fan == 0.f) {
      w[i] = 0.f;
      continue;
    }
    const uint64_t r = splitmix64((seed + (uint64_t)m) * 0x100000000ULL + (uint64_t)j);
    const float u = (float)((r >> 40) * (1.0 / 16777216.0));  // [0, 1)
    w[i] = (2.0f * u - 1.0f) * rsqrtf(fan);
  }
}

__global__ void gather_kernel(int64_t n, const int32_t* idx, const float* x, const float* y, float* xb, float* yb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = idx[i];
    xb[2 * i] = x[2 * s];
    xb[2 * i + 1] = x[2 * s + 1];
    yb[2 * i] = y[2 * s];
    yb[2 * i + 1] = y[2 * s + 1];
  }
}

static unsigned grid_1d(int64_t n) {
  int64_t g = (n + 255) / 256;
  g = g < 1 ? 1 : (g > 8192 ? 8192 : g);
  return (unsigned)g;
}

cudaError_t set_smem_limits() {
  cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_forward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBwdSmem);
  return e;
}

cudaError_t launch_forward_train(const FwdArgs& a, cudaStream_t s) {
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  mlp_forward_kernel<true><<<dim3((unsigned)tiles, a.members), kThreads, kFwdSmem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_forward_screen(const FwdArgs& a, cudaStream_t s) {
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  if (tiles > 0x7fffffffLL || a.members > kMaxMembers) return cudaErrorInvalidValue;
  mlp_forward_kernel<false><<<(unsigned)tiles, kThreads, kFwdSmem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_backward(const BwdArgs& a, int members, cudaStream_t s) {
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  mlp_backward_kernel<<<dim3((unsigned)tiles, members), kThreads, kBwdSmem, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const GradArgs& a, int members, int splits, cudaStream_t s) {
  if (splits < 1 || splits > kMaxSplits || a.rows % kChunk != 0 || (int64_t)splits * a.rows < a.n)
    return cudaErrorInvalidValue;
  mlp_wgrad_kernel<<<dim3(members, 5, splits), kThreads, kGradSmem, s>>>(a);
  return cudaGetLastError();
}

__global__ void mlp_grad_reduce_kernel(int64_t total, int splits, const float* part, float* grad) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    float acc = part[i];
    for (int k = 1; k < splits; ++k) acc += part[(int64_t)k * total + i];
    grad[i] = acc;
  }
}

cudaError_t launch_grad_reduce(int members, int splits, const float* part, float* grad, cudaStream_t s) {
  const int64_t total = (int64_t)members * kP;
  mlp_grad_reduce_kernel<<<grid_1d(total), 256, 0, s>>>(total, splits, part, grad);
  return cudaGetLastError();
}

cudaError_t launch_adam(int64_t total, float* w, __nv_bfloat16* wb, const float* part, int splits, float* m1,
                        float* m2, float lr, float b1, float b2, float eps, float c1, float c2, cudaStream_t s) {
  adam_kernel<<<grid_1d(total), 256, 0, s>>>(total, w, wb, part, splits, m1, m2, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_to_bf16(int64_t total, const float* w, __nv_bfloat16* wb, cudaStream_t s) {
  to_bf16_kernel<<<grid_1d(total), 256, 0, s>>>(total, w, wb);
  return cudaGetLastError();
}

cudaError_t launch_init(int members, uint64_t seed, float* w, cudaStream_t s) {
  init_kernel<<<grid_1d((int64_t)members * kP), 256, 0, s>>>(members, seed, w);
  return cudaGetLastError();
}

cudaError_t launch_gather(int64_t n, const int32_t* idx, const float* x, const float* y, float* xb, float* yb,
                          cudaStream_t s) {
  gather_kernel<<<grid_1d(n), 256, 0, s>>>(n, idx, x, y, xb, yb);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace ens
