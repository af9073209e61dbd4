// mlp.cuh -- shared declarations of the surrogate-network kernels (mlp.cu)
// and their host driver (abi_mlp.cu).
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "common.cuh"

namespace ens {
namespace mlp {

constexpr int H = 128;
constexpr int kTile = 128;       // samples per block
constexpr int kThreads = 256;    // 8 warps
constexpr int LDA = H + 8;       // padded bf16 row stride (conflict-free fragments)
constexpr int LDC = 64 + 8;      // padded stride of the weight-gradient chunks
constexpr int kChunk = 64;       // samples per weight-gradient chunk
constexpr int kMaxMembers = 8;

constexpr int64_t oW1 = 0, ob1 = 256, oW2 = 384, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + H * H,
                  oW4 = ob3 + H, ob4 = oW4 + H * H, oW5 = ob4 + H, ob5 = oW5 + 2 * H, kP = ob5 + 2;
static_assert(kP == 50178, "parameter layout");
// member stride of the bf16 weight copies: a multiple of 8 elements, so the
// 16-byte vector loads of the weight tiles stay aligned for every member
constexpr int64_t kPS = 50184;
static_assert(kPS % 8 == 0 && kPS >= kP, "bf16 member stride");

constexpr size_t kFwdSmem = (size_t)3 * H * LDA * sizeof(__nv_bfloat16) + (size_t)kMaxMembers * kTile * 2 * sizeof(float);
constexpr size_t kBwdSmem = (size_t)2 * H * LDA * sizeof(__nv_bfloat16) + (size_t)kTile * 2 * sizeof(float);
constexpr size_t kGradSmem = (size_t)2 * H * LDC * sizeof(__nv_bfloat16) + kThreads * sizeof(float) + 16;

struct FwdArgs {
  int64_t n;
  int members;
  const float* x;              // [n][2]
  const float* master;         // [members][kP] (biases read in fp32)
  const __nv_bfloat16* wbf;    // [members][kPS] bf16 copies of the weights
  // training outputs
  float* z;                    // [members][n][4][128] pre-activations
  float* out;                  // [members][n][2]
  // screening outputs
  float* mean;                 // [n] mean of output 0 over members
  float* stdv;                 // [n] population standard deviation of output 0
  float* p1;                   // [n] mean of sigmoid(output 1)
};

struct BwdArgs {
  int64_t n;          // batch size
  const float* y;     // [n][2] targets
  const float* master;
  const __nv_bfloat16* wbf;
  const float* z;     // [members][n][4][128]
  const float* out;   // [members][n][2]
  float* dout;        // [members][n][2]
  float* dz;          // [members][4][n][128]
  float* loss;        // [members] (sum over samples of the per-sample loss)
};

constexpr int kMaxSplits = 8;     // batch slices of the weight-gradient kernel

struct GradArgs {
  int64_t n;
  const float* x;     // [n][2]
  const float* z;     // [members][n][4][128]
  const float* dz;    // [members][4][n][128]
  const float* dout;  // [members][n][2]
  float* grad;        // [splits][members][kP]: one partial gradient per batch slice
  int64_t rows;       // samples per slice (a multiple of kChunk)
};

// GELU, erf form, and its derivative: gelu(z) = z Phi(z), gelu'(z) = Phi(z) +
// z phi(z), with Phi and phi the standard normal distribution and density
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}
// both from one erf evaluation (the same expressions as gelu and gelu_grad)
__device__ __forceinline__ void gelu_and_grad(float z, float& h, float& g) {
  const float phi2 = 1.0f + erff(z * 0.70710678118654752f);
  h = 0.5f * z * phi2;
  g = 0.5f * phi2 + z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

// Weight and bias gradients of one 2-wide FP32 layer of member m over the
// samples r0 .. r1 - 1 into the parameter partial G:
//   l = 1: dW1[f][i] = sum_b dz_1[b][f] x[b][i],  db1[f] = sum_b dz_1[b][f];
//   l = 5: dW5[j][f] = sum_b dout[b][j] gelu(z_4[b][f]),  db5[j] = sum_b dout[b][j].
// 256 threads: thread = (feature f = tid % 128, half of the samples); part is
// 768 floats of shared scratch.  z [members][n][4][128], dz [members][4][n][128],
// dout [members][n][2], x [n][2].
__device__ __forceinline__ void wgrad_fp32_layer(int l, int m, int64_t n, int64_t r0, int64_t r1, const float* x,
                                                 const float* z, const float* dz, const float* dout, float* G,
                                                 float* part) {
  const int tid = threadIdx.x;
  const int f = tid & (H - 1), half = tid >> 7;
  const int64_t mid = r0 + (r1 - r0) / 2;
  const int64_t b0 = half ? mid : r0, b1 = half ? r1 : mid;
  float s0 = 0.f, s1 = 0.f, sb = 0.f;
  if (l == 1) {
    for (int64_t b = b0; b < b1; ++b) {
      const float d = dz[(((int64_t)m * 4 + 0) * n + b) * H + f];
      s0 = fmaf(d, x[2 * b], s0);
      s1 = fmaf(d, x[2 * b + 1], s1);
      sb += d;
    }
  } else {
    for (int64_t b = b0; b < b1; ++b) {
      const float h = gelu(z[(((int64_t)m * n + b) * 4 + 3) * H + f]);
      s0 = fmaf(dout[((int64_t)m * n + b) * 2], h, s0);
      s1 = fmaf(dout[((int64_t)m * n + b) * 2 + 1], h, s1);
    }
    if (f < 2) {
      for (int64_t b = b0; b < b1; ++b) sb += dout[((int64_t)m * n + b) * 2 + f];
    }
  }
  part[tid * 3 + 0] = s0;
  part[tid * 3 + 1] = s1;
  part[tid * 3 + 2] = sb;
  __syncthreads();
  if (tid < H) {
    const float w0 = part[tid * 3] + part[(tid + H) * 3];
    const float w1 = part[tid * 3 + 1] + part[(tid + H) * 3 + 1];
    const float bb = part[tid * 3 + 2] + part[(tid + H) * 3 + 2];
    if (l == 1) {
      G[oW1 + 2 * tid] = w0;
      G[oW1 + 2 * tid + 1] = w1;
      G[ob1 + tid] = bb;
    } else {
      G[oW5 + tid] = w0;
      G[oW5 + H + tid] = w1;
      if (tid < 2) G[ob5 + tid] = bb;
    }
  }
}

// batch slices for n samples: one per 128 samples, at most kMaxSplits
inline int grad_splits(int64_t n) {
  const int64_t s = (n + 127) / 128;
  return (int)(s < 1 ? 1 : (s > kMaxSplits ? kMaxSplits : s));
}

// Host launchers (the kernels live in mlp.cu).
cudaError_t set_smem_limits();
cudaError_t launch_forward_train(const FwdArgs& a, cudaStream_t s);
cudaError_t launch_forward_screen(const FwdArgs& a, cudaStream_t s);
cudaError_t launch_backward(const BwdArgs& a, int members, cudaStream_t s);
cudaError_t launch_wgrad(const GradArgs& a, int members, int splits, cudaStream_t s);
// grad[m][i] = sum over slices of part[s][m][i], slices in order (deterministic)
cudaError_t launch_grad_reduce(int members, int splits, const float* part, float* grad, cudaStream_t s);
// Adam step on the gradient sum over the slice partials part[splits][total]
cudaError_t launch_adam(int64_t total, float* w, __nv_bfloat16* wb, const float* part, int splits, float* m1,
                        float* m2, float lr, float b1, float b2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t launch_to_bf16(int64_t total, const float* w, __nv_bfloat16* wb, cudaStream_t s);
cudaError_t launch_init(int members, uint64_t seed, float* w, cudaStream_t s);
cudaError_t launch_gather(int64_t n, const int32_t* idx, const float* x, const float* y, float* xb, float* yb,
                          cudaStream_t s);

struct TrainTcArgs {
  int64_t n;
  int members;
  const float* x;            // [n][2]
  const float* y;            // [n][2] targets
  const float* master;       // [members][kP]
  const __nv_bfloat16* wbf;  // [members][kPS]
  __nv_bfloat16* wbfT;       // [members][3][128][128] W_2..W_4 transposed (written by step 1)
  float* z;                  // [members][n][4][128] pre-activations
  float* gp;                 // [members][n][4][128] gelu'(z), written by the forward for the backward
  float* out;                // [members][n][2]
  float* dout;               // [members][n][2]
  float* dz;                 // [members][4][n][128]
  float* loss;               // [members]
  float* grad;               // [splits][members][kP] slice partials
  int64_t rows;              // samples per weight-gradient slice
  unsigned* error;
};

// tcgen05 training (mlp_tc05_train.cu): step 0 forward (z, out), 1 the
// transposed weights (wbfT) then loss and input gradients (dout, dz, loss),
// 2 weight and bias gradients of all five layers into the slice partials.
cudaError_t launch_train_tc05(int step, const TrainTcArgs& a, int splits, cudaStream_t s);

// tcgen05 screening forward (mlp_tc05.cu): per-member outputs into out
// [members][n][2], then mean / spread / period-1 probability.
cudaError_t launch_screen_tc05(int64_t n, int members, const float* x, const float* master, const __nv_bfloat16* wbf,
                               float* out, unsigned* error, float* mean, float* stdv, float* p1, int sms,
                               cudaStream_t s);

// splitmix64 (Steele, Lea & Flood 2014): counter-based generator of the
// initial weights and of the shuffles.
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ULL;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
  return x ^ (x >> 31);
}

}  // namespace mlp
}  // namespace ens
