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
cudaError_t launch_adam(int64_t total, float* w, __nv_bfloat16* wb, const float* g, float* m1, float* m2, float lr,
                        float b1, float b2, float eps, float c1, float c2, cudaStream_t s);
cudaError_t launch_to_bf16(int64_t total, const float* w, __nv_bfloat16* wb, cudaStream_t s);
cudaError_t launch_init(int members, uint64_t seed, float* w, cudaStream_t s);
cudaError_t launch_gather(int64_t n, const int32_t* idx, const float* x, const float* y, float* xb, float* yb,
                          cudaStream_t s);

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
