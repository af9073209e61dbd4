// mlp_tc05.cu -- ensemble screening forward on the 5th-generation tensor
// cores (tcgen05): accumulators in tensor memory, operands in shared memory.
//
// One CTA per SM, 128 threads (the four warps that own the 128 TMEM lanes).
// A CTA serves one ensemble member: it stages that member's three 128 x 128
// BF16 weight matrices in shared memory once, then walks its share of the
// 128-point tiles.  Per tile:
//   layer 1 (2 -> 128)  FP32 FMAs, thread = point, GELU, BF16 into the
//                       activation tile (shared memory, UMMA K-major layout);
//   layers 2..4         one thread issues 8 tcgen05.mma (M = N = 128, K = 16,
//                       BF16 x BF16 -> FP32 in TMEM), commits to an mbarrier;
//                       the four warps read their 32 TMEM lanes (tcgen05.ld
//                       32x32b), add the bias, apply GELU and write the next
//                       activation tile;
//   layer 5 (128 -> 2)  folded into the layer-4 epilogue as FP32 dot products.
// The per-member outputs [members][n][2] are reduced to mean / spread /
// period-1 probability by a second, elementwise kernel.
//
// Shared-memory operand layout (no swizzle, K-major): 8-row x 16-byte core
// matrices; core (r/8, k/8) of a 128 x 128 BF16 matrix starts at byte
// ((r/8) * 16 + k/8) * 128, so the K-direction core stride (leading byte
// offset) is 128 B and the row-group stride (stride byte offset) 2048 B.
// Waits on the mbarrier are bounded; on expiry the kernel records an error,
// waits (bounded) for its MMAs, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "mlp.cuh"
#include "tc05.cuh"

namespace ens {
namespace mlp {

namespace {

using namespace tc05;
constexpr int kTcThreads = tc05::kThreads;
// shared memory map (bytes from the 1024-aligned base)
constexpr size_t kSW = 0;                      // W2, W3, W4 (3 x 32 KB)
constexpr size_t kSA = kSW + 3 * kMatBytes;    // activation tile (32 KB)
constexpr size_t kSF = kSA + kMatBytes;        // fp32 W1[256], b1..b4[4][128], W5[256], b5[2]
constexpr size_t kSFFloats = 256 + 4 * 128 + 256 + 2;
constexpr size_t kSBar = kSF + ((kSFFloats * 4 + 15) / 16) * 16;   // mbarrier (8 B) + TMEM slot (4 B)
constexpr size_t kTcSmem = kSBar + 64 + 1024;  // + alignment slack

}  // namespace

struct TcArgs {
  int64_t n;
  int members;
  int ctas_per_member;
  const float* x;            // [n][2]
  const float* master;       // [members][kP]
  const __nv_bfloat16* wbf;  // [members][kPS]
  float* out;                // [members][n][2]
  unsigned* error;           // set to 1 if a wait expired
};

__global__ void __launch_bounds__(kTcThreads, 1) mlp_screen_tc05_kernel(TcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = blockIdx.x % a.members;
  const int g = blockIdx.x / a.members;
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  float* sf = reinterpret_cast<float*>(smem + kSF);
  float* sW1 = sf;              // [128][2]
  float* sB = sf + 256;         // b1..b4 [4][128]
  float* sW5 = sf + 256 + 512;  // [2][128]
  float* sB5 = sW5 + 256;       // [2]
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kSBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kSBar + 8);
  const uint32_t bar_a = smem_u32(bar);

  // stage this member's parameters
  const float* P = a.master + (int64_t)m * kP;
  const __nv_bfloat16* Pb = a.wbf + (int64_t)m * kPS;
  for (int i = tid; i < 256; i += kTcThreads) {
    sW1[i] = __bfloat162float(Pb[oW1 + i]);
    sW5[i] = __bfloat162float(Pb[oW5 + i]);
  }
  for (int i = tid; i < 128; i += kTcThreads) {
    sB[i] = P[ob1 + i];
    sB[128 + i] = P[ob2 + i];
    sB[256 + i] = P[ob3 + i];
    sB[384 + i] = P[ob4 + i];
  }
  if (tid < 2) sB5[tid] = P[ob5 + tid];
  for (int l = 0; l < 3; ++l) {
    const __nv_bfloat16* W = Pb + (l == 0 ? oW2 : l == 1 ? oW3 : oW4);
    unsigned char* dst = smem + kSW + l * kMatBytes;
    for (int idx = tid; idx < H * (H / 8); idx += kTcThreads) {   // 16-byte chunks: row n, k-chunk kc
      const int n = idx >> 4, kc = idx & 15;
      *reinterpret_cast<uint4*>(dst + core_off(n, kc * 8)) = *reinterpret_cast<const uint4*>(W + n * H + kc * 8);
    }
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar_a));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t sA = smem_u32(smem + kSA), sW = smem_u32(smem + kSW);
  uint32_t parity = 0;
  bool failed = false;

  for (int64_t t = g; t < tiles && !failed; t += a.ctas_per_member) {
    const int64_t p = t * kTile + tid;
    const bool live = p < a.n;
    const float x0 = live ? a.x[2 * p] : 0.f, x1 = live ? a.x[2 * p + 1] : 0.f;
    // layer 1: thread = point (row tid), 16 chunks of 8 features
    for (int kc = 0; kc < 16; ++kc) {
      uint32_t pk[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int f = kc * 8 + 2 * j;
        const float z0 = fmaf(sW1[2 * f + 1], x1, fmaf(sW1[2 * f], x0, sB[f]));
        const float z1 = fmaf(sW1[2 * f + 3], x1, fmaf(sW1[2 * f + 2], x0, sB[f + 1]));
        __nv_bfloat162 h2 = __floats2bfloat162_rn(gelu(z0), gelu(z1));
        pk[j] = *reinterpret_cast<uint32_t*>(&h2);
      }
      *reinterpret_cast<uint4*>(smem + kSA + core_off(tid, kc * 8)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
    float o0 = sB5[0], o1 = sB5[1];
    for (int l = 0; l < 3 && !failed; ++l) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (tid == 0) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          mma_bf16(tmem, make_desc(sA + k * 256), make_desc(sW + l * (uint32_t)kMatBytes + k * 256), k > 0);
        mma_commit(bar_a);
      }
      const bool ok = bar_wait(bar_a, parity);
      if (__syncthreads_or(!ok)) {  // block-uniform decision
        failed = true;
        if (tid == 0) atomicOr(a.error, 1u);
        break;
      }
      parity ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float* bl = sB + (l + 1) * 128;
      for (int c = 0; c < 4; ++c) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
        if (l < 2) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            uint32_t pk[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int col = c * 32 + q * 8 + 2 * j;
              __nv_bfloat162 h2 = __floats2bfloat162_rn(gelu(v[q * 8 + 2 * j] + bl[col]),
                                                        gelu(v[q * 8 + 2 * j + 1] + bl[col + 1]));
              pk[j] = *reinterpret_cast<uint32_t*>(&h2);
            }
            *reinterpret_cast<uint4*>(smem + kSA + core_off(tid, c * 32 + q * 8)) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = c * 32 + j;
            // round to BF16 like the activations of the hidden layers
            const float h = __bfloat162float(__float2bfloat16(gelu(v[j] + bl[col])));
            o0 = fmaf(h, sW5[col], o0);
            o1 = fmaf(h, sW5[128 + col], o1);
          }
        }
      }
    }
    if (live && !failed) {
      a.out[((int64_t)m * a.n + p) * 2] = o0;
      a.out[((int64_t)m * a.n + p) * 2 + 1] = o1;
    }
  }
  if (failed && tid == 0) {
    // give the MMAs in flight a bounded chance to land before the TMEM is freed
    bar_wait(bar_a, parity);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// mean / population spread of output 0 and mean sigmoid of output 1 over members
__global__ void mlp_reduce_members_kernel(int64_t n, int members, const float* out, float* mean, float* stdv,
                                          float* p1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.f, p = 0.f;
    for (int m = 0; m < members; ++m) {
      s += out[((int64_t)m * n + i) * 2];
      p += 1.0f / (1.0f + __expf(-out[((int64_t)m * n + i) * 2 + 1]));
    }
    const float mu = s / members;
    float s2 = 0.f;
    for (int m = 0; m < members; ++m) {
      const float d = out[((int64_t)m * n + i) * 2] - mu;
      s2 += d * d;
    }
    mean[i] = mu;
    stdv[i] = sqrtf(s2 / members);
    p1[i] = p / members;
  }
}

cudaError_t launch_screen_tc05(int64_t n, int members, const float* x, const float* master, const __nv_bfloat16* wbf,
                               float* out, unsigned* error, float* mean, float* stdv, float* p1, int sms,
                               cudaStream_t s) {
  // once per process (thread-safe static initialisation)
  static const cudaError_t attr = cudaFuncSetAttribute(mlp_screen_tc05_kernel,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
  if (attr != cudaSuccess) return attr;
  if (n == 0) return cudaSuccess;
  TcArgs a{};
  a.n = n;
  a.members = members;
  a.ctas_per_member = (sms + members - 1) / members;
  a.x = x;
  a.master = master;
  a.wbf = wbf;
  a.out = out;
  a.error = error;
  mlp_screen_tc05_kernel<<<a.ctas_per_member * members, kTcThreads, kTcSmem, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int64_t blocks = (n + 255) / 256;
  blocks = blocks > 8192 ? 8192 : blocks;
  mlp_reduce_members_kernel<<<(unsigned)blocks, 256, 0, s>>>(n, members, out, mean, stdv, p1);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace ens
