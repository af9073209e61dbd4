// tc05.cuh -- 5th-generation tensor-core (tcgen05) building blocks shared by
// the surrogate-network kernels: the no-swizzle K-major shared-memory operand
// layout and its descriptor, the BF16 MMA with FP32 accumulation in tensor
// memory, the commit to an mbarrier, a bounded mbarrier wait and the 32-column
// tensor-memory load.
//
// Operand layout: 8-row x 16-byte core matrices; core (r/8, k/8) of a
// 128 x 128 BF16 matrix starts at byte ((r/8) * 16 + k/8) * 128, so the
// K-direction core stride (leading byte offset) is 128 B and the row-group
// stride (stride byte offset) 2048 B.  A K = 16 step advances the descriptor
// start by two cores, 256 B.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "mlp.cuh"

namespace ens {
namespace mlp {
namespace tc05 {

constexpr int kThreads = 128;                                       // the four warps of the 128 TMEM lanes
constexpr uint32_t kTmemCols = 128;
constexpr size_t kMatBytes = (size_t)H * H * sizeof(__nv_bfloat16);  // 32 KB
constexpr uint32_t kWaitLimit = 1u << 20;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// byte offset of element (r, k) of a 128 x 128 BF16 operand in core-matrix layout
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)(((r >> 3) * 16 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

// shared-memory matrix descriptor: start >> 4, LBO = 128 B, SBO = 2048 B,
// descriptor version 1 (bit 46), no swizzle
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(2048u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major,
// N = 128 (bits 17-22 = N >> 3), M = 128 (bits 24-28 = M >> 4)
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

// D (TMEM) = A (128 x 128, K-major at sa) * B^T (128 x 128, K-major at sb),
// accumulating onto D when acc != 0: eight K = 16 steps.  One thread issues.
__device__ __forceinline__ void mma_128(uint32_t d_tmem, uint32_t sa, uint32_t sb, bool acc) {
#pragma unroll
  for (int k = 0; k < 8; ++k) mma_bf16(d_tmem, make_desc(sa + k * 256), make_desc(sb + k * 256), (acc || k > 0) ? 1u : 0u);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// bounded wait for the mbarrier phase `parity`; returns false on expiry
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// make shared-memory writes of the generic proxy visible to the tensor cores
// and order them against the thread barrier that follows
__device__ __forceinline__ void fence_to_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

}  // namespace tc05
}  // namespace mlp
}  // namespace ens
