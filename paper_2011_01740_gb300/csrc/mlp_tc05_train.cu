// mlp_tc05_train.cu -- surrogate-network training on the 5th-generation
// tensor cores (tcgen05): forward with stored pre-activations, input
// gradients and weight gradients of the three 128 x 128 layers, accumulators
// in tensor memory, operands in shared memory (layout in tc05.cuh).
//
// Every CTA has 256 threads in two warpgroups.  Warp w reads TMEM lanes
// 32 (w % 4) .. + 31 (a warp may only touch its own quarter of the lanes) and
// columns 64 (w / 4) .. + 63, so the two warpgroups split each epilogue.  One
// thread issues the MMAs and commits them to an mbarrier; all threads wait on
// it (bounded) before reading TMEM with tcgen05.ld.  The products:
//   forward      Z_l[sample][out] = H_{l-1}[sample][in] W_l[out][in]
//                (A = activations, B = W_l as stored: [out][in] is K-major);
//   input grad.  G[sample][in] = D_l[sample][out] W_l[out][in]
//                (A = output gradients, B = the transposed copy W_l^T[in][out],
//                written once per batch by mlp_transpose_w_kernel);
//   weight grad. dW_l[out][in] = sum_b D_l[b][out] H_{l-1}[b][in]
//                (K = samples: both operands transposed while staging).
// BF16 operands, FP32 accumulation, as the mma.sync kernels of mlp.cu, whose
// buffers (z, dz, dout, out) and conventions these kernels share; layers 1 and
// 5 (2-wide) stay in FP32.  A wait that expires sets the error word; the CTA
// then waits (bounded) for its MMAs, frees its tensor memory and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include "mlp.cuh"
#include "tc05.cuh"

namespace ens {
namespace mlp {

namespace {

using namespace tc05;
constexpr int kT = 256;   // two warpgroups

__host__ __device__ constexpr int64_t w_of(int l) { return l == 2 ? oW2 : l == 3 ? oW3 : oW4; }
__host__ __device__ constexpr int64_t b_of(int l) { return l == 1 ? ob1 : l == 2 ? ob2 : l == 3 ? ob3 : ob4; }
static_assert(kP % 2 == 0 && oW2 % 2 == 0 && oW3 % 2 == 0 && oW4 % 2 == 0, "8-byte gradient stores");
static_assert(kPS % 8 == 0 && oW2 % 8 == 0 && oW3 % 8 == 0 && oW4 % 8 == 0, "16-byte weight loads");
static_assert(ob3 - ob2 == ob2 - ob1 && ob4 - ob3 == ob2 - ob1, "evenly spaced hidden biases");

// shared memory of the forward and input-gradient kernels
constexpr size_t kFW = 0;                                // three 128 x 128 BF16 operands
constexpr size_t kFA = kFW + 3 * kMatBytes;              // activation / gradient tile
constexpr size_t kFF = kFA + kMatBytes;                  // fp32 side data
constexpr int kFO = 1032;                                // output partials of the second warpgroup
constexpr size_t kFFloats = kFO + 2 * 128;
constexpr size_t kFBar = kFF + ((kFFloats * 4 + 15) / 16) * 16;
constexpr size_t kFSmem = kFBar + 64 + 1024;
// shared memory of the weight-gradient kernel
constexpr size_t kGA = 0;
constexpr size_t kGB = kGA + kMatBytes;
constexpr size_t kGR = kGB + kMatBytes;                  // [256] bias partials
constexpr size_t kGBar = kGR + 256 * 4;
constexpr size_t kGSmem = kGBar + 64 + 1024;

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return reinterpret_cast<unsigned char*>(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
}

// TMEM address of the 32 columns c * 32 .. + 31 in this warp's lane quarter
__device__ __forceinline__ uint32_t tmem_at(uint32_t tmem, int c) {
  return tmem + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + (uint32_t)(c * 32);
}

// barrier init and TMEM allocation at kernel start (all threads call)
__device__ __forceinline__ uint32_t tc_setup(uint32_t bar, uint32_t* tslot) {
  const int tid = threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((tid >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_to_mma();
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return *tslot;
}

// TMEM release at kernel end (all threads call); after a failed wait the
// MMAs in flight get a bounded chance to land first
__device__ __forceinline__ void tc_teardown(uint32_t tmem, uint32_t bar, uint32_t parity, bool failed) {
  if (failed && threadIdx.x == 0) bar_wait(bar, parity);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
  }
}

// issue one 128 x 128 x 128 product into TMEM (all threads call: the
// operands written by every thread are fenced and published first)
__device__ __forceinline__ void tc_issue(uint32_t tmem, uint32_t sa, uint32_t sb, bool acc, uint32_t bar) {
  fence_to_mma();
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    mma_128(tmem, sa, sb, acc);
    mma_commit(bar);
  }
}

// wait for the product issued last; returns false (block-uniformly) when the
// wait expired
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t& parity, unsigned* error) {
  const bool ok = bar_wait(bar, parity);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) atomicOr(error, 1u);
    return false;
  }
  parity ^= 1u;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  return true;
}

__device__ __forceinline__ bool tc_product(uint32_t tmem, uint32_t sa, uint32_t sb, bool acc, uint32_t bar,
                                           uint32_t& parity, unsigned* error) {
  tc_issue(tmem, sa, sb, acc, bar);
  return tc_wait(bar, parity, error);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h2 = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&h2);
}

__device__ __forceinline__ void store_bf16x8(unsigned char* base, int r, int k, const float* v) {
  *reinterpret_cast<uint4*>(base + core_off(r, k)) =
      make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]), pack_bf16x2(v[6], v[7]));
}

// eight consecutive floats (16-byte aligned) as two 16-byte loads; zeros when !live
__device__ __forceinline__ void load8(const float* src, bool live, float* v) {
  float4 lo = make_float4(0.f, 0.f, 0.f, 0.f), hi = lo;
  if (live) {
    lo = reinterpret_cast<const float4*>(src)[0];
    hi = reinterpret_cast<const float4*>(src)[1];
  }
  v[0] = lo.x, v[1] = lo.y, v[2] = lo.z, v[3] = lo.w, v[4] = hi.x, v[5] = hi.y, v[6] = hi.z, v[7] = hi.w;
}

// eight consecutive floats to a 16-byte aligned address
__device__ __forceinline__ void store8(float* dst, const float* v) {
  reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// output gradients D[b][f] and pre-activations Z[b * 512 + f] of the samples
// b0 .. b0 + 7 (0 past r1)
__device__ __forceinline__ void load_group(const float* D, const float* Z, int64_t b0, int64_t r1, int f, float* d,
                                           float* z) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t smp = b0 + j;
    d[j] = smp < r1 ? D[smp * H + f] : 0.f;
    z[j] = smp < r1 ? Z[smp * 4 * H + f] : 0.f;
  }
}

// Stage three row-major 128 x 128 BF16 matrices M_i[n][k] as K-major
// operands at dst + i * kMatBytes.  Thread index bits: 0-2 the row within a
// core matrix, 3-6 the 16-byte chunk of the row, 7 and up the row group; a
// phase of 8 threads then writes one whole 128-byte core matrix (no bank
// conflict) and a warp reads 8 rows x 64 contiguous bytes.  All 24 loads of
// a thread are issued before its stores.
__device__ __forceinline__ void stage3_kmajor(unsigned char* dst, const __nv_bfloat16* M0, const __nv_bfloat16* M1,
                                              const __nv_bfloat16* M2) {
  constexpr int kIt = H * (H / 8) / kT;   // 8 chunks per thread and matrix
  const __nv_bfloat16* Ms[3] = {M0, M1, M2};
  uint4 v[3][kIt];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int idx = it * kT + (int)threadIdx.x;
      const int n = (idx >> 7) * 8 + (idx & 7), kc = (idx >> 3) & 15;
      v[i][it] = *reinterpret_cast<const uint4*>(Ms[i] + n * H + kc * 8);
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int it = 0; it < kIt; ++it) {
      const int idx = it * kT + (int)threadIdx.x;
      const int n = (idx >> 7) * 8 + (idx & 7), kc = (idx >> 3) & 15;
      *reinterpret_cast<uint4*>(dst + i * kMatBytes + core_off(n, kc * 8)) = v[i][it];
    }
  }
}

}  // namespace

// W_l^T of layers 2..4 of every member: wbfT[m][l - 2][in][out] = W_l[out][in].
// grid = members * 3, 256 threads; thread = one 8 x 8 block, transposed in
// registers (pairs of BF16 values regrouped with byte permutes).
__global__ void __launch_bounds__(256) mlp_transpose_w_kernel(const __nv_bfloat16* wbf, __nv_bfloat16* wbfT) {
  const int m = blockIdx.x / 3, l = blockIdx.x % 3 + 2;
  const __nv_bfloat16* W = wbf + (int64_t)m * kPS + w_of(l);
  __nv_bfloat16* T = wbfT + (int64_t)blockIdx.x * H * H;
  const int ob = threadIdx.x & 15, ib = threadIdx.x >> 4;
  uint32_t r[8][4];   // r[j] = W[ob*8 + j][ib*8 .. ib*8 + 7]
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint4 q = *reinterpret_cast<const uint4*>(W + (ob * 8 + j) * H + ib * 8);
    r[j][0] = q.x;
    r[j][1] = q.y;
    r[j][2] = q.z;
    r[j][3] = q.w;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    // row ib*8 + i of the transpose: element j = W[ob*8 + j][ib*8 + i], the
    // low (i even) or high (i odd) half of word i/2 of r[j]
    const uint32_t sel = (i & 1) ? 0x7632u : 0x5410u;
    uint4 o;
    o.x = __byte_perm(r[0][i >> 1], r[1][i >> 1], sel);
    o.y = __byte_perm(r[2][i >> 1], r[3][i >> 1], sel);
    o.z = __byte_perm(r[4][i >> 1], r[5][i >> 1], sel);
    o.w = __byte_perm(r[6][i >> 1], r[7][i >> 1], sel);
    *reinterpret_cast<uint4*>(T + (ib * 8 + i) * H + ob * 8) = o;
  }
}

// Forward of one 128-sample tile of one member: grid = (tiles, members).
// Stores the pre-activations z (for the weight gradients) and gelu'(z) (for
// the backward) of the four hidden layers, and the outputs.
// Sample s = tid % 128 is TMEM lane s; warpgroup hf = tid / 128 takes the
// features 64 hf .. + 63 of every layer.
__global__ void __launch_bounds__(kT, 1) mlp_forward_train_tc05_kernel(TrainTcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  const int tid = threadIdx.x, s = tid & 127, hf = tid >> 7;
  const int m = blockIdx.y;
  const int64_t p = (int64_t)blockIdx.x * kTile + s;
  const bool live = p < a.n;
  float* sf = reinterpret_cast<float*>(smem + kFF);
  float* sW1 = sf;              // [128][2]
  float* sB = sf + 256;         // b1..b4
  float* sW5 = sf + 256 + 512;  // [2][128]
  float* sB5 = sW5 + 256;
  float* sO = sf + kFO;         // [128][2] output partials of features 64..127
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kFBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kFBar + 8);
  const uint32_t bar_a = smem_u32(bar);
  const float* P = a.master + (int64_t)m * kP;
  const __nv_bfloat16* Pb = a.wbf + (int64_t)m * kPS;
  for (int i = tid; i < 256; i += kT) {
    sW1[i] = __bfloat162float(Pb[oW1 + i]);
    sW5[i] = __bfloat162float(Pb[oW5 + i]);
  }
  for (int i = tid; i < 512; i += kT) sB[i] = P[ob1 + (i >> 7) * (ob2 - ob1) + (i & 127)];
  if (tid < 2) sB5[tid] = P[ob5 + tid];
  // W_l [out][in] is the K-major B operand as stored
  stage3_kmajor(smem + kFW, Pb + w_of(2), Pb + w_of(3), Pb + w_of(4));
  const uint32_t tmem = tc_setup(bar_a, tslot);   // its barrier also publishes sf
  const uint32_t sA = smem_u32(smem + kFA), sW = smem_u32(smem + kFW);
  uint32_t parity = 0;
  bool failed = false;
  const int64_t row = ((int64_t)m * a.n + (live ? p : 0)) * 4 * H;   // [4][128] of this sample
  float* zrow = a.z + row;
  float* grow = a.gp + row;
  // layer 1 in FP32
  {
    const float x0 = live ? a.x[2 * p] : 0.f, x1 = live ? a.x[2 * p + 1] : 0.f;
    for (int kc = hf * 8; kc < hf * 8 + 8; ++kc) {
      float zv[8], hv[8], gv[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int f = kc * 8 + j;
        zv[j] = fmaf(sW1[2 * f + 1], x1, fmaf(sW1[2 * f], x0, sB[f]));
        gelu_and_grad(zv[j], hv[j], gv[j]);
      }
      store_bf16x8(smem + kFA, s, kc * 8, hv);
      if (live) {
        store8(zrow + kc * 8, zv);
        store8(grow + kc * 8, gv);
      }
    }
  }
  float o0 = hf ? 0.f : sB5[0], o1 = hf ? 0.f : sB5[1];
  for (int l = 2; l <= 4 && !failed; ++l) {
    if (!tc_product(tmem, sA, sW + (uint32_t)((l - 2) * kMatBytes), false, bar_a, parity, a.error)) {
      failed = true;
      break;
    }
    const float* bl = sB + (l - 1) * 128;
    for (int c = 2 * hf; c < 2 * hf + 2; ++c) {
      float v[32];
      tmem_ld32(tmem_at(tmem, c), v);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] += bl[c * 32 + j];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int col0 = c * 32 + q * 8;
        float hv[8], gv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) gelu_and_grad(v[q * 8 + j], hv[j], gv[j]);
        if (live) {
          store8(zrow + (l - 1) * H + col0, v + q * 8);
          store8(grow + (l - 1) * H + col0, gv);
        }
        if (l < 4) {
          store_bf16x8(smem + kFA, s, col0, hv);
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // the output layer reads the BF16-rounded activations, as the MMAs do
            const float h = __bfloat162float(__float2bfloat16(hv[j]));
            o0 = fmaf(h, sW5[col0 + j], o0);
            o1 = fmaf(h, sW5[128 + col0 + j], o1);
          }
        }
      }
    }
  }
  if (hf == 1) {
    sO[2 * s] = o0;
    sO[2 * s + 1] = o1;
  }
  __syncthreads();   // failed is block-uniform: every thread gets here
  if (hf == 0 && live && !failed) {
    a.out[((int64_t)m * a.n + p) * 2] = o0 + sO[2 * s];
    a.out[((int64_t)m * a.n + p) * 2 + 1] = o1 + sO[2 * s + 1];
  }
  tc_teardown(tmem, bar_a, parity, failed);
}

// Loss, output gradient and the gradients of the pre-activations of one
// 128-sample tile of one member: grid = (tiles, members).  dz_4 = (dout W5)
// * gelu'(z_4) in FP32; dz_{l-1} = (dz_l W_l) * gelu'(z_{l-1}) for l = 4, 3, 2
// (gelu'(z) as the forward wrote it)
// on the tensor cores with W_l^T (a.wbfT) as the B operand.  Warpgroup hf
// takes features 64 hf .. + 63; the first one also owns loss and dout.
__global__ void __launch_bounds__(kT, 1) mlp_backward_tc05_kernel(TrainTcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, s = tid & 127, hf = tid >> 7;
  const int m = blockIdx.y;
  const int64_t p = (int64_t)blockIdx.x * kTile + s;
  const bool live = p < a.n;
  float* sf = reinterpret_cast<float*>(smem + kFF);
  float* sW5 = sf;            // [2][128]
  float* red = sf + 256;      // [8] loss partials of the warps
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kFBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kFBar + 8);
  const uint32_t bar_a = smem_u32(bar);
  const __nv_bfloat16* Pb = a.wbf + (int64_t)m * kPS;
  for (int i = tid; i < 256; i += kT) sW5[i] = __bfloat162float(Pb[oW5 + i]);
  // B operand of the input gradient: element (n = in, k = out) = W_l^T[in][out]
  const __nv_bfloat16* WT = a.wbfT + (int64_t)m * 3 * H * H;
  stage3_kmajor(smem + kFW, WT, WT + H * H, WT + 2 * H * H);
  const uint32_t tmem = tc_setup(bar_a, tslot);
  const uint32_t sA = smem_u32(smem + kFA), sW = smem_u32(smem + kFW);
  uint32_t parity = 0;
  bool failed = false;
  const float inv_n = 1.0f / (float)a.n;
  const float* grow = a.gp + ((int64_t)m * a.n + (live ? p : 0)) * 4 * H;   // gelu'(z) of this sample
  // loss and output gradient of sample s (both warpgroups need dout)
  float d0 = 0.f, d1 = 0.f, lsum = 0.f;
  if (live) {
    const float o0 = a.out[((int64_t)m * a.n + p) * 2], o1 = a.out[((int64_t)m * a.n + p) * 2 + 1];
    const float y0 = a.y[2 * p], y1 = a.y[2 * p + 1];
    d0 = 2.0f * (o0 - y0) * inv_n;
    d1 = (1.0f / (1.0f + __expf(-o1)) - y1) * inv_n;
    if (hf == 0) {
      lsum = (o0 - y0) * (o0 - y0) + fmaxf(o1, 0.f) - o1 * y1 + log1pf(__expf(-fabsf(o1)));
      a.dout[((int64_t)m * a.n + p) * 2] = d0;
      a.dout[((int64_t)m * a.n + p) * 2 + 1] = d1;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
  if (lane == 0) red[warp] = lsum;
  // dz_4 in FP32; gelu'(z_4) of this thread's 64 features is loaded first
  // (16 independent 16-byte loads)
  float gz[64];
#pragma unroll
  for (int q = 0; q < 8; ++q) load8(grow + 3 * H + hf * 64 + q * 8, live, gz + q * 8);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int kc = hf * 8 + q;
    float dv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int f = kc * 8 + j;
      dv[j] = live ? fmaf(d0, sW5[f], d1 * sW5[128 + f]) * gz[q * 8 + j] : 0.f;
    }
    store_bf16x8(smem + kFA, s, kc * 8, dv);
    if (live) {
      float4* dd = reinterpret_cast<float4*>(a.dz + (((int64_t)m * 4 + 3) * a.n + p) * H + kc * 8);
      dd[0] = make_float4(dv[0], dv[1], dv[2], dv[3]);
      dd[1] = make_float4(dv[4], dv[5], dv[6], dv[7]);
    }
  }
  __syncthreads();
  if (tid == 0) {
    float t = 0.f;
    for (int w = 0; w < kT / 32; ++w) t += red[w];
    atomicAdd(&a.loss[m], t);
  }
  for (int l = 4; l >= 2 && !failed; --l) {
    tc_issue(tmem, sA, sW + (uint32_t)((l - 2) * kMatBytes), false, bar_a);
    // gelu'(z_{l-1}) of this thread's features, loaded while the product runs
#pragma unroll
    for (int q = 0; q < 8; ++q) load8(grow + (l - 2) * H + hf * 64 + q * 8, live, gz + q * 8);
    if (!tc_wait(bar_a, parity, a.error)) {
      failed = true;
      break;
    }
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
      const int c = 2 * hf + cc;
      float v[32];
      tmem_ld32(tmem_at(tmem, c), v);
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = live ? v[j] * gz[cc * 32 + j] : 0.f;
      if (live) {
        float4* dd = reinterpret_cast<float4*>(a.dz + (((int64_t)m * 4 + (l - 2)) * a.n + p) * H + c * 32);
#pragma unroll
        for (int q = 0; q < 8; ++q) dd[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
      if (l > 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) store_bf16x8(smem + kFA, s, c * 32 + q * 8, v + q * 8);
      }
    }
  }
  tc_teardown(tmem, bar_a, parity, failed);
}

// Weight and bias gradients of one batch slice of one member: grid =
// (members, 5, slices); blockIdx.y = 0..2 layers 2..4 on the tensor cores,
// 3 and 4 the FP32 layers 1 and 5 (wgrad_fp32_layer).  Per 128-sample chunk
// the output gradients (A: element (out, b)) and the activations (B: element
// (in, b)) are transposed into shared memory; the chunks accumulate in TMEM.
// Staging: thread = (feature f = tid % 128, half of the chunk), 8 samples
// packed per 16-byte store.  Writes the slice's partial dW_l and db_l.
__global__ void __launch_bounds__(kT, 3) mlp_wgrad_tc05_kernel(TrainTcArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = align1024(smem_raw);
  const int tid = threadIdx.x, f = tid & 127, hf = tid >> 7;
  const int m = blockIdx.x;
  float* G = a.grad + ((int64_t)blockIdx.z * a.members + m) * kP;
  const int64_t r0 = (int64_t)blockIdx.z * a.rows;
  const int64_t r1 = r0 + a.rows < a.n ? r0 + a.rows : a.n;
  if (blockIdx.y >= 3) {   // layers 1 and 5 in FP32, no tensor memory
    wgrad_fp32_layer(blockIdx.y == 3 ? 1 : 5, m, a.n, r0, r1, a.x, a.z, a.dz, a.dout, G,
                     reinterpret_cast<float*>(smem));
    return;
  }
  const int l = blockIdx.y + 2;
  float* red = reinterpret_cast<float*>(smem + kGR);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kGBar);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + kGBar + 8);
  const uint32_t bar_a = smem_u32(bar);
  const uint32_t tmem = tc_setup(bar_a, tslot);
  const uint32_t sA = smem_u32(smem + kGA), sB = smem_u32(smem + kGB);
  uint32_t parity = 0;
  bool failed = false, any = false;
  float bsum = 0.f;  // bias gradient of feature f over this thread's samples
  const float* D = a.dz + (((int64_t)m * 4 + (l - 1)) * a.n) * H;      // dz_l [n][128]
  const float* Z = a.z + (int64_t)m * a.n * 4 * H + (l - 2) * H;        // z_{l-1} of sample b at Z[b * 512]
  for (int64_t c0 = r0; c0 < r1 && !failed; c0 += kTile) {
    // groups of 8 samples; the loads of group g + 1 are in flight while
    // group g is converted and stored (samples past r1 read as 0, gelu(0) = 0)
    float dn[8], zn[8];
    load_group(D, Z, c0 + hf * 64, r1, f, dn, zn);
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int b0 = hf * 64 + g * 8;
      float d[8], h[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        d[j] = dn[j];
        h[j] = zn[j];
      }
      if (g < 7) load_group(D, Z, c0 + b0 + 8, r1, f, dn, zn);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        h[j] = gelu(h[j]);
        bsum += d[j];
      }
      store_bf16x8(smem + kGA, f, b0, d);
      store_bf16x8(smem + kGB, f, b0, h);
    }
    if (!tc_product(tmem, sA, sB, any, bar_a, parity, a.error)) {
      failed = true;
      break;
    }
    any = true;
  }
  red[tid] = bsum;
  __syncthreads();   // failed is block-uniform
  if (!failed) {
    if (hf == 0) G[b_of(l) + f] = red[f] + red[f + 128];
    float* Wg = G + w_of(l) + (int64_t)f * H;   // row out = f (TMEM lane)
    for (int c = 2 * hf; c < 2 * hf + 2; ++c) {
      float v[32];
      if (any) {
        tmem_ld32(tmem_at(tmem, c), v);
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = 0.f;
      }
      // 8-byte stores: the member stride kP is even but not a multiple of 4
      float2* wd = reinterpret_cast<float2*>(Wg + c * 32);
#pragma unroll
      for (int q = 0; q < 16; ++q) wd[q] = make_float2(v[2 * q], v[2 * q + 1]);
    }
  }
  tc_teardown(tmem, bar_a, parity, failed);
}

cudaError_t launch_train_tc05(int step, const TrainTcArgs& a, int splits, cudaStream_t s) {
  // once per process (thread-safe static initialisation)
  static const cudaError_t attr = [] {
    cudaError_t e = cudaFuncSetAttribute(mlp_forward_train_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kFSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mlp_backward_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(mlp_wgrad_tc05_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGSmem);
    return e;
  }();
  if (attr != cudaSuccess) return attr;
  const int64_t tiles = (a.n + kTile - 1) / kTile;
  if (a.n <= 0 || tiles > 0x7fffffffLL || a.members < 1 || a.members > kMaxMembers) return cudaErrorInvalidValue;
  if (step == 0) {
    mlp_forward_train_tc05_kernel<<<dim3((unsigned)tiles, a.members), kT, kFSmem, s>>>(a);
  } else if (step == 1) {
    if (!a.wbfT) return cudaErrorInvalidValue;
    mlp_transpose_w_kernel<<<a.members * 3, 256, 0, s>>>(a.wbf, a.wbfT);
    mlp_backward_tc05_kernel<<<dim3((unsigned)tiles, a.members), kT, kFSmem, s>>>(a);
  } else {
    if (splits < 1 || splits > kMaxSplits || (int64_t)splits * a.rows < a.n) return cudaErrorInvalidValue;
    mlp_wgrad_tc05_kernel<<<dim3(a.members, 5, splits), kT, kGSmem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace ens
