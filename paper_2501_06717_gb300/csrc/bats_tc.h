// bats_tc.h -- device helpers shared by the learned correction's kernels
// (bats_mlp.cu) and the fused learned stage (bats_stage.cu): BF16 packing,
// the tanh-form GELU, and the tcgen05 building blocks (shared-memory matrix
// descriptors of the no-swizzle K-major canonical layout, the BF16 MMA with
// an FP32 accumulator in tensor memory, commit to an mbarrier, tensor-memory
// loads, bounded mbarrier waits).
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "bats_internal.h"

namespace batsk {

__device__ __forceinline__ uint32_t tc_saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf16_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ float tanh_approx(float x) {
  float r;
  asm("tanh.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// GELU, tanh form, and its derivative.
__device__ __forceinline__ float gelu_f(float x) {
  const float k = 0.7978845608028654f;
  return 0.5f * x * (1.0f + tanh_approx(k * (x + 0.044715f * x * x * x)));
}
// Two GELUs (tanh form) rounded to a BF16 pair (x0 in the low half), in
// packed FP32 arithmetic around one tanh.approx.f32 per value:
// u = x (k + k 0.044715 x^2), gelu = h + h tanh(u) with h = x / 2.  The
// hardware tanh has an absolute error of a few 2^-12, so
// |gelu2 - gelu| <= 0.5 |x| 1e-3 + the final BF16 rounding (2^-9 relative),
// the size of the BF16 rounding every hidden activation gets anyway.  For
// |x| beyond the FP32 range of x^2 the argument is +-inf and tanh +-1: the
// GELU's limits.
__device__ __forceinline__ float2 gelu_arg2(float2 x) {
  const float k = 0.7978845608028654f, c = 0.7978845608028654f * 0.044715f;
  return __fmul2_rn(x, __ffma2_rn(__fmul2_rn(x, x), make_float2(c, c), make_float2(k, k)));
}
__device__ __forceinline__ uint32_t gelu2_pack(float x0, float x1) {
  const float2 u = gelu_arg2(make_float2(x0, x1));
  const float2 t = make_float2(tanh_approx(u.x), tanh_approx(u.y));
  const float2 h = __fmul2_rn(make_float2(0.5f, 0.5f), make_float2(x0, x1));
  const float2 g = __ffma2_rn(h, t, h);
  return pack_bf16(g.x, g.y);
}
// Twice the GELU pair, x (1 + tanh(u)), for a layer whose next layer takes
// weights halved (exactly, in BF16): one multiplication fewer per pair, and
// BF16(2 g) = 2 BF16(g), so the next layer's products are the same.
__device__ __forceinline__ uint32_t gelu2x_pack(float x0, float x1) {
  const float2 x = make_float2(x0, x1);
  const float2 u = gelu_arg2(x);
  const float2 t = make_float2(tanh_approx(u.x), tanh_approx(u.y));
  const float2 g = __ffma2_rn(x, t, x);
  return pack_bf16(g.x, g.y);
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float k = 0.7978845608028654f;
  float t = tanh_approx(k * (x + 0.044715f * x * x * x));
  return 0.5f * (1.0f + t) + 0.5f * x * (1.0f - t * t) * k * (1.0f + 3.0f * 0.044715f * x * x);
}

// ---------------------------------------------------------------------------
// Inference on tcgen05.  Operands in shared memory use the no-swizzle K-major
// canonical layout: "core matrices" of 8 rows x 16 bytes (8 BF16 along K)
// stored as 128 contiguous bytes; core matrices adjacent along K are LBO =
// 128 bytes apart, those adjacent along M (or N) SBO = 16 K bytes apart.

// byte offset of the 16-byte chunk (row r, K chunk kc) in a canonical tile
__device__ __forceinline__ uint32_t cm_off(int r, int kc, uint32_t sbo) {
  return static_cast<uint32_t>(r >> 3) * sbo + static_cast<uint32_t>(kc) * 128u + static_cast<uint32_t>(r & 7) * 16u;
}
// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), LBO >> 4
// (16-29), SBO >> 4 (32-45), the fixed value 1 in bits 46-48, base offset 0,
// relative LBO, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t umma_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4) | (static_cast<uint64_t>(lbo >> 4) << 16) |
         (static_cast<uint64_t>(sbo >> 4) << 32) | (1ull << 46);
}
// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9 and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t umma_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(N >> 3) << 17) |
         (static_cast<uint32_t>(M >> 4) << 24);
}
// D[tmem] (+)= A B^T for one K = 16 slice; accum = 0 overwrites D.
__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
// The mbarrier completes one phase once every tcgen05.mma this thread issued
// before has finished.
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(tc_saddr(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void proxy_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// 16 consecutive FP32 columns of this thread's tensor-memory lane (the wait
// for the load sits in the same statement, so no use of the registers can be
// scheduled ahead of it).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; i++) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void mbar_init_tc(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_saddr(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait_tc(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(tc_saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for an mbarrier phase for at most ~1 s of wall time; on expiry record
// ERR_TIMEOUT and return false.
static __device__ __noinline__ bool mbar_wait_bounded_tc(uint64_t* bar, uint32_t parity, int32_t* err) {
  if (mbar_try_wait_tc(bar, parity)) return true;
  uint64_t t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    if (mbar_try_wait_tc(bar, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) {
      atomicOr(err, ERR_TIMEOUT);
      return false;
    }
  }
}

constexpr uint32_t SBO_K48 = 768;        // 16 bytes x K = 48
constexpr uint32_t SBO_K64 = 1024;       // 16 bytes x K = 64
constexpr uint32_t SBO_K80 = 1280;       // 16 bytes x K = 80

// true in one lane of the (converged) warp
__device__ __forceinline__ bool elect_one() {
  uint32_t pred;
  asm volatile(
      "{\n .reg .b32 r;\n .reg .pred p;\n elect.sync r|p, 0xffffffff;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(pred));
  return pred != 0;
}

// 32 consecutive FP32 columns of this thread's tensor-memory lane, the wait
// for the load in the same statement.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

}  // namespace batsk
