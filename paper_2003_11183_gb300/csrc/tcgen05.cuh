// tcgen05 / TMA building blocks of the tensor-core products (sm_103a): stage
// shapes and instruction descriptors, shared-memory matrix descriptors, bounded
// mbarrier waits, 2-D TMA loads, the 16-bit (bf16 or fp16) MMA and its commit.  Used by the
// whole-tile sweep of the BF16-shift integrand (sweep_tc.cuh), whose products are
//
//   D (M x N) += A (M x K) * B (N x K)^T     bf16 or fp16 operands (both the same type):
//                                             B K-major; A K-major,
//                                             or MN-major (A_MN: stored K x M, M contiguous)
//
// with M = 128 (TMEM lanes = samples), fp32 accumulation in TMEM, operands staged
// by TMA with 128-byte (64-deep stages) or 64-byte (32-deep) swizzle.  Every
// mbarrier wait is bounded: on expiry the caller records an error code and gives up.
#pragma once
#include <cuda.h>
#include "common.cuh"

namespace tlrmvn {
namespace tc {

constexpr int BM = 128;
constexpr uint32_t WAIT_LIMIT = 1u << 24;  // polls before a wait gives up (seconds)

// Shape of one product configuration: K depth of a stage (KB = 64 with 128-byte
// swizzle, or 32 with 64-byte swizzle), tile bytes, stage bytes (SPLIT stages
// hold hi and lo tiles of both operands), stage count and shared memory.  By
// default SPLIT configurations take one stage and others two or four; NSTQ > 0
// fixes the stage count.
template <int BN, bool SPLIT, bool A_MN = false, int KB = 64, int NSTQ = 0>
struct Cfg {
  static constexpr int BK = KB;
  static constexpr int A_BYTES = BM * KB * 2;
  static constexpr int B_BYTES = BN * KB * 2;
  static constexpr int HALF = A_BYTES + B_BYTES;  // [A][B] of one precision part
  static constexpr int SB = SPLIT ? 2 * HALF : HALF;
  static constexpr int NST = NSTQ > 0 ? NSTQ : (SPLIT ? 1 : ((4 * SB <= 100 * 1024) ? 4 : 2));
  static constexpr int SMEM = NST * SB + 1024 /*align*/ + 256 /*barriers*/;
  // instruction descriptor of tcgen05.mma kind::f16: fp32 accumulator, bf16 A
  // and B (bits 7-9 and 10-12: format 1), both K-major, N = BN (bits 17-22 hold
  // N/8), M = 128 (bits 24-28 hold M/16) (bit 15 set: A is MN-major); IDESC_F16:
  // the same with fp16 A and B (format 0)
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((A_MN ? 1u : 0u) << 15) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static constexpr uint32_t IDESC_F16 = IDESC & ~((7u << 7) | (7u << 10));
  static_assert(BN == 32 || BN == 64 || BN == 128 || BN == 256, "N of the MMA");
  static_assert(KB == 64 || KB == 32, "stage depth");
  static_assert(!A_MN || KB == 64, "the MN-major operand uses 64-deep stages");
  static_assert(HALF % (16 * KB) == 0 && A_BYTES % (16 * KB) == 0, "swizzle atoms (8 rows) must stay aligned");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, rows of 2 KB bytes (KB = 64: 128-byte
// swizzle, 8-row groups 1024 bytes apart; KB = 32: 64-byte swizzle, 8-row
// groups 512 bytes apart), descriptor version 1.
template <int KB = 64>
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused with swizzling)
  d |= (uint64_t)((16 * KB) >> 4) << 32;   // stride byte offset: 8 rows of 2 KB bytes
  d |= (uint64_t)1 << 46;                  // version
  d |= (uint64_t)(KB == 64 ? 2 : 4) << 61;  // 128-byte or 64-byte swizzle
  return d;
}

// MN-major operand (A_MN): TMA writes each 64-element-wide MN slice of the tile
// as 64 K-rows of 128 bytes (128-byte swizzle); the two slices of a 128-row tile
// sit 8 KB apart (leading byte offset, between MN atoms) and the 8-row K groups
// 1 KB apart (stride byte offset).  One 16-deep K step spans two K groups (2 KB).
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)(8192 >> 4) << 16;  // leading byte offset: next 64-element MN slice
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: next 8-row K group
  d |= (uint64_t)1 << 46;            // version
  d |= (uint64_t)2 << 61;            // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false (and the error code set) when the limit expires.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err, int code,
                                          uint32_t limit = WAIT_LIMIT) {
  for (uint32_t i = 0; i < limit; i++)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, code);
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

}  // namespace tc
}  // namespace tlrmvn
