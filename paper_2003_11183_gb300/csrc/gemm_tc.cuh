// BF16 x BF16 -> FP32 GEMM on the 5th-generation tensor cores (tcgen05, sm_103a)
// for the low-rank limit shifts, the projections and the in-tile coupling of the
// BF16-shift integrand.
//
//   D (M x N) = A (M x K) * B (N x K)^T      bf16 operands: B K-major; A K-major,
//                                             or MN-major (A_MN: stored K x M, M contiguous)
//
// One 128 x BN output tile per CTA of 128 threads (BN = 64, 128 or 256, a
// template parameter).  Operands are staged by TMA (128-byte swizzle) through a
// ring of shared-memory stages; one thread issues tcgen05.mma (M=128, N=BN,
// K=16) into a TMEM accumulator of BN columns; after the last k-block all four
// warps read their 32 TMEM lanes (one output row each) and run the epilogue:
//   EPI_TRANS_F32:    D[col * ldd + row] = acc, or += acc  (fp32; the rows are
//                     samples, so a warp's stores cover 32 consecutive samples)
//   EPI_TRANS_BF16:   W[map[col] * ldw + row] = bf16(acc)   (projections, bf16; the rows
//                     are samples, so a warp's stores cover 32 consecutive samples)
// Every mbarrier wait is bounded; on expiry the CTA records an error code,
// skips the remaining work, frees its TMEM and returns.
#pragma once
#include <cuda.h>
#include "common.cuh"

namespace tlrmvn {
namespace tc {

constexpr int BM = 128;
constexpr uint32_t WAIT_LIMIT = 1u << 24;  // polls before a wait gives up (seconds)

enum { EPI_TRANS_F32 = 0, EPI_TRANS_BF16 = 1 };

// Shape of one kernel configuration: K depth of a stage (KB = 64 with 128-byte
// swizzle, or 32 with 64-byte swizzle), tile bytes, stage bytes (SPLIT stages
// hold hi and lo tiles of both operands), stage count and shared memory.  By
// default stages are sized so that two CTAs share an SM where they fit in about
// 100 KB each, and SPLIT configurations (short-K products: the in-tile coupling,
// K <= 448) take one stage, so that several CTAs share an SM and overlap one
// another; NSTQ > 0 fixes the stage count.
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
  // and B, both K-major, N = BN (bits 17-22 hold N/8), M = 128 (bits 24-28 hold M/16)
  // (bit 15 set: A is MN-major)
  static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((A_MN ? 1u : 0u) << 15) |
                                    ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
  static_assert(BN == 64 || BN == 128 || BN == 256, "N of the MMA");
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

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
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

// 32 consecutive fp32 columns of this warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; i++) v[i] = __uint_as_float(r[i]);
}

struct GemmTcArgs {
  int M, N, K;          // logical sizes; rows >= M and cols >= N are not stored
  int ax0, ay0;         // A tile origin in its tensor map (x = K, y = M)
  int bx0, by0;         // B tile origin (x = K, y = N)
  float* D;             // EPI_TRANS_F32
  int64_t ldd;
  __nv_bfloat16* W;     // EPI_TRANS_BF16
  int64_t ldw;
  const int32_t* map;
  int* err;             // nonzero after a wait expired
  // SPLIT kernels: operands x = hi + lo with the lo halves at x offsets alo (A)
  // and blo (B) of the same tensors; acc = A_hi B_hi + A_hi B_lo + A_lo B_hi
  int alo = 0, blo = 0;
  int accumulate = 0;   // EPI_TRANS_F32: D += acc
  int rows_fast = 0;    // grid: blockIdx.x walks the M blocks (CTAs that share a B tile run together)
};

// A's tensor map has a box of KB x 128 (BM rows; A_MN: 64 M-elements x 64 K-rows,
// loaded twice per stage), B's a box of KB x BN; the maps' swizzle is 128-byte
// for KB = 64 and 64-byte for KB = 32.
// PREF (EPI_TRANS_F32, N = 64): the epilogue's old output values are loaded
// while the MMAs run (64 registers; four CTAs per SM); without it they are loaded
// 32 at a time just before their stores, and six CTAs fit per SM.
template <int EPI, bool SPLIT, int BN, bool A_MN = false, int KB = 64, int NSTQ = 0, bool PREF = true>
__global__ void __launch_bounds__(128, SPLIT ? (PREF ? 4 : 6) : 1) k_gemm_tc(const __grid_constant__ CUtensorMap mapA,
                                                 const __grid_constant__ CUtensorMap mapB, GemmTcArgs p) {
  static_assert(!(A_MN && SPLIT), "MN-major A is used without split operands");
  using G = Cfg<BN, SPLIT, A_MN, KB, NSTQ>;
  constexpr int BK = G::BK, A_BYTES = G::A_BYTES;
  constexpr int NST = G::NST;
  constexpr uint32_t SB = G::SB;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + NST * SB);
  uint64_t* empty = full + NST;
  uint64_t* done = empty + NST;
  uint32_t* tmem_slot = (uint32_t*)(done + 1);
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = (p.rows_fast ? blockIdx.x : blockIdx.y) * BM, n0 = (p.rows_fast ? blockIdx.y : blockIdx.x) * BN;
  const int nk = (p.K + BK - 1) / BK;

  pdl_trigger();
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < NST; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  pdl_wait();  // operands and outputs belong to the preceding kernels until they finish

  if (warp == 0 && lane == 0) {
    // TMA producer
    int issued = 0;
    for (int kb = 0; kb < nk; kb++) {
      const int s = kb % NST;
      if (kb >= NST && !mbar_wait(&empty[s], ((kb / NST) - 1) & 1, p.err, 2)) {
        abort_flag = 1;
        break;
      }
      if (*(volatile int*)&abort_flag) break;
      unsigned char* sa = smem + s * SB;
      mbar_expect_tx(&full[s], SB);
      if (A_MN) {  // x = M, y = K: two 64-wide M slices
        tma_load_2d(sa, &mapA, &full[s], p.ay0 + m0, p.ax0 + kb * BK);
        tma_load_2d(sa + A_BYTES / 2, &mapA, &full[s], p.ay0 + m0 + 64, p.ax0 + kb * BK);
      } else {
        tma_load_2d(sa, &mapA, &full[s], p.ax0 + kb * BK, p.ay0 + m0);
      }
      tma_load_2d(sa + A_BYTES, &mapB, &full[s], p.bx0 + kb * BK, p.by0 + n0);
      if (SPLIT) {
        tma_load_2d(sa + G::HALF, &mapA, &full[s], p.ax0 + p.alo + kb * BK, p.ay0 + m0);
        tma_load_2d(sa + G::HALF + A_BYTES, &mapB, &full[s], p.bx0 + p.blo + kb * BK, p.by0 + n0);
      }
      issued = kb + 1;
    }
    if (*(volatile int*)&abort_flag) {
      // drain: wait (bounded) for the copies still in flight before the CTA exits
      for (int kb = (issued > NST ? issued - NST : 0); kb < issued; kb++)
        mbar_wait(&full[kb % NST], (kb / NST) & 1, p.err, 5);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    bool ok = true;
    for (int kb = 0; kb < nk && ok; kb++) {
      const int s = kb % NST;
      if (!mbar_wait(&full[s], (kb / NST) & 1, p.err, 3)) {
        abort_flag = 1;
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(smem + s * SB);
      const uint64_t da = A_MN ? sdesc_mn(sa) : sdesc<BK>(sa), db = sdesc<BK>(sa + A_BYTES);
      // per 16-deep k-step, in the descriptor's 16-byte units: K-major +32 bytes
      // (+2), MN-major two 1 KB K groups (+128)
      constexpr uint64_t ASTEP = A_MN ? 128 : 2;
#pragma unroll
      for (int kk = 0; kk < BK / 16; kk++) {
        mma_bf16(tmem, da + ASTEP * kk, db + (uint64_t)(kk * 2), G::IDESC, (kb > 0 || kk > 0) ? 1u : 0u);
        if (SPLIT) {
          const uint64_t dal = sdesc<BK>(sa + G::HALF), dbl = sdesc<BK>(sa + G::HALF + A_BYTES);
          mma_bf16(tmem, da + (uint64_t)(kk * 2), dbl + (uint64_t)(kk * 2), G::IDESC, 1u);
          mma_bf16(tmem, dal + (uint64_t)(kk * 2), db + (uint64_t)(kk * 2), G::IDESC, 1u);
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();
  const int row = m0 + 32 * warp + lane;
  // PRE: the output row's old values (accumulate) are loaded while the MMAs run;
  // the epilogue warps have nothing else to do until the accumulator is ready
  constexpr bool PRE = PREF && (EPI == EPI_TRANS_F32) && BN <= 64;
  float pre[PRE ? BN : 1];
  if (PRE) {
    const bool ld = p.accumulate && row < p.M;
    const float* src = p.D + (int64_t)n0 * p.ldd + row;
#pragma unroll
    for (int q = 0; q < (PRE ? BN : 1); q++) pre[q] = (ld && n0 + q < p.N) ? __ldcs(src + (int64_t)q * p.ldd) : 0.0f;
  }
  // epilogue: every warp reads its 32 TMEM lanes (rows m0 + 32*warp + lane)
  const bool ready = mbar_wait(done, 0, p.err, 4);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready && !*(volatile int*)&abort_flag) {
    const uint32_t tbase = tmem + ((uint32_t)(32 * warp) << 16);
    if (EPI == EPI_TRANS_F32) {
#pragma unroll
      for (int c = 0; c < BN / 32; c++) {
        float v[32];
        tmem_ld32(tbase + c * 32, v);
        const int col0 = n0 + c * 32;
        if (row < p.M) {
          float* dst = p.D + (int64_t)col0 * p.ldd + row;
          if (PRE) {
#pragma unroll
            for (int q = 0; q < 32; q++) v[q] += pre[(c * 32 + q) % (PRE ? BN : 1)];
          } else if (p.accumulate) {
            // all 32 old values are loaded before any store, so the loads overlap
            float old[32];
#pragma unroll
            for (int q = 0; q < 32; q++) old[q] = (col0 + q < p.N) ? __ldcs(dst + (int64_t)q * p.ldd) : 0.0f;
#pragma unroll
            for (int q = 0; q < 32; q++) v[q] += old[q];
          }
#pragma unroll
          for (int q = 0; q < 32; q++)
            if (col0 + q < p.N) dst[(int64_t)q * p.ldd] = v[q];
        }
      }
    } else {
#pragma unroll
      for (int c = 0; c < BN / 32; c++) {
        float v[32];
        tmem_ld32(tbase + c * 32, v);
        const int col0 = n0 + c * 32;
        if (row < p.M) {
#pragma unroll
          for (int q = 0; q < 32; q++)
            if (col0 + q < p.N) p.W[(int64_t)p.map[col0 + q] * p.ldw + row] = __float2bfloat16_rn(v[q]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

// The bounded-wait path on its own: one thread waits on an mbarrier that nothing
// arrives at, `polls` times, and records code 6 when it gives up.
__global__ void k_wait_selftest(int* err, uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_wait(&bar, 0, err, 6, polls);
}

}  // namespace tc
}  // namespace tlrmvn
