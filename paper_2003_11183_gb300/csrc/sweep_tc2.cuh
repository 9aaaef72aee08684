// The whole-tile sweep of the BF16/FP16-shift paths with its products overlapped
// (Algorithm 6's per-tile step with eq. 2 over the tile, as k_sweep_tc), in
// sub-tiles of 32 variables whose products are double-buffered in TMEM.
//
// One CTA of 128 threads owns 128 samples (one per thread and TMEM lane) and 64
// TMEM columns: two buffers of 32.  Sub-tile q (variables q0 = 32q ..) takes its
// sums from buffer q & 1:
//     T[c][v] = sum_k U_i[q0 + v][k] W[k][c]            (the low-rank shifts)
//             + sum_{u < q0} B_i[q0 + v][u] y_u[c]      (the coupling to the earlier
//               sub-tiles, split hi/lo operands, hi*hi + hi*lo + lo*hi)
// While the four warps sweep sub-tile q from its buffer, thread 0 - between its
// own variables, by non-blocking mbarrier tests (test_wait) - streams the products of
// sub-tile q + 1 that do not depend on sub-tile q into the other buffer: its
// low-rank shifts and its coupling to sub-tiles 0 .. q-1, one k-block at a time
// through one shared-memory stage (TMA copy, then the MMAs).  Only the coupling
// to sub-tile q itself (one 32-deep k-block) waits for the end of q's sweep.
// The sweep of a sub-tile is k_sweep_tc's: the 16-variable blocks read their
// sums from the thread's lane, each y goes into the lane's column whose sum has
// been read, and the block's y are stored sample-major (hi, lo) for the later
// products.  After the last sub-tile the tile's projections run through all 64
// columns in passes of 64 ranks, as in k_sweep_tc.
//
// Shared memory: one 24 KB stage (coupling k-block: y rows hi/lo 128 x 32 and B
// rows hi/lo 32 x 32, 64-byte swizzle; shift k-block: two MN-major boxes of W and
// 32 U rows, 128-byte swizzle; projection k-block: y rows 128 x 64 and 64 V rows),
// the sub-tile's transposed triangle (32 x 32) and band copy (32 x 16) - not in
// the stage, which is busy during the sweep - and the per-variable constants:
// ~31 KB, so six CTAs still share an SM.  Every wait is bounded; on expiry the
// CTA records an error code, skips the rest, waits (bounded) for its copies and
// products in flight, frees its TMEM and returns.
#pragma once
#include "sweep_tc.cuh"

namespace tlrmvn {

constexpr int ST2_SUB = 32;  // variables per sub-tile (= TMEM columns per buffer)
constexpr uint32_t ST2_STAGE = 24576;
// coupling k-block: [y hi 8 KB][B hi 2 KB][y lo 8 KB][B lo 2 KB]
constexpr uint32_t ST2_CA = 128 * 32 * 2, ST2_CB = 32 * 32 * 2, ST2_CHALF = ST2_CA + ST2_CB;  // 10 KB
constexpr uint32_t ST2_CBYTES = 2 * ST2_CHALF;                                                   // 20 KB
// shift k-block: [W box 8 KB][W box 8 KB][U rows 4 KB]
constexpr uint32_t ST2_SA = 128 * 64 * 2, ST2_SBYTES = ST2_SA + 32 * 64 * 2;                     // 20 KB
// projection k-block: [y hi 16 KB][V rows 8 KB]
constexpr uint32_t ST2_PA = 128 * 64 * 2, ST2_PBYTES = ST2_PA + 64 * 64 * 2;                     // 24 KB
static_assert(ST2_CBYTES <= ST2_STAGE && ST2_SBYTES <= ST2_STAGE && ST2_PBYTES <= ST2_STAGE, "stage size");
static_assert(ST2_CA % 1024 == 0 && ST2_CHALF % 1024 == 0 && ST2_SA % 1024 == 0 && ST2_PA % 1024 == 0,
              "swizzled operands start on 1 KB boundaries");

// instruction descriptors (kind::f16, fp32 accumulator, M = 128): coupling N = 32
// (K-major A, B); shift N = 32 (MN-major A); projection N = 64 (K-major); bf16
// operands (bits 7-12 format 1), or fp16 (format 0)
template <bool F16>
struct St2Desc {
  static constexpr uint32_t base(int n, bool a_mn) {
    return (1u << 4) | (F16 ? 0u : ((1u << 7) | (1u << 10))) | ((a_mn ? 1u : 0u) << 15) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  }
  static constexpr uint32_t COUPLE = base(32, false), SHIFT = base(32, true), PROJ = base(64, false);
};

__host__ __device__ constexpr size_t sweep_tc2_smem_bytes() {
  return 1024 /*align*/ + ST2_STAGE + ST2_SUB * ST2_SUB * 4 + ST2_SUB * 16 * 4 +
         ST2_SUB * (sizeof(float4) + sizeof(uint64_t)) + 64;
}

// Thread 0's product pipeline for the next sub-tile: jobs 0 .. n_pre - 1 are the
// shift k-blocks (nks of them) and then the coupling k-blocks to sub-tiles
// 0 .. n_pre - nks - 1; `post` is one more coupling k-block (to the sub-tile just
// swept).  st: 0 stage free, 1 copies in flight, 2 products in flight.
struct St2Pipe {
  int job, n_pre, nks, q0n, buf, st;
  uint32_t ph;  // bit 0: full parity, bit 1: freeb parity
};

template <int FLAGS, bool F16>
__global__ void __launch_bounds__(STC_NS, 6)
    k_sweep_tc2(const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapB,
                const __grid_constant__ CUtensorMap mapW, const __grid_constant__ CUtensorMap mapU,
                const __grid_constant__ CUtensorMap mapY64, const __grid_constant__ CUtensorMap mapV, SweepTcArgs p) {
  constexpr bool PER = FLAGS & SWEEP_PERIODIZE, ONE = FLAGS & SWEEP_ONE_SIDED;
  using Op = Op16<F16>;
  using Dsc = St2Desc<F16>;
  extern __shared__ __align__(1024) unsigned char st2_smem[];
  unsigned char* smem = st2_smem + ((1024u - (tc::smem_u32(st2_smem) & 1023u)) & 1023u);
  unsigned char* stage = smem;
  float* s_bt = reinterpret_cast<float*>(smem + ST2_STAGE);     // s_bt[u * 32 + v] = B_i[q0 + v][q0 + u]
  float* s_band = s_bt + ST2_SUB * ST2_SUB;                      // s_band[v * 16 + k] = B_i[q0 + v + 1 + k][q0 + v]
  float4* s_abi = reinterpret_cast<float4*>(s_band + ST2_SUB * 16);
  uint64_t* s_q = reinterpret_cast<uint64_t*>(s_abi + ST2_SUB);
  uint64_t* full = s_q + ST2_SUB;  // the stage's copies landed
  uint64_t* freeb = full + 1;      // the products reading the stage are done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(freeb + 1);
  __shared__ int abort_flag;
  __shared__ St2Pipe P;  // thread 0's product pipeline (shared memory: no registers in the other threads)

  const DiagArgs32& d = p.d;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = d.mt;
  const int c0 = blockIdx.x * STC_NS;

  if (tid == 0) {
    abort_flag = 0;
    tc::mbar_init(full, 1);
    tc::mbar_init(freeb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                 "r"(2 * ST2_SUB)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *tmem_slot;
  const uint32_t tl = tbase + ((uint32_t)(32 * warp) << 16);  // this warp's 32 lanes
  pdl_trigger();
  pdl_wait();

  const bool act = c0 + tid < d.C;
  const int cs = act ? c0 + tid : (int)d.C - 1;
  const uint64_t* Ds;
  uint32_t ks;
  {
    const int64_t g = d.sample0 + cs, sh = g / d.N;
    ks = (uint32_t)(g - sh * d.N) + 1u;
    Ds = d.D + sh * d.ldD + d.coord0;
  }
  const float rs = d.rs ? d.rs[cs] : 1.0f;
  float prod = 1.0f, lsum = 0.0f;
  int pe = 0;

  const int nks = (p.kr + 63) / 64;
  const uint32_t sa = tc::smem_u32(stage);
  // thread 0: issue the copies of job j of the pipe into the stage
  auto issue_copy = [&](const St2Pipe& P, int j) {
    if (j < P.nks) {
      const int y = p.krow0 + j * 64;
      tc::mbar_expect_tx(full, ST2_SBYTES);
      tc::tma_load_2d(stage, &mapW, full, c0, y);
      tc::tma_load_2d(stage + ST2_SA / 2, &mapW, full, c0 + 64, y);
      tc::tma_load_2d(stage + ST2_SA, &mapU, full, j * 64, p.urow0 + P.q0n);
    } else {
      const int x = (j - P.nks) * ST2_SUB;  // the earlier sub-tile's first variable
      tc::mbar_expect_tx(full, ST2_CBYTES);
      tc::tma_load_2d(stage, &mapY, full, x, c0);
      tc::tma_load_2d(stage + ST2_CA, &mapB, full, x, p.brow0 + P.q0n);
      tc::tma_load_2d(stage + ST2_CHALF, &mapY, full, p.alo + x, c0);
      tc::tma_load_2d(stage + ST2_CHALF + ST2_CA, &mapB, full, p.blo + x, p.brow0 + P.q0n);
    }
  };
  // thread 0: the MMAs of job j (the stage holds its operands) into the pipe's buffer
  auto issue_mma = [&](const St2Pipe& P, int j) {
    const uint32_t dst = tbase + (uint32_t)(P.buf * ST2_SUB);
    if (j < P.nks) {
      const uint64_t dw = tc::sdesc_mn(sa), du = tc::sdesc<64>(sa + ST2_SA);
#pragma unroll
      for (int kk = 0; kk < 4; kk++)
        tc::mma_f16(dst, dw + (uint64_t)(128 * kk), du + (uint64_t)(2 * kk), Dsc::SHIFT, (j > 0 || kk > 0) ? 1u : 0u);
    } else {
      const uint64_t dah = tc::sdesc<32>(sa), dbh = tc::sdesc<32>(sa + ST2_CA);
      const uint64_t dal = tc::sdesc<32>(sa + ST2_CHALF), dbl = tc::sdesc<32>(sa + ST2_CHALF + ST2_CA);
#pragma unroll
      for (int kk = 0; kk < 2; kk++) {
        const uint64_t o = (uint64_t)(kk * 2);
        tc::mma_f16(dst, dah + o, dbh + o, Dsc::COUPLE, (j > 0 || kk > 0) ? 1u : 0u);
        tc::mma_f16(dst, dah + o, dbl + o, Dsc::COUPLE, 1u);
        tc::mma_f16(dst, dal + o, dbh + o, Dsc::COUPLE, 1u);
      }
    }
    tc::mma_commit(freeb);
  };
  // thread 0: advance the pipe without blocking (one step per call)
  auto poll = [&](St2Pipe& P) {
    if (P.st == 1) {
      if (tc::mbar_test_wait(full, P.ph & 1)) {
        P.ph ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue_mma(P, P.job);
        P.st = 2;
      }
    } else if (P.st == 2) {
      if (tc::mbar_test_wait(freeb, (P.ph >> 1) & 1)) {
        P.ph ^= 2;
        P.st = 0;
        P.job++;
      }
    }
    if (P.st == 0 && P.job < P.n_pre) {
      issue_copy(P, P.job);
      P.st = 1;
    }
  };
  // thread 0: run the pipe to completion (bounded waits); false on expiry (abort set,
  // the copies or products in flight waited for)
  auto drain = [&](St2Pipe& P) -> bool {
    for (;;) {
      if (P.st == 1) {
        if (!tc::mbar_wait(full, P.ph & 1, p.err, 8)) {
          tc::mbar_wait(full, P.ph & 1, p.err, 5);  // (the copies in flight, bounded)
          abort_flag = 1;
          return false;
        }
        P.ph ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue_mma(P, P.job);
        P.st = 2;
      }
      if (P.st == 2) {
        if (!tc::mbar_wait(freeb, (P.ph >> 1) & 1, p.err, 9)) {
          tc::mbar_wait(freeb, (P.ph >> 1) & 1, p.err, 5);  // (the products in flight, bounded)
          abort_flag = 1;
          return false;
        }
        P.ph ^= 2;
        P.st = 0;
        P.job++;
      }
      if (P.job >= P.n_pre) return true;
      issue_copy(P, P.job);
      P.st = 1;
    }
  };

  const int nsub = (mt + ST2_SUB - 1) / ST2_SUB;
  // sub-tile 0's products: its low-rank shifts (no earlier sub-tile)
  if (tid == 0) {
    P = St2Pipe{0, nks, nks, 0, 0, 0, 0u};
    if (P.n_pre > 0) drain(P);
  }
  for (int q = 0; q < nsub; q++) {
    const int q0 = q * ST2_SUB, mq = min(ST2_SUB, mt - q0), buf = q & 1;
    const bool has_sum = q > 0 || p.kr > 0;
    // constants and the sub-tile's triangle and band (every thread is past the previous sub-tile's reads)
    for (int t = tid; t < mq; t += STC_NS) {
      s_abi[t] = make_float4(d.a[q0 + t], d.b[q0 + t], d.inv[q0 + t], 0.0f);
      s_q[t] = d.Q[d.coord0 + q0 + t];
    }
    {
      const int w4 = ((mq + 15) & ~15) >> 2;
      for (int t = tid; t < mq * w4; t += STC_NS) {
        const int u = t / w4, c = t - u * w4;
        reinterpret_cast<float4*>(s_bt + u * ST2_SUB)[c] =
            __ldg(reinterpret_cast<const float4*>(d.BT + (int64_t)(q0 + u) * d.ldbt + q0) + c);
      }
      for (int t = tid; t < mq * 4; t += STC_NS)
        reinterpret_cast<float4*>(s_band)[t] = __ldg(reinterpret_cast<const float4*>(d.band + (int64_t)q0 * 16) + t);
    }
    if (tid == 0 && !*(volatile int*)&abort_flag) {
      // sub-tile q's products are complete (the pipe drained); start sub-tile q + 1's
      // independent products into the other buffer: shifts, coupling to sub-tiles < q
      P.job = 0;
      P.nks = nks;
      P.n_pre = (q + 1 < nsub) ? nks + q : 0;
      P.q0n = q0 + ST2_SUB;
      P.buf = buf ^ 1;
      P.st = 0;
      if (P.n_pre > 0) poll(P);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // sums of sub-tile q in TMEM, constants and triangle staged
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (*(volatile int*)&abort_flag) break;
    const uint32_t tq = tl + (uint32_t)(buf * ST2_SUB);

    for (int v0 = 0; v0 < mq; v0 += DIAG_VB) {
      const int nb = min(DIAG_VB, mq - v0);
      float acc[DIAG_VB], dl[DIAG_VB];
      if (has_sum) {
        uint32_t r[DIAG_VB];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tq + (uint32_t)v0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < DIAG_VB; j++) dl[j] = F16 ? __uint_as_float(r[j]) * p.tscale : __uint_as_float(r[j]);
      } else {
#pragma unroll
        for (int j = 0; j < DIAG_VB; j++) dl[j] = 0.0f;
      }
#pragma unroll
      for (int j = 0; j < DIAG_VB; j++) acc[j] = 0.0f;
      uint64_t dnext = Ds[q0 + v0];
      for (int u0 = 0; u0 < v0; u0 += 4) {
        uint32_t r[4];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                     : "r"(tq + (uint32_t)u0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int uu = 0; uu < 4; uu++) {
          const float yu = __uint_as_float(r[uu]);
          const float4* b4 = reinterpret_cast<const float4*>(s_bt + (u0 + uu) * ST2_SUB + v0);
          const float4 qb[4] = {b4[0], b4[1], b4[2], b4[3]};
#pragma unroll
          for (int h = 0; h < 4; h++) {
            acc[4 * h] = fmaf(qb[h].x, yu, acc[4 * h]);
            acc[4 * h + 1] = fmaf(qb[h].y, yu, acc[4 * h + 1]);
            acc[4 * h + 2] = fmaf(qb[h].z, yu, acc[4 * h + 2]);
            acc[4 * h + 3] = fmaf(qb[h].w, yu, acc[4 * h + 3]);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < DIAG_VB; j++) acc[j] += dl[j];
#pragma unroll 1
      for (int j = 0; j < nb; j++) {
        const int v = v0 + j;
        // thread 0 moves the next sub-tile's products on (never blocks; twice per variable)
        if (tid == 0 && P.job < P.n_pre) poll(P);
        const float4 abi = s_abi[v];
        const uint64_t qv = s_q[v];
        const uint64_t dv = dnext;
        dnext = Ds[q0 + ((j + 1 < nb) ? v + 1 : v)];
        const float sum = acc[0];
        const float bt = (abi.y * rs - sum) * abi.z;
        float w, wc, f, la, y;
        lattice_wf((uint64_t)ks * qv + dv, PER ? 1 : 0, w, wc);
        if (ONE) {
          sov_step_f32_upper(bt, w, wc, f, la, y);
        } else {
          const float at = (abi.x * rs - sum) * abi.z;
          sov_step_f32_prod(at, bt, w, wc, f, la, y);
        }
        lsum += la;
        prod *= f;
        const int pb = __float_as_int(prod);
        pe += (pb >> 23) - 127;
        prod = __int_as_float((pb & 0x007FFFFF) | 0x3F800000);
        // thread 0 moves the next sub-tile's products on (never blocks)
        if (tid == 0 && P.job < P.n_pre) poll(P);
        __syncwarp();
        asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(tq + (uint32_t)v), "r"(__float_as_uint(y))
                     : "memory");
        const float4* b4 = reinterpret_cast<const float4*>(s_band + v * 16);
        const float4 qb[4] = {b4[0], b4[1], b4[2], b4[3]};
        const float bcur[DIAG_VB] = {qb[0].x, qb[0].y, qb[0].z, qb[0].w, qb[1].x, qb[1].y, qb[1].z, qb[1].w,
                                     qb[2].x, qb[2].y, qb[2].z, qb[2].w, qb[3].x, qb[3].y, qb[3].z, qb[3].w};
#pragma unroll
        for (int i = 0; i < DIAG_VB - 1; i++) acc[i] = fmaf(bcur[i], y, acc[i + 1]);
        acc[DIAG_VB - 1] = 0.0f;
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      {
        uint32_t r[DIAG_VB];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tq + (uint32_t)v0));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (act) {
          unsigned short* row = reinterpret_cast<unsigned short*>(d.Ys) + (int64_t)cs * d.ldys + q0 + v0;
          uint32_t hi2[DIAG_VB / 2], lo2[DIAG_VB / 2];
#pragma unroll
          for (int j = 0; j < DIAG_VB; j += 2) {
            const float y0 = __uint_as_float(r[j]), y1 = __uint_as_float(r[j + 1]);
            float h0, h1, l0, l1;
            hi2[j / 2] = Op::pack(y0, y1, h0, h1);
            lo2[j / 2] = Op::pack(y0 - h0, y1 - h1, l0, l1);
          }
          if (nb == DIAG_VB) {
            uint4* dh = reinterpret_cast<uint4*>(row);
            uint4* dlo = reinterpret_cast<uint4*>(row + d.ys_lo);
            dh[0] = make_uint4(hi2[0], hi2[1], hi2[2], hi2[3]);
            dh[1] = make_uint4(hi2[4], hi2[5], hi2[6], hi2[7]);
            dlo[0] = make_uint4(lo2[0], lo2[1], lo2[2], lo2[3]);
            dlo[1] = make_uint4(lo2[4], lo2[5], lo2[6], lo2[7]);
          } else {
#pragma unroll
            for (int j = 0; j < DIAG_VB; j++)
              if (j < nb) {
                row[j] = (unsigned short)(hi2[j / 2] >> (16 * (j & 1)));
                row[d.ys_lo + j] = (unsigned short)(lo2[j / 2] >> (16 * (j & 1)));
              }
          }
        }
      }
    }
    // sub-tile q's y stored and visible to the copies; its TMEM columns read
    asm volatile("fence.proxy.async;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && q + 1 < nsub && !*(volatile int*)&abort_flag) {
      // finish sub-tile q + 1's independent products, then its coupling to sub-tile q
      if (drain(P)) {
        P.n_pre = P.job + 1;  // one more job: the coupling k-block to sub-tile q (x = q0)
        if (drain(P)) {
        }
      }
    }
  }
  // the tile's projections for the later tiles, 64 ranks a pass through all 64
  // columns: W[vmap[r]][c] = sum_v V[kcol0 + r][v] y_v[c] (y hi parts)
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  uint32_t ph = P.ph;
  for (int r0 = 0; r0 < p.kc && !*(volatile int*)&abort_flag; r0 += 64) {
    if (tid == 0) {
      const uint64_t da = tc::sdesc<64>(sa), db = tc::sdesc<64>(sa + ST2_PA);
      int bad = 0;
      for (int kb = 0; kb < (mt + 63) / 64; kb++) {
        tc::mbar_expect_tx(full, ST2_PBYTES);
        tc::tma_load_2d(stage, &mapY64, full, kb * 64, c0);
        tc::tma_load_2d(stage + ST2_PA, &mapV, full, kb * 64, p.kcol0 + r0);
        if (!tc::mbar_wait(full, ph & 1, p.err, 8)) {
          bad = 1;
          break;
        }
        ph ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int kk = 0; kk < 4; kk++)
          tc::mma_f16(tbase, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), Dsc::PROJ, (kb > 0 || kk > 0) ? 1u : 0u);
        tc::mma_commit(freeb);
        if (!tc::mbar_wait(freeb, (ph >> 1) & 1, p.err, 9)) {
          bad = 2;
          break;
        }
        ph ^= 2;
      }
      if (bad) {
        if (bad == 1) tc::mbar_wait(full, ph & 1, p.err, 5);
        else tc::mbar_wait(freeb, (ph >> 1) & 1, p.err, 5);
        abort_flag = 1;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (*(volatile int*)&abort_flag) break;
#pragma unroll 1
    for (int h = 0; h < 64; h += 16) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tl + (uint32_t)h));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (act) {
#pragma unroll
        for (int j = 0; j < 16; j++)
          if (r0 + h + j < p.kc)
            p.W[(int64_t)p.vmap[r0 + h + j] * p.ldw + cs] =
                Op::one(F16 ? __uint_as_float(r[j]) * p.wscale[r0 + h + j] : __uint_as_float(r[j]));
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  if (!*(volatile int*)&abort_flag && act) {
    const double lp = (double)(logf(prod) + lsum) + (double)pe * 0.69314718055994530942;
    const int64_t g = d.sample0 + cs;
    if (d.first) d.logP[g] = lp;
    else d.logP[g] += lp;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(2 * ST2_SUB) : "memory");
  }
}

}  // namespace tlrmvn
