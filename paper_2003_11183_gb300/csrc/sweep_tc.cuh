// The BF16-path integrand of a whole diagonal tile i in one kernel (Algorithm 6's
// per-tile step with eq. 2 over the tile): the tile's low-rank limit shifts, the
// sweep with its in-tile coupling, and the tile's projections for the later
// tiles, the products on the tensor cores.
//
// One CTA of 128 threads owns 128 samples, one per thread and per TMEM lane, and
// 64 TMEM columns.  The tile runs in sub-tiles of 64 variables.  Before sub-tile
// q, one thread accumulates into the columns, by tcgen05 products,
//     T[c][v] = sum_k U_i[q0 + v][k] W[k][c]           (the low-rank shifts: W the
//               rank-major projections of the earlier tiles, read MN-major; U
//               the tile's rows of the row factors; bf16, fp32 accumulation)
//             + sum_{u < q0} B_i[q0 + v][u] y_u[c]     (the coupling to the tile's
//               earlier sub-tiles: the CTA's own rows of the sample-major y, hi
//               and lo bf16 parts, times the split copy of B_i, hi*hi + hi*lo +
//               lo*hi)
// for v < 64, the same sums as eq. 2 regrouped.  Each thread then runs the
// sub-tile's chain for its sample as the sub-tile sweep k_diag_f32 does, with
// three differences of place: the sums of each 16-variable block come from the
// thread's TMEM lane (tcgen05.ld); the y of the sub-tile go to the same lane,
// into the columns whose sums have been read (tcgen05.st), instead of shared
// memory; and the sub-tile's transposed triangle and band copy are staged in
// shared memory, in the space the MMA operands use before the sweep.  After
// each 16-variable block its y are stored, sample-major bf16 hi and lo, for the
// later products.  After the last sub-tile the CTA computes the tile's
// projections W[k][c] = sum_v V_i[k][v] y_v[c] in passes of 64 ranks through
// the same columns and writes them as rows of W.  So neither the shifts nor the
// coupling go through global memory, the per-variable loads of B are
// shared-memory broadcasts, and the sample's log P is closed once per tile.
//
// The MMA operands are staged by TMA into one stage of 24 KB (shift and
// projection k-blocks 64 deep, 128-byte swizzle; coupling k-blocks 32 deep,
// 64-byte swizzle), so a CTA needs ~27 KB of shared memory and 64 TMEM columns;
// six share an SM.  (A ring of two 16-deep coupling stages measured slower:
// twice the copies for the same bytes in flight.)  Every wait is bounded; on
// expiry the CTA records an error code, skips the rest, waits (bounded) for its
// copies and products in flight, frees its TMEM and returns.
#pragma once
#include "tcgen05.cuh"
#include "sweep.cuh"

namespace tlrmvn {

constexpr int STC_SUB = 64;   // variables per sub-tile
constexpr int STC_NS = 128;   // samples per CTA (TMEM lanes)
constexpr int STC_KB = 32;    // K depth of a coupling k-block
using StcCfg = tc::Cfg<64, true, false, STC_KB, 1>;

// The 16-bit operand type of the products: bf16 (BF16-shift path) or fp16
// (FP16-shift path), as raw 16-bit words.  pack rounds two floats to the type
// (round to nearest even) and returns them packed low word first, with their
// rounded values in ra, rb.
template <bool F16>
struct Op16;
template <>
struct Op16<false> {
  static __device__ __forceinline__ uint32_t pack(float a, float b, float& ra, float& rb) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    ra = __low2float(h);
    rb = __high2float(h);
    return ((uint32_t)__bfloat16_as_ushort(h.y) << 16) | __bfloat16_as_ushort(h.x);
  }
  static __device__ __forceinline__ unsigned short one(float a) { return __bfloat16_as_ushort(__float2bfloat16_rn(a)); }
};
template <>
struct Op16<true> {
  static __device__ __forceinline__ uint32_t pack(float a, float b, float& ra, float& rb) {
    const __half2 h = __floats2half2_rn(a, b);
    ra = __low2float(h);
    rb = __high2float(h);
    return ((uint32_t)__half_as_ushort(h.y) << 16) | __half_as_ushort(h.x);
  }
  static __device__ __forceinline__ unsigned short one(float a) { return __half_as_ushort(__float2half_rn(a)); }
};

struct SweepTcArgs {
  DiagArgs32 d;  // pointers at the tile's first variable; d.mt = tile size; d.Ys and d.ys_lo required
                 // (d.Delta unused: the low-rank shifts are products of this kernel)
  int brow0;     // row of the tile's first variable in the split-B map
  int alo, blo;  // x offsets of the lo halves in the y and split-B maps
  int urow0;     // row of the tile's first variable in the U map
  int krow0, kr; // the tile's rank rows in the W map (first, count; 0: no low-rank shift)
  int kcol0, kc; // the tile's column ranks: first row in the V map, count (0: no projection)
  unsigned short* W;      // projections (16-bit words of the operand type), rank-major: W[vmap[r] * ldw + sample]
  int64_t ldw;
  const int32_t* vmap;    // at the tile's first column rank
  const float* wscale;    // FP16 path: per column rank, the factor applied to a projection before it is
                          // stored (the inverse of the per-tile scales of U and V); null on the BF16 path
  float tscale;           // FP16 path: 1 / g, undoing the products' global scale g where the sweep reads them
  int* err;
};
using StcProjCfg = tc::Cfg<64, false, false, 64, 1>;  // projection k-block: y rows x V rows, 64 deep
static_assert(StcProjCfg::SB == StcCfg::SB, "a projection k-block fills the same stage");
using StcShiftCfg = tc::Cfg<64, false, true, 64, 1>;  // shift k-block: W (MN-major) x U rows, 64 deep
static_assert(StcShiftCfg::SB == StcCfg::SB, "a shift k-block fills the same stage");

// Stage layout for SPT samples per thread (a CTA owns 128 x SPT samples: thread t
// the samples t, 128 + t, ...; slot s's sums in TMEM columns [64 s, 64 s + 64) of the
// thread's lane).  Each k-block loads SPT A operands (one per slot, samples as rows)
// and one B operand shared by the slots:
//   coupling (32 deep, split):  [A hi x SPT][B hi] [A lo x SPT][B lo]
//   shift (64 deep, A MN-major): [A x SPT][U rows]
//   projection (64 deep):       [A x SPT][V rows]
// During the sweep the stage holds the transposed triangle (64 x 64) and the band copy (64 x 16).
template <int SPT>
struct StcLayout {
  static constexpr uint32_t CA = StcCfg::A_BYTES, CB = StcCfg::B_BYTES;
  static constexpr uint32_t CHALF = SPT * CA + CB;
  static constexpr uint32_t SA = StcShiftCfg::A_BYTES, PA = StcProjCfg::A_BYTES;
  static constexpr uint32_t SB = 2 * CHALF;
  static constexpr uint32_t TMEM_COLS = STC_SUB * SPT;
  static_assert(SPT == 1 || SPT == 2, "samples per thread");
  static_assert(SPT * SA + StcShiftCfg::B_BYTES == SB && SPT * PA + StcProjCfg::B_BYTES == SB,
                "every k-block fills the same stage");
  static_assert(CHALF % 1024 == 0, "operand bases stay on swizzle atoms");
};
constexpr int STC_BT_FLOATS = STC_SUB * STC_SUB, STC_BAND_FLOATS = STC_SUB * 16;
static_assert((STC_BT_FLOATS + STC_BAND_FLOATS) * 4 <= StcCfg::SB, "the sweep's B copies fit in the stage");
// [stage][constants (a, b, 1/B_vv), lattice generators][barriers, TMEM slot]
template <int SPT = 1>
__host__ __device__ constexpr size_t sweep_tc_smem_bytes() {
  return 1024 /*align*/ + (size_t)StcLayout<SPT>::SB + STC_SUB * (sizeof(float4) + sizeof(uint64_t)) + 64;
}

// Shared-memory layout and per-CTA state of the whole-tile sweep (set up once per
// kernel: a persistent kernel runs many tiles through the same stage, barriers
// and TMEM columns).
struct StcCta {
  unsigned char* stage;
  float4* s_abi;
  uint64_t* s_q;
  uint64_t* full;        // the stage's copies landed
  uint64_t* freeb;       // the products reading the stage are done
  uint32_t tmem;         // first of the CTA's TMEM columns
  uint32_t* phases;      // thread 0's barrier parities (bit 0: full, bit 1: freeb)
  int* abort_flag;
};

// Where the CTA's samples sit in the operand maps and the result buffers (slot s of
// the thread: the sample 128 s + thread of the CTA).
struct StcPlace {
  int wx;                   // x coordinate of the CTA's first sample in the W map (samples are columns)
  int wy;                   // row added to the tile's rank rows in the W map
  int yrow;                 // row coordinate of the CTA's first sample in the y maps (samples are rows)
  unsigned short* ysrow[2]; // each slot's row of sample-major y (hi; lo at + d.ys_lo)
  unsigned short* wcol[2];  // each slot's column of W (row k at wcol[k * p.ldw])
};

// One diagonal tile for the CTA's samples: the low-rank shifts and in-tile
// coupling on tcgen05, the float sweep of eq. 2, the projections.  act[s]: slot
// s's sample exists (else it shadows one and writes nothing); Ds[s], ks[s]: its
// lattice shift row and point index; rs[s]: its MVT scale (1 for MVN).  The
// tile's log P is added to (prod[s], pe[s], lsum[s]).  Returns false when a
// bounded wait expired.
template <int FLAGS, bool F16, int SPT>
__device__ __forceinline__ bool stc_tile(const CUtensorMap* mapY, const CUtensorMap* mapB, const CUtensorMap* mapW,
                                         const CUtensorMap* mapU, const CUtensorMap* mapY64, const CUtensorMap* mapV,
                                         const SweepTcArgs& p, const StcCta& k, const StcPlace& pl,
                                         const bool (&act)[SPT], const uint64_t* const (&Ds)[SPT],
                                         const uint32_t (&ks)[SPT], const float (&rs)[SPT], float (&prod)[SPT],
                                         float (&lsum)[SPT], int (&pe)[SPT]) {
  constexpr bool PER = FLAGS & SWEEP_PERIODIZE, ONE = FLAGS & SWEEP_ONE_SIDED;
  using Op = Op16<F16>;
  using Lay = StcLayout<SPT>;
  constexpr uint32_t ID_C = F16 ? StcCfg::IDESC_F16 : StcCfg::IDESC;
  constexpr uint32_t ID_S = F16 ? StcShiftCfg::IDESC_F16 : StcShiftCfg::IDESC;
  constexpr uint32_t ID_P = F16 ? StcProjCfg::IDESC_F16 : StcProjCfg::IDESC;
  constexpr uint32_t CA = Lay::CA, CHALF = Lay::CHALF, SA = Lay::SA, PA = Lay::PA, SB = Lay::SB;
  unsigned char* stage = k.stage;
  float* s_bt = reinterpret_cast<float*>(stage);  // sweep: s_bt[u * 64 + v] = B_i[q0 + v][q0 + u]
  float* s_band = s_bt + STC_BT_FLOATS;           // sweep: s_band[v * 16 + k] = B_i[q0 + v + 1 + k][q0 + v]
  float4* s_abi = k.s_abi;
  uint64_t* s_q = k.s_q;
  uint64_t* full = k.full;
  uint64_t* freeb = k.freeb;
  volatile int* abort_flag = k.abort_flag;
  const DiagArgs32& d = p.d;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int mt = d.mt;
  const uint32_t tmem = k.tmem;
  const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);  // this warp's 32 lanes (slot s: columns + 64 s)

  for (int q0 = 0; q0 < mt; q0 += STC_SUB) {
    const int mq = min(STC_SUB, mt - q0);
    // every thread is past the previous sub-tile's reads of the shared copies and its TMEM accesses;
    // threads 1..64 stage the constants while thread 0 issues the copies and products at once
    for (int t = tid - 1; t >= 0 && t < mq; t += STC_NS - 1) {
      s_abi[t] = make_float4(d.a[q0 + t], d.b[q0 + t], d.inv[q0 + t], 0.0f);
      s_q[t] = d.Q[d.coord0 + q0 + t];
    }
    if ((q0 > 0 || p.kr > 0) && tid == 0) {
      // T = W[ranks of row tile i, samples]^T U_i[q0 + v, ranks]^T     (the low-rank shifts,
      //     64-deep stages: two 64-sample MN-major boxes of W per slot, one box of U rows)
      //   + y[:, <q0] B_i[q0 + v, <q0]^T                              (the coupling, 32-deep split stages)
      const uint32_t sa = tc::smem_u32(stage);
      const uint64_t dbh = tc::sdesc<STC_KB>(sa + SPT * CA), dbl = tc::sdesc<STC_KB>(sa + CHALF + SPT * CA);
      const uint64_t du = tc::sdesc<64>(sa + SPT * SA);
      const int nks = (p.kr + 63) / 64, nk = nks + q0 / STC_KB;
      uint32_t ph = *k.phases;
      int bad = 0;  // 1: copies left in flight, 2: products left in flight
      for (int kb = 0; kb < nk; kb++) {
        tc::mbar_expect_tx(full, SB);
        if (kb < nks) {
          const int y = pl.wy + p.krow0 + kb * 64;
#pragma unroll
          for (int s = 0; s < SPT; s++) {
            tc::tma_load_2d(stage + s * SA, mapW, full, pl.wx + 128 * s, y);
            tc::tma_load_2d(stage + s * SA + SA / 2, mapW, full, pl.wx + 128 * s + 64, y);
          }
          tc::tma_load_2d(stage + SPT * SA, mapU, full, kb * 64, p.urow0 + q0);
        } else {
          const int x = (kb - nks) * STC_KB;
#pragma unroll
          for (int s = 0; s < SPT; s++) {
            tc::tma_load_2d(stage + s * CA, mapY, full, x, pl.yrow + 128 * s);
            tc::tma_load_2d(stage + CHALF + s * CA, mapY, full, p.alo + x, pl.yrow + 128 * s);
          }
          tc::tma_load_2d(stage + SPT * CA, mapB, full, x, p.brow0 + q0);
          tc::tma_load_2d(stage + CHALF + SPT * CA, mapB, full, p.blo + x, p.brow0 + q0);
        }
        if (!tc::mbar_wait(full, ph & 1, p.err, 8)) {
          bad = 1;
          break;
        }
        ph ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (kb < nks) {
          // per 16-deep step: MN-major W two 1 KB K groups on (+128), U rows 32 bytes on (+2)
#pragma unroll
          for (int s = 0; s < SPT; s++) {
            const uint64_t dw = tc::sdesc_mn(sa + s * SA);
#pragma unroll
            for (int kk = 0; kk < 4; kk++)
              tc::mma_f16(tmem + STC_SUB * s, dw + (uint64_t)(128 * kk), du + (uint64_t)(2 * kk), ID_S,
                          (kb > 0 || kk > 0) ? 1u : 0u);
          }
        } else {
#pragma unroll
          for (int s = 0; s < SPT; s++) {
            const uint64_t dah = tc::sdesc<STC_KB>(sa + s * CA), dal = tc::sdesc<STC_KB>(sa + CHALF + s * CA);
#pragma unroll
            for (int kk = 0; kk < STC_KB / 16; kk++) {
              const uint64_t o = (uint64_t)(kk * 2);  // 32 bytes per 16-deep step, in 16-byte units
              tc::mma_f16(tmem + STC_SUB * s, dah + o, dbh + o, ID_C, (kb > 0 || kk > 0) ? 1u : 0u);
              tc::mma_f16(tmem + STC_SUB * s, dah + o, dbl + o, ID_C, 1u);
              tc::mma_f16(tmem + STC_SUB * s, dal + o, dbh + o, ID_C, 1u);
            }
          }
        }
        tc::mma_commit(freeb);
        if (!tc::mbar_wait(freeb, (ph >> 1) & 1, p.err, 9)) {
          bad = 2;
          break;
        }
        ph ^= 2;
      }
      if (bad) {
        // wait (bounded) for the copies or products still in flight
        if (bad == 1) tc::mbar_wait(full, ph & 1, p.err, 5);
        else tc::mbar_wait(freeb, (ph >> 1) & 1, p.err, 5);
        *abort_flag = 1;
      }
      *k.phases = ph;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // constants staged; shifts and coupling are in TMEM and the stage is free
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (*abort_flag) return false;
    {
      // the sub-tile's transposed triangle (rows u < mq, columns v < mq rounded up to 16) and band copy
      const int w4 = ((mq + 15) & ~15) >> 2;  // float4 per row
      for (int t = tid; t < mq * w4; t += STC_NS) {
        const int u = t / w4, c = t - u * w4;
        reinterpret_cast<float4*>(s_bt + u * STC_SUB)[c] =
            __ldg(reinterpret_cast<const float4*>(d.BT + (int64_t)(q0 + u) * d.ldbt + q0) + c);
      }
      // band rows of odd variables as stored (B[v+1+k][v] at k); of even variables moved
      // one place down (B[v+2+k][v] at k < 14) with B[v+1][v] at 14, so that the pair
      // update of the sweep below reads aligned pairs
      for (int t = tid; t < mq * 16; t += STC_NS) {
        const int v = t >> 4, kk = t & 15;
        const float* src = d.band + (int64_t)(q0 + v) * 16;
        s_band[t] = (v & 1) ? __ldg(src + kk) : (kk < 14 ? __ldg(src + kk + 1) : (kk == 14 ? __ldg(src) : 0.0f));
      }
    }
    __syncthreads();

    for (int v0 = 0; v0 < mq; v0 += DIAG_VB) {
      const int nb = min(DIAG_VB, mq - v0);
      // acc[s][i] = sums of the block's variables 2i (x) and 2i + 1 (y), as pairs for the
      // paired float32 FMAs (each pair FMA rounds as two fmaf)
      float2 acc[SPT][DIAG_VB / 2];
#pragma unroll
      for (int s = 0; s < SPT; s++) {
        if (q0 > 0 || p.kr > 0) {
          uint32_t r[DIAG_VB];
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];"
              : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
              : "r"(tl + (uint32_t)(STC_SUB * s + v0)));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
          for (int j = 0; j < DIAG_VB / 2; j++)
            acc[s][j] = F16 ? make_float2(__uint_as_float(r[2 * j]) * p.tscale, __uint_as_float(r[2 * j + 1]) * p.tscale)
                            : make_float2(__uint_as_float(r[2 * j]), __uint_as_float(r[2 * j + 1]));
        } else {
#pragma unroll
          for (int j = 0; j < DIAG_VB / 2; j++) acc[s][j] = make_float2(0.0f, 0.0f);
        }
      }
      uint64_t dnext[SPT];
#pragma unroll
      for (int s = 0; s < SPT; s++) dnext[s] = Ds[s][q0 + v0];
      // sums over the sub-tile's earlier variables for the block's 16 variables:
      // y_u from this lane's TMEM columns, four at a time, the B rows shared by the slots
      for (int u0 = 0; u0 < v0; u0 += 4) {
        uint32_t r[SPT][4];
#pragma unroll
        for (int s = 0; s < SPT; s++)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(r[s][0]), "=r"(r[s][1]), "=r"(r[s][2]), "=r"(r[s][3])
                       : "r"(tl + (uint32_t)(STC_SUB * s + u0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int uu = 0; uu < 4; uu++) {
          const float4* b4 = reinterpret_cast<const float4*>(s_bt + (u0 + uu) * STC_SUB + v0);
          const float4 q[4] = {b4[0], b4[1], b4[2], b4[3]};
#pragma unroll
          for (int s = 0; s < SPT; s++) {
            const float yu = __uint_as_float(r[s][uu]);
            const float2 yy = make_float2(yu, yu);
#pragma unroll
            for (int h = 0; h < 4; h++) {
              acc[s][2 * h] = __ffma2_rn(make_float2(q[h].x, q[h].y), yy, acc[s][2 * h]);
              acc[s][2 * h + 1] = __ffma2_rn(make_float2(q[h].z, q[h].w), yy, acc[s][2 * h + 1]);
            }
          }
        }
      }
      // one variable of eq. 2 for each slot: sum[s] = its sum over the earlier variables
      // and the shifts; returns its y and stores it into this lane's column v (whose sum
      // has been read), warp-wide after the step's divergent branches
      auto step = [&](int j, const float (&sum)[SPT], float (&y)[SPT]) {
        const int v = v0 + j;
        const float4 abi = s_abi[v];
        const uint64_t qv = s_q[v];
        const int vn = q0 + ((j + 1 < nb) ? v + 1 : v);  // next variable (the last one reloads its own)
#pragma unroll
        for (int s = 0; s < SPT; s++) {
          const uint64_t dv = dnext[s];
          dnext[s] = Ds[s][vn];
          const float bt = (abi.y * rs[s] - sum[s]) * abi.z;
          float w, wc, f, la;
          lattice_wf((uint64_t)ks[s] * qv + dv, PER ? 1 : 0, w, wc);
          if (ONE) {
            sov_step_f32_upper(bt, w, wc, f, la, y[s]);
          } else {
            const float at = (abi.x * rs[s] - sum[s]) * abi.z;
            sov_step_f32_prod(at, bt, w, wc, f, la, y[s]);
          }
          lsum[s] += la;
          prod[s] *= f;  // prod in [1, 2) and f >= Phi(-12): a normal float
          const int pb = __float_as_int(prod[s]);
          pe[s] += (pb >> 23) - 127;
          prod[s] = __int_as_float((pb & 0x007FFFFF) | 0x3F800000);
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < SPT; s++)
          asm volatile("tcgen05.st.sync.aligned.32x32b.x1.b32 [%0], {%1};" ::"r"(tl + (uint32_t)(STC_SUB * s + v)),
                       "r"(__float_as_uint(y[s]))
                       : "memory");
      };
      // the block's variables in pairs (v even, v + 1): after y_v the pair's second sum
      // takes B[v+1][v] y_v and the window moves two places, the later sums taking
      // B[v+2+k][v] y_v; after y_{v+1} they take B[v+2+k][v+1] y_{v+1} (k < 14: the
      // rest of the block).  Each sum receives its terms in the order of the variables.
#pragma unroll 1
      for (int j = 0; j < nb; j += 2) {
        const int v = v0 + j;
        float sum[SPT], y0[SPT];
#pragma unroll
        for (int s = 0; s < SPT; s++) sum[s] = acc[s][0].x;
        step(j, sum, y0);
        if (j + 1 == nb) break;  // (a ragged block's last variable: the window is not needed)
        {
          const float4* b4 = reinterpret_cast<const float4*>(s_band + v * 16);
          const float4 q[4] = {b4[0], b4[1], b4[2], b4[3]};
#pragma unroll
          for (int s = 0; s < SPT; s++) {
            sum[s] = fmaf(q[3].z, y0[s], acc[s][0].y);
            const float2 yy = make_float2(y0[s], y0[s]);
#pragma unroll
            for (int h = 0; h < 3; h++) {
              acc[s][2 * h] = __ffma2_rn(make_float2(q[h].x, q[h].y), yy, acc[s][2 * h + 1]);
              acc[s][2 * h + 1] = __ffma2_rn(make_float2(q[h].z, q[h].w), yy, acc[s][2 * h + 2]);
            }
            acc[s][6] = __ffma2_rn(make_float2(q[3].x, q[3].y), yy, acc[s][7]);
            acc[s][7] = make_float2(0.0f, 0.0f);
          }
        }
        float y1[SPT];
        step(j + 1, sum, y1);
        {
          const float4* b4 = reinterpret_cast<const float4*>(s_band + (v + 1) * 16);
          const float4 q[4] = {b4[0], b4[1], b4[2], b4[3]};
#pragma unroll
          for (int s = 0; s < SPT; s++) {
            const float2 yy = make_float2(y1[s], y1[s]);
#pragma unroll
            for (int h = 0; h < 3; h++) {
              acc[s][2 * h] = __ffma2_rn(make_float2(q[h].x, q[h].y), yy, acc[s][2 * h]);
              acc[s][2 * h + 1] = __ffma2_rn(make_float2(q[h].z, q[h].w), yy, acc[s][2 * h + 1]);
            }
            acc[s][6] = __ffma2_rn(make_float2(q[3].x, q[3].y), yy, acc[s][6]);
          }
        }
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      // the block's y, sample-major bf16 hi and lo (32 bytes each per sample), for
      // the later sub-tiles' products (read back by TMA: async proxy) and the projection
#pragma unroll
      for (int s = 0; s < SPT; s++) {
        uint32_t r[DIAG_VB];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tl + (uint32_t)(STC_SUB * s + v0)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (act[s]) {
          unsigned short* row = pl.ysrow[s] + q0 + v0;
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
            unsigned short* rh = row;
            unsigned short* rl = row + d.ys_lo;
#pragma unroll
            for (int j = 0; j < DIAG_VB; j++)
              if (j < nb) {
                rh[j] = (unsigned short)(hi2[j / 2] >> (16 * (j & 1)));
                rl[j] = (unsigned short)(lo2[j / 2] >> (16 * (j & 1)));
              }
          }
        }
      }
    }
    // y stored and visible to the copies (global), the shared copies free for the next copies into the stage
    // (shared), the TMEM columns free for the next products
    asm volatile("fence.proxy.async;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
  }
  // the tile's projections for the later tiles, 64 ranks a pass through the same
  // TMEM columns: W[vmap[r]][c] = sum_v V[kcol0 + r][v] y_v[c] (y hi parts, 64-deep
  // stages of the CTA's y rows and of V rows)
  for (int r0 = 0; r0 < p.kc; r0 += 64) {
    if (tid == 0) {
      const uint32_t sa = tc::smem_u32(stage);
      const uint64_t db = tc::sdesc<64>(sa + SPT * PA);
      uint32_t ph = *k.phases;
      int bad = 0;
      for (int kb = 0; kb < (mt + 63) / 64; kb++) {
        tc::mbar_expect_tx(full, SB);
#pragma unroll
        for (int s = 0; s < SPT; s++) tc::tma_load_2d(stage + s * PA, mapY64, full, kb * 64, pl.yrow + 128 * s);
        tc::tma_load_2d(stage + SPT * PA, mapV, full, kb * 64, p.kcol0 + r0);
        if (!tc::mbar_wait(full, ph & 1, p.err, 8)) {
          bad = 1;
          break;
        }
        ph ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int s = 0; s < SPT; s++) {
          const uint64_t da = tc::sdesc<64>(sa + s * PA);
#pragma unroll
          for (int kk = 0; kk < 4; kk++)
            tc::mma_f16(tmem + STC_SUB * s, da + (uint64_t)(2 * kk), db + (uint64_t)(2 * kk), ID_P,
                        (kb > 0 || kk > 0) ? 1u : 0u);
        }
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
        *abort_flag = 1;
      }
      *k.phases = ph;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (*abort_flag) return false;
#pragma unroll 1
    for (int h = 0; h < 64; h += 16) {
#pragma unroll
      for (int s = 0; s < SPT; s++) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
            "%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tl + (uint32_t)(STC_SUB * s + h)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (act[s]) {
#pragma unroll
          for (int j = 0; j < 16; j++)
            if (r0 + h + j < p.kc)
              pl.wcol[s][(int64_t)p.vmap[r0 + h + j] * p.ldw] =
                  Op::one(F16 ? __uint_as_float(r[j]) * p.wscale[r0 + h + j] : __uint_as_float(r[j]));
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // the TMEM columns and the stage free for the next pass
  }
  return true;
}

// The CTA's stage, constants, barriers and TMEM columns (dynamic shared memory of
// sweep_tc_smem_bytes<SPT>()); the barriers initialised and the columns allocated.
// Ends with every thread past the allocation.
template <int SPT>
__device__ __forceinline__ StcCta stc_cta_setup(unsigned char* smem_raw, uint32_t* phases, int* abort_flag) {
  // (offset within the shared window, so that the accesses stay shared-memory ones)
  unsigned char* smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  StcCta k;
  k.stage = smem;
  k.s_abi = reinterpret_cast<float4*>(smem + StcLayout<SPT>::SB);
  k.s_q = reinterpret_cast<uint64_t*>(k.s_abi + STC_SUB);
  k.full = k.s_q + STC_SUB;
  k.freeb = k.full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(k.freeb + 1);
  k.phases = phases;
  k.abort_flag = abort_flag;
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    *phases = 0;
    tc::mbar_init(k.full, 1);
    tc::mbar_init(k.freeb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(tmem_slot)),
                 "r"(StcLayout<SPT>::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  k.tmem = *tmem_slot;
  return k;
}

// Frees the CTA's TMEM columns once every thread is done with them.
template <int SPT>
__device__ __forceinline__ void stc_cta_release(const StcCta& k) {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(k.tmem), "r"(StcLayout<SPT>::TMEM_COLS)
                 : "memory");
}

// One launch per diagonal tile of one problem: CTA x owns samples [128 SPT x, 128 SPT (x + 1)) of the
// chunk.  SPT = 1: six CTAs per SM, 80 registers each (the 72 that seven would allow measured 17%
// slower); SPT = 2: two samples per thread, 128 TMEM columns and a 40 KB stage per CTA, four per SM.
template <int FLAGS, bool F16, int SPT>
__global__ void __launch_bounds__(STC_NS, SPT == 1 ? 6 : 4)
    k_sweep_tc(const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapB,
               const __grid_constant__ CUtensorMap mapW, const __grid_constant__ CUtensorMap mapU,
               const __grid_constant__ CUtensorMap mapY64, const __grid_constant__ CUtensorMap mapV, SweepTcArgs p) {
  extern __shared__ __align__(1024) unsigned char stc_smem[];
  __shared__ uint32_t phases;
  __shared__ int abort_flag;
  const StcCta k = stc_cta_setup<SPT>(stc_smem, &phases, &abort_flag);
  pdl_trigger();  // (after the allocation: a successor's CTAs never hold TMEM this grid still needs)
  pdl_wait();  // limit shifts, y and log P of the preceding kernels

  const DiagArgs32& d = p.d;
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * STC_NS * SPT;  // (a chunk holds fewer than 2^31 samples)
  bool act[SPT];
  int cs[SPT];
  const uint64_t* Ds[SPT];
  uint32_t ks[SPT];  // lattice point index k = 1..N (N < 2^31)
  float rs[SPT], prod[SPT], lsum[SPT];
  int pe[SPT];
  StcPlace pl;
  pl.wx = c0;
  pl.wy = 0;
  pl.yrow = c0;
#pragma unroll
  for (int s = 0; s < SPT; s++) {
    act[s] = c0 + STC_NS * s + tid < d.C;
    cs[s] = act[s] ? c0 + STC_NS * s + tid : (int)d.C - 1;  // inactive lanes shadow a valid sample, write nothing
    const int64_t g = d.sample0 + cs[s], sh = g / d.N;
    ks[s] = (uint32_t)(g - sh * d.N) + 1u;
    Ds[s] = d.D + sh * d.ldD + d.coord0;
    rs[s] = d.rs ? d.rs[cs[s]] : 1.0f;
    // log P of the tile = log(prod) + pe log 2 + lsum, prod kept in [1, 2)
    prod[s] = 1.0f;
    lsum[s] = 0.0f;
    pe[s] = 0;
    pl.ysrow[s] = reinterpret_cast<unsigned short*>(d.Ys) + (int64_t)cs[s] * d.ldys;
    pl.wcol[s] = p.W + cs[s];
  }
  const bool ok = stc_tile<FLAGS, F16, SPT>(&mapY, &mapB, &mapW, &mapU, &mapY64, &mapV, p, k, pl, act, Ds, ks, rs,
                                            prod, lsum, pe);
#pragma unroll
  for (int s = 0; s < SPT; s++)
    if (ok && act[s]) {
      const double lp = (double)(logf(prod[s]) + lsum[s]) + (double)pe[s] * 0.69314718055994530942;
      const int64_t g = d.sample0 + cs[s];
      if (d.first) d.logP[g] = lp;
      else d.logP[g] += lp;
    }
  stc_cta_release<SPT>(k);
}

}  // namespace tlrmvn
