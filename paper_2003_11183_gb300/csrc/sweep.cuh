// The float32 diagonal-tile sweep (eq. 2 over one sub-tile of a diagonal tile
// B_i, Algorithm 6's per-tile step), one chain of variables per sample.
#pragma once
#include "common.cuh"
#include "sov_device.cuh"

namespace tlrmvn {

// Arguments of one float32 sweep over a (sub-)tile of mt variables.  All
// pointers are already offset to the sub-tile's first variable.
struct DiagArgs32 {
  const float* BT;   // transposed diagonal block, BT[u * ldbt + v] = B[v][u]
  const float* inv;  // 1 / B[v][v]
  const float* band; // band[v * 16 + k] = B[v+1+k][v] (k < 15; zero past the tile), 16-byte aligned
  int mt;
  int64_t ldbt;
  const float* Delta;  // limit shifts, variable-major (ldd), or null
  int64_t ldd;
  const float* a;
  const float* b;
  const float* rs;
  const uint64_t* Q;
  const uint64_t* D;
  int64_t ldD, coord0, sample0, N, C;
  int periodize, first;
  float* Yv;             // y variable-major, Yv[v * ldyv + c], or null
  int64_t ldyv;
  __nv_bfloat16* Ys;     // y sample-major bf16, Ys[c * ldys + v], or null
  int64_t ldys;
  int64_t ys_lo;         // > 0: also the low part bf16(y - hi) at Ys[c * ldys + ys_lo + v]
  double* logP;
};

// 16 variables per pass: the partial sums of a block of 16 variables over all
// earlier variables of the (sub-)tile are accumulated together (each y_u read
// once per block, B read as four broadcast float4 per u); then the block's
// variables run in order in a rolled loop, each pushing its y into the partial
// sums of the block's later variables through a shifting window of
// accumulators (so the special-function code exists once).
constexpr int DIAG_VB = 16;
// Largest sub-tile, and the sub-tile of the SIMT coupling (FP32 path).
constexpr int DIAG_SUB = 128;
// Extra floats after the transposed tiles: the accumulator window may read up
// to DIAG_VB - 1 entries past the last row.
constexpr int DIAG_PAD = 32;

// Shared memory of one block of `ns` samples: the sub-tile's y of each sample
// (ns + 1 floats per variable), the sub-tile's transposed triangle (mt rows of mt
// rounded up to 16 floats) and band copy (mt x 16; every per-variable load of B a
// shared-memory broadcast),
// then the per-variable constants: (a, b, 1/B_vv) as one float4 per variable (one
// 16-byte load), then the lattice generators.
__host__ __device__ inline size_t sweep_ys_bytes(int mt, int ns) {
  return ((size_t)mt * (ns + 1) * sizeof(float) + 15) / 16 * 16;
}
__host__ __device__ inline size_t sweep_bt_bytes(int mt) {
  return (size_t)mt * ((mt + 15) & ~15) * sizeof(float) + (size_t)mt * 16 * sizeof(float);  // (+ the band copy)
}
__host__ __device__ inline size_t sweep_smem_bytes(int mt, int ns) {
  return sweep_ys_bytes(mt, ns) + sweep_bt_bytes(mt) + (size_t)mt * (sizeof(float4) + sizeof(uint64_t));
}

// FLAGS, fixed for a launch: SWEEP_PERIODIZE (tent-periodised lattice),
// SWEEP_YV (also write y as float to Yv), SWEEP_ONE_SIDED (every lower limit of
// the problem is -inf: the one-sided step only).
enum { SWEEP_PERIODIZE = 1, SWEEP_YV = 2, SWEEP_ONE_SIDED = 4 };

// SPT samples per thread (samples c0 + tid + s * blockDim.x): every broadcast
// load of B and of the per-variable constants serves SPT chains, and the SPT
// chains are independent instruction streams for the scheduler.  Each
// variable's lattice offsets are loaded one variable ahead and its window
// column before its special functions, and the block's limit shifts are added
// after its sums over earlier variables, so that those loads are in flight
// while other work runs.
template <int SPT, int FLAGS>
__global__ void k_diag_f32(DiagArgs32 p) {
  constexpr bool PER = FLAGS & SWEEP_PERIODIZE, YV = FLAGS & SWEEP_YV, ONE = FLAGS & SWEEP_ONE_SIDED;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int bd = blockDim.x, tid = threadIdx.x, ns = SPT * bd, ld = ns + 1;
  const int mt = p.mt;
  float* ys = reinterpret_cast<float*>(smem_raw);
  const int wbt = (mt + 15) & ~15;  // row length of the staged triangle
  float* s_bt = reinterpret_cast<float*>(smem_raw + sweep_ys_bytes(mt, ns));
  float4* s_abi = reinterpret_cast<float4*>(smem_raw + sweep_ys_bytes(mt, ns) + sweep_bt_bytes(mt));
  uint64_t* s_q = reinterpret_cast<uint64_t*>(s_abi + mt);
  const int64_t c0 = (int64_t)blockIdx.x * ns;
  pdl_trigger();
  // limits, diagonal, triangle and generators are not written by the preceding kernels
  for (int t = tid; t < mt; t += bd) {
    s_abi[t] = make_float4(p.a[t], p.b[t], p.inv[t], 0.0f);
    s_q[t] = p.Q[p.coord0 + t];
  }
  for (int t = tid; t < mt * (wbt >> 2); t += bd) {
    const int u = t / (wbt >> 2), c = t - u * (wbt >> 2);
    reinterpret_cast<float4*>(s_bt + u * wbt)[c] = __ldg(reinterpret_cast<const float4*>(p.BT + (int64_t)u * p.ldbt) + c);
  }
  // s_band[v * 16 + k] = B[v+1+k][v] for odd v; for even v moved one place down
  // (B[v+2+k][v] at k < 14) with B[v+1][v] at 14, so that the pair update of the
  // sweep below reads aligned pairs
  float* s_band = s_bt + mt * wbt;
  for (int t = tid; t < mt * 16; t += bd) {
    const int v = t >> 4, kk = t & 15;
    const float* src = p.band + (int64_t)v * 16;
    s_band[t] = (v & 1) ? __ldg(src + kk) : (kk < 14 ? __ldg(src + kk + 1) : (kk == 14 ? __ldg(src) : 0.0f));
  }
  __syncthreads();
  pdl_wait();  // the limit shifts, y and log P of the preceding kernels
  bool act[SPT];
  int64_t cs[SPT];
  uint32_t ks[SPT];  // lattice point index k = 1..N (N < 2^31)
  const uint64_t* Ds[SPT];
  float rs[SPT];
  // log P of the sub-tile = log(prod) + pe log 2 + lsum: prod is kept in [1, 2)
  // with its binary exponent in pe, so it neither underflows nor needs a log per variable
  float prod[SPT], lsum[SPT];
  int pe[SPT];
#pragma unroll
  for (int s = 0; s < SPT; s++) {
    act[s] = c0 + tid + s * bd < p.C;
    cs[s] = act[s] ? c0 + tid + s * bd : p.C - 1;  // inactive lanes shadow a valid sample, write nothing
    const int64_t g = p.sample0 + cs[s];
    const int64_t sh = g / p.N;
    ks[s] = (uint32_t)(g - sh * p.N) + 1u;
    Ds[s] = p.D + sh * p.ldD + p.coord0;
    rs[s] = p.rs ? p.rs[cs[s]] : 1.0f;
    prod[s] = 1.0f;
    lsum[s] = 0.0f;
    pe[s] = 0;
  }
  for (int v0 = 0; v0 < mt; v0 += DIAG_VB) {
    const int nb = min(DIAG_VB, mt - v0);
    // acc[s][i] = sums of the block's variables 2i (x) and 2i + 1 (y), as pairs for the
    // paired float32 FMAs (each pair FMA rounds as two fmaf)
    float2 acc[SPT][DIAG_VB / 2], dl[SPT][DIAG_VB / 2];
#pragma unroll
    for (int s = 0; s < SPT; s++)
#pragma unroll
      for (int j = 0; j < DIAG_VB / 2; j++) {
        dl[s][j].x = (p.Delta && 2 * j < nb) ? p.Delta[(int64_t)(v0 + 2 * j) * p.ldd + cs[s]] : 0.0f;
        dl[s][j].y = (p.Delta && 2 * j + 1 < nb) ? p.Delta[(int64_t)(v0 + 2 * j + 1) * p.ldd + cs[s]] : 0.0f;
        acc[s][j] = make_float2(0.0f, 0.0f);
      }
    // lattice offsets of the block's first variable
    uint64_t dnext[SPT];
#pragma unroll
    for (int s = 0; s < SPT; s++) dnext[s] = Ds[s][v0];
    // sums over the sub-tile's earlier variables for the block's 16 variables
    const float* bcol = s_bt + v0;
#pragma unroll 2
    for (int u = 0; u < v0; u++) {
      float yu[SPT];
#pragma unroll
      for (int s = 0; s < SPT; s++) yu[s] = ys[u * ld + tid + s * bd];
      const float4* b4 = reinterpret_cast<const float4*>(bcol + u * wbt);
      const float4 q[4] = {b4[0], b4[1], b4[2], b4[3]};
#pragma unroll
      for (int s = 0; s < SPT; s++) {
        const float2 yy = make_float2(yu[s], yu[s]);
#pragma unroll
        for (int h = 0; h < 4; h++) {
          acc[s][2 * h] = __ffma2_rn(make_float2(q[h].x, q[h].y), yy, acc[s][2 * h]);
          acc[s][2 * h + 1] = __ffma2_rn(make_float2(q[h].z, q[h].w), yy, acc[s][2 * h + 1]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < SPT; s++)
#pragma unroll
      for (int j = 0; j < DIAG_VB / 2; j++) acc[s][j] = __fadd2_rn(acc[s][j], dl[s][j]);
    // one variable of eq. 2 for each slot: sum[s] = its sum over the earlier variables
    // and the shifts; returns its y (also stored for the later variables and blocks)
    auto step = [&](int j, const float (&sum)[SPT], float (&y)[SPT]) {
      const int v = v0 + j;
      const float4 abi = s_abi[v];
      const float av = abi.x, bv = abi.y, iv = abi.z;
      const uint64_t qv = s_q[v];
#pragma unroll
      for (int s = 0; s < SPT; s++) {
        const uint64_t dv = dnext[s];
        dnext[s] = Ds[s][(j + 1 < nb) ? v + 1 : v];  // next variable's offset (the last one reloads its own)
        const float bt = (bv * rs[s] - sum[s]) * iv;
        float w, wc;
        lattice_wf((uint64_t)ks[s] * qv + dv, PER ? 1 : 0, w, wc);
        float f, la;
        if (ONE) {
          sov_step_f32_upper(bt, w, wc, f, la, y[s]);
        } else {
          const float at = (av * rs[s] - sum[s]) * iv;
          sov_step_f32_prod(at, bt, w, wc, f, la, y[s]);
        }
        lsum[s] += la;
        prod[s] *= f;  // prod in [1, 2) and f >= Phi(-12): a normal float
        const int pb = __float_as_int(prod[s]);
        pe[s] += (pb >> 23) - 127;
        prod[s] = __int_as_float((pb & 0x007FFFFF) | 0x3F800000);
        ys[v * ld + tid + s * bd] = y[s];
        if (YV && act[s]) p.Yv[(int64_t)v * p.ldyv + cs[s]] = y[s];
      }
    };
    // the block's variables in pairs (v even, v + 1): after y_v the pair's second sum
    // takes B[v+1][v] y_v and the window moves two places, the later sums taking
    // B[v+2+k][v] y_v; after y_{v+1} they take B[v+2+k][v+1] y_{v+1} (k < 14: the rest
    // of the block).  Each sum receives its terms in the order of the variables.  The
    // window columns are loaded before the steps, so that the loads are in flight
    // during their special functions.
#pragma unroll 1
    for (int j = 0; j < nb; j += 2) {
      const int v = v0 + j;
      const float4* b4 = reinterpret_cast<const float4*>(s_band + v * 16);
      const float4 q[4] = {b4[0], b4[1], b4[2], b4[3]};
      float sum[SPT], y0[SPT];
#pragma unroll
      for (int s = 0; s < SPT; s++) sum[s] = acc[s][0].x;
      step(j, sum, y0);
      if (j + 1 == nb) break;  // (a ragged block's last variable: the window is not needed)
      const float4* c4 = reinterpret_cast<const float4*>(s_band + (v + 1) * 16);
      const float4 r[4] = {c4[0], c4[1], c4[2], c4[3]};
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
      float y1[SPT];
      step(j + 1, sum, y1);
#pragma unroll
      for (int s = 0; s < SPT; s++) {
        const float2 yy = make_float2(y1[s], y1[s]);
#pragma unroll
        for (int h = 0; h < 3; h++) {
          acc[s][2 * h] = __ffma2_rn(make_float2(r[h].x, r[h].y), yy, acc[s][2 * h]);
          acc[s][2 * h + 1] = __ffma2_rn(make_float2(r[h].z, r[h].w), yy, acc[s][2 * h + 1]);
        }
        acc[s][6] = __ffma2_rn(make_float2(r[3].x, r[3].y), yy, acc[s][6]);
      }
    }
  }
#pragma unroll
  for (int s = 0; s < SPT; s++) {
    if (!act[s]) continue;
    const int64_t g = p.sample0 + cs[s];
    const double lp = (double)(logf(prod[s]) + lsum[s]) + (double)pe[s] * 0.69314718055994530942;
    if (p.first) p.logP[g] = lp;
    else p.logP[g] += lp;
  }
  if (p.Ys) {
    __syncthreads();
    const int nw = bd >> 5, warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < ns; j += nw) {
      if (c0 + j >= p.C) break;
      __nv_bfloat16* row = p.Ys + (c0 + j) * p.ldys;
      for (int v = lane; v < p.mt; v += 32) {
        const float yv = ys[v * ld + j];
        const __nv_bfloat16 hi = __float2bfloat16_rn(yv);
        row[v] = hi;
        if (p.ys_lo) row[p.ys_lo + v] = __float2bfloat16_rn(yv - __bfloat162float(hi));
      }
    }
  }
}

}  // namespace tlrmvn
