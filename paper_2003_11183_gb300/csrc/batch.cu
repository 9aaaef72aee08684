// Many MVN/MVT problems of uneven dimension in one persistent launch.
//
// A work item is (problem, chunk of up to 128 samples).  Persistent CTAs take
// items from an atomic counter, largest problems first, and run the whole TLR
// integrand of Algorithms 6/7 for their chunk: for every diagonal tile, the
// low-rank limit shift sum_{j<i} U_ij (V_ij^T y_j) (from the chunk's projections
// W, kept in a CTA-private global buffer), the float32 SOV sweep of eq. (2),
// then the projections V_col,i^T y_i of the tile for the later tiles.  Items
// never wait on one another, so the kernel has no inter-CTA spin.  A plan
// captures the launch sequence (limit permutation, persistent kernel,
// estimator) in a CUDA graph, replayed for every new set of limits.
//
// Two persistent kernels: k_batch (TLRMVN_FP32: the shifts and projections as
// float SIMT loops, W float) and k_batch_tc (TLRMVN_BF16_SHIFT: every tile runs
// the whole-tile sweep of the single-problem path, stc_tile, with the shifts,
// in-tile coupling and projections on tcgen05; W and the sample-major y in
// CTA-private bf16 regions read back by TMA through one tensor map each, the
// per-problem factor operands through three tensor maps per problem kept in
// global memory).
#include "common.cuh"
#include "sov_device.cuh"
#include "sweep_tc.cuh"

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <numeric>
#include <string>

namespace tlrmvn {

__global__ void k_shift_reduce(const double* logP, int64_t N, double* ell);
__global__ void k_final(const double* ell, int M, double* logp, double* errp);

constexpr int BATCH_T = 128;     // samples per work item = threads per CTA
constexpr int BATCH_MMAX = 128;  // largest tile size of a batched problem
constexpr int BATCH_VB = 16;     // variables per register block

struct BatchProblem {
  int n, r, m, n_shifts;
  int64_t n_points, ldbt, ktot, logp_off;
  double nu;
  int periodize;
  const int64_t* tile_off;
  const int64_t* krow_off;
  const int64_t* kcol_off;
  const int64_t* vt_off;
  const int32_t* kcpad;
  const float* BT;
  const float* inv;
  const float* band;  // band[(i*m + v)*16 + k] = B_i[v+1+k][v] (the factor's band32)
  const float* UT;  // UT[(krow_off[i] + k) * ldbt + v] = Ucat_i[v][k]
  const float* VT;  // VT[vt_off[j] + u * kcpad[j] + k] = Vcat_j[k][u]
  const int32_t* vmap;
  const uint64_t* Q;
  const uint64_t* D;
  const float* a;
  const float* b;
};
struct BatchItem {
  int prob, count;
  int64_t sample0;
};

__device__ __forceinline__ void fma16(float* acc, const float* row, float x) {
  const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
  for (int q = 0; q < 4; q++) {
    const float4 v = __ldg(r4 + q);
    acc[4 * q] = fmaf(v.x, x, acc[4 * q]);
    acc[4 * q + 1] = fmaf(v.y, x, acc[4 * q + 1]);
    acc[4 * q + 2] = fmaf(v.z, x, acc[4 * q + 2]);
    acc[4 * q + 3] = fmaf(v.w, x, acc[4 * q + 3]);
  }
}

__global__ void __launch_bounds__(BATCH_T) k_batch(const BatchProblem* __restrict__ probs,
                                                   const BatchItem* __restrict__ items, int n_items, int* next,
                                                   float* Wbase, int64_t wstride, double* logP) {
  extern __shared__ __align__(16) float ys[];  // [BATCH_MMAX][BATCH_T + 1]
  __shared__ int cur;
  const int tid = threadIdx.x, ld = BATCH_T + 1;
  float* W = Wbase + (int64_t)blockIdx.x * wstride;  // [ktot][BATCH_T]
  for (;;) {
    __syncthreads();
    if (tid == 0) cur = atomicAdd(next, 1);
    __syncthreads();
    const int it = cur;
    if (it >= n_items) break;
    const BatchItem item = items[it];
    if (tid >= item.count) continue;
    const BatchProblem& P = probs[item.prob];
    const int64_t g = item.sample0 + tid;
    const int64_t s = g / P.n_points;
    const uint64_t k = (uint64_t)(g - s * P.n_points) + 1;
    const uint64_t* Ds = P.D + s * (int64_t)(P.n + 1);
    float rs = 1.0f;
    if (isfinite(P.nu)) {
      double w, wc;
      lattice_w(k * P.Q[P.n] + Ds[P.n], P.periodize, w, wc);
      rs = (float)sqrt(2.0 * gamma_p_inv(0.5 * P.nu, w, wc) / P.nu);
    }
    // log P = log(prod) + pe log 2 + lsum, prod kept in [1, 2) (see the float sweep)
    float prod = 1.0f, lsum = 0.0f;
    int pe = 0;
    for (int i = 0; i < P.r; i++) {
      const int64_t t0 = P.tile_off[i];
      const int mt = (int)(P.tile_off[i + 1] - t0);
      const int64_t kr0 = P.krow_off[i], Kr = P.krow_off[i + 1] - kr0;
      const float* BTi = P.BT + (int64_t)i * P.m * P.ldbt;
      const float* invi = P.inv + (int64_t)i * P.m;
      for (int v0 = 0; v0 < mt; v0 += BATCH_VB) {
        float acc[BATCH_VB];
#pragma unroll
        for (int j = 0; j < BATCH_VB; j++) acc[j] = 0.0f;
        for (int64_t kk = 0; kk < Kr; kk++)  // low-rank shift of the limits
          fma16(acc, P.UT + (kr0 + kk) * P.ldbt + v0, W[(kr0 + kk) * BATCH_T + tid]);
        for (int u = 0; u < v0; u++)  // earlier variables of the tile
          fma16(acc, BTi + (int64_t)u * P.ldbt + v0, ys[u * ld + tid]);
        const int nb = min(BATCH_VB, mt - v0);
        // per-variable values of the block's first variable; later ones one variable ahead
        float an = P.a[t0 + v0], bn = P.b[t0 + v0], ivn = __ldg(invi + v0);
        uint64_t xn = k * P.Q[t0 + v0] + Ds[t0 + v0];
#pragma unroll 1
        for (int j = 0; j < nb; j++) {  // the block in order; acc[0] belongs to variable v
          const int v = v0 + j;
          const float av = an, bv = bn, iv = ivn;
          const uint64_t xv = xn;
          {
            const int vn = (j + 1 < nb) ? v + 1 : v;  // the last one reloads its own (in bounds)
            an = P.a[t0 + vn];
            bn = P.b[t0 + vn];
            ivn = __ldg(invi + vn);
            xn = k * P.Q[t0 + vn] + Ds[t0 + vn];
          }
          float bcur[BATCH_VB];  // B[v+1+i][v] from the band copy, loaded before the step's special functions
          {
            const float4* b4 = reinterpret_cast<const float4*>(P.band + ((int64_t)i * P.m + v) * 16);
#pragma unroll
            for (int h = 0; h < 4; h++) {
              const float4 x = __ldg(b4 + h);
              bcur[4 * h] = x.x;
              bcur[4 * h + 1] = x.y;
              bcur[4 * h + 2] = x.z;
              bcur[4 * h + 3] = x.w;
            }
          }
          const float sum = acc[0];
          const float at = (av * rs - sum) * iv;
          const float bt = (bv * rs - sum) * iv;
          float w, wc;
          lattice_wf(xv, P.periodize, w, wc);
          float f, la, y;
          sov_step_f32_prod(at, bt, w, wc, f, la, y);
          lsum += la;
          prod *= f;
          const int pb = __float_as_int(prod);
          pe += (pb >> 23) - 127;
          prod = __int_as_float((pb & 0x007FFFFF) | 0x3F800000);
          ys[v * ld + tid] = y;
#pragma unroll
          for (int i = 0; i < BATCH_VB - 1; i++) acc[i] = fmaf(bcur[i], y, acc[i + 1]);
          acc[BATCH_VB - 1] = 0.0f;
        }
      }
      const int64_t kc0 = P.kcol_off[i], Kc = P.kcol_off[i + 1] - kc0;
      if (Kc > 0) {  // projections of this tile for the later tiles
        const float* VTi = P.VT + P.vt_off[i];
        const int kcp = P.kcpad[i];
        const int32_t* vm = P.vmap + kc0;
        for (int64_t q0 = 0; q0 < Kc; q0 += BATCH_VB) {
          float acc[BATCH_VB];
#pragma unroll
          for (int j = 0; j < BATCH_VB; j++) acc[j] = 0.0f;
          for (int u = 0; u < mt; u++) fma16(acc, VTi + (int64_t)u * kcp + q0, ys[u * ld + tid]);
#pragma unroll
          for (int j = 0; j < BATCH_VB; j++)
            if (q0 + j < Kc) W[(int64_t)vm[q0 + j] * BATCH_T + tid] = acc[j];
        }
      }
    }
    logP[P.logp_off + g] = (double)(logf(prod) + lsum) + (double)pe * 0.69314718055994530942;
  }
}

// ---- tensor-core batched integrand (BF16-shift precision) ----------------------------------
constexpr int BATCH_TC_MAPS = 3;  // per problem: split B (32-deep boxes), U rows, V rows (64 x 64 boxes)

struct BatchTcProblem {
  int n, r, m, my;  // my: the factor's split-B lo offset (m rounded up to 64)
  int64_t n_points, ldbt, logp_off;
  double nu;
  const int64_t* tile_off;
  const int64_t* kpad_off;  // first W row of each row tile's ranks (multiples of 64)
  const int64_t* krow_off;
  const int64_t* kcol_off;
  const int32_t* vmap16;    // W row of each column rank
  const float* BT;
  const float* inv;
  const float* band;
  const uint64_t* Q;
  const uint64_t* D;
  const float* a;
  const float* b;
};

template <int FLAGS>
__global__ void __launch_bounds__(STC_NS, 6)
    k_batch_tc(const BatchTcProblem* __restrict__ probs, const CUtensorMap* __restrict__ pmaps,
               const BatchItem* __restrict__ items, int n_items, int* next, const __grid_constant__ CUtensorMap mapW,
               const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapY64,
               unsigned short* Wbase, int64_t kwmax, unsigned short* Ybase, int my, double* logP, int* err) {
  constexpr bool PER = FLAGS & SWEEP_PERIODIZE;
  extern __shared__ __align__(1024) unsigned char stc_smem[];
  __shared__ uint32_t phases;
  __shared__ int abort_flag;
  __shared__ int cur;
  const StcCta k = stc_cta_setup<1>(stc_smem, &phases, &abort_flag);
  const int tid = threadIdx.x;
  StcPlace pl;
  pl.wx = 0;
  pl.wy = (int)(blockIdx.x * kwmax);
  pl.yrow = blockIdx.x * STC_NS;
  pl.ysrow[0] = Ybase + ((int64_t)blockIdx.x * STC_NS + tid) * (2 * my);  // (hi at 0, lo at my)
  pl.wcol[0] = Wbase + (int64_t)blockIdx.x * kwmax * STC_NS + tid;
  for (;;) {
    __syncthreads();  // every thread is done with the previous item
    if (tid == 0) cur = atomicAdd(next, 1);
    __syncthreads();
    const int it = cur;
    if (it >= n_items || *(volatile int*)&abort_flag) break;
    const BatchItem item = items[it];
    const BatchTcProblem& P = probs[item.prob];
    const bool act[1] = {tid < item.count};
    const int64_t g = item.sample0 + (act[0] ? tid : item.count - 1);  // inactive lanes shadow a valid sample
    const int64_t sh = g / P.n_points;
    const uint32_t ks[1] = {(uint32_t)(g - sh * P.n_points) + 1u};
    const uint64_t* Drow = P.D + sh * (int64_t)(P.n + 1);
    float rs[1] = {1.0f};
    if (isfinite(P.nu)) {
      double w, wc;
      lattice_w((uint64_t)ks[0] * P.Q[P.n] + Drow[P.n], PER ? 1 : 0, w, wc);
      rs[0] = (float)sqrt(2.0 * gamma_p_inv(0.5 * P.nu, w, wc) / P.nu);
    }
    const CUtensorMap* mp = pmaps + (int64_t)BATCH_TC_MAPS * item.prob;
    float prod[1] = {1.0f}, lsum[1] = {0.0f};
    int pe[1] = {0};
    bool ok = true;
    for (int i = 0; i < P.r && ok; i++) {
      const int64_t t0 = P.tile_off[i];
      SweepTcArgs p;
      DiagArgs32& d = p.d;
      d.BT = P.BT + (int64_t)i * P.m * P.ldbt;
      d.inv = P.inv + (int64_t)i * P.m;
      d.band = P.band + (int64_t)i * P.m * 16;
      d.mt = (int)(P.tile_off[i + 1] - t0);
      d.ldbt = P.ldbt;
      d.a = P.a + t0;
      d.b = P.b + t0;
      d.Q = P.Q;
      d.coord0 = t0;
      d.ys_lo = my;
      p.brow0 = i * P.m;
      p.alo = my;
      p.blo = P.my;
      p.urow0 = i * P.m;
      p.krow0 = (int)P.kpad_off[i];
      p.kr = (int)(P.krow_off[i + 1] - P.krow_off[i]);
      p.kcol0 = (int)P.kcol_off[i];
      p.kc = (int)(P.kcol_off[i + 1] - P.kcol_off[i]);
      p.W = Wbase;
      p.ldw = STC_NS;
      p.vmap = P.vmap16 ? P.vmap16 + P.kcol_off[i] : nullptr;
      p.wscale = nullptr;
      p.tscale = 1.0f;
      p.err = err;
      const uint64_t* const Ds[1] = {Drow + t0};
      ok = stc_tile<FLAGS, false, 1>(&mapY, mp, &mapW, mp + 1, &mapY64, mp + 2, p, k, pl, act, Ds, ks, rs, prod,
                                     lsum, pe);
    }
    if (ok && act[0])
      logP[P.logp_off + g] = (double)(logf(prod[0]) + lsum[0]) + (double)pe[0] * 0.69314718055994530942;
  }
  stc_cta_release<1>(k);
}
static const void* batch_tc_kernel(int periodize) {
  return periodize ? (const void*)k_batch_tc<SWEEP_PERIODIZE> : (const void*)k_batch_tc<0>;
}

// limits of all problems: original order (staged) -> factor order, float; validation
__global__ void k_permute_batch(const double* a, const double* b, const int64_t* perm_g, int64_t total, float* a32,
                                float* b32, int* bad) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int64_t src = perm_g[t];  // global index into the staged limits
  const double av = a[src], bv = b[src];
  if (isnan(av) || isnan(bv) || av > bv || av == INFINITY || bv == -INFINITY) atomicExch(bad, 1);
  a32[t] = (float)av;
  b32[t] = (float)bv;
}

// UT row g (global rank index) = column g - krow_off[i] of Ucat_i, padded to ldbt
__global__ void k_make_ut(const double* Ucat, const int32_t* ktile, const int64_t* krow_off, int m, int64_t ldbt,
                          int64_t count, float* UT) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t g = t / ldbt, v = t % ldbt;
  const int i = ktile[g];
  const int64_t Kr = krow_off[i + 1] - krow_off[i];
  UT[t] = (v < m) ? (float)Ucat[(int64_t)m * krow_off[i] + v * Kr + (g - krow_off[i])] : 0.0f;
}
// VT block of column tile j: VT[u * kcp + k] = Vcat_j[k][u], zero for k >= Kc
__global__ void k_make_vt(const double* Vcat_j, int m, int64_t Kc, int kcp, float* VT) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * kcp) return;
  const int64_t u = t / kcp, kk = t % kcp;
  VT[t] = (kk < Kc) ? (float)Vcat_j[kk * m + u] : 0.0f;
}

// per-problem estimates: block p reduces the shifts of problem p
__global__ void k_final_batch(const double* ell, int M, double* out);

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// The float copies used by the batched kernel, made once per factor.
struct BatchCopies {
  float* UT = nullptr;
  float* VT = nullptr;
  int64_t *tile_off = nullptr, *krow_off = nullptr, *kcol_off = nullptr, *vt_off = nullptr, *kpad_off = nullptr;
  int32_t* kcpad = nullptr;
  ~BatchCopies() {
    dfree(UT);
    dfree(VT);
    dfree(tile_off);
    dfree(krow_off);
    dfree(kcol_off);
    dfree(vt_off);
    dfree(kpad_off);
    dfree(kcpad);
  }
};
int ensure_precision_copies(Factor& F, int precision, cudaStream_t st);  // prob.cu
int make_tensor_map_16(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch,
                       uint32_t box_outer, uint32_t box_inner, bool f16);  // prob.cu

int ensure_float_tiles(Factor& F, cudaStream_t st);  // prob.cu: BT32 / inv32

// tc: the tensor-core kernel's operands (the factor's bf16 copies and the padded
// rank offsets) instead of the float SIMT copies UT / VT.
static int make_batch_copies(Factor& F, BatchCopies& C, bool tc, cudaStream_t st) {
  const int r = F.r, m = F.m;
  if (tc) {
    TLR_CHECK(ensure_precision_copies(F, TLRMVN_BF16_SHIFT, st));
    TLR_CHECK(dalloc(&C.kpad_off, r + 1));
    TLR_CUDA(cudaMemcpyAsync(C.kpad_off, F.kpad_off.data(), (r + 1) * 8, cudaMemcpyHostToDevice, st));
  } else {
    std::lock_guard<std::mutex> lk(F.copy_mu);
    TLR_CHECK(ensure_float_tiles(F, st));
    TLR_CUDA(cudaStreamSynchronize(st));
  }
  std::vector<int64_t> vt_off(r + 1, 0);
  std::vector<int32_t> kcpad(r);
  for (int j = 0; j < r; j++) {
    kcpad[j] = (int32_t)((F.kcol(j) + 15) / 16 * 16);
    vt_off[j + 1] = vt_off[j] + (int64_t)m * kcpad[j];
  }
  TLR_CHECK(dalloc(&C.tile_off, r + 1));
  TLR_CHECK(dalloc(&C.krow_off, r + 1));
  TLR_CHECK(dalloc(&C.kcol_off, r + 1));
  TLR_CHECK(dalloc(&C.vt_off, r + 1));
  TLR_CHECK(dalloc(&C.kcpad, r));
  TLR_CUDA(cudaMemcpyAsync(C.tile_off, F.tile_off.data(), (r + 1) * 8, cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaMemcpyAsync(C.krow_off, F.krow_off.data(), (r + 1) * 8, cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaMemcpyAsync(C.kcol_off, F.kcol_off.data(), (r + 1) * 8, cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaMemcpyAsync(C.vt_off, vt_off.data(), (r + 1) * 8, cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaMemcpyAsync(C.kcpad, kcpad.data(), r * 4, cudaMemcpyHostToDevice, st));
  if (F.ktot && !tc) {
    std::vector<int32_t> ktile(F.ktot);
    for (int i = 0; i < r; i++)
      for (int64_t g = F.krow_off[i]; g < F.krow_off[i + 1]; g++) ktile[g] = i;
    int32_t* dkt = nullptr;
    TLR_CHECK(dalloc(&dkt, (size_t)F.ktot));
    TLR_CUDA(cudaMemcpyAsync(dkt, ktile.data(), ktile.size() * 4, cudaMemcpyHostToDevice, st));
    const int64_t nut = F.ktot * F.ldbt;
    TLR_CHECK(dalloc(&C.UT, (size_t)nut));
    k_make_ut<<<nblk(nut, 256), 256, 0, st>>>(F.Ucat, dkt, C.krow_off, m, F.ldbt, nut, C.UT);
    TLR_CHECK(dalloc(&C.VT, (size_t)std::max<int64_t>(vt_off[r], 1)));
    for (int j = 0; j < r; j++)
      if (F.kcol(j))
        k_make_vt<<<nblk((int64_t)m * kcpad[j], 256), 256, 0, st>>>(F.Vcat + (size_t)m * F.kcol_off[j], m, F.kcol(j),
                                                                      kcpad[j], C.VT + vt_off[j]);
    TLR_CUDA(cudaStreamSynchronize(st));
    dfree(dkt);
  }
  TLR_CUDA(cudaStreamSynchronize(st));
  TLR_CUDA(cudaGetLastError());
  return TLRMVN_OK;
}

struct Batch {
  int count = 0, M = 0, device = 0;
  int64_t N = 0, total_n = 0, total_samples = 0, ktot_max = 0;
  int periodize = 1;
  cudaStream_t st = nullptr;
  std::vector<Factor*> F;
  std::vector<int64_t> n_off;  // limits offsets of each problem (host)
  std::vector<BatchCopies> copies;
  BatchProblem* dprobs = nullptr;
  BatchItem* ditems = nullptr;
  int n_items = 0, grid = 0, grid_max = 0, per_sm = 0, per_sm_max = 0, sms = 0;
  int* dnext = nullptr;
  int* dbad = nullptr;
  float* W = nullptr;
  // tensor-core kernel (TLRMVN_BF16_SHIFT)
  bool tc = false;
  int64_t kwmax = 0;          // W rows of one CTA's region (the largest padded rank space)
  int my = 64;                // y hi columns of one sample's row in the CTA-private y (lo at + my)
  BatchTcProblem* dtprobs = nullptr;
  CUtensorMap* dmaps = nullptr;
  unsigned short *W16 = nullptr, *Y16 = nullptr;
  CUtensorMap mapW{}, mapY{}, mapY64{};
  int* derr = nullptr;
  double *logP = nullptr, *ell = nullptr, *out = nullptr, *a_st = nullptr, *b_st = nullptr;
  float *a32 = nullptr, *b32 = nullptr;
  int64_t* perm_g = nullptr;
  uint64_t* D = nullptr;
  double* h_ab = nullptr;   // pinned staging of the limits
  double* h_out = nullptr;  // pinned results
  cudaGraphExec_t exec = nullptr;
  ~Batch() {
    if (exec) cudaGraphExecDestroy(exec);
    dfree(dprobs);
    dfree(dtprobs);
    dfree(dmaps);
    dfree(W16);
    dfree(Y16);
    dfree(derr);
    dfree(ditems);
    dfree(dnext);
    dfree(dbad);
    dfree(W);
    dfree(logP);
    dfree(ell);
    dfree(out);
    dfree(a_st);
    dfree(b_st);
    dfree(a32);
    dfree(b32);
    dfree(perm_g);
    dfree(D);
    if (h_ab) cudaFreeHost(h_ab);
    if (h_out) cudaFreeHost(h_out);
    if (st) cudaStreamDestroy(st);
  }
};

uint64_t splitmix64_seed_at(uint64_t seed, uint64_t t);  // prob.cu

static size_t batch_smem() { return (size_t)BATCH_MMAX * (BATCH_T + 1) * sizeof(float); }

// CTAs of `threads` threads and `dyn_smem` dynamic shared memory that one SM holds at
// once, from the kernel's registers and static shared memory and the device's limits.
static int resident_ctas(const void* kernel, int threads, size_t dyn_smem, int dev, int* out) {
  cudaFuncAttributes fa;
  TLR_CUDA(cudaFuncGetAttributes(&fa, kernel));
  int regs_sm = 0, smem_sm = 0, res_blk = 0, thr_sm = 0, blk_sm = 0;
  TLR_CUDA(cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
  TLR_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  TLR_CUDA(cudaDeviceGetAttribute(&res_blk, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  TLR_CUDA(cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev));
  TLR_CUDA(cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev));
  const int warps = (threads + 31) / 32;
  const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;  // (allocated per warp in units of 256)
  int n = std::min(thr_sm / threads, blk_sm);
  if (regs_warp > 0) n = std::min(n, regs_sm / (regs_warp * warps));
  const size_t smem = (dyn_smem + fa.sharedSizeBytes + 127) / 128 * 128 + (size_t)res_blk;
  n = std::min<int>(n, (int)((size_t)smem_sm / smem));
  *out = std::max(n, 1);
  return TLRMVN_OK;
}

// Captures the plan's launch sequence (permute limits -> persistent integrand
// with `per_sm` CTAs per SM -> estimator) into a CUDA graph, replacing any
// earlier one.
static int batch_capture(Batch& B, int per_sm) {
  cudaStream_t st = B.st;
  const int grid = std::max(1, std::min(std::min(per_sm, B.per_sm_max) * B.sms, B.n_items));
  cudaGraph_t graph;
  TLR_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(B.dbad, 0, sizeof(int), st);
  cudaMemsetAsync(B.dnext, 0, sizeof(int), st);
  if (B.tc) cudaMemsetAsync(B.derr, 0, sizeof(int), st);
  k_permute_batch<<<nblk(B.total_n, 256), 256, 0, st>>>(B.a_st, B.b_st, B.perm_g, B.total_n, B.a32, B.b32, B.dbad);
  if (B.tc) {
    if (B.periodize)
      k_batch_tc<SWEEP_PERIODIZE><<<grid, STC_NS, sweep_tc_smem_bytes<1>(), st>>>(
          B.dtprobs, B.dmaps, B.ditems, B.n_items, B.dnext, B.mapW, B.mapY, B.mapY64, B.W16, B.kwmax, B.Y16, B.my,
          B.logP, B.derr);
    else
      k_batch_tc<0><<<grid, STC_NS, sweep_tc_smem_bytes<1>(), st>>>(B.dtprobs, B.dmaps, B.ditems, B.n_items, B.dnext,
                                                                 B.mapW, B.mapY, B.mapY64, B.W16, B.kwmax, B.Y16,
                                                                 B.my, B.logP, B.derr);
  } else {
    k_batch<<<grid, BATCH_T, batch_smem(), st>>>(B.dprobs, B.ditems, B.n_items, B.dnext, B.W,
                                                std::max<int64_t>(B.ktot_max, 1) * BATCH_T, B.logP);
  }
  k_shift_reduce<<<(unsigned)(B.count * B.M), 256, 0, st>>>(B.logP, B.N, B.ell);
  k_final_batch<<<B.count, 256, 0, st>>>(B.ell, B.M, B.out);
  cudaError_t ec = cudaStreamEndCapture(st, &graph);
  if (ec != cudaSuccess) return cuda_fail(ec, "capture of the batched integrand");
  cudaGraphExec_t exec = nullptr;
  ec = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ec != cudaSuccess) return cuda_fail(ec, "instantiate the batched integrand graph");
  if (B.exec) cudaGraphExecDestroy(B.exec);
  B.exec = exec;
  B.grid = grid;
  B.per_sm = std::min(per_sm, B.per_sm_max);
  return TLRMVN_OK;
}

static int batch_build(Batch& B, int count, const tlrmvn_factor_t* factors, const double* nu,
                       const tlrmvn_opts& o) {
  B.count = count;
  B.M = o.n_shifts;
  B.N = o.n_points;
  B.periodize = o.periodize;
  B.tc = o.precision == TLRMVN_BF16_SHIFT;
  TLR_CUDA(cudaGetDevice(&B.device));
  TLR_CUDA(cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking));
  cudaStream_t st = B.st;
  B.F.resize(count);
  B.copies.resize(count);
  B.n_off.assign(count + 1, 0);
  for (int p = 0; p < count; p++) {
    Factor* F = reinterpret_cast<Factor*>(factors[p]);
    if (!F) return fail(TLRMVN_E_INVAL, "null factor in batch");
    if (!B.tc && F->m > BATCH_MMAX) return fail(TLRMVN_E_NOTSUP, "FP32 batched problems need tile size <= 128");
    if (!(nu[p] > 0.0)) return fail(TLRMVN_E_INVAL, "nu must be > 0");
    B.F[p] = F;
    B.n_off[p + 1] = B.n_off[p] + F->n;
    B.ktot_max = std::max(B.ktot_max, F->ktot);
    TLR_CHECK(make_batch_copies(*F, B.copies[p], B.tc, st));
    if (B.tc) {
      B.kwmax = std::max(B.kwmax, F->kw16);
      B.my = std::max<int>(B.my, (int)F->my16);
    }
  }
  B.total_n = B.n_off[count];
  const int64_t S = (int64_t)B.M * B.N;
  B.total_samples = S * count;
  // device tables
  std::vector<BatchProblem> probs(count);
  std::vector<int64_t> perm_g(B.total_n);
  std::vector<int64_t> d_off(count + 1, 0);
  for (int p = 0; p < count; p++) d_off[p + 1] = d_off[p] + (int64_t)B.M * (B.F[p]->n + 1);
  TLR_CHECK(dalloc(&B.D, (size_t)d_off[count]));
  TLR_CHECK(dalloc(&B.a32, (size_t)B.total_n));
  TLR_CHECK(dalloc(&B.b32, (size_t)B.total_n));
  {
    std::vector<uint64_t> hD((size_t)d_off[count]);
    for (int p = 0; p < count; p++) {
      const Factor& F = *B.F[p];
      for (int64_t t = 0; t < (int64_t)B.M * (F.n + 1); t++) hD[d_off[p] + t] = splitmix64_seed_at(o.seed + p, t);
      for (int64_t t = 0; t < F.n; t++) perm_g[B.n_off[p] + t] = B.n_off[p] + F.perm[t];
      const BatchCopies& C = B.copies[p];
      BatchProblem& P = probs[p];
      P.n = (int)F.n;
      P.r = F.r;
      P.m = F.m;
      P.n_shifts = B.M;
      P.n_points = B.N;
      P.ldbt = F.ldbt;
      P.ktot = F.ktot;
      P.logp_off = S * p;
      P.nu = nu[p];
      P.periodize = B.periodize;
      P.tile_off = C.tile_off;
      P.krow_off = C.krow_off;
      P.kcol_off = C.kcol_off;
      P.vt_off = C.vt_off;
      P.kcpad = C.kcpad;
      P.BT = F.BT32;
      P.inv = F.inv32;
      P.band = F.band32;
      P.UT = C.UT;
      P.VT = C.VT;
      P.vmap = F.vmap;
      P.Q = F.Q;
      P.D = B.D + d_off[p];
      P.a = B.a32 + B.n_off[p];
      P.b = B.b32 + B.n_off[p];
    }
    TLR_CUDA(cudaMemcpyAsync(B.D, hD.data(), hD.size() * 8, cudaMemcpyHostToDevice, st));
    TLR_CUDA(cudaStreamSynchronize(st));
  }
  // work items, largest problems first
  std::vector<int> order(count);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return B.F[x]->n > B.F[y]->n; });
  std::vector<BatchItem> items;
  for (int p : order)
    for (int64_t c0 = 0; c0 < S; c0 += BATCH_T) items.push_back(BatchItem{p, (int)std::min<int64_t>(BATCH_T, S - c0), c0});
  B.n_items = (int)items.size();
  TLR_CHECK(dalloc(&B.dprobs, count));
  TLR_CHECK(dalloc(&B.ditems, items.size()));
  TLR_CHECK(dalloc(&B.perm_g, (size_t)B.total_n));
  TLR_CUDA(cudaMemcpyAsync(B.dprobs, probs.data(), probs.size() * sizeof(BatchProblem), cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaMemcpyAsync(B.ditems, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaMemcpyAsync(B.perm_g, perm_g.data(), perm_g.size() * 8, cudaMemcpyHostToDevice, st));
  // persistent grid (all the CTAs that fit, until tuned) and its private projection buffers
  TLR_CUDA(cudaDeviceGetAttribute(&B.sms, cudaDevAttrMultiProcessorCount, B.device));
  if (B.tc) {
    const void* kt = batch_tc_kernel(B.periodize);
    TLR_CUDA(cudaFuncSetAttribute(kt, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared));
    // resident CTAs from the kernel's registers and shared memory (the occupancy query
    // reported one CTA per SM for this kernel where the launches fit six), and at most
    // 512 / 64 per SM: each holds its 64 TMEM columns until the end
    TLR_CHECK(resident_ctas(kt, STC_NS, sweep_tc_smem_bytes<1>(), B.device, &B.per_sm_max));
    B.per_sm_max = std::min(B.per_sm_max, 512 / STC_SUB);
  } else {
    const size_t smem = batch_smem();
    TLR_CHECK(raise_smem_limit((const void*)k_batch, (size_t)smem));
    TLR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&B.per_sm_max, k_batch, BATCH_T, smem));
  }
  B.per_sm_max = std::max(B.per_sm_max, 1);
  B.grid_max = std::max(1, std::min(B.per_sm_max * B.sms, B.n_items));
  if (B.tc) {
    // CTA-private W (kwmax rank rows x 128 samples) and sample-major y (128 rows of
    // 2 x 128 hi / lo columns), zeroed once: padding rows and columns meet zero
    // operand entries and must stay finite
    B.kwmax = std::max<int64_t>(B.kwmax, 64);
    if ((int64_t)B.grid_max * B.kwmax >= ((int64_t)1 << 31))
      return fail(TLRMVN_E_NOTSUP, "batched projections exceed the tensor map's coordinate range");
    const size_t nw = (size_t)B.grid_max * B.kwmax * STC_NS, ny = (size_t)B.grid_max * STC_NS * 2 * B.my;
    TLR_CHECK(dalloc(&B.W16, nw));
    TLR_CHECK(dalloc(&B.Y16, ny));
    TLR_CHECK(dalloc(&B.derr, 1));
    TLR_CUDA(cudaMemsetAsync(B.W16, 0, nw * 2, st));
    TLR_CUDA(cudaMemsetAsync(B.Y16, 0, ny * 2, st));
    TLR_CUDA(cudaMemsetAsync(B.derr, 0, sizeof(int), st));
    TLR_CHECK(make_tensor_map_16(&B.mapW, B.W16, STC_NS, (uint64_t)B.grid_max * B.kwmax, STC_NS * 2, 64, 64, false));
    TLR_CHECK(make_tensor_map_16(&B.mapY, B.Y16, 2 * B.my, (uint64_t)B.grid_max * STC_NS, 2 * B.my * 2,
                                 STC_NS, 32, false));
    TLR_CHECK(make_tensor_map_16(&B.mapY64, B.Y16, 2 * B.my, (uint64_t)B.grid_max * STC_NS, 2 * B.my * 2, STC_NS,
                                 64, false));
    // per problem: the split B, U and V maps, and its table entry
    std::vector<CUtensorMap> maps((size_t)BATCH_TC_MAPS * count);
    std::vector<BatchTcProblem> tp(count);
    for (int p = 0; p < count; p++) {
      const Factor& F = *B.F[p];
      const int64_t ly = 2 * F.my16;
      CUtensorMap* mp = &maps[(size_t)BATCH_TC_MAPS * p];
      TLR_CHECK(make_tensor_map_16(&mp[0], F.B16x2, ly, (uint64_t)F.r * F.m, ly * 2, 64, 32, false));
      if (F.ktot) {
        TLR_CHECK(make_tensor_map_16(&mp[1], F.U16, F.kmax16, (uint64_t)F.r * F.m, F.kmax16 * 2, 64, 64, false));
        TLR_CHECK(make_tensor_map_16(&mp[2], F.V16, F.my16, F.ktot, F.my16 * 2, 64, 64, false));
      } else {
        mp[1] = B.mapW;  // (never read: no tile has ranks)
        mp[2] = B.mapW;
      }
      const BatchProblem& P = probs[p];
      BatchTcProblem& T = tp[p];
      T.n = P.n;
      T.r = P.r;
      T.m = P.m;
      T.my = (int)F.my16;
      T.n_points = P.n_points;
      T.ldbt = P.ldbt;
      T.logp_off = P.logp_off;
      T.nu = P.nu;
      T.tile_off = P.tile_off;
      T.kpad_off = B.copies[p].kpad_off;
      T.krow_off = P.krow_off;
      T.kcol_off = P.kcol_off;
      T.vmap16 = F.vmap16;
      T.BT = P.BT;
      T.inv = P.inv;
      T.band = P.band;
      T.Q = P.Q;
      T.D = P.D;
      T.a = P.a;
      T.b = P.b;
    }
    TLR_CHECK(dalloc(&B.dmaps, maps.size()));
    TLR_CHECK(dalloc(&B.dtprobs, count));
    TLR_CUDA(cudaMemcpyAsync(B.dmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice, st));
    TLR_CUDA(cudaMemcpyAsync(B.dtprobs, tp.data(), tp.size() * sizeof(BatchTcProblem), cudaMemcpyHostToDevice, st));
  } else {
    TLR_CHECK(dalloc(&B.W, (size_t)B.grid_max * std::max<int64_t>(B.ktot_max, 1) * BATCH_T));
  }
  TLR_CHECK(dalloc(&B.dnext, 1));
  TLR_CHECK(dalloc(&B.dbad, 1));
  TLR_CHECK(dalloc(&B.logP, (size_t)B.total_samples));
  TLR_CHECK(dalloc(&B.ell, (size_t)count * B.M));
  TLR_CHECK(dalloc(&B.out, (size_t)count * 2));
  TLR_CHECK(dalloc(&B.a_st, (size_t)B.total_n));
  TLR_CHECK(dalloc(&B.b_st, (size_t)B.total_n));
  TLR_CUDA(cudaMallocHost(&B.h_ab, (size_t)B.total_n * 2 * 8));
  TLR_CUDA(cudaMallocHost(&B.h_out, (size_t)count * 2 * 8 + 16));
  TLR_CUDA(cudaStreamSynchronize(st));
  return batch_capture(B, B.per_sm_max);
}

static int batch_run(Batch& B, const double* const* a, const double* const* b, double* logp, double* err) {
  int cur = 0;
  cudaGetDevice(&cur);
  TLR_CUDA(cudaSetDevice(B.device));
  for (int p = 0; p < B.count; p++) {
    if (!a[p] || !b[p]) return fail(TLRMVN_E_INVAL, "null limits in batch");
    std::copy(a[p], a[p] + B.F[p]->n, B.h_ab + B.n_off[p]);
    std::copy(b[p], b[p] + B.F[p]->n, B.h_ab + B.total_n + B.n_off[p]);
  }
  cudaStream_t st = B.st;
  TLR_CUDA(cudaMemcpyAsync(B.a_st, B.h_ab, B.total_n * 8, cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaMemcpyAsync(B.b_st, B.h_ab + B.total_n, B.total_n * 8, cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaGraphLaunch(B.exec, st));
  TLR_CUDA(cudaMemcpyAsync(B.h_out, B.out, (size_t)B.count * 2 * 8, cudaMemcpyDeviceToHost, st));
  TLR_CUDA(cudaMemcpyAsync(B.h_out + 2 * B.count, B.dbad, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (B.tc) TLR_CUDA(cudaMemcpyAsync(B.h_out + 2 * B.count + 1, B.derr, sizeof(int), cudaMemcpyDeviceToHost, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  int bad = 0, terr = 0;
  memcpy(&bad, B.h_out + 2 * B.count, sizeof(int));
  if (B.tc) memcpy(&terr, B.h_out + 2 * B.count + 1, sizeof(int));
  cudaSetDevice(cur);
  if (bad) return fail(TLRMVN_E_INVAL, "limits must satisfy a_i <= b_i, a_i < +inf, b_i > -inf, no NaN");
  if (terr)
    return fail(TLRMVN_E_TIMEOUT, "tensor-core batched kernel gave up waiting (code " + std::to_string(terr) + ")");
  for (int p = 0; p < B.count; p++) {
    logp[p] = B.h_out[2 * p];
    err[p] = B.h_out[2 * p + 1];
  }
  return TLRMVN_OK;
}

static int check_batch_opts(int count, const tlrmvn_factor_t* f, const double* nu, const tlrmvn_opts* o) {
  if (count < 1 || !f || !nu || !o) return fail(TLRMVN_E_INVAL, "bad batch arguments");
  if (o->n_shifts < 1 || o->n_points < 1) return fail(TLRMVN_E_INVAL, "n_shifts and n_points must be >= 1");
  if (o->precision != TLRMVN_FP32 && o->precision != TLRMVN_BF16_SHIFT)
    return fail(TLRMVN_E_NOTSUP, "the batched integrand runs in TLRMVN_FP32 or TLRMVN_BF16_SHIFT");
  if (o->shifts) return fail(TLRMVN_E_NOTSUP, "batched problems draw their shifts from opts.seed + problem index");
  return TLRMVN_OK;
}

}  // namespace tlrmvn

using namespace tlrmvn;

extern "C" int tlrmvn_batch_create(int count, const tlrmvn_factor_t* factors, const double* nu,
                                   const tlrmvn_opts* opts, tlrmvn_batch_t* out) {
  if (!out) return fail(TLRMVN_E_INVAL, "null output");
  TLR_CHECK(check_batch_opts(count, factors, nu, opts));
  Batch* B = new Batch();
  int s = batch_build(*B, count, factors, nu, *opts);
  if (s != TLRMVN_OK) {
    delete B;
    return s;
  }
  *out = reinterpret_cast<tlrmvn_batch_t>(B);
  return TLRMVN_OK;
}

extern "C" int tlrmvn_batch_run(tlrmvn_batch_t plan, const double* const* a, const double* const* b, double* logp,
                                double* err) {
  if (!plan || !a || !b || !logp || !err) return fail(TLRMVN_E_INVAL, "null argument");
  return batch_run(*reinterpret_cast<Batch*>(plan), a, b, logp, err);
}

extern "C" int tlrmvn_batch_tune(tlrmvn_batch_t plan, const double* const* a, const double* const* b,
                                 const char* cache_path, int force, int* ctas_per_sm, double* ms) {
  if (!plan || !a || !b) return fail(TLRMVN_E_INVAL, "null argument");
  Batch& B = *reinterpret_cast<Batch*>(plan);
  // cache key: device, problems, total dimension, total rank, shifts x points
  std::string key;
  {
    cudaDeviceProp prop;
    std::string dev = "unknown";
    if (cudaGetDeviceProperties(&prop, B.device) == cudaSuccess) dev = prop.name;
    for (char& c : dev)
      if (c == ' ') c = '_';
    int64_t ksum = 0;
    for (Factor* F : B.F) ksum += F->ktot;
    key = dev + (B.tc ? " batch-bf16 c" : " batch c") + std::to_string(B.count) + " n" + std::to_string(B.total_n) + " k" +
          std::to_string(ksum) + " s" + std::to_string((int64_t)B.M * B.N);
  }
  int best = -1;
  double best_ms = -1.0;
  if (!force && cache_path && *cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      const size_t bar = line.find(" | ");
      if (bar == key.size() && line.compare(0, bar, key) == 0) best = atoi(line.c_str() + bar + 3);
    }
  }
  if (best >= 1) {
    TLR_CHECK(batch_capture(B, best));
  } else {
    std::vector<double> lp(B.count), er(B.count);
    cudaEvent_t e0, e1;
    TLR_CUDA(cudaEventCreate(&e0));
    TLR_CUDA(cudaEventCreate(&e1));
    int s = TLRMVN_OK;
    for (int k = 1; k <= B.per_sm_max && s == TLRMVN_OK; k++) {
      s = batch_capture(B, k);
      if (s == TLRMVN_OK) s = batch_run(B, a, b, lp.data(), er.data());  // untimed
      float t = 0.0f;
      if (s == TLRMVN_OK) {
        cudaEventRecord(e0, B.st);
        s = batch_run(B, a, b, lp.data(), er.data());
        cudaEventRecord(e1, B.st);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t, e0, e1);
      }
      if (s == TLRMVN_OK && (best < 0 || t < best_ms)) {
        best = k;
        best_ms = t;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    TLR_CHECK(s);
    TLR_CHECK(batch_capture(B, best));
    if (cache_path && *cache_path) {
      FILE* f = fopen(cache_path, "a");
      if (f) {
        fprintf(f, "%s | %d # %.4f ms\n", key.c_str(), best, best_ms);
        fclose(f);
      }
    }
  }
  if (ctas_per_sm) *ctas_per_sm = B.per_sm;
  if (ms) *ms = best_ms;
  return TLRMVN_OK;
}

extern "C" int tlrmvn_batch_free(tlrmvn_batch_t plan) {
  delete reinterpret_cast<Batch*>(plan);
  return TLRMVN_OK;
}

extern "C" int tlrmvn_prob_batch(int count, const tlrmvn_factor_t* factors, const double* const* a,
                                 const double* const* b, const double* nu, const tlrmvn_opts* opts, double* logp,
                                 double* err) {
  tlrmvn_batch_t plan = nullptr;
  TLR_CHECK(tlrmvn_batch_create(count, factors, nu, opts, &plan));
  int s = tlrmvn_batch_run(plan, a, b, logp, err);
  tlrmvn_batch_free(plan);
  return s;
}
