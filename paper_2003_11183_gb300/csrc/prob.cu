// The TLR quasi-Monte Carlo integrand (Algorithms 6 and 7) and its estimator.
//
// For a chunk of C samples (shift-major sample index g = s*N + k-1) the
// integrand walks the diagonal tiles i = 0..r-1:
//   1. low-rank shift   Delta_i = Ucat_i * W_row_i         (m x C)   [Algorithm 6, shift of the limits]
//   2. diagonal sweep   per sample, eq. (2) on tile B_i with limits r_s b - Delta - s
//                       -> y_i (m x C) and the log of the tile's product
//   3. projection       W_col_i = Vcat_i * y_i   scattered into W (ktot x C)
// Step 1 accumulates, in one product, the sums that Algorithm 6 adds tile by
// tile after every diagonal block: sum_{j<i} U_ij (V_ij^T y_j).  Student-t
// problems first scale the limits by chi_nu^-1(w0)/sqrt(nu) per sample (Algorithm 7).
// Per-sample logs are reduced per shift by a log-sum-exp and then across shifts (Section 2.1).
#include "common.cuh"
#include "gemm.cuh"
#include "sov_device.cuh"
#include "sweep.cuh"
#include "sweep_tc.cuh"
#include "tcgen05.cuh"

#include <cudaTypedefs.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

namespace tlrmvn {

// ---- Student-t scale (Algorithm 7): chi_nu^-1(w0)/sqrt(nu) ------------------------
__global__ void k_chi_scale(double* rs, float* rs32, const uint64_t* Q, const uint64_t* D, int64_t ldD,
                            int64_t coord, int64_t sample0, int64_t N, int64_t C, double nu, int periodize) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  int64_t g = sample0 + c, s = g / N;
  uint64_t k = (uint64_t)(g - s * N) + 1;
  double w, wc;
  lattice_w(k * Q[coord] + D[s * ldD + coord], periodize, w, wc);
  double x = gamma_p_inv(0.5 * nu, w, wc);
  double r = sqrt(2.0 * x / nu);
  if (rs) rs[c] = r;
  if (rs32) rs32[c] = (float)r;
}

// ---- limits: permute to factor order and validate ---------------------------------
__global__ void k_permute_limits(const double* a, const double* b, const int64_t* perm, int64_t n, double* ap,
                                 double* bp, float* ap32, float* bp32, int* bad) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  double av = a[perm[t]], bv = b[perm[t]];
  if (isnan(av) || isnan(bv) || av > bv || av == INFINITY || bv == -INFINITY) atomicExch(bad, 1);
  if (av != -INFINITY) atomicExch(bad + 1, 1);  // a finite lower limit: not a one-sided problem
  ap[t] = av;
  bp[t] = bv;
  if (ap32) {
    ap32[t] = (float)av;
    bp32[t] = (float)bv;
  }
}

// ---- diagonal-tile sweep (eq. 2 on B_i, Algorithm 6 inner call) -------------------
template <typename T, typename YT>
struct DiagArgs {
  const T* B;
  int mt, ldb;
  const T* Delta;   // m x C sample-major, or null (no earlier tiles)
  int64_t ldd;
  const double* a;  // the tile's limits, factor order
  const double* b;
  const double* rs;  // per-sample Student-t scale or null
  const uint64_t* Q;
  const uint64_t* D;
  int64_t ldD, coord0, sample0, N, C;
  int periodize, first;
  YT* Y;
  int64_t ldy;
  double* logP;  // all samples
};

__device__ __forceinline__ void put_y(double* Y, int64_t i, double y) { Y[i] = y; }
__device__ __forceinline__ void put_y(float* Y, int64_t i, float y) { Y[i] = y; }
__device__ __forceinline__ void put_y(__nv_bfloat16* Y, int64_t i, float y) { Y[i] = __float2bfloat16_rn(y); }

// One thread per sample; the tile's y values of the thread's sample live in shared
// memory (column tid of a [mt][blockDim+1] array); B_i rows are read through L1
// as warp-uniform broadcasts.  Y layout:
//   SAMPLE_MAJOR = false: Y[v * ldy + c]  (variable-major, written as produced)
//   SAMPLE_MAJOR = true:  Y[c * ldy + v]  (each sample's y contiguous: the K-major
//                         operand of the tensor-core projection), written at the
//                         end of the tile from shared memory, a row per warp pass.
template <typename T, typename YT, bool SAMPLE_MAJOR>
__global__ void k_diag(DiagArgs<T, YT> p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ys = reinterpret_cast<T*>(smem_raw);
  const int bd = blockDim.x, tid = threadIdx.x, ld = bd + 1;
  const int64_t c0 = (int64_t)blockIdx.x * bd;
  const int64_t c = c0 + tid;
  const bool active = c < p.C;
  if (active) {
    const int64_t g = p.sample0 + c;
    const int64_t s = g / p.N;
    const uint64_t k = (uint64_t)(g - s * p.N) + 1;
    const uint64_t* Ds = p.D + s * p.ldD + p.coord0;
    const uint64_t* Qt = p.Q + p.coord0;
    const T rs = p.rs ? (T)p.rs[c] : (T)1;
    T lp = 0;
    for (int v = 0; v < p.mt; v++) {
      const T* Brow = p.B + (int64_t)v * p.ldb;
      T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
      int u = 0;
      for (; u + 4 <= v; u += 4) {
        s0 = fma(__ldg(Brow + u), ys[(u)*ld + tid], s0);
        s1 = fma(__ldg(Brow + u + 1), ys[(u + 1) * ld + tid], s1);
        s2 = fma(__ldg(Brow + u + 2), ys[(u + 2) * ld + tid], s2);
        s3 = fma(__ldg(Brow + u + 3), ys[(u + 3) * ld + tid], s3);
      }
      for (; u < v; u++) s0 = fma(__ldg(Brow + u), ys[u * ld + tid], s0);
      const T sum = (s0 + s1) + (s2 + s3);
      const T dl = p.Delta ? p.Delta[(int64_t)v * p.ldd + c] : (T)0;
      const T lvv = __ldg(Brow + v);
      const T at = ((T)p.a[v] * rs - dl - sum) / lvv;
      const T bt = ((T)p.b[v] * rs - dl - sum) / lvv;
      double w, wc;
      lattice_w(k * Qt[v] + Ds[v], p.periodize, w, wc);
      T lv, y;
      sov_step<T>(at, bt, (T)w, (T)wc, lv, y);
      lp += lv;
      ys[v * ld + tid] = y;
      if (!SAMPLE_MAJOR) put_y(p.Y, (int64_t)v * p.ldy + c, y);
    }
    if (p.first) p.logP[g] = (double)lp;
    else p.logP[g] += (double)lp;
  }
  if (SAMPLE_MAJOR) {
    __syncthreads();
    const int nw = bd >> 5, warp = tid >> 5, lane = tid & 31;
    for (int j = warp; j < bd; j += nw) {
      if (c0 + j >= p.C) break;
      YT* row = p.Y + (c0 + j) * p.ldy;
      for (int v = lane; v < p.mt; v += 32) put_y(row, v, ys[v * ld + j]);
    }
  }
}

// BT32[i][u][v] = B[i][v][u] (zero for v >= m), inv32[i][v] = 1 / B[i][v][v]
__global__ void k_transpose_tiles(const double* B, int m, int64_t ldbt, int64_t count, float* BT, float* inv) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int64_t i = t / ((int64_t)m * ldbt), rem = t % ((int64_t)m * ldbt);
  int64_t u = rem / ldbt, v = rem % ldbt;
  const double* Bi = B + i * (int64_t)m * m;
  BT[t] = (v < m) ? (float)Bi[v * m + u] : 0.0f;
  if (v == u && v < m) inv[i * m + v] = (float)(1.0 / Bi[v * m + v]);
}

// ---- reductions (Section 2.1 estimator, in logs) -----------------------------------
// Block-wide reduction; `ident` pads the lanes beyond the warp count.
template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T* sh, T ident) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  v = threadIdx.x < nw ? sh[threadIdx.x] : ident;
  if (wid == 0)
    for (int o = 16; o; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (threadIdx.x == 0) sh[0] = v;
  __syncthreads();
  v = sh[0];
  __syncthreads();
  return v;
}
struct MaxOp {
  __device__ double operator()(double a, double b) const { return a > b ? a : b; }
};
struct SumOp {
  __device__ double operator()(double a, double b) const { return a + b; }
};

// ell_s = log((1/N) sum_k exp(logP_{s,k})) for shift s = blockIdx.x.
__global__ void k_shift_reduce(const double* logP, int64_t N, double* ell) {
  __shared__ double sh[32];
  const double* L = logP + (int64_t)blockIdx.x * N;
  double mx = -INFINITY;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) mx = fmax(mx, L[i]);
  mx = block_reduce(mx, MaxOp(), sh, (double)-INFINITY);
  double sum = 0.0;
  if (mx > -INFINITY)
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) sum += exp(L[i] - mx);
  sum = block_reduce(sum, SumOp(), sh, 0.0);
  if (threadIdx.x == 0) ell[blockIdx.x] = (mx > -INFINITY) ? mx + log(sum) - log((double)N) : -INFINITY;
}

// log p_hat = log((1/M) sum_s exp(ell_s)); err = SD_s(exp ell_s)/(sqrt(M) p_hat).
__device__ void final_estimate(const double* ell, int M, double* logp, double* errp) {
  __shared__ double sh[32];
  double mx = -INFINITY;
  for (int s = threadIdx.x; s < M; s += blockDim.x) mx = fmax(mx, ell[s]);
  mx = block_reduce(mx, MaxOp(), sh, (double)-INFINITY);
  double sum = 0.0;
  if (mx > -INFINITY)
    for (int s = threadIdx.x; s < M; s += blockDim.x) sum += exp(ell[s] - mx);
  sum = block_reduce(sum, SumOp(), sh, 0.0);
  double mean = sum / M;
  double sq = 0.0;
  if (mx > -INFINITY)
    for (int s = threadIdx.x; s < M; s += blockDim.x) {
      double d = exp(ell[s] - mx) - mean;
      sq += d * d;
    }
  sq = block_reduce(sq, SumOp(), sh, 0.0);
  if (threadIdx.x == 0) {
    *logp = (mx > -INFINITY) ? mx + log(sum) - log((double)M) : -INFINITY;
    *errp = (M > 1 && mx > -INFINITY) ? sqrt(sq / (M - 1) / M) / mean : NAN;
  }
}
__global__ void k_final(const double* ell, int M, double* logp, double* errp) { final_estimate(ell, M, logp, errp); }
// one problem per block: ell + blockIdx.x * M -> out[2 * blockIdx.x], out[2 * blockIdx.x + 1]
__global__ void k_final_batch(const double* ell, int M, double* out) {
  final_estimate(ell + (int64_t)blockIdx.x * M, M, out + 2 * blockIdx.x, out + 2 * blockIdx.x + 1);
}

template <typename S, typename D>
__global__ void k_convert(const S* src, D* dst, int64_t count) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = (D)src[i];
}
// U16[(i*m + v) * kmax + k] = Ucat_i[v][k] for k < Krow_i, else 0
__global__ void k_pad_u16(const double* Ucat, const int64_t* krow_off, int m, int64_t kmax, int64_t count,
                          __nv_bfloat16* U16) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int64_t row = t / kmax, k = t % kmax;
  int64_t i = row / m, v = row % m;
  int64_t Kr = krow_off[i + 1] - krow_off[i];
  U16[t] = (k < Kr) ? __double2bfloat16(Ucat[(int64_t)m * krow_off[i] + v * Kr + k]) : __float2bfloat16(0.f);
}
// V16[row * my + u] = Vcat[row][u] for u < m, else 0
__global__ void k_pad_v16(const double* Vcat, int m, int64_t my, int64_t count, __nv_bfloat16* V16) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  int64_t row = t / my, u = t % my;
  V16[t] = (u < m) ? __double2bfloat16(Vcat[row * m + u]) : __float2bfloat16(0.f);
}

// B16x2[(i*m + v) * 2my + h*my + u]: h = 0 hi = bf16(B_i[v][u]), h = 1 lo = bf16(B_i[v][u] - hi)
__global__ void k_split_b16(const double* B, int m, int64_t my, int64_t count, __nv_bfloat16* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t row = t / (2 * my), c = t % (2 * my);
  const int64_t u = c % my, h = c / my, i = row / m, v = row % m;
  const double b = (u < m) ? B[(i * m + v) * m + u] : 0.0;
  const __nv_bfloat16 hi = __double2bfloat16(b);
  out[t] = h ? __double2bfloat16(b - (double)__bfloat162float(hi)) : hi;
}

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Largest |B| over all diagonal tiles (non-negative doubles order as their bit patterns).
__global__ void k_absmax(const double* x, int64_t count, unsigned long long* out) {
  double mx = 0.0;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(x[t]));
  for (int o = 16; o; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// FP16-shift operands.  Largest |entry| of each Ucat column (rank) of every row
// tile, and of each Vcat row: out[g] for global rank index g (Ucat columns in
// krow order, Vcat rows in kcol order).
__global__ void k_rank_absmax_u(const double* Ucat, const int64_t* krow_off, const int32_t* ktile, int m,
                                int64_t ktot, double* out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ktot) return;
  const int i = ktile[g];
  const int64_t Kr = krow_off[i + 1] - krow_off[i], k = g - krow_off[i];
  const double* col = Ucat + (int64_t)m * krow_off[i] + k;
  double mx = 0.0;
  for (int v = 0; v < m; v++) mx = fmax(mx, fabs(col[(int64_t)v * Kr]));
  out[g] = mx;
}
__global__ void k_rank_absmax_v(const double* Vcat, int m, int64_t ktot, double* out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ktot) return;
  double mx = 0.0;
  for (int u = 0; u < m; u++) mx = fmax(mx, fabs(Vcat[g * m + u]));
  out[g] = mx;
}
// U16h[(i*m + v) * kmax + k] = fp16(Ucat_i[v][k] su[krow_off[i] + k]) for k < Krow_i, else 0
__global__ void k_pad_u16h(const double* Ucat, const int64_t* krow_off, const float* su, int m, int64_t kmax,
                           int64_t count, __half* U16h) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t row = t / kmax, k = t % kmax, i = row / m, v = row % m;
  const int64_t Kr = krow_off[i + 1] - krow_off[i];
  U16h[t] = (k < Kr) ? __double2half(Ucat[(int64_t)m * krow_off[i] + v * Kr + k] * (double)su[krow_off[i] + k])
                     : __float2half(0.f);
}
// V16h[row * my + u] = fp16(Vcat[row][u] sv[row]) for u < m, else 0
__global__ void k_pad_v16h(const double* Vcat, const float* sv, int m, int64_t my, int64_t count, __half* V16h) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t row = t / my, u = t % my;
  V16h[t] = (u < m) ? __double2half(Vcat[row * m + u] * (double)sv[row]) : __float2half(0.f);
}
// B16x2h: as B16x2 for B g, fp16 hi = fp16(B_i[v][u] g) and lo = fp16(B_i[v][u] g - hi)
__global__ void k_split_b16h(const double* B, double g, int m, int64_t my, int64_t count, __half* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t row = t / (2 * my), c = t % (2 * my);
  const int64_t u = c % my, h = c / my, i = row / m, v = row % m;
  const double b = (u < m) ? B[(i * m + v) * m + u] * g : 0.0;
  const __half hi = __double2half(b);
  out[t] = h ? __double2half(b - (double)__half2float(hi)) : hi;
}

// float32 diagonal tiles: row-major B32, transposed BT32 (ld ldbt), reciprocal diagonal inv32
// band32[(i*m + v)*16 + k] = B_i[v+1+k][v] (k < 15, v+1+k < m), else 0
__global__ void k_make_band(const double* B, int m, int64_t count, float* band) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  const int64_t row = t / 16, k = t % 16, i = row / m, v = row % m, u = v + 1 + k;
  band[t] = (k < 15 && u < m) ? (float)B[(i * m + u) * m + v] : 0.0f;
}

int ensure_float_tiles(Factor& F, cudaStream_t st) {
  if (F.B32 && F.BT32 && F.inv32 && F.band32) return TLRMVN_OK;
  dfree(F.B32);  // a failed earlier attempt may have left some of these behind
  dfree(F.BT32);
  dfree(F.inv32);
  dfree(F.band32);
  const int64_t nb = (int64_t)F.r * F.m * F.m;
  TLR_CHECK(dalloc(&F.B32, nb));
  k_convert<double, float><<<blocks_for(nb, 256), 256, 0, st>>>(F.B, F.B32, nb);
  F.ldbt = ((int64_t)F.m + DIAG_VB - 1) / DIAG_VB * DIAG_VB;
  const int64_t nt = (int64_t)F.r * F.m * F.ldbt;
  TLR_CHECK(dalloc(&F.BT32, nt + DIAG_PAD));
  TLR_CUDA(cudaMemsetAsync(F.BT32 + nt, 0, DIAG_PAD * sizeof(float), st));
  TLR_CHECK(dalloc(&F.inv32, (size_t)F.r * F.m));
  k_transpose_tiles<<<blocks_for(nt, 256), 256, 0, st>>>(F.B, F.m, F.ldbt, nt, F.BT32, F.inv32);
  const int64_t nw = (int64_t)F.r * F.m * 16;
  TLR_CHECK(dalloc(&F.band32, nw));
  k_make_band<<<blocks_for(nw, 256), 256, 0, st>>>(F.B, F.m, nw, F.band32);
  TLR_CUDA(cudaGetLastError());
  return TLRMVN_OK;
}

// out[k * m + v] = U[v * kr + k] for k < kr, else 0 (one row tile's U, float, k-major,
// its ranks padded to a multiple of 8: ld8 rows)
__global__ void k_pad_u32t(const double* U, int64_t kr, int64_t m, int64_t cnt, float* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t k = t / m, v = t % m;
  out[t] = k < kr ? (float)U[v * kr + k] : 0.0f;
}
// out[v * kc4 + r] = Vt[r * m + v] for r < kc, else 0 (one column tile's V, float,
// variable-major, its ranks padded to a multiple of 4)
__global__ void k_pad_v32(const double* Vt, int64_t kc, int64_t kc4, int64_t m, int64_t cnt, float* out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int64_t v = t / kc4, r = t % kc4;
  out[t] = r < kc ? (float)Vt[r * m + v] : 0.0f;
}

// Makes the copies a precision needs; the first caller makes them (and waits for
// them) under the factor's lock, so concurrent streams never see a partial copy.
static int ensure_copies_locked(Factor& F, int precision, cudaStream_t st);
static bool bf16_ready(const Factor& F) {
  return !F.kpad_off.empty() && (F.ktot == 0 || (F.U16 && F.V16 && F.vmap16)) && F.B16x2;
}
static bool fp16_ready(const Factor& F) {
  return bf16_ready(F) && (F.ktot == 0 || (F.U16h && F.V16h && F.wscale16)) && F.B16x2h;
}
static bool copies_ready(const Factor& F, int precision) {
  if (precision == TLRMVN_FP64) return true;
  if (!F.B32 || !F.BT32 || !F.inv32 || !F.band32) return false;
  if (precision == TLRMVN_FP32) return (F.U32 && F.V32) || F.ktot == 0;
  if (precision == TLRMVN_FP16_SHIFT) return fp16_ready(F);
  return bf16_ready(F);
}
static int ensure_copies(Factor& F, int precision, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(F.copy_mu);
  if (copies_ready(F, precision)) return TLRMVN_OK;  // made and completed by an earlier call
  TLR_CHECK(ensure_copies_locked(F, precision, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  return TLRMVN_OK;
}
// FP16-shift operands with per-tile scaling (the factor's bf16 layout must exist).
// All products are of the factor scaled by one power of two g with max |B g| in
// (1/2, 1] (the probability and every y are unchanged by scaling the factor and
// the limits alike, and the sweep undoes g where it reads the products), so a
// covariance far from unit scale keeps fp16's range.  For each off-diagonal tile
// (i, j) with rank > 0: c_ij = 2^-ceil(log2 max|V_ij|) brings max |V c| into
// (1/2, 1]; a_ij = 2^-ceil(log2 max|U_ij g|) does the same for U g, and is
// raised, when needed, until the tile's projections fit fp16: a projection of
// the scaled V times the inverse 1 / (a c) is bounded by mt_j * 9 * max|V c| /
// (a c) (|y| < 9: the quantile of the lattice's smallest point), kept below
// 2^15.  A tile whose raised a would take max |U g a| above 2^15 cannot be held
// in fp16: TLRMVN_E_NOTSUP.
static int make_fp16_copies(Factor& F, cudaStream_t st) {
  dfree(F.U16h);
  dfree(F.V16h);
  dfree(F.B16x2h);
  dfree(F.wscale16);
  const int r = F.r, m = F.m;
  double g = 1.0;  // global scale: max |B g| in (1/2, 1]
  {
    unsigned long long* dmx = nullptr;
    TLR_CHECK(dalloc(&dmx, 1));
    unsigned long long hmx = 0;
    cudaError_t e = cudaMemsetAsync(dmx, 0, 8, st);
    if (e == cudaSuccess) {
      k_absmax<<<1024, 256, 0, st>>>(F.B, (int64_t)r * m * m, dmx);
      e = cudaMemcpyAsync(&hmx, dmx, 8, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(dmx);
    if (e != cudaSuccess) return cuda_fail(e, "fp16 copies: largest |B|");
    double mb;
    memcpy(&mb, &hmx, 8);
    if (mb > 0.0) g = std::ldexp(1.0, -(int)std::ceil(std::log2(mb)));
    const int64_t nb2 = (int64_t)r * m * 2 * F.my16;
    TLR_CHECK(dalloc(&F.B16x2h, nb2));
    k_split_b16h<<<blocks_for(nb2, 256), 256, 0, st>>>(F.B, g, m, F.my16, nb2, F.B16x2h);
    F.inv_g16 = (float)(1.0 / g);
  }
  if (F.ktot == 0) return TLRMVN_OK;
  std::vector<int32_t> ktile(F.ktot);
  for (int i = 0; i < r; i++)
    for (int64_t g = F.krow_off[i]; g < F.krow_off[i + 1]; g++) ktile[g] = i;
  int32_t* dkt = nullptr;
  int64_t* dkro = nullptr;
  double* dmax = nullptr;
  float *dsu = nullptr, *dsv = nullptr;
  auto cleanup = [&] {
    dfree(dkt);
    dfree(dkro);
    dfree(dmax);
    dfree(dsu);
    dfree(dsv);
  };
  int s = dalloc(&dkt, (size_t)F.ktot);
  if (s == TLRMVN_OK) s = dalloc(&dkro, (size_t)r + 1);
  if (s == TLRMVN_OK) s = dalloc(&dmax, (size_t)2 * F.ktot);
  if (s != TLRMVN_OK) {
    cleanup();
    return s;
  }
  std::vector<double> hmax(2 * F.ktot);
  cudaError_t e = cudaMemcpyAsync(dkt, ktile.data(), ktile.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dkro, F.krow_off.data(), (r + 1) * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_rank_absmax_u<<<blocks_for(F.ktot, 256), 256, 0, st>>>(F.Ucat, dkro, dkt, m, F.ktot, dmax);
    k_rank_absmax_v<<<blocks_for(F.ktot, 256), 256, 0, st>>>(F.Vcat, m, F.ktot, dmax + F.ktot);
    e = cudaMemcpyAsync(hmax.data(), dmax, hmax.size() * 8, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "fp16 copies: rank maxima");
  }
  std::vector<float> su(F.ktot), sv(F.ktot), ws(F.ktot);
  for (int j = 0; j < r; j++) {
    int64_t vrow = F.kcol_off[j];
    for (int i = j + 1; i < r; i++) {
      const int k = F.rank[(size_t)i * r + j];
      if (!k) continue;
      int64_t ucol = F.krow_off[i];
      for (int t = 0; t < j; t++) ucol += F.rank[(size_t)i * r + t];
      double mu = 0.0, mv = 0.0;
      for (int q = 0; q < k; q++) {
        mu = std::max(mu, hmax[ucol + q]);
        mv = std::max(mv, hmax[F.ktot + vrow + q]);
      }
      const double c = mv > 0.0 ? std::ldexp(1.0, -(int)std::ceil(std::log2(mv))) : 1.0;
      const double mug = mu * g;  // (the products are of the factor scaled by g)
      double a = mug > 0.0 ? std::ldexp(1.0, -(int)std::ceil(std::log2(mug))) : 1.0;
      const double bound = (double)F.tsize(j) * 9.0 * mv * c;  // |projection| before the inverse scale
      while (bound / (a * c) > 32768.0 && mug * a <= 16384.0) a *= 2.0;
      if (bound / (a * c) > 32768.0) {
        cleanup();
        return fail(TLRMVN_E_NOTSUP, "FP16 shifts: tile (" + std::to_string(i) + ", " + std::to_string(j) +
                                         ") exceeds fp16's range after scaling");
      }
      for (int q = 0; q < k; q++) {
        su[ucol + q] = (float)(a * g);
        sv[vrow + q] = (float)c;
        ws[vrow + q] = (float)(1.0 / (a * c));
      }
      vrow += k;
    }
  }
  s = dalloc(&dsu, (size_t)F.ktot);
  if (s == TLRMVN_OK) s = dalloc(&dsv, (size_t)F.ktot);
  if (s == TLRMVN_OK) s = dalloc(&F.wscale16, (size_t)F.ktot);
  const int64_t nu16 = (int64_t)r * m * F.kmax16, nv16 = F.ktot * F.my16;
  if (s == TLRMVN_OK) s = dalloc(&F.U16h, (size_t)nu16);
  if (s == TLRMVN_OK) s = dalloc(&F.V16h, (size_t)nv16);
  if (s != TLRMVN_OK) {
    cleanup();
    return s;
  }
  e = cudaMemcpyAsync(dsu, su.data(), su.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dsv, sv.data(), sv.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(F.wscale16, ws.data(), ws.size() * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_pad_u16h<<<blocks_for(nu16, 256), 256, 0, st>>>(F.Ucat, dkro, dsu, m, F.kmax16, nu16, F.U16h);
    k_pad_v16h<<<blocks_for(nv16, 256), 256, 0, st>>>(F.Vcat, dsv, m, F.my16, nv16, F.V16h);
    e = cudaStreamSynchronize(st);
  }
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "fp16 copies");
  return TLRMVN_OK;
}

static int ensure_copies_locked(Factor& F, int precision, cudaStream_t st) {
  const int64_t nu = (int64_t)F.m * F.ktot;
  if (precision != TLRMVN_FP64) TLR_CHECK(ensure_float_tiles(F, st));
  if (precision == TLRMVN_FP32 && !(F.U32 && F.V32) && nu) {
    dfree(F.U32);
    dfree(F.V32);
    // the first factors of the float products, k-major (a k-step of them is one plain
    // copy): U32 each row tile's U transposed, its rank count padded to a multiple of 8
    // (zero rows); V32 each column tile's V, its rank count padded to a multiple of 4
    F.u32_off.assign(F.r + 1, 0);
    F.v32_off.assign(F.r + 1, 0);
    for (int i = 0; i < F.r; i++) {
      F.u32_off[i + 1] = F.u32_off[i] + (int64_t)F.m * ((F.krow(i) + 7) / 8 * 8);
      F.v32_off[i + 1] = F.v32_off[i] + (int64_t)F.m * ((F.kcol(i) + 3) / 4 * 4);
    }
    TLR_CHECK(dalloc(&F.U32, (size_t)std::max<int64_t>(F.u32_off[F.r], 1)));
    TLR_CHECK(dalloc(&F.V32, (size_t)std::max<int64_t>(F.v32_off[F.r], 1)));
    for (int i = 0; i < F.r; i++) {
      const int64_t kr = F.krow(i), cnt = F.u32_off[i + 1] - F.u32_off[i];
      if (cnt)
        k_pad_u32t<<<blocks_for(cnt, 256), 256, 0, st>>>(F.Ucat + (size_t)F.m * F.krow_off[i], kr, F.m, cnt,
                                                         F.U32 + F.u32_off[i]);
      const int64_t kc = F.kcol(i), cntv = F.v32_off[i + 1] - F.v32_off[i];
      if (cntv)
        k_pad_v32<<<blocks_for(cntv, 256), 256, 0, st>>>(F.Vcat + (size_t)F.m * F.kcol_off[i], kc, (kc + 3) / 4 * 4,
                                                         F.m, cntv, F.V32 + F.v32_off[i]);
    }
  }
  if ((precision == TLRMVN_BF16_SHIFT || precision == TLRMVN_FP16_SHIFT) && !bf16_ready(F)) {
    // (a failed earlier attempt may have left some of these behind)
    dfree(F.U16);
    dfree(F.V16);
    dfree(F.vmap16);
    dfree(F.B16x2);
    // padded rank space: row tile i starts at a multiple of 64
    const int r = F.r, m = F.m;
    F.kpad_off.assign(r + 1, 0);
    int64_t kmax = 0;
    for (int i = 0; i < r; i++) {
      F.kpad_off[i + 1] = F.kpad_off[i] + (F.krow(i) + 63) / 64 * 64;
      kmax = std::max(kmax, F.krow(i));
    }
    F.kw16 = std::max<int64_t>(F.kpad_off[r], 64);
    F.kmax16 = std::max<int64_t>((kmax + 63) / 64 * 64, 64);
    F.my16 = ((int64_t)m + 63) / 64 * 64;
    {
      const int64_t nb2 = (int64_t)r * m * 2 * F.my16;
      TLR_CHECK(dalloc(&F.B16x2, nb2));
      k_split_b16<<<blocks_for(nb2, 256), 256, 0, st>>>(F.B, m, F.my16, nb2, F.B16x2);
    }
    if (F.ktot) {
      // vmap16: for each Vcat row, its column in the padded rank space
      std::vector<int32_t> v16(F.ktot);
      for (int j = 0; j < r; j++) {
        int64_t row = F.kcol_off[j];
        for (int i = j + 1; i < r; i++) {
          int64_t local = 0;
          for (int t = 0; t < j; t++) local += F.rank[(size_t)i * r + t];
          for (int c = 0; c < F.rank[(size_t)i * r + j]; c++) v16[row++] = (int32_t)(F.kpad_off[i] + local + c);
        }
      }
      TLR_CHECK(dalloc(&F.vmap16, (size_t)F.ktot));
      TLR_CUDA(cudaMemcpyAsync(F.vmap16, v16.data(), v16.size() * 4, cudaMemcpyHostToDevice, st));
      std::vector<int64_t> kro(F.krow_off);
      int64_t* dkro = nullptr;
      TLR_CHECK(dalloc(&dkro, kro.size()));
      TLR_CUDA(cudaMemcpyAsync(dkro, kro.data(), kro.size() * 8, cudaMemcpyHostToDevice, st));
      const int64_t nu16 = (int64_t)r * m * F.kmax16, nv16 = F.ktot * F.my16;
      TLR_CHECK(dalloc(&F.U16, nu16));
      TLR_CHECK(dalloc(&F.V16, nv16));
      k_pad_u16<<<blocks_for(nu16, 256), 256, 0, st>>>(F.Ucat, dkro, m, F.kmax16, nu16, F.U16);
      k_pad_v16<<<blocks_for(nv16, 256), 256, 0, st>>>(F.Vcat, m, F.my16, nv16, F.V16);
      TLR_CUDA(cudaStreamSynchronize(st));
      dfree(dkro);
    }
  }
  if (precision == TLRMVN_FP16_SHIFT && !fp16_ready(F)) TLR_CHECK(make_fp16_copies(F, st));
  TLR_CUDA(cudaGetLastError());
  return TLRMVN_OK;
}

// The bounded-wait path on its own: one thread waits on an mbarrier that nothing
// arrives at, `polls` times, and records code 6 when it gives up.
__global__ void k_wait_selftest(int* err, uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  tc::mbar_init(&bar, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc::mbar_wait(&bar, 0, err, 6, polls);
}

// ---- tensor maps for the tcgen05 shifts ---------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}
// 2-D map of a 16-bit tensor (bf16, or fp16 when f16; inner x outer, row pitch in
// bytes) with a box of box_inner (64: 128-byte swizzle, 32: 64-byte swizzle) x
// box_outer elements.
static int make_map(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch,
                    uint32_t box_outer, uint32_t box_inner = 64, bool f16 = false) {
  auto enc = tensor_map_encoder();
  if (!enc) return fail(TLRMVN_E_CUDA, "cuTensorMapEncodeTiled is not available");
  cuuint64_t dims[2] = {inner, outer};
  cuuint64_t strides[1] = {pitch};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t es[2] = {1, 1};
  CUresult r = enc(map, f16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void*>(base), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, box_inner == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TLRMVN_E_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
  return TLRMVN_OK;
}

// (for the batched integrand)
int ensure_precision_copies(Factor& F, int precision, cudaStream_t st) { return ensure_copies(F, precision, st); }
int make_tensor_map_16(CUtensorMap* map, const void* base, uint64_t inner, uint64_t outer, uint64_t pitch,
                       uint32_t box_outer, uint32_t box_inner, bool f16) {
  return make_map(map, base, inner, outer, pitch, box_outer, box_inner, f16);
}

// splitmix64 (S. Vigna): output number t of the generator started at `seed`.
uint64_t splitmix64_seed_at(uint64_t seed, uint64_t t);
static uint64_t splitmix64_at(uint64_t seed, uint64_t t) { return splitmix64_seed_at(seed, t); }
uint64_t splitmix64_seed_at(uint64_t seed, uint64_t t) {
  uint64_t z = seed + (t + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Freed scratch stays in the device's default memory pool between calls: a
// solve's scratch is several GB (the projections of all samples), and handing it
// back to the driver at every synchronisation, to map it again in the next call,
// cost more than 10% of a solve.
static void keep_pool_memory(int dev) {
  static std::mutex mu;
  static std::vector<int> done;
  std::lock_guard<std::mutex> g(mu);
  if (std::find(done.begin(), done.end(), dev) != done.end()) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  cudaGetLastError();
  done.push_back(dev);
}

// Scratch of one call, freed on every exit path (into the pool kept by keep_pool_memory).
struct Scratch {
  std::vector<void*> ptrs;
  cudaStream_t st;
  explicit Scratch(cudaStream_t s) : st(s) {
    int dev = 0;
    cudaGetDevice(&dev);
    keep_pool_memory(dev);
  }
  template <typename T>
  int get(T** p, size_t count) {
    *p = nullptr;
    if (!count) return TLRMVN_OK;
    cudaError_t e = cudaMallocAsync((void**)p, count * sizeof(T), st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(TLRMVN_E_NOMEM, "scratch allocation of " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    ptrs.push_back(*p);
    return TLRMVN_OK;
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
    cudaStreamSynchronize(st);
  }
};

// Samples per pass: opts.sample_chunk, else the factor's tuned chunk, else as
// many as keep the projection buffer W within 8 GiB (SIMT paths) or 32 GiB (bf16
// path); a multiple of 256.
static int64_t round_chunk(int64_t C, int64_t S) {
  C = std::min<int64_t>(C, S);
  return (C + 255) / 256 * 256;
}
static int64_t chunk_simt(const tlrmvn_opts& o, const Tuning& tu, int64_t S, int64_t ktot, int m, int64_t es) {
  if (o.sample_chunk > 0) return round_chunk(o.sample_chunk, S);
  if (tu.chunk > 0) return round_chunk(tu.chunk, S);
  const double budget = 8.0 * (1ull << 30);
  const double per = (double)(ktot + 2 * m) * es + 16.0;
  return round_chunk((int64_t)std::max(256.0, std::min((double)S, budget / per)), S);
}
static int64_t chunk_bf16(const tlrmvn_opts& o, const Tuning& tu, int64_t S, int64_t kw, int64_t ly) {
  if (o.sample_chunk > 0) return round_chunk(o.sample_chunk, S);
  if (tu.chunk > 0) return round_chunk(tu.chunk, S);
  const double budget = 32.0 * (1ull << 30);
  const double per = (double)kw * 2 + (double)ly * 2 + 16.0;
  return round_chunk((int64_t)std::max(256.0, std::min((double)S, budget / per)), S);
}

// Limits in factor order, in float64 and (for the float paths) float32.
struct Lims {
  const double* a;
  const double* b;
  const float* a32;
  const float* b32;
  bool one_sided;  // every lower limit is -inf
};

// Threads per block of the float64 sweep: as many as keep the sub-tile's y values
// of the block's samples within 64 KB of shared memory (at least one warp).
template <typename T>
static int diag_threads(int m) {
  int bd = 256;
  while (bd > 32 && (size_t)m * bd * sizeof(T) > 65536) bd >>= 1;
  return bd;
}

// Launch shape of the float sweep: samples per thread (spt) and per block (ns).
// Each sample's chain of special functions is latency-bound, so a launch takes
// (waves) x (time of one block) and a second wave for a few leftover blocks
// nearly doubles it.  Unless the factor's tuning fixes the block size, this
// takes, among blocks of 2 to 8 warps, the fewest waves over C samples
// (occupancy from the CUDA occupancy calculator, which accounts for registers
// and shared memory), and among those the one nearest 128 samples per block.
// One sample per thread (two per thread, k_diag_f32<2, .>, measured slower).
struct SweepShape {
  int spt, threads, ns;
};
typedef void (*SweepKernel)(DiagArgs32);
static SweepKernel sweep_kernel(int flags) {
  static const SweepKernel table[8] = {k_diag_f32<1, 0>, k_diag_f32<1, 1>, k_diag_f32<1, 2>, k_diag_f32<1, 3>,
                                       k_diag_f32<1, 4>, k_diag_f32<1, 5>, k_diag_f32<1, 6>, k_diag_f32<1, 7>};
  return table[flags & 7];
}
static SweepShape sweep_shape(int64_t C, int mt, int forced) {
  const int spt = 1;
  if (forced >= 32 && forced <= 256 && forced % 32 == 0) return SweepShape{spt, forced, forced * spt};
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  // one-entry memo per thread: a solve asks for the same (C, mt) once per sub-tile
  thread_local int64_t memo_c = -1;
  thread_local int memo_mt = -1, memo_dev = -1;
  thread_local SweepShape memo{1, 128, 128};
  if (memo_c == C && memo_mt == mt && memo_dev == dev) return memo;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  SweepShape best{spt, 128 / spt, 128};
  int64_t best_waves = INT64_MAX;
  for (int bd = 64 / spt; bd <= 256 / spt; bd += 32) {
    const int ns = bd * spt;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel(SWEEP_PERIODIZE | SWEEP_ONE_SIDED), bd,
                                                      sweep_smem_bytes(mt, ns)) !=
            cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      continue;
    }
    const int64_t blocks = (C + ns - 1) / ns, slots = (int64_t)per_sm * std::max(sms, 1);
    const int64_t waves = (blocks + slots - 1) / slots;
    if (waves < best_waves || (waves == best_waves && std::abs(ns - 128) < std::abs(best.ns - 128))) {
      best_waves = waves;
      best = SweepShape{spt, bd, ns};
    }
  }
  memo_c = C;
  memo_mt = mt;
  memo_dev = dev;
  memo = best;
  return best;
}
// The whole-tile sweep of the BF16- and FP16-shift paths, by (periodisation,
// one-sided) flags and operand type.
typedef void (*SweepTcKernel)(const CUtensorMap, const CUtensorMap, const CUtensorMap, const CUtensorMap,
                              const CUtensorMap, const CUtensorMap, SweepTcArgs);
static SweepTcKernel sweep_tc_kernel(int flags, bool f16, int spt) {
  static const SweepTcKernel table[16] = {
      k_sweep_tc<0, false, 1>, k_sweep_tc<SWEEP_PERIODIZE, false, 1>, k_sweep_tc<SWEEP_ONE_SIDED, false, 1>,
      k_sweep_tc<SWEEP_PERIODIZE | SWEEP_ONE_SIDED, false, 1>, k_sweep_tc<0, true, 1>,
      k_sweep_tc<SWEEP_PERIODIZE, true, 1>, k_sweep_tc<SWEEP_ONE_SIDED, true, 1>,
      k_sweep_tc<SWEEP_PERIODIZE | SWEEP_ONE_SIDED, true, 1>, k_sweep_tc<0, false, 2>,
      k_sweep_tc<SWEEP_PERIODIZE, false, 2>, k_sweep_tc<SWEEP_ONE_SIDED, false, 2>,
      k_sweep_tc<SWEEP_PERIODIZE | SWEEP_ONE_SIDED, false, 2>, k_sweep_tc<0, true, 2>,
      k_sweep_tc<SWEEP_PERIODIZE, true, 2>, k_sweep_tc<SWEEP_ONE_SIDED, true, 2>,
      k_sweep_tc<SWEEP_PERIODIZE | SWEEP_ONE_SIDED, true, 2>};
  return table[((flags & SWEEP_PERIODIZE) ? 1 : 0) | ((flags & SWEEP_ONE_SIDED) ? 2 : 0) | (f16 ? 4 : 0) |
               (spt == 2 ? 8 : 0)];
}
// Dynamic shared memory of a whole-tile sweep launch with `ctas` CTAs per SM: the
// kernel's own need, or more so that no more than `ctas` fit (tuning; with two
// samples per thread at most four fit by TMEM, so the shared memory keeps it there).
static size_t sweep_tc_launch_smem(int ctas, int spt) {
  size_t need = spt == 2 ? sweep_tc_smem_bytes<2>() : sweep_tc_smem_bytes<1>();
  const int cap_ctas = spt == 2 ? 4 : 6;
  ctas = std::min(std::max(ctas, 1), cap_ctas);
  if (ctas < cap_ctas || spt == 2) {
    int dev = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    // (1 KB of each CTA's shared memory is reserved by the system)
    const size_t cap = (size_t)per_sm / (size_t)(ctas + 1) - 1024 + 16;
    need = std::max(need, (cap + 15) / 16 * 16);
  }
  return need;
}
static int set_sweep_smem(int sub) {
  for (int flags = 0; flags < 8; flags++)
    TLR_CHECK(raise_smem_limit((const void*)sweep_kernel(flags), sweep_smem_bytes(sub, 256)));
  for (int t = 0; t < 16; t++) {  // every (periodisation, one-sided, operand type, samples per thread) variant
    const int spt = (t & 8) ? 2 : 1;
    const void* kf = (const void*)sweep_tc_kernel(((t & 1) ? SWEEP_PERIODIZE : 0) | ((t & 2) ? SWEEP_ONE_SIDED : 0),
                                                  (t & 4) != 0, spt);
    TLR_CHECK(raise_smem_limit(kf, sweep_tc_launch_smem(1, spt)));
  }
  return TLRMVN_OK;
}

// Operands of the whole-tile sweep (BF16-shift path): tensor maps of the split
// copy of B and of the sample-major hi/lo y buffer (32-deep boxes, 64-byte
// swizzle), of W and of the row and column factors (64 x 64 boxes), of the y hi
// halves for the projection; the projections W, the offset of the lo halves and
// the error flag.
struct TcOperands {
  CUtensorMap mapB32, mapY32, mapY64;
  CUtensorMap mapW{}, mapU64{}, mapV64{};
  unsigned short* W = nullptr;
  int64_t ldw = 0;
  int64_t my;
  int* err;
  bool f16 = false;  // fp16 operands (FP16-shift path), else bf16
};

// Whole diagonal tile i on the BF16-shift path: one launch of k_sweep_tc
// (low-rank shifts, in-tile coupling, sweep and projections).
static void sweep_tile_tc(const Factor& F, int i, int64_t C, const Lims& L, const float* rs32, const uint64_t* dD,
                          int64_t c0, int64_t N, int64_t Cc, int periodize, unsigned short* Ys, int64_t ldys,
                          double* logP, const TcOperands& tco, const Tuning& tu, cudaStream_t st, Prof& pf) {
  const int m = F.m, mt = (int)F.tsize(i);
  SweepTcArgs t;
  DiagArgs32& a = t.d;
  a.BT = F.BT32 + (size_t)i * m * F.ldbt;
  a.inv = F.inv32 + (size_t)i * m;
  a.band = F.band32 + (size_t)i * m * 16;
  a.mt = mt;
  a.ldbt = F.ldbt;
  a.Delta = nullptr;  // (the shifts are products of the kernel)
  a.ldd = C;
  a.a = L.a32 + F.tile_off[i];
  a.b = L.b32 + F.tile_off[i];
  a.rs = rs32;
  a.Q = F.Q;
  a.D = dD;
  a.ldD = F.n + 1;
  a.coord0 = F.tile_off[i];
  a.sample0 = c0;
  a.N = N;
  a.C = Cc;
  a.periodize = periodize;
  a.first = (i == 0);
  a.Yv = nullptr;
  a.ldyv = 0;
  a.Ys = reinterpret_cast<__nv_bfloat16*>(Ys);  // (16-bit words of the operand type)
  a.ldys = ldys;
  a.ys_lo = tco.my;
  a.logP = logP;
  t.brow0 = i * m;
  t.alo = (int)tco.my;
  t.blo = (int)tco.my;
  t.urow0 = i * m;
  t.krow0 = (int)F.kpad_off[i];
  t.kr = (int)F.krow(i);
  t.kcol0 = (int)F.kcol_off[i];
  t.kc = (int)F.kcol(i);
  t.W = tco.W;
  t.ldw = tco.ldw;
  t.vmap = F.vmap16 ? F.vmap16 + F.kcol_off[i] : nullptr;
  t.wscale = (tco.f16 && F.wscale16) ? F.wscale16 + F.kcol_off[i] : nullptr;
  t.tscale = tco.f16 ? F.inv_g16 : 1.0f;
  t.err = tco.err;
  const int flags = (periodize ? SWEEP_PERIODIZE : 0) | (L.one_sided ? SWEEP_ONE_SIDED : 0);
  pf.begin(TLRMVN_KC_DIAG);
  const int spt = tu.spt == 2 ? 2 : 1;
  launch_pdl(sweep_tc_kernel(flags, tco.f16, spt), dim3((unsigned)((Cc + STC_NS * spt - 1) / (STC_NS * spt))),
             dim3(STC_NS), sweep_tc_launch_smem(tu.tc_ctas, spt), st, tco.mapY32, tco.mapB32, tco.mapW, tco.mapU64, tco.mapY64,
             tco.mapV64, t);
  pf.end();
}

// Float sweep of diagonal tile i (FP32 path), `sub` variables at a time.  Before
// each sub-tile q > 0, the coupling to the tile's earlier sub-tiles,
// B_i[q, <q] y_i[<q], is added to the limit shifts Dl (variable-major, ld C) by
// a dense SIMT product; y goes to Yv (float, variable-major, ld C).  has_shift:
// Dl already holds the low-rank shifts of this tile.
static void sweep_tile_f32(const Factor& F, int i, bool has_shift, float* Dl, int64_t C, const Lims& L,
                           const float* rs32, const uint64_t* dD, int64_t c0, int64_t N, int64_t Cc, int periodize,
                           float* Yv, double* logP, const Tuning& tu, cudaStream_t st, Prof& pf) {
  const int m = F.m, mt = (int)F.tsize(i);
  const int sub = tu.sub;
  const SweepShape sh = sweep_shape(Cc, std::min(mt, sub), tu.threads);
  for (int q0 = 0; q0 < mt; q0 += sub) {
    const int mq = std::min(sub, mt - q0);
    if (q0 > 0) {
      // B_i[q0 + v][u] = BT32 row u, column q0 + v: the transposed tile is the k-major operand
      pf.begin(TLRMVN_KC_COUPLE);
      gemm_tn_f32(st, mq, Cc, q0, F.BT32 + (size_t)i * m * F.ldbt + q0, F.ldbt, Yv, C, Dl + (size_t)q0 * C, C,
                  nullptr, has_shift ? 1 : 0);
      pf.end();
    }
    DiagArgs32 a;
    a.BT = F.BT32 + (size_t)i * m * F.ldbt + (size_t)q0 * F.ldbt + q0;
    a.inv = F.inv32 + (size_t)i * m + q0;
    a.band = F.band32 + ((size_t)i * m + q0) * 16;
    a.mt = mq;
    a.ldbt = F.ldbt;
    a.Delta = (has_shift || q0 > 0) ? Dl + (size_t)q0 * C : nullptr;
    a.ldd = C;
    a.a = L.a32 + F.tile_off[i] + q0;
    a.b = L.b32 + F.tile_off[i] + q0;
    a.rs = rs32;
    a.Q = F.Q;
    a.D = dD;
    a.ldD = F.n + 1;
    a.coord0 = F.tile_off[i] + q0;
    a.sample0 = c0;
    a.N = N;
    a.C = Cc;
    a.periodize = periodize;
    a.first = (i == 0 && q0 == 0);
    a.Yv = Yv + (size_t)q0 * C;
    a.ldyv = C;
    a.Ys = nullptr;
    a.ldys = 0;
    a.ys_lo = 0;
    a.logP = logP;
    pf.begin(TLRMVN_KC_DIAG);
    const int flags = (periodize ? SWEEP_PERIODIZE : 0) | SWEEP_YV | (L.one_sided ? SWEEP_ONE_SIDED : 0);
    launch_pdl(sweep_kernel(flags), dim3((unsigned)blocks_for(Cc, sh.ns)), dim3(sh.threads), sweep_smem_bytes(mq, sh.ns), st,
               a);
    pf.end();
  }
}

template <typename T, typename YT>
static int run_chunks(Factor& F, const T* Bt, const T* Ut, const T* Vt, const Lims& L, double nu,
                      const tlrmvn_opts& o, const Tuning& tu, const uint64_t* dD, double* logP, Scratch& sc,
                      cudaStream_t st, Prof& pf) {
  const int64_t M = o.n_shifts, N = o.n_points, S = M * N;
  const int m = F.m;
  const bool f32 = sizeof(T) == 4;
  const int64_t C = chunk_simt(o, tu, S, F.ktot, m, sizeof(T));
  T *W = nullptr, *Dl = nullptr;
  YT* Y = nullptr;
  double* rs = nullptr;
  float* rs32 = nullptr;
  // (float: eight spare rows and a zeroed start, since a tile's shift reads its rank rows
  // rounded up to 8, past rows a projection may not have written yet)
  TLR_CHECK(sc.get(&W, (size_t)(F.ktot + (f32 ? 8 : 0)) * C));
  if (f32) TLR_CUDA(cudaMemsetAsync(W, 0, (size_t)(F.ktot + 8) * C * sizeof(T), st));
  TLR_CHECK(sc.get(&Dl, (size_t)m * C));
  TLR_CHECK(sc.get(&Y, (size_t)m * C));
  const bool mvt = std::isfinite(nu);
  if (mvt) TLR_CHECK(f32 ? sc.get(&rs32, (size_t)C) : sc.get(&rs, (size_t)C));

  // float64: sub-tiles of tu.sub variables, each sample keeping only the sub-tile's y in shared memory
  const int sub64 = std::min(m, tu.sub);
  const int bd = diag_threads<T>(sub64);
  const size_t smem = (size_t)sub64 * (bd + 1) * sizeof(T);
  if (f32)
    TLR_CHECK(set_sweep_smem(tu.sub));
  else
    TLR_CHECK(raise_smem_limit((const void*)k_diag<T, YT, false>, (size_t)smem));

  for (int64_t c0 = 0; c0 < S; c0 += C) {
    const int64_t Cc = std::min(C, S - c0);
    if (mvt) {
      pf.begin(TLRMVN_KC_CHI);
      k_chi_scale<<<blocks_for(Cc, 128), 128, 0, st>>>(rs, rs32, F.Q, dD, F.n + 1, F.n, c0, N, Cc, nu, o.periodize);
      pf.end();
    }
    for (int i = 0; i < F.r; i++) {
      const int mt = (int)F.tsize(i);
      const int64_t Kr = F.krow(i), Kc = F.kcol(i);
      const T* Delta = nullptr;
      if (Kr > 0) {
        pf.begin(TLRMVN_KC_SHIFT);
        if constexpr (sizeof(T) == 4) {
          const int64_t ld8 = (Kr + 7) / 8 * 8;
          gemm_tn_f32(st, mt, Cc, ld8, (const float*)Ut + F.u32_off[i], m, (const float*)W + (size_t)F.krow_off[i] * C,
                      C, (float*)Dl, C, nullptr);
        } else {
          gemm_nn<T>(st, mt, Cc, Kr, Ut + (size_t)m * F.krow_off[i], Kr, W + (size_t)F.krow_off[i] * C, C, Dl, C,
                     nullptr);
        }
        pf.end();
        Delta = Dl;
      }
      if constexpr (sizeof(T) == 4) {
        sweep_tile_f32(F, i, Kr > 0, (float*)Dl, C, L, rs32, dD, c0, N, Cc, o.periodize, (float*)Y, logP, tu, st,
                       pf);
      } else {
        // the coupling to the tile's earlier sub-tiles, B_i[q, <q] y_i[<q], is added
        // to the limit shifts by a dense product first (the same sums as eq. 2, regrouped)
        const T* Bi = Bt + (size_t)i * m * m;
        for (int q0 = 0; q0 < mt; q0 += sub64) {
          const int mq = std::min(sub64, mt - q0);
          if (q0 > 0) {
            pf.begin(TLRMVN_KC_COUPLE);
            gemm_nn<T>(st, mq, Cc, q0, Bi + (size_t)q0 * m, m, Y, C, Dl + (size_t)q0 * C, C, nullptr,
                       Delta ? 1 : 0);
            pf.end();
          }
          pf.begin(TLRMVN_KC_DIAG);
          DiagArgs<T, YT> a;
          a.B = Bi + (size_t)q0 * m + q0;
          a.mt = mq;
          a.ldb = m;
          a.Delta = (Delta || q0 > 0) ? Dl + (size_t)q0 * C : nullptr;
          a.ldd = C;
          a.a = L.a + F.tile_off[i] + q0;
          a.b = L.b + F.tile_off[i] + q0;
          a.rs = rs;
          a.Q = F.Q;
          a.D = dD;
          a.ldD = F.n + 1;
          a.coord0 = F.tile_off[i] + q0;
          a.sample0 = c0;
          a.N = N;
          a.C = Cc;
          a.periodize = o.periodize;
          a.first = (i == 0 && q0 == 0);
          a.Y = Y + (size_t)q0 * C;
          a.ldy = C;
          a.logP = logP;
          k_diag<T, YT, false><<<blocks_for(Cc, bd), bd, smem, st>>>(a);
          pf.end();
        }
      }
      if (Kc > 0) {
        pf.begin(TLRMVN_KC_VPROJ);
        if constexpr (sizeof(T) == 4)
          gemm_tn_f32(st, (int)Kc, Cc, mt, (const float*)Vt + F.v32_off[i], (Kc + 3) / 4 * 4, (const float*)Y, C,
                      (float*)W, C, F.vmap + F.kcol_off[i]);
        else
          gemm_nn<T>(st, (int)Kc, Cc, mt, Vt + (size_t)m * F.kcol_off[i], m, Y, C, W, C, F.vmap + F.kcol_off[i]);
        pf.end();
      }
    }
    TLR_CUDA(cudaGetLastError());
  }
  return TLRMVN_OK;
}

// BF16-shift integrand: one whole-tile sweep per diagonal tile (k_sweep_tc): the
// low-rank shifts, the in-tile coupling between 64-variable sub-tiles (split
// bf16 operands: x = hi + lo, hi*hi + hi*lo + lo*hi, relative error ~1e-5) and
// the projections on tcgen05 with fp32 accumulation in TMEM, the sweep itself in
// float32.  Layouts (C = samples in the chunk):
//   W16  kw16 x ldw bf16, rank-major (ldw = C rounded up to 64): row k holds
//        projection k of every sample (written as whole rows by the tile that
//        owns the rank, read as an MN-major operand by the later tiles' shifts)
//   Y16  C x 2 my16 bf16, sample-major: the tile's y (hi) in columns [0, my16) and
//        bf16(y - hi) in [my16, 2 my16)
static int run_chunks_bf16(Factor& F, const Lims& L, double nu, const tlrmvn_opts& o, const Tuning& tu,
                           const uint64_t* dD, double* logP, Scratch& sc, cudaStream_t st, Prof& pf) {
  const int64_t M = o.n_shifts, N = o.n_points, S = M * N;
  const int m = F.m;
  const bool f16 = o.precision == TLRMVN_FP16_SHIFT;
  const int64_t ly = 2 * F.my16;  // Y16 row: hi halves, then lo halves
  const int64_t C = chunk_bf16(o, tu, S, F.kw16, ly);
  unsigned short *W = nullptr, *Y = nullptr;
  float* rs32 = nullptr;
  int* err = nullptr;
  const int64_t ldw = (C + 63) / 64 * 64;
  TLR_CHECK(sc.get(&W, (size_t)F.kw16 * ldw));
  TLR_CHECK(sc.get(&Y, (size_t)ly * C));
  TLR_CHECK(sc.get(&err, 1));
  const bool mvt = std::isfinite(nu);
  if (mvt) TLR_CHECK(sc.get(&rs32, (size_t)C));
  // padding columns of W and Y must hold finite values: they meet zero operand columns
  TLR_CUDA(cudaMemsetAsync(W, 0, (size_t)F.kw16 * ldw * 2, st));
  TLR_CUDA(cudaMemsetAsync(Y, 0, (size_t)ly * C * 2, st));
  TLR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));

  // tensor maps: A operands (samples) take 128-row boxes, B operands 64-row boxes
  //   shift      T = W16^T (A, MN-major) x U16 rows (B)
  //   coupling   T += Y16 rows (A, hi/lo) x B16x2 rows (B, hi/lo)
  //   projection T = Y16 rows (A, hi) x V16 rows (B)
  TcOperands tco;
  tco.f16 = f16;
  const void* B2 = f16 ? (const void*)F.B16x2h : (const void*)F.B16x2;
  TLR_CHECK(make_map(&tco.mapB32, B2, ly, (uint64_t)F.r * m, ly * 2, 64, 32, f16));
  TLR_CHECK(make_map(&tco.mapY32, Y, ly, C, ly * 2, STC_NS, 32, f16));
  TLR_CHECK(make_map(&tco.mapY64, Y, ly, C, ly * 2, STC_NS, 64, f16));
  TLR_CHECK(make_map(&tco.mapW, W, ldw, F.kw16, ldw * 2, 64, 64, f16));
  if (F.ktot) {
    const void* U = f16 ? (const void*)F.U16h : (const void*)F.U16;
    const void* V = f16 ? (const void*)F.V16h : (const void*)F.V16;
    TLR_CHECK(make_map(&tco.mapU64, U, F.kmax16, (uint64_t)F.r * m, F.kmax16 * 2, 64, 64, f16));
    TLR_CHECK(make_map(&tco.mapV64, V, F.my16, F.ktot, F.my16 * 2, 64, 64, f16));
  } else {
    tco.mapU64 = tco.mapW;  // (never read: no tile has ranks)
    tco.mapV64 = tco.mapW;
  }
  tco.W = W;
  tco.ldw = ldw;
  tco.my = F.my16;
  tco.err = err;
  TLR_CHECK(set_sweep_smem(64));

  for (int64_t c0 = 0; c0 < S; c0 += C) {
    const int64_t Cc = std::min(C, S - c0);
    if (mvt) {
      pf.begin(TLRMVN_KC_CHI);
      k_chi_scale<<<blocks_for(Cc, 128), 128, 0, st>>>(nullptr, rs32, F.Q, dD, F.n + 1, F.n, c0, N, Cc, nu,
                                                       o.periodize);
      pf.end();
    }
    for (int i = 0; i < F.r; i++)
      sweep_tile_tc(F, i, C, L, rs32, dD, c0, N, Cc, o.periodize, Y, ly, logP, tco, tu, st, pf);
    TLR_CUDA(cudaGetLastError());
  }
  int herr = 0;
  TLR_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  if (herr) return fail(TLRMVN_E_TIMEOUT, "tensor-core kernel gave up waiting (code " + std::to_string(herr) + ")");
  return TLRMVN_OK;
}

// Bytes of stream-ordered scratch one tlrmvn_prob call takes (used for admission
// by the serving loop); mirrors the buffers of prob_impl and the chunk loops.
int64_t prob_scratch_bytes(const Factor& F, const tlrmvn_opts& o) {
  const int64_t M = o.n_shifts, N = o.n_points, S = M * N, n = F.n, m = F.m;
  const Tuning tu = F.tuning(o.precision);
  int64_t bytes = n * (8 * 2 + 4 * 2) + M * (n + 1) * 8 + M * 8 + S * 8 + 256;
  if (o.precision == TLRMVN_BF16_SHIFT || o.precision == TLRMVN_FP16_SHIFT) {
    int64_t kw = 0;
    for (int i = 0; i < F.r; i++) kw += (F.krow(i) + 63) / 64 * 64;
    kw = std::max<int64_t>(kw, 64);
    const int64_t my = (m + 63) / 64 * 64, ly = 2 * my;
    const int64_t C = chunk_bf16(o, tu, S, kw, ly);
    bytes += C * (kw * 2 + ly * 2 + 4);
  } else {
    const int64_t es = o.precision == TLRMVN_FP64 ? 8 : 4;
    const int64_t C = chunk_simt(o, tu, S, F.ktot, m, es);
    bytes += C * ((F.ktot + 2 * m) * es + 8);
  }
  return bytes;
}

int prob_impl(Factor& F, const double* a_dev, const double* b_dev, double nu, const tlrmvn_opts& o,
              double* logp_dev, double* err_dev, double* ell_dev_out, double* per_sample_dev, cudaStream_t st) {
  const int64_t M = o.n_shifts, N = o.n_points, S = M * N, n = F.n;
  Scratch sc(st);
  double *ap = nullptr, *bp = nullptr, *logP = nullptr, *ell = nullptr;
  float *ap32 = nullptr, *bp32 = nullptr;
  uint64_t* dD = nullptr;
  int* bad = nullptr;
  TLR_CHECK(sc.get(&ap, n));
  TLR_CHECK(sc.get(&bp, n));
  if (o.precision != TLRMVN_FP64) {
    TLR_CHECK(sc.get(&ap32, n));
    TLR_CHECK(sc.get(&bp32, n));
  }
  TLR_CHECK(sc.get(&bad, 2));  // invalid limits; a finite lower limit
  TLR_CHECK(sc.get(&dD, (size_t)M * (n + 1)));
  TLR_CHECK(sc.get(&ell, M));
  if (per_sample_dev) logP = per_sample_dev;
  else TLR_CHECK(sc.get(&logP, S));
  // lattice shifts
  {
    std::vector<uint64_t> hD;
    const uint64_t* src = o.shifts;
    if (!src) {
      hD.resize((size_t)M * (n + 1));
      for (size_t t = 0; t < hD.size(); t++) hD[t] = splitmix64_at(o.seed, t);
      src = hD.data();
    }
    TLR_CUDA(cudaMemcpyAsync(dD, src, (size_t)M * (n + 1) * 8, cudaMemcpyHostToDevice, st));
    if (!hD.empty()) TLR_CUDA(cudaStreamSynchronize(st));
  }
  TLR_CUDA(cudaMemsetAsync(bad, 0, 2 * sizeof(int), st));
  Prof pf(st);
  pf.begin(TLRMVN_KC_PREP);
  k_permute_limits<<<blocks_for(n, 256), 256, 0, st>>>(a_dev, b_dev, F.dperm, n, ap, bp, ap32, bp32, bad);
  pf.end();
  int hbad[2] = {0, 0};
  TLR_CUDA(cudaMemcpyAsync(hbad, bad, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  if (hbad[0]) {
    pf.collect();
    return fail(TLRMVN_E_INVAL, "limits must satisfy a_i <= b_i, a_i < +inf, b_i > -inf, no NaN");
  }
  TLR_CHECK(ensure_copies(F, o.precision, st));
  int s;
  const Lims L{ap, bp, ap32, bp32, hbad[1] == 0};
  const Tuning tu = F.tuning(o.precision);
  if (o.precision == TLRMVN_FP64)
    s = run_chunks<double, double>(F, F.B, F.Ucat, F.Vcat, L, nu, o, tu, dD, logP, sc, st, pf);
  else if (o.precision == TLRMVN_FP32)
    s = run_chunks<float, float>(F, F.B32, F.U32, F.V32, L, nu, o, tu, dD, logP, sc, st, pf);
  else
    s = run_chunks_bf16(F, L, nu, o, tu, dD, logP, sc, st, pf);
  TLR_CHECK(s);
  pf.begin(TLRMVN_KC_REDUCE);
  k_shift_reduce<<<(unsigned)M, 256, 0, st>>>(logP, N, ell);
  pf.end();
  pf.begin(TLRMVN_KC_REDUCE);
  k_final<<<1, 256, 0, st>>>(ell, (int)M, logp_dev, err_dev);
  pf.end();
  if (ell_dev_out) TLR_CUDA(cudaMemcpyAsync(ell_dev_out, ell, M * 8, cudaMemcpyDeviceToDevice, st));
  TLR_CUDA(cudaGetLastError());
  TLR_CUDA(cudaStreamSynchronize(st));
  return pf.collect();
}

static int check_opts(const Factor& F, double nu, const tlrmvn_opts* o) {
  if (!o) return fail(TLRMVN_E_INVAL, "null options");
  if (o->n_shifts < 1 || o->n_points < 1) return fail(TLRMVN_E_INVAL, "n_shifts and n_points must be >= 1");
  if (o->precision < TLRMVN_FP64 || o->precision > TLRMVN_FP16_SHIFT) return fail(TLRMVN_E_INVAL, "bad precision");
  if (!(nu > 0.0)) return fail(TLRMVN_E_INVAL, "nu must be > 0 (INFINITY for the normal case)");
  (void)F;
  return TLRMVN_OK;
}

}  // namespace tlrmvn

using namespace tlrmvn;

extern "C" int tlrmvn_prob_device(tlrmvn_factor_t f, const double* a, const double* b, double nu,
                                  const tlrmvn_opts* opts, double* logp, double* err, double* per_shift,
                                  double* per_sample) {
  if (!f || !a || !b || !logp || !err) return fail(TLRMVN_E_INVAL, "null argument");
  Factor& F = *reinterpret_cast<Factor*>(f);
  TLR_CHECK(check_opts(F, nu, opts));
  int cur = 0;
  cudaGetDevice(&cur);
  TLR_CUDA(cudaSetDevice(F.device));
  cudaStream_t st = pick_stream(opts->stream);
  // (the estimate is written straight into the caller's device outputs: no allocation here)
  const int s = prob_impl(F, a, b, nu, *opts, logp, err, per_shift, per_sample, st);
  cudaSetDevice(cur);
  return s;
}

extern "C" int tlrmvn_prob(tlrmvn_factor_t f, const double* a, const double* b, double nu, const tlrmvn_opts* opts,
                           double* logp, double* err, double* per_shift, double* per_sample) {
  if (!f || !a || !b || !logp || !err) return fail(TLRMVN_E_INVAL, "null argument");
  Factor& F = *reinterpret_cast<Factor*>(f);
  TLR_CHECK(check_opts(F, nu, opts));
  int cur = 0;
  cudaGetDevice(&cur);
  TLR_CUDA(cudaSetDevice(F.device));
  cudaStream_t st = pick_stream(opts->stream);
  const int64_t n = F.n, M = opts->n_shifts, S = M * (int64_t)opts->n_points;
  double *da = nullptr, *db = nullptr, *out2 = nullptr, *dell = nullptr, *dps = nullptr;
  int s = dalloc(&da, n);
  if (s == TLRMVN_OK) s = dalloc(&db, n);
  if (s == TLRMVN_OK) s = dalloc(&out2, 2);
  if (s == TLRMVN_OK && per_shift) s = dalloc(&dell, M);
  if (s == TLRMVN_OK && per_sample) s = dalloc(&dps, S);
  if (s == TLRMVN_OK) {
    cudaError_t e = cudaMemcpyAsync(da, a, n * 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db, b, n * 8, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) s = cuda_fail(e, "copy limits");
  }
  if (s == TLRMVN_OK) s = prob_impl(F, da, db, nu, *opts, out2, out2 + 1, dell, dps, st);
  if (s == TLRMVN_OK) {
    double h[2];
    cudaError_t e = cudaMemcpyAsync(h, out2, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && per_shift) e = cudaMemcpyAsync(per_shift, dell, M * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && per_sample) e = cudaMemcpyAsync(per_sample, dps, S * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "copy results");
    else {
      *logp = h[0];
      *err = h[1];
    }
  }
  dfree(da);
  dfree(db);
  dfree(out2);
  dfree(dell);
  dfree(dps);
  cudaSetDevice(cur);
  return s;
}

extern "C" int tlrmvn_selftest_wait_timeout(int polls, void* stream) {
  if (polls < 1 || polls > (1 << 20)) return fail(TLRMVN_E_INVAL, "polls must be in [1, 2^20]");
  cudaStream_t st = pick_stream(stream);
  int* err = nullptr;
  TLR_CUDA(cudaMallocAsync((void**)&err, sizeof(int), st));
  int herr = 0;
  cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    k_wait_selftest<<<1, 32, 0, st>>>(err, (uint32_t)polls);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(err, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test");
  if (herr) return fail(TLRMVN_E_TIMEOUT, "wait self-test gave up after " + std::to_string(polls) + " polls (code " +
                                              std::to_string(herr) + ")");
  return TLRMVN_OK;
}

// Evaluates the sweep's float32 Phi(-x) (phi_neg_f32) on n host values.
__global__ void k_phi_neg_selftest(const float* x, int n, float* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = phi_neg_f32(x[t]);
}

extern "C" int tlrmvn_selftest_phi_neg(const float* x, int n, float* out) {
  if (!x || !out || n < 1 || n > (1 << 24)) return fail(TLRMVN_E_INVAL, "bad arguments");
  cudaStream_t st = pick_stream(nullptr);
  float* d = nullptr;
  TLR_CUDA(cudaMallocAsync((void**)&d, (size_t)2 * n * sizeof(float), st));
  cudaError_t e = cudaMemcpyAsync(d, x, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_phi_neg_selftest<<<(n + 255) / 256, 256, 0, st>>>(d, n, d + n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "phi self-test");
  return TLRMVN_OK;
}

// Evaluates the float path's normal quantile (ndtri_f32) on n host values.
__global__ void k_ndtri_selftest(const float* p, const float* lp, int n, float* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) out[t] = ndtri_f32(p[t], lp[t]);
}

// Eight independent FMA chains per thread, `iters` x 8 steps each; the sum is
// written only when it takes a value it never takes, which keeps the chains live.
__global__ void __launch_bounds__(256) k_fma_peak(float m, float c, int iters, float* sink) {
  float x[8];
#pragma unroll
  for (int j = 0; j < 8; j++) x[j] = (float)(threadIdx.x + j) * 1e-3f;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 8; u++)
#pragma unroll
      for (int j = 0; j < 8; j++) x[j] = fmaf(x[j], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < 8; j++) s += x[j];
  if (s == -1.0f) sink[blockIdx.x] = s;
}

extern "C" int tlrmvn_measure_fp32_peak(void* stream, double* tflops) {
  if (!tflops) return fail(TLRMVN_E_INVAL, "null output");
  cudaStream_t st = pick_stream(stream);
  int dev = 0, sms = 0;
  TLR_CUDA(cudaGetDevice(&dev));
  TLR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8, threads = 256, iters = 2048;
  float* sink = nullptr;
  TLR_CUDA(cudaMallocAsync((void**)&sink, (size_t)blocks * sizeof(float), st));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.0f;
  if (e == cudaSuccess) {
    k_fma_peak<<<blocks, threads, 0, st>>>(0.99999994f, 1e-7f, iters, sink);  // untimed
    cudaEventRecord(e0, st);
    k_fma_peak<<<blocks, threads, 0, st>>>(0.99999994f, 1e-7f, iters, sink);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFreeAsync(sink, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "float32 FMA throughput");
  const double flops = 2.0 * 64.0 * (double)iters * (double)blocks * (double)threads;
  *tflops = flops / ((double)ms * 1e-3) / 1e12;
  return TLRMVN_OK;
}

extern "C" int tlrmvn_selftest_ndtri(const float* p, const float* lp, int n, float* out) {
  if (!p || !lp || !out || n < 1 || n > (1 << 24)) return fail(TLRMVN_E_INVAL, "bad arguments");
  cudaStream_t st = pick_stream(nullptr);
  float* d = nullptr;
  TLR_CUDA(cudaMallocAsync((void**)&d, (size_t)3 * n * sizeof(float), st));
  cudaError_t e = cudaMemcpyAsync(d, p, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d + n, lp, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_ndtri_selftest<<<(n + 255) / 256, 256, 0, st>>>(d, d + n, n, d + 2 * n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + 2 * n, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "quantile self-test");
  return TLRMVN_OK;
}
