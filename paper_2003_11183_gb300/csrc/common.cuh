// Shared internals of the tlrmvn library: status plumbing, the factor handle,
// and the device-side univariate functions of the SOV integrand.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <math.h>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/tlrmvn.h"

namespace tlrmvn {

// ---- error plumbing --------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define TLR_CUDA(call)                                              \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ::tlrmvn::cuda_fail(e_, #call);   \
  } while (0)

#define TLR_CHECK(st)            \
  do {                           \
    int s_ = (st);               \
    if (s_ != TLRMVN_OK) return s_; \
  } while (0)

// Device allocation owned by the caller of dalloc.
template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) return TLRMVN_OK;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(TLRMVN_E_NOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  return TLRMVN_OK;
}
template <typename T>
void dfree(T*& p) {
  if (p) cudaFree((void*)p);
  p = nullptr;
}

// ---- launch choices ----------------------------------------------------------
// Launch choices of the integrand for one factor and precision, made by the
// autotuner (tlrmvn_autotune) or left at these defaults:
//   sub      variables per sub-tile of the float32 and float64 sweeps (64 or 128;
//            the in-tile coupling between sub-tiles is a dense product)
//   threads  threads per block of the float32 sweep (0: the occupancy rule)
//   chunk    samples in flight per pass (0: as many as the memory rule allows)
//   tc_ctas  whole-tile sweeps (BF16-/FP16-shift paths) sharing an SM: 6 (all that
//            fit: 80 registers, 28 KB of shared memory and 64 TMEM columns each), or
//            fewer by reserving shared memory
//   spt      samples per thread of the whole-tile sweep: 1, or 2 (256 samples per
//            CTA, two independent chains per thread, 128 TMEM columns, four CTAs per SM)
struct Tuning {
  int sub = 64;
  int threads = 0;
  int64_t chunk = 0;
  int tc_ctas = 6;
  int spt = 1;
};

// ---- factor handle -----------------------------------------------------------
// L ~ tile-low-rank Cholesky factor of Sigma[perm][:, perm] (Section 3.3).
// Compact device layout used by the integrand:
//   B     r x m x m float64, diagonal tiles by position, row-major, zero above the diagonal
//   Ucat  for row tile i: an m x Krow_i row-major block at offset m*krow_off[i]; its
//         columns are the ranks of (i,0), (i,1), ..., (i,i-1) in that order
//   Vcat  for column tile j: a Kcol_j x m row-major block at offset m*kcol_off[j];
//         its rows are the ranks of (j+1,j), (j+2,j), ..., (r-1,j), stored as V^T
//   vmap  Vcat row -> global rank index (the row-grouped index of Ucat columns)
struct Factor {
  int64_t n = 0;
  int r = 0, m = 0;
  int64_t ktot = 0;
  int capped = 0;
  int device = 0;
  std::vector<int64_t> tile_off, perm;   // host
  std::vector<int32_t> rank;             // host, r*r, rank[i*r+j] for i > j
  std::vector<int64_t> krow_off, kcol_off;
  double* B = nullptr;
  double* Ucat = nullptr;
  double* Vcat = nullptr;
  int32_t* vmap = nullptr;
  // lazily made copies for the reduced-precision integrands
  //   BT32  r x m x ldbt: transposed diagonal tiles, BT32[i][u][v] = B_i[v][u]
  //   inv32 r x m: 1 / B_i[v][v]
  float* BT32 = nullptr;
  float* inv32 = nullptr;
  //   band32 r x m x 16: band32[(i*m + v)*16 + k] = B_i[v+1+k][v] for k < 15 and
  //         v+1+k < m, else 0 (each variable's window column, contiguous)
  float* band32 = nullptr;
  int64_t ldbt = 0;
  float* B32 = nullptr;
  float* U32 = nullptr;  // row tile i at u32_off[i]: (Krow_i rounded up to 8) x m, U_i transposed, zero rows
  std::vector<int64_t> u32_off;
  float* V32 = nullptr;  // column tile i at v32_off[i]: m x (Kcol_i rounded up to 4), V_i, zero columns
  std::vector<int64_t> v32_off;
  // bf16 operands of the tensor-core shifts (K-major, padded for TMA):
  //   U16   (r*m) x kmax16: row i*m+v holds row v of Ucat_i, zero beyond Krow_i
  //   V16   ktot x my16:    Vcat rows, zero beyond m
  //   vmap16 Vcat row -> column of the padded rank space, whose row tile i starts at
  //          kpad_off[i] (a multiple of 64) and spans kw16 columns in all
  //   B16x2 (r*m) x (2*my16): row i*m+v holds bf16 hi(B_i[v][u]) at column u and
  //         lo = bf16(B_i[v][u] - hi) at column my16 + u (zero for u >= m); the
  //         in-tile coupling operand of the tensor-core path
  __nv_bfloat16* U16 = nullptr;
  __nv_bfloat16* V16 = nullptr;
  __nv_bfloat16* B16x2 = nullptr;
  int32_t* vmap16 = nullptr;
  std::vector<int64_t> kpad_off;
  int64_t kmax16 = 0, kw16 = 0, my16 = 0;
  // fp16 operands of the FP16-shift path, same layouts: U16h = U g a_ij and V16h = V c_ij
  // with per-tile powers of two a_ij, c_ij (max |U g a| and max |V c| in (1/2, 1], a_ij
  // raised where the projections' range needs it), B16x2h the fp16 split of B g; wscale16
  // (per Vcat row) = 1 / (a_ij c_ij), the factor applied to a projection before it is stored
  __half* U16h = nullptr;
  __half* V16h = nullptr;
  __half* B16x2h = nullptr;
  float* wscale16 = nullptr;
  // the fp16 products are of the factor scaled by g (a power of two with max |B g| in
  // (1/2, 1], so that badly scaled covariances keep fp16's range); the sweep multiplies
  // what it reads from the products by inv_g16 = 1 / g
  float inv_g16 = 1.0f;
  // lattice generators for n + 1 coordinates (device), and the permutation (device)
  uint64_t* Q = nullptr;
  int64_t* dperm = nullptr;
  // guards the lazily made copies when several streams use the factor at once
  std::mutex copy_mu;
  // launch choices per precision (TLRMVN_FP64 / FP32 / BF16_SHIFT / FP16_SHIFT), set by the autotuner
  Tuning tune[4];
  mutable std::mutex tune_mu;
  Tuning tuning(int precision) const {
    std::lock_guard<std::mutex> lk(tune_mu);
    return tune[precision < 0 || precision > 3 ? 0 : precision];
  }

  int64_t tsize(int t) const { return tile_off[t + 1] - tile_off[t]; }
  int64_t krow(int i) const { return krow_off[i + 1] - krow_off[i]; }
  int64_t kcol(int j) const { return kcol_off[j + 1] - kcol_off[j]; }
  ~Factor();
};

// Fills krow_off/kcol_off/ktot from rank and allocates Ucat/Vcat/vmap/B (not filled).
int factor_alloc_compact(Factor& F, cudaStream_t st);
// Host tables: lattice generators Q_i = floor(frac(sqrt(p_i)) 2^64) for the first d primes.
std::vector<uint64_t> richtmyer_generators(int64_t d);
// Uploads Q and perm, called once the factor is complete.
int factor_finish(Factor& F, cudaStream_t st);

cudaStream_t pick_stream(void* s);
// Raise `kernel`'s dynamic shared memory limit on the current device to at least
// `bytes`.  The limit is per function and process-wide, so it is only ever
// raised: a caller with a smaller tile never lowers it under another thread that
// is about to launch with a larger one.
int raise_smem_limit(const void* kernel, size_t bytes);

// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while its predecessor in the stream is still running.  Every kernel that can
// be launched that way calls pdl_trigger() on entry (its own successor may then
// be scheduled once all of its CTAs are running) and pdl_wait() before it reads
// anything the predecessor wrote or writes any global memory (pdl_wait returns
// once the predecessor grid has completed and its writes are visible).  Both are
// no-ops for a kernel launched the ordinary way.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Kernel-class timing (tlrmvn_profile_*): Prof brackets launches with events.
struct Prof {
  bool on;
  cudaStream_t st;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
  explicit Prof(cudaStream_t s);
  void begin(int cls);
  void end();
  int collect();  // after the stream is synchronised: add to the global accumulators
  ~Prof();
};

// ---- device univariate functions ------------------------------------------------
#define TLR_RSQRT2 0.70710678118654752440
#define TLR_SQRT2PI 2.50662827463100050242
#define TLR_LOG_SQRT2PI 0.91893853320467274178

// Rational approximation of the standard normal quantile by P. J. Acklam
// (2003; relative error below 1.15e-9 on (0,1)): central branch in p - 1/2,
// tail branch in q = sqrt(-2 log p).  Coefficients as published.
struct Acklam {
  static constexpr double a1 = -3.969683028665376e+01, a2 = 2.209460984245205e+02, a3 = -2.759285104469687e+02,
                          a4 = 1.383577518672690e+02, a5 = -3.066479806614716e+01, a6 = 2.506628277459239e+00;
  static constexpr double b1 = -5.447609879822406e+01, b2 = 1.615858368580409e+02, b3 = -1.556989798598866e+02,
                          b4 = 6.680131188771972e+01, b5 = -1.328068155288572e+01;
  static constexpr double c1 = -7.784894002430293e-03, c2 = -3.223964580411365e-01, c3 = -2.400758277161838e+00,
                          c4 = -2.549732539343734e+00, c5 = 4.374664141464968e+00, c6 = 2.938163982698783e+00;
  static constexpr double d1 = 7.784695709041462e-03, d2 = 3.224671290700398e-01, d3 = 2.445134137142996e+00,
                          d4 = 3.754408661907416e+00;
  static constexpr double p_low = 0.02425;
};

// log Phi(x), accurate in both tails.
__device__ __forceinline__ double log_Phi(double x) {
  if (x < -1.0) return log(0.5 * erfcx(-x * TLR_RSQRT2)) - 0.5 * x * x;
  if (x < 0.0) return log(0.5 * erfc(-x * TLR_RSQRT2));
  return log1p(-0.5 * erfc(x * TLR_RSQRT2));
}
__device__ __forceinline__ float log_Phi(float x) {
  if (x < -1.0f) return logf(0.5f * erfcxf(-x * (float)TLR_RSQRT2)) - 0.5f * x * x;
  if (x < 0.0f) return logf(0.5f * erfcf(-x * (float)TLR_RSQRT2));
  return log1pf(-0.5f * erfcf(x * (float)TLR_RSQRT2));
}

// Phi^-1(p) for p in (0, 1/2]; lp = log p (finite even when p underflows).
// float64: Acklam start, then one Newton step on log Phi(x) - log p in the tail
// or one Halley step on Phi(x) - p in the centre, which brings the relative
// error to the level of the erfc evaluation.
__device__ __forceinline__ double ndtri_lower(double p, double lp) {
  double x;
  if (p < Acklam::p_low) {
    double q = sqrt(-2.0 * lp);
    x = (((((Acklam::c1 * q + Acklam::c2) * q + Acklam::c3) * q + Acklam::c4) * q + Acklam::c5) * q + Acklam::c6) /
        ((((Acklam::d1 * q + Acklam::d2) * q + Acklam::d3) * q + Acklam::d4) * q + 1.0);
    double lphi = log_Phi(x);
    double f = lphi - lp;
    double dfdx = exp(-0.5 * x * x - TLR_LOG_SQRT2PI - lphi);
    x -= f / dfdx;
  } else {
    double q = p - 0.5, rr = q * q;
    x = (((((Acklam::a1 * rr + Acklam::a2) * rr + Acklam::a3) * rr + Acklam::a4) * rr + Acklam::a5) * rr + Acklam::a6) * q /
        (((((Acklam::b1 * rr + Acklam::b2) * rr + Acklam::b3) * rr + Acklam::b4) * rr + Acklam::b5) * rr + 1.0);
    double e = 0.5 * erfc(-x * TLR_RSQRT2) - p;
    double u = e * TLR_SQRT2PI * exp(0.5 * x * x);
    x = x - u / (1.0 + 0.5 * x * u);
  }
  return x;
}
// float32 normal quantile, lower half.  Two regions:
//  * p > 0.0017 (w = -log(4 p (1 - p)) < 5; all but about 1 in 300 calls):
//    Phi^-1(p) = -sqrt(2) (1 - 2p) R(w), R(w) = erfinv(1 - 2p) / (1 - 2p) as a
//    degree-8 polynomial in w - 2.5 (the variable of M. Giles, Approximating the
//    erfinv function, GPU Computing Gems, 2011; coefficients from the library's
//    own fit, csrc/fit_ndtri.py, relative error about 2.2e-7 in float32);
//  * below: Wichura's tail forms in t = sqrt(-log p) (M. J. Wichura, Algorithm AS
//    241, Applied Statistics 37 (1988) 477-484, PPND7, coefficients as
//    published: t <= 5 and t > 5), from log p, so that the quantile stays finite
//    when p underflows (to log p = -700: relative error about 4e-7 in float32).
// lp_tiny = log p is read only when p < 1e-30 (p may then be 0); above that the
// log is taken here.  A warp takes the tail branch only when one of its lanes
// falls there.
__device__ __forceinline__ float ndtri_tail_f32(float lp) {
  const float nl = fminf(fmaxf(-lp, 0.0f), 3.0e38f);
  const float t = nl * rsqrtf(fmaxf(nl, 1e-30f));  // sqrt(-log p)
  if (t <= 5.0f) {
    const float s = t - 1.6f;
    const float num = fmaf(fmaf(fmaf(1.7023821103e-01f, s, 1.3067284816e+00f), s, 2.7568153900e+00f), s,
                           1.4234372777e+00f);
    const float den = fmaf(fmaf(1.2021132975e-01f, s, 7.3700164250e-01f), s, 1.0f);
    return -num / den;
  }
  const float s = t - 5.0f;
  const float num =
      fmaf(fmaf(fmaf(1.7337203997e-02f, s, 4.2868294337e-01f), s, 3.0812263860e+00f), s, 6.6579051150e+00f);
  const float den = fmaf(fmaf(1.2258202635e-02f, s, 2.4197894225e-01f), s, 1.0f);
  return -num / den;
}
__device__ __forceinline__ float ndtri_f32(float p, float lp_tiny) {
  const float w = -__logf(p * fmaf(-4.0f, p, 4.0f));  // -log(4 p (1 - p))
  if (w < 5.0f) {
    // -sqrt(2) R(w) (the fitted coefficients times -sqrt(2)), times x = 1 - 2p
    const float z = w - 2.5f;
    float r = -3.958320960e-08f;
    r = fmaf(r, z, -4.851791005e-07f);
    r = fmaf(r, z, 4.981194706e-06f);
    r = fmaf(r, z, 6.207880233e-06f);
    r = fmaf(r, z, -3.091151011e-04f);
    r = fmaf(r, z, 1.773041789e-03f);
    r = fmaf(r, z, 5.908129737e-03f);
    r = fmaf(r, z, -3.488026857e-01f);
    r = fmaf(r, z, -2.123313665e+00f);
    return r * fmaf(-2.0f, p, 1.0f);
  }
  return ndtri_tail_f32(p >= 1e-30f ? __logf(p) : lp_tiny);
}
// (the float overload used by the general step: lp = log p)
__device__ __forceinline__ float ndtri_lower(float p, float lp) { return ndtri_f32(p, lp); }

__device__ __forceinline__ double dev_log(double x) { return log(x); }
__device__ __forceinline__ float dev_log(float x) { return logf(x); }
__device__ __forceinline__ double dev_erfc(double x) { return erfc(x); }
__device__ __forceinline__ float dev_erfc(float x) { return erfcf(x); }
__device__ __forceinline__ double dev_exp(double x) { return exp(x); }
__device__ __forceinline__ float dev_exp(float x) { return expf(x); }
__device__ __forceinline__ double dev_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float dev_expm1(float x) { return expm1f(x); }

// Phi^-1 given u and its complement uc = 1 - u (both accurate) and lu = log u.
template <typename T>
__device__ __forceinline__ T ndtri2(T u, T uc, T lu) {
  if (u <= (T)0.5) return ndtri_lower(u, lu);
  return -ndtri_lower(uc, dev_log(uc));
}

// One variable of eq. (2) on standardised limits (at, bt), lattice value w with
// complement wc = 1 - w: returns log(e - d) and y = Phi^-1(d + w (e - d)),
// with d = Phi(at), e = Phi(bt).  Upper-half intervals (at > 0) are handled
// through the complements Phi(-at), Phi(-bt); one-sided intervals through log Phi.
template <typename T>
__device__ __forceinline__ void sov_step(T at, T bt, T w, T wc, T& ld, T& y) {
  const T rs2 = (T)TLR_RSQRT2;
  const T INF = (T)INFINITY;
  if (at == -INF) {
    if (bt == INF) {
      ld = (T)0;
      y = ndtri2(w, wc, dev_log(w));
      return;
    }
    T e, ec, le;
    if (bt < (T)0) {
      e = (T)0.5 * dev_erfc(-bt * rs2);
      ec = (T)1 - e;
      le = log_Phi(bt);
    } else {
      ec = (T)0.5 * dev_erfc(bt * rs2);
      e = (T)1 - ec;
      le = log_Phi(bt);
    }
    T u = w * e, uc = ec + wc * e;
    y = ndtri2(u, uc, dev_log(w) + le);
    ld = le;
    return;
  }
  if (at > (T)0) {
    // upper half, in logs of the complements Phi(-at) >= Phi(-bt): finite when both underflow
    const T lca = log_Phi(-at);
    const T dl = (bt == INF) ? -INF : log_Phi(-bt) - lca;
    ld = lca + dev_log(-dev_expm1(dl));
    const T luc = lca + dev_log(wc + w * dev_exp(dl));  // log(1 - u) = log((1-w) Phi(-at) + w Phi(-bt))
    y = -ndtri_lower(dev_exp(luc), luc);
    return;
  }
  if (bt <= (T)0) {
    // lower half, in logs: Phi(at) <= Phi(bt) <= 1/2
    const T lb = log_Phi(bt);
    const T dl = log_Phi(at) - lb;
    ld = lb + dev_log(-dev_expm1(dl));
    const T lu = lb + dev_log(w + wc * dev_exp(dl));  // log u = log((1-w) Phi(at) + w Phi(bt))
    y = ndtri_lower(dev_exp(lu), lu);
    return;
  }
  // straddles 0 (at <= 0 < bt): e - d >= e - 1/2 > 0
  const T d = (T)0.5 * dev_erfc(-at * rs2);
  const T ec = (bt == INF) ? (T)0 : (T)0.5 * dev_erfc(bt * rs2);
  const T e = (T)1 - ec;
  T diff = e - d;
  T u = d + w * diff, uc = ec + wc * diff;
  y = ndtri2(u, uc, dev_log(u));
  ld = dev_log(diff);
}

// Lattice coordinate -> (w, 1 - w), exactly (see the lattice definition:
// tent transform of the cell midpoint of the top 53 bits, or the midpoint of
// the top 52 bits without periodisation).
__device__ __forceinline__ void lattice_w(uint64_t x, int periodize, double& w, double& wc) {
  const double s53 = 1.1102230246251565e-16;  // 2^-53
  if (periodize) {
    int64_t h = (int64_t)(x >> 11);
    int64_t num = 2 * h + 1 - (int64_t(1) << 53);
    if (num < 0) num = -num;
    w = (double)num * s53;
    wc = (double)((int64_t(1) << 53) - num) * s53;
  } else {
    int64_t h = (int64_t)(x >> 12);
    int64_t num = 2 * h + 1;
    w = (double)num * s53;
    wc = (double)((int64_t(1) << 53) - num) * s53;
  }
}

}  // namespace tlrmvn
