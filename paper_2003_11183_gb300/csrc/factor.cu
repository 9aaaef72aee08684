// Block-reordered tile-low-rank Cholesky factorisation in float64 on the GPU
// (Section 3.3, Algorithms 4 and 5).
//
// Blocks (tile-sized clusters of the geometric order) carry a block id; the
// factor is built position by position j = 0..r-1:
//   * Algorithm 5 (iterative): univariate conditioning (UC) of every remaining
//     block on its current Schur complement and conditioned limits; the block
//     with the smallest estimate takes position j, and its UC pivot order is its
//     within-block order.  Algorithm 4 (one-shot): UC of the original blocks
//     once, blocks sorted by the estimate.
//   * L_jj = Cholesky(S_jj); S_ij = Sigma_ij - sum_{k<j} U_ik (V_ik^T V_jk) U_jk^T
//     (left-looking, so no dense Schur complement of the off-diagonal part is
//     ever stored); L_ij = S_ij L_jj^-T; L_ij ~ U_ij V_ij^T by adaptive cross
//     approximation with full pivoting at absolute tolerance tol.
//   * Algorithm 5 only: limits of the remaining blocks are conditioned by
//     U_ij (V_ij^T y_j); these steer the ordering only.
//   * The diagonal Schur blocks S_ii -= U_ij (V_ij^T V_ij) U_ij^T are kept current.
#include "common.cuh"
#include "gemm.cuh"

#include <algorithm>
#include <cstring>
#include <functional>
#include <numeric>

namespace tlrmvn {

// ---- device helpers (float64) -------------------------------------------------------
// log(Phi(bt) - Phi(at)) for at <= bt.  Intervals inside one half are taken in
// logs, log Phi(bt) + log(-expm1(log Phi(at) - log Phi(bt))) (complements in the
// upper half), which stays finite when both probabilities underflow; intervals
// that straddle 0 take the plain difference.
__device__ double log_interval_d(double at, double bt) {
  if (at == -INFINITY) return (bt == INFINITY) ? 0.0 : log_Phi(bt);
  if (at > 0.0) {
    const double lca = log_Phi(-at);
    if (bt == INFINITY) return lca;
    return lca + log(-expm1(log_Phi(-bt) - lca));
  }
  if (bt <= 0.0) {
    const double lb = log_Phi(bt);
    return lb + log(-expm1(log_Phi(at) - lb));
  }
  const double d = 0.5 * erfc(-at * TLR_RSQRT2);
  const double e = (bt == INFINITY) ? 1.0 : 1.0 - 0.5 * erfc(bt * TLR_RSQRT2);
  return log(e - d);
}
// Mean of N(0,1) truncated to (at, bt).
__device__ double trunc_mean_d(double at, double bt) {
  double ld = log_interval_d(at, bt);
  double ta = (at > -INFINITY && at < INFINITY) ? exp(-0.5 * at * at - TLR_LOG_SQRT2PI - ld) : 0.0;
  double tb = (bt > -INFINITY && bt < INFINITY) ? exp(-0.5 * bt * bt - TLR_LOG_SQRT2PI - ld) : 0.0;
  return ta - tb;
}

__device__ __forceinline__ void argmin_merge(double& q, int& i, double q2, int i2) {
  if (q2 < q || (q2 == q && i2 < i)) {
    q = q2;
    i = i2;
  }
}
// block-wide (min q, lowest index); every thread gets the result
__device__ void block_argmin(double& q, int& i, double* shq, int* shi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o; o >>= 1) {
    double q2 = __shfl_xor_sync(0xffffffffu, q, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    argmin_merge(q, i, q2, i2);
  }
  if (lane == 0) {
    shq[wid] = q;
    shi[wid] = i;
  }
  __syncthreads();
  if (wid == 0) {
    q = lane < nw ? shq[lane] : INFINITY;
    i = lane < nw ? shi[lane] : 0x7fffffff;
    for (int o = 16; o; o >>= 1) {
      double q2 = __shfl_xor_sync(0xffffffffu, q, o);
      int i2 = __shfl_xor_sync(0xffffffffu, i, o);
      argmin_merge(q, i, q2, i2);
    }
    if (lane == 0) {
      shq[0] = q;
      shi[0] = i;
    }
  }
  __syncthreads();
  q = shq[0];
  i = shi[0];
  __syncthreads();
}
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < nw ? sh[lane] : 0.0;
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) sh[0] = v;
  }
  __syncthreads();
  v = sh[0];
  __syncthreads();
  return v;
}

// ---- covariance tiles -----------------------------------------------------------------
struct TileJob {
  double* out;              // m x m row-major (ld m)
  const int64_t* rows;      // original indices of the tile rows
  const int64_t* cols;
  int nr, nc;
};
struct CovSrc {
  const double* xy;    // n x 2 (kernel source) or null
  const double* dense; // column-major n x n, leading dimension ld (dense source) or null
  int64_t ld;
  int kernel;
  double p0, p1, nugget;
};
__device__ __forceinline__ double cov_value(const CovSrc& s, int64_t i, int64_t j) {
  if (s.dense) return s.dense[i + j * s.ld];
  double dx = s.xy[2 * i] - s.xy[2 * j], dy = s.xy[2 * i + 1] - s.xy[2 * j + 1];
  double d = sqrt(dx * dx + dy * dy);
  double v;
  if (s.kernel == TLRMVN_KERNEL_EXP) v = exp(-d / s.p0);
  else if (s.kernel == TLRMVN_KERNEL_MATERN15) {
    double t = 1.7320508075688772 * d / s.p0;
    v = (1.0 + t) * exp(-t);
  } else {
    double t = 1.7320508075688772 * d / s.p1;
    v = exp(-d / s.p0) + (1.0 + t) * exp(-t);
  }
  if (i == j) v += s.nugget;
  return v;
}
__global__ void k_cov_tiles(const TileJob* jobs, CovSrc src, int m) {
  const TileJob jb = jobs[blockIdx.y];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m * m; t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / m), j = (int)(t % m);
    jb.out[t] = (i < jb.nr && j < jb.nc) ? cov_value(src, jb.rows[i], jb.cols[j]) : 0.0;
  }
}

// ---- univariate conditioning (Trinh & Genz) of diagonal blocks --------------------------
// One block per CTA; right-looking pivoted Cholesky of a copy of the block in
// `work`.  Writes log of the estimate; with emit, also the pivot order and the
// truncated expectations in the new order.
__global__ void __launch_bounds__(512) k_uc(const int* blist, const double* diagS, const int* bsize, int m,
                                            const double* acur, const double* bcur, double* work, double* logp_out,
                                            int emit, int* order_out, double* y_out, int* status) {
  extern __shared__ double shm[];
  double* sa = shm;
  double* sb = sa + m;
  double* ss = sb + m;
  double* lcol = ss + m;
  double* sy = lcol + m;
  int* so = (int*)(sy + m);
  __shared__ double shq[32];
  __shared__ int shi[32];
  __shared__ double shy;
  const int b = blist[blockIdx.x];
  const int mb = bsize[b];
  double* A = work + (size_t)blockIdx.x * m * m;
  const double* S = diagS + (size_t)b * m * m;
  for (int t = threadIdx.x; t < mb * mb; t += blockDim.x) A[(t / mb) * m + t % mb] = S[(t / mb) * m + t % mb];
  for (int t = threadIdx.x; t < mb; t += blockDim.x) {
    sa[t] = acur[(size_t)b * m + t];
    sb[t] = bcur[(size_t)b * m + t];
    ss[t] = 0.0;
    so[t] = t;
  }
  __syncthreads();
  double logp = 0.0;
  for (int k = 0; k < mb; k++) {
    double bq = INFINITY;
    int bi = 0x7fffffff;
    for (int i = k + threadIdx.x; i < mb; i += blockDim.x) {
      double var = A[(size_t)i * m + i];
      double q;
      if (!(var > 0.0)) {
        atomicExch(status, TLRMVN_E_NOT_SPD);
        q = INFINITY;
      } else {
        double sig = sqrt(var);
        q = log_interval_d((sa[i] - ss[i]) / sig, (sb[i] - ss[i]) / sig);
      }
      argmin_merge(bq, bi, q, i);
    }
    block_argmin(bq, bi, shq, shi);
    const int piv = (bi < mb) ? bi : k;
    if (threadIdx.x == 0) {
      if (piv != k) {
        double t;
        t = sa[k]; sa[k] = sa[piv]; sa[piv] = t;
        t = sb[k]; sb[k] = sb[piv]; sb[piv] = t;
        t = ss[k]; ss[k] = ss[piv]; ss[piv] = t;
        int ti = so[k]; so[k] = so[piv]; so[piv] = ti;
      }
      logp += bq;
    }
    // (only the lower triangle of the symmetric block is kept: swapping variables k < piv
    // exchanges A(k,t) with A(piv,t) for t < k, A(t,k) with A(piv,t) for k < t < piv,
    // A(t,k) with A(t,piv) for t > piv, and the two diagonal entries)
    if (piv != k) {
      for (int t = threadIdx.x; t < mb; t += blockDim.x) {
        double *x0, *x1;
        if (t < k) {
          x0 = A + (size_t)k * m + t;
          x1 = A + (size_t)piv * m + t;
        } else if (t == k) {
          x0 = A + (size_t)k * m + k;
          x1 = A + (size_t)piv * m + piv;
        } else if (t < piv) {
          x0 = A + (size_t)t * m + k;
          x1 = A + (size_t)piv * m + t;
        } else if (t > piv) {
          x0 = A + (size_t)t * m + k;
          x1 = A + (size_t)t * m + piv;
        } else {
          continue;  // A(piv,k) stays
        }
        const double x = *x0;
        *x0 = *x1;
        *x1 = x;
      }
    }
    __syncthreads();
    const double dkk = A[(size_t)k * m + k];
    const double lkk = sqrt(dkk > 0.0 ? dkk : 1.0);
    for (int i = k + 1 + threadIdx.x; i < mb; i += blockDim.x) lcol[i] = A[(size_t)i * m + k] / lkk;
    if (threadIdx.x == 0) {
      double y = trunc_mean_d((sa[k] - ss[k]) / lkk, (sb[k] - ss[k]) / lkk);
      sy[k] = y;
      shy = y;
    }
    __syncthreads();
    const double yk = shy;
    for (int i = k + 1 + threadIdx.x; i < mb; i += blockDim.x) ss[i] += lcol[i] * yk;
    // the Schur update of the lower triangle, a row per warp
    {
      const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
      for (int i = k + 1 + (threadIdx.x >> 5); i < mb; i += nw) {
        double* row = A + (size_t)i * m;
        const double li = lcol[i];
        int jj = k + 1 + lane;
        for (; jj + 96 <= i; jj += 128) {  // (four loads per lane in flight)
          double x0 = row[jj], x1 = row[jj + 32], x2 = row[jj + 64], x3 = row[jj + 96];
          x0 -= li * lcol[jj];
          x1 -= li * lcol[jj + 32];
          x2 -= li * lcol[jj + 64];
          x3 -= li * lcol[jj + 96];
          row[jj] = x0;
          row[jj + 32] = x1;
          row[jj + 64] = x2;
          row[jj + 96] = x3;
        }
        for (; jj <= i; jj += 32) row[jj] -= li * lcol[jj];
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) logp_out[blockIdx.x] = logp;
  if (emit) {
    for (int t = threadIdx.x; t < mb; t += blockDim.x) {
      order_out[(size_t)blockIdx.x * m + t] = so[t];
      y_out[(size_t)blockIdx.x * m + t] = sy[t];
    }
  }
}

// ---- plain Cholesky of one block, in place (lower), zero above -------------------------
// (grid x: independent blocks A + x * m * m, sizes from mbs when given)
__global__ void __launch_bounds__(512) k_potrf(double* A, int mb, int m, int* status, const int* mbs) {
  extern __shared__ double col[];
  A += (size_t)blockIdx.x * m * m;
  if (mbs) mb = mbs[blockIdx.x];
  for (int k = 0; k < mb; k++) {
    const double d = A[(size_t)k * m + k];
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) atomicExch(status, TLRMVN_E_NOT_SPD);
      return;
    }
    const double lkk = sqrt(d);
    for (int i = k + 1 + threadIdx.x; i < mb; i += blockDim.x) {
      double l = A[(size_t)i * m + k] / lkk;
      A[(size_t)i * m + k] = l;
      col[i] = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) A[(size_t)k * m + k] = lkk;
    const int w = mb - k - 1;
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      int i = k + 1 + t / w, jj = k + 1 + t % w;
      if (jj <= i) A[(size_t)i * m + jj] -= col[i] * col[jj];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
    int i = t / m, jj = t % m;
    if (jj > i || i >= mb) A[t] = 0.0;
  }
}

// ---- inverse of a lower triangular block, column-parallel: one warp per column of X = L^-1 --
// Column c by forward substitution, x_c = 1 / L_cc, x_i = -(sum_{c <= t < i} L_it x_t) / L_ii
// (the dot product across the warp's lanes, x in the warp's shared-memory row).  X rows and
// columns in [0, ncols); zero above the diagonal and past mb.  L with leading dimension ldl,
// X with ldx; 8 warps per 256-thread block, 8 x ncols doubles of shared memory.  Grid y:
// independent blocks, L and X advanced by sL and sX per block, mb from mbs[y] when mbs is given.
__global__ void __launch_bounds__(256) k_trinv_cols(const double* L, int ldl, size_t sL, double* X, int ldx, size_t sX,
                                                    int mb, const int* mbs, int ncols) {
  extern __shared__ double xs[];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  L += blockIdx.y * sL;
  X += blockIdx.y * sX;
  if (mbs) mb = mbs[blockIdx.y];
  const int c = blockIdx.x * 8 + wl;
  if (c >= ncols) return;  // (whole warps; the kernel has no block-wide barrier)
  double* x = xs + (size_t)wl * ncols;
  const int top = c < mb ? c : ncols;
  for (int i = lane; i < top; i += 32) X[(size_t)i * ldx + c] = 0.0;
  if (c >= mb) return;
  for (int i = mb + lane; i < ncols; i += 32) X[(size_t)i * ldx + c] = 0.0;
  if (lane == 0) {
    const double xc = 1.0 / L[(size_t)c * ldl + c];
    x[c] = xc;
    X[(size_t)c * ldx + c] = xc;
  }
  __syncwarp();
  for (int i = c + 1; i < mb; i++) {
    const double* Li = L + (size_t)i * ldl;
    double sum = 0.0;
    for (int t = c + lane; t < i; t += 32) sum = fma(Li[t], x[t], sum);
#pragma unroll
    for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) {
      const double xi = -sum / Li[i];
      x[i] = xi;
      X[(size_t)i * ldx + c] = xi;
    }
    __syncwarp();
  }
}

// ---- blocked Cholesky pieces: one diagonal block of at most 64 in place ------------------
// (lower; its strict upper triangle zeroed; the rest of the matrix untouched)
__global__ void __launch_bounds__(256) k_potrf_diag(double* A, int nb, int ld, int* status) {
  __shared__ double col[64];
  for (int k = 0; k < nb; k++) {
    const double d = A[(size_t)k * ld + k];
    if (!(d > 0.0)) {
      if (threadIdx.x == 0) atomicExch(status, TLRMVN_E_NOT_SPD);
      return;
    }
    const double lkk = sqrt(d);
    for (int i = k + 1 + threadIdx.x; i < nb; i += blockDim.x) {
      const double l = A[(size_t)i * ld + k] / lkk;
      A[(size_t)i * ld + k] = l;
      col[i] = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) A[(size_t)k * ld + k] = lkk;
    const int w = nb - k - 1;
    for (int t = threadIdx.x; t < w * w; t += blockDim.x) {
      const int i = k + 1 + t / w, jj = k + 1 + t % w;
      if (jj <= i) A[(size_t)i * ld + jj] -= col[i] * col[jj];
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nb * nb; t += blockDim.x) {
    const int i = t / nb, jj = t % nb;
    if (jj > i) A[(size_t)i * ld + jj] = 0.0;
  }
}
// zero the strict upper triangle of the mb x mb block and every row and column past mb (m x m, ld m)
__global__ void k_zero_upper(double* A, int mb, int m) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m * m;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / m), jj = (int)(t % m);
    if (jj > i || i >= mb) A[t] = 0.0;
  }
}

// ---- adaptive cross approximation with full pivoting, in place on R --------------------
// R (mi x mj, ld m) ~ U V^T with max|R - U V^T| <= tol or rank == cap.
// U, V: m x cap row-major slots; each rank-one term balanced (|u| = |v|).
struct AcaJob {
  double* R;
  double* U;
  double* V;
  int mi, mj;
};
// |x| compared through its bit pattern (for non-negative doubles the integer order is the
// numeric order): the pivot search runs on the integer pipes, not the float64 one.
__device__ __forceinline__ long long abs_key(double x) { return __double_as_longlong(fabs(x)); }
__device__ __forceinline__ void keymax_merge(long long& a, int& i, long long a2, int i2) {
  if (a2 > a || (a2 == a && i2 < i)) {
    a = a2;
    i = i2;
  }
}
__device__ void block_keymax(long long& a, int& i, long long* sha, int* shi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o; o >>= 1) {
    long long a2 = __shfl_xor_sync(0xffffffffu, a, o);
    int i2 = __shfl_xor_sync(0xffffffffu, i, o);
    keymax_merge(a, i, a2, i2);
  }
  if (lane == 0) {
    sha[wid] = a;
    shi[wid] = i;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < nw ? sha[lane] : -1LL;
    i = lane < nw ? shi[lane] : 0x7fffffff;
    for (int o = 16; o; o >>= 1) {
      long long a2 = __shfl_xor_sync(0xffffffffu, a, o);
      int i2 = __shfl_xor_sync(0xffffffffu, i, o);
      keymax_merge(a, i, a2, i2);
    }
    if (lane == 0) {
      sha[0] = a;
      shi[0] = i;
    }
  }
  __syncthreads();
  a = sha[0];
  i = shi[0];
  __syncthreads();
}
__global__ void __launch_bounds__(512) k_aca(const AcaJob* jobs, int m, int cap, double tol, int* ranks, int* capped) {
  extern __shared__ double sm[];
  double* u = sm;
  double* v = sm + m;
  __shared__ long long shk[32];
  __shared__ double shs[32];
  __shared__ int shi[32];
  const AcaJob jb = jobs[blockIdx.x];
  const int mi = jb.mi, mj = jb.mj, tot = mi * mj;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  // entries by (row i over warps, column jj over lanes); t = i * mj + jj orders the ties
  long long akey = -1;
  int aidx = 0x7fffffff;
  // (rows are streamed four loads per lane at a time: the passes are bound by memory latency)
  for (int i = wid; i < mi; i += nw) {
    const double* row = jb.R + (size_t)i * m;
    int jj = lane;
    for (; jj + 96 < mj; jj += 128) {
      const double x0 = row[jj], x1 = row[jj + 32], x2 = row[jj + 64], x3 = row[jj + 96];
      keymax_merge(akey, aidx, abs_key(x0), i * mj + jj);
      keymax_merge(akey, aidx, abs_key(x1), i * mj + jj + 32);
      keymax_merge(akey, aidx, abs_key(x2), i * mj + jj + 64);
      keymax_merge(akey, aidx, abs_key(x3), i * mj + jj + 96);
    }
    for (; jj < mj; jj += 32) keymax_merge(akey, aidx, abs_key(row[jj]), i * mj + jj);
  }
  int rank = 0, cp = 0;
  for (;;) {
    block_keymax(akey, aidx, shk, shi);
    const double amax = akey >= 0 ? __longlong_as_double(akey) : -1.0;
    if (!(amax > tol) || aidx >= tot) break;
    if (rank >= cap) {
      cp = 1;
      break;
    }
    const int pi = aidx / mj, pj = aidx % mj;
    const double piv = jb.R[(size_t)pi * m + pj];
    for (int t = threadIdx.x; t < mi; t += blockDim.x) u[t] = jb.R[(size_t)t * m + pj];
    for (int t = threadIdx.x; t < mj; t += blockDim.x) v[t] = jb.R[(size_t)pi * m + t] / piv;
    __syncthreads();
    double nu2 = 0.0, nv2 = 0.0;
    for (int t = threadIdx.x; t < mi; t += blockDim.x) nu2 += u[t] * u[t];
    nu2 = block_sum(nu2, shs);
    for (int t = threadIdx.x; t < mj; t += blockDim.x) nv2 += v[t] * v[t];
    nv2 = block_sum(nv2, shs);
    const double f = sqrt(sqrt(nv2) / sqrt(nu2));
    for (int t = threadIdx.x; t < mi; t += blockDim.x) jb.U[(size_t)t * cap + rank] = u[t] * f;
    for (int t = threadIdx.x; t < mj; t += blockDim.x) jb.V[(size_t)t * cap + rank] = v[t] / f;
    akey = -1;
    aidx = 0x7fffffff;
    for (int i = wid; i < mi; i += nw) {
      double* row = jb.R + (size_t)i * m;
      const double ui = u[i];
      int jj = lane;
      for (; jj + 96 < mj; jj += 128) {
        double x0 = row[jj], x1 = row[jj + 32], x2 = row[jj + 64], x3 = row[jj + 96];
        x0 -= ui * v[jj];
        x1 -= ui * v[jj + 32];
        x2 -= ui * v[jj + 64];
        x3 -= ui * v[jj + 96];
        row[jj] = x0;
        row[jj + 32] = x1;
        row[jj + 64] = x2;
        row[jj + 96] = x3;
        keymax_merge(akey, aidx, abs_key(x0), i * mj + jj);
        keymax_merge(akey, aidx, abs_key(x1), i * mj + jj + 32);
        keymax_merge(akey, aidx, abs_key(x2), i * mj + jj + 64);
        keymax_merge(akey, aidx, abs_key(x3), i * mj + jj + 96);
      }
      for (; jj < mj; jj += 32) {
        const double x = row[jj] - ui * v[jj];
        row[jj] = x;
        keymax_merge(akey, aidx, abs_key(x), i * mj + jj);
      }
    }
    __syncthreads();
    rank++;
  }
  if (threadIdx.x == 0) {
    ranks[blockIdx.x] = rank;
    if (cp) atomicAdd(capped, 1);
  }
}

// ---- limit conditioning (Algorithm 5): a_i -= U_ij (V_ij^T y_j) --------------------------
struct CondJob {
  const double* U;
  const double* V;
  double* a;
  double* b;
  int mi, mj, k;
};
__global__ void k_condition(const CondJob* jobs, const double* y, int cap) {
  __shared__ double t[1024];
  const CondJob jb = jobs[blockIdx.x];
  for (int c = threadIdx.x; c < jb.k; c += blockDim.x) {
    double s = 0.0;
    for (int u = 0; u < jb.mj; u++) s += jb.V[(size_t)u * cap + c] * y[u];
    t[c] = s;
  }
  __syncthreads();
  for (int v = threadIdx.x; v < jb.mi; v += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < jb.k; c++) s += jb.U[(size_t)v * cap + c] * t[c];
    jb.a[v] -= s;
    jb.b[v] -= s;
  }
}

// ---- within-block permutation of a chosen block ------------------------------------------
// rows/cols of the diagonal block, its index list and limits, and the rows of
// the finished factor tiles U_jk (k < j).
__global__ void k_permute_block(double* S, double* tmp, int64_t* idx, double* a, double* b, const int* order, int mb,
                                int m, double* const* Urows, int nU, int cap) {
  for (int t = threadIdx.x; t < mb * mb; t += blockDim.x) {
    int i = t / mb, jj = t % mb;
    tmp[(size_t)i * m + jj] = S[(size_t)order[i] * m + order[jj]];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < mb * mb; t += blockDim.x) {
    int i = t / mb, jj = t % mb;
    S[(size_t)i * m + jj] = tmp[(size_t)i * m + jj];
  }
  __syncthreads();
  // idx, a, b via tmp as staging (3 * mb doubles)
  double* ti = tmp;
  double* ta = tmp + m;
  double* tb = tmp + 2 * m;
  for (int t = threadIdx.x; t < mb; t += blockDim.x) {
    ti[t] = (double)idx[order[t]];
    ta[t] = a[order[t]];
    tb[t] = b[order[t]];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < mb; t += blockDim.x) {
    idx[t] = (int64_t)ti[t];
    a[t] = ta[t];
    b[t] = tb[t];
  }
  __syncthreads();
  for (int q = 0; q < nU; q++) {
    double* U = Urows[q];
    for (int t = threadIdx.x; t < mb * cap; t += blockDim.x) tmp[t] = U[(size_t)order[t / cap] * cap + t % cap];
    __syncthreads();
    for (int t = threadIdx.x; t < mb * cap; t += blockDim.x) U[t] = tmp[t];
    __syncthreads();
  }
}

// ---- a cluster's variables reordered in every tile that involves it ------------------------
// M[v][c] <- M[order[v]][c] for v < mb, c < k (one m x cap slot side per CTA, 4 columns at a time)
struct PermJob {
  double* M;
  int k;
};
__global__ void __launch_bounds__(256) k_permute_rows(const PermJob* jobs, const int* order, int mb, int cap) {
  __shared__ double sh[1024 * 4];
  const PermJob jb = jobs[blockIdx.x];
  for (int c0 = 0; c0 < jb.k; c0 += 4) {
    const int w = min(4, jb.k - c0);
    for (int t = threadIdx.x; t < mb * 4; t += blockDim.x)
      if ((t & 3) < w) sh[t] = jb.M[(size_t)(t >> 2) * cap + c0 + (t & 3)];
    __syncthreads();
    for (int t = threadIdx.x; t < mb * 4; t += blockDim.x)
      if ((t & 3) < w) jb.M[(size_t)(t >> 2) * cap + c0 + (t & 3)] = sh[order[t >> 2] * 4 + (t & 3)];
    __syncthreads();
  }
}

// ---- pack slots into the compact factor layout ---------------------------------------------
struct PackJob {
  const double* U;   // slot, m x cap
  const double* V;
  double* Ucat;      // row block base of tile i: m x Krow_i, ld Krow
  int64_t ldu, col0; // column offset of (i,j) within row block i
  double* Vcat;      // first row of (i,j) in column block j: k x m
  int32_t* vmap;
  int64_t g0;        // global rank index of component 0
  int mi, mj, k;
};
__global__ void k_pack(const PackJob* jobs, int m, int cap) {
  const PackJob jb = jobs[blockIdx.x];
  for (int t = threadIdx.x; t < jb.mi * jb.k; t += blockDim.x) {
    int v = t / jb.k, c = t % jb.k;
    jb.Ucat[(int64_t)v * jb.ldu + jb.col0 + c] = jb.U[(size_t)v * cap + c];
  }
  for (int t = threadIdx.x; t < jb.k * m; t += blockDim.x) {
    int c = t / m, u = t % m;
    jb.Vcat[(int64_t)c * m + u] = (u < jb.mj) ? jb.V[(size_t)u * cap + c] : 0.0;
  }
  for (int c = threadIdx.x; c < jb.k; c += blockDim.x) jb.vmap[c] = (int32_t)(jb.g0 + c);
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------

// k-d bisection ordering (Section 3.2 geometric indexing, cardinality balanced):
// a set spanning t tiles splits into the first ceil(t/2)*m points and the rest,
// along the coordinate of larger extent (x on a tie), ranked by (that
// coordinate, the other one, original index); leaves depth first.
static void kd_order(const double* xy, int64_t n, int m, std::vector<int64_t>& perm, std::vector<int>& sizes) {
  perm.resize(n);
  std::iota(perm.begin(), perm.end(), 0);
  sizes.clear();
  std::function<void(int64_t, int64_t)> split = [&](int64_t lo, int64_t hi) {
    int64_t cnt = hi - lo;
    int64_t t = (cnt + m - 1) / m;
    if (t <= 1) {
      sizes.push_back((int)cnt);
      return;
    }
    int64_t nl = ((t + 1) / 2) * m;
    double mn[2] = {INFINITY, INFINITY}, mx[2] = {-INFINITY, -INFINITY};
    for (int64_t q = lo; q < hi; q++)
      for (int d = 0; d < 2; d++) {
        mn[d] = std::min(mn[d], xy[2 * perm[q] + d]);
        mx[d] = std::max(mx[d], xy[2 * perm[q] + d]);
      }
    int ax = (mx[0] - mn[0] >= mx[1] - mn[1]) ? 0 : 1, ot = 1 - ax;
    std::sort(perm.begin() + lo, perm.begin() + hi, [&](int64_t p, int64_t q) {
      double pa = xy[2 * p + ax], qa = xy[2 * q + ax];
      if (pa != qa) return pa < qa;
      double po = xy[2 * p + ot], qo = xy[2 * q + ot];
      if (po != qo) return po < qo;
      return p < q;
    });
    split(lo, lo + nl);
    split(lo + nl, hi);
  };
  split(0, n);
}

// Device buffers of one factorisation; freed on every exit path.
struct Build {
  std::vector<void*> ptrs;
  template <typename T>
  int get(T** p, size_t count) {
    TLR_CHECK(dalloc(p, std::max<size_t>(count, 1)));
    ptrs.push_back(*p);
    return TLRMVN_OK;
  }
  ~Build() {
    for (void* p : ptrs) cudaFree(p);
  }
};

template <typename T>
static int upload(T* dst, const std::vector<T>& src, cudaStream_t st) {
  if (src.empty()) return TLRMVN_OK;
  TLR_CUDA(cudaMemcpyAsync(dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  return TLRMVN_OK;
}

static int check_status(int* d_status, cudaStream_t st, const char* what) {
  int h = 0;
  TLR_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  if (h) return fail(h, std::string(what) + ": covariance block is not positive definite");
  return TLRMVN_OK;
}

template <bool TA, bool TB>
static int run_batched(std::vector<GemmEntry>& ent, std::vector<GemmSeg>& seg, GemmEntry* d_ent, GemmSeg* d_seg,
                       size_t ent_cap, size_t seg_cap, cudaStream_t st) {
  if (ent.empty()) return TLRMVN_OK;
  if (ent.size() > ent_cap || seg.size() > seg_cap) return fail(TLRMVN_E_CUDA, "internal: gemm job list overflow");
  int maxM = 0, maxN = 0;
  for (auto& e : ent) {
    maxM = std::max(maxM, e.M);
    maxN = std::max(maxN, e.N);
  }
  TLR_CHECK(upload(d_ent, ent, st));
  TLR_CHECK(upload(d_seg, seg, st));
  for (size_t z0 = 0; z0 < ent.size(); z0 += 65535) {
    unsigned nz = (unsigned)std::min<size_t>(65535, ent.size() - z0);
    dim3 grid((unsigned)((maxN + 63) / 64), (unsigned)((maxM + 63) / 64), nz);
    k_gemm_batched<TA, TB><<<grid, 256, 0, st>>>(d_ent + z0, d_seg);
  }
  TLR_CUDA(cudaGetLastError());
  // the host vectors are reused right away: wait for the uploads
  TLR_CUDA(cudaStreamSynchronize(st));
  return TLRMVN_OK;
}

// Cholesky factor of the leading mb x mb part of the m x m block A, in place (lower, zero
// elsewhere), and its inverse Linv: right-looking in panels of 64 -- the panel's diagonal
// block by one CTA, the panel below it through that block's inverse and the trailing update
// as GEMMs over the whole GPU -- then the inverse with one warp per column.  P (m x 64) and
// Pinv (64 x 64) are scratch.  (One CTA for the whole block is bound by one SM's float64
// rate: ~20 ms at m = 512, against ~1 ms this way.)
static int chol_inverse(double* A, int mb, int m, double* Linv, double* P, double* Pinv, GemmEntry* d_ent,
                        GemmSeg* d_seg, size_t ent_cap, size_t seg_cap, int* d_status, cudaStream_t st,
                        const char* what) {
  std::vector<GemmEntry> ent;
  std::vector<GemmSeg> seg;
  for (int k0 = 0; k0 < mb; k0 += 64) {
    const int nb = std::min(64, mb - k0), rest = mb - k0 - nb;
    double* Akk = A + (size_t)k0 * m + k0;
    k_potrf_diag<<<1, 256, 0, st>>>(Akk, nb, m, d_status);
    TLR_CUDA(cudaGetLastError());
    if (rest == 0) break;
    k_trinv_cols<<<(nb + 7) / 8, 256, 8 * (size_t)nb * sizeof(double), st>>>(Akk, m, 0, Pinv, 64, 0, nb, nullptr, nb);
    TLR_CUDA(cudaGetLastError());
    double* Apan = A + (size_t)(k0 + nb) * m + k0;
    ent.clear();
    seg.clear();
    seg.push_back(GemmSeg{Apan, Pinv, m, 64, nb});  // P = A_21 L_11^-T
    ent.push_back(GemmEntry{P, 64, rest, nb, 0, 1, 1.0, 0.0});
    TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
    ent.clear();
    seg.clear();
    seg.push_back(GemmSeg{P, P, 64, 64, nb});  // A_22 -= P P^T
    ent.push_back(GemmEntry{A + (size_t)(k0 + nb) * m + k0 + nb, m, rest, rest, 0, 1, -1.0, 1.0});
    TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
    TLR_CUDA(cudaMemcpy2DAsync(Apan, (size_t)m * sizeof(double), P, 64 * sizeof(double), (size_t)nb * sizeof(double),
                               (size_t)rest, cudaMemcpyDeviceToDevice, st));
  }
  k_zero_upper<<<std::max(1, std::min(1024, (m * m + 255) / 256)), 256, 0, st>>>(A, mb, m);
  TLR_CUDA(cudaGetLastError());
  TLR_CHECK(check_status(d_status, st, what));
  k_trinv_cols<<<(m + 7) / 8, 256, 8 * (size_t)m * sizeof(double), st>>>(A, m, 0, Linv, m, 0, mb, nullptr, m);
  TLR_CUDA(cudaGetLastError());
  return TLRMVN_OK;
}

static int factor_build(const CovSrc& src, int64_t n, std::vector<int64_t> geo, std::vector<int> sizes,
                        const double* a_ref, const double* b_ref, const tlrmvn_factor_opts& o, Factor& F) {
  cudaStream_t st = pick_stream(o.stream);
  const int m = o.tile;
  const int r = (int)sizes.size();
  const int cap = (o.max_rank > 0) ? std::min(o.max_rank, m) : m;
  const bool reorder = o.reorder != TLRMVN_REORDER_NONE;
  Build bd;
  // block-id layout: block b's variables at [b*m, b*m + sizes[b])
  std::vector<int64_t> idx_h((size_t)r * m, 0);
  {
    int64_t off = 0;
    for (int b = 0; b < r; b++) {
      for (int t = 0; t < sizes[b]; t++) idx_h[(size_t)b * m + t] = geo[off + t];
      off += sizes[b];
    }
  }
  int64_t* d_idx;
  int* d_bsize;
  double *d_a, *d_b, *diagS, *work, *Sij, *Lij, *Linv, *pool, *Xs, *Ys, *d_y;
  int *d_status, *d_order, *d_ranks, *d_capped, *d_blist;
  double* d_logp;
  TLR_CHECK(bd.get(&d_idx, (size_t)r * m));
  TLR_CHECK(bd.get(&d_bsize, r));
  TLR_CHECK(bd.get(&d_a, (size_t)r * m));
  TLR_CHECK(bd.get(&d_b, (size_t)r * m));
  TLR_CHECK(bd.get(&diagS, (size_t)r * m * m));
  TLR_CHECK(bd.get(&d_status, 1));
  double* ptmp;
  TLR_CHECK(bd.get(&d_order, (size_t)r * m));
  TLR_CHECK(bd.get(&d_y, (size_t)r * m));
  TLR_CHECK(bd.get(&ptmp, std::max<size_t>((size_t)m * std::max(m, cap), 3 * (size_t)m)));
  const bool tlr = o.schur == TLRMVN_SCHUR_TLR;
  const size_t max_pairs_step = (size_t)(r / 2 + 1) * (size_t)(r / 2 + 1);
  // TLR arithmetic: tiles truncated per batch, each written out densely first (<= 1 GiB of them)
  const size_t tbatch =
      tlr ? std::max<size_t>(1, std::min<size_t>({max_pairs_step, (size_t)16384, ((size_t)1 << 30) / ((size_t)m * m * 8)}))
          : (size_t)r;
  const size_t jcap = std::max<size_t>(tbatch, (size_t)r);
  TLR_CHECK(bd.get(&d_ranks, jcap));
  TLR_CHECK(bd.get(&d_capped, 1));
  TLR_CHECK(bd.get(&d_blist, r));
  TLR_CHECK(bd.get(&d_logp, r));
  TLR_CHECK(bd.get(&Linv, (size_t)m * m));
  double *Pch = nullptr, *Pinv = nullptr;  // scratch of the blocked Cholesky
  TLR_CHECK(bd.get(&Pch, (size_t)m * 64));
  TLR_CHECK(bd.get(&Pinv, (size_t)64 * 64));
  const size_t npairs = (size_t)r * (r - 1) / 2;
  TLR_CHECK(bd.get(&pool, std::max<size_t>(npairs, 1) * 2 * (size_t)m * cap));
  if (tlr) {
    TLR_CHECK(bd.get(&Sij, tbatch * m * m));  // the batch of dense tiles to truncate
    Lij = nullptr;
  } else {
    TLR_CHECK(bd.get(&Sij, (size_t)std::max(r - 1, 1) * m * m));
    TLR_CHECK(bd.get(&Lij, (size_t)std::max(r - 1, 1) * m * m));
  }
  const size_t uc_par = reorder ? (size_t)r : 1;
  TLR_CHECK(bd.get(&work, uc_par * m * m));
  TLR_CHECK(bd.get(&Xs, max_pairs_step * cap * cap));
  TLR_CHECK(bd.get(&Ys, max_pairs_step * cap * m));
  const size_t ent_cap = std::max<size_t>(max_pairs_step, (size_t)r) + 8, seg_cap = 2 * ent_cap;
  GemmEntry* d_ent;
  GemmSeg* d_seg;
  TileJob* d_tj;
  AcaJob* d_aj;
  CondJob* d_cj;
  PackJob* d_pj;
  double** d_urows;
  TLR_CHECK(bd.get(&d_ent, ent_cap));
  TLR_CHECK(bd.get(&d_seg, seg_cap));
  TLR_CHECK(bd.get(&d_tj, jcap));
  TLR_CHECK(bd.get(&d_aj, jcap));
  PermJob* d_pmj;
  TLR_CHECK(bd.get(&d_pmj, (size_t)r));
  TLR_CHECK(bd.get(&d_cj, (size_t)r));
  TLR_CHECK(bd.get(&d_pj, std::max<size_t>(npairs, 1)));
  TLR_CHECK(bd.get(&d_urows, (size_t)r));
  TLR_CHECK(upload(d_idx, idx_h, st));
  TLR_CHECK(upload(d_bsize, sizes, st));
  TLR_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  TLR_CUDA(cudaMemsetAsync(d_capped, 0, sizeof(int), st));
  if (reorder) {
    std::vector<double> ah((size_t)r * m, 0.0), bh((size_t)r * m, 0.0);
    for (int b = 0; b < r; b++)
      for (int t = 0; t < sizes[b]; t++) {
        ah[(size_t)b * m + t] = a_ref[idx_h[(size_t)b * m + t]];
        bh[(size_t)b * m + t] = b_ref[idx_h[(size_t)b * m + t]];
      }
    TLR_CHECK(upload(d_a, ah, st));
    TLR_CHECK(upload(d_b, bh, st));
  }
  // diagonal blocks of Sigma
  {
    std::vector<TileJob> tj(r);
    for (int b = 0; b < r; b++)
      tj[b] = TileJob{diagS + (size_t)b * m * m, d_idx + (size_t)b * m, d_idx + (size_t)b * m, sizes[b], sizes[b]};
    TLR_CHECK(upload(d_tj, tj, st));
    k_cov_tiles<<<dim3(std::max(1, (m * m + 255) / 256 / 4), r), 256, 0, st>>>(d_tj, src, m);
    TLR_CUDA(cudaGetLastError());
  }
  std::vector<int> pos2blk(r);
  std::iota(pos2blk.begin(), pos2blk.end(), 0);
  const size_t uc_smem = (size_t)m * (5 * sizeof(double) + sizeof(int));
  TLR_CHECK(raise_smem_limit((const void*)k_uc, (size_t)uc_smem));
  TLR_CHECK(raise_smem_limit((const void*)k_aca, 2 * m * sizeof(double)));
  TLR_CHECK(raise_smem_limit((const void*)k_potrf, m * sizeof(double)));
  TLR_CHECK(raise_smem_limit((const void*)k_trinv_cols, 8 * (size_t)m * sizeof(double)));
  const int uc_threads = m >= 256 ? 512 : 256;

  if (o.reorder == TLRMVN_REORDER_BLOCK) {
    // Algorithm 4: one UC estimate per original block, then a selection sort
    std::vector<int> bl(r);
    std::iota(bl.begin(), bl.end(), 0);
    TLR_CHECK(upload(d_blist, bl, st));
    k_uc<<<r, uc_threads, uc_smem, st>>>(d_blist, diagS, d_bsize, m, d_a, d_b, work, d_logp, 1, d_order, d_y,
                                          d_status);
    TLR_CUDA(cudaGetLastError());
    TLR_CHECK(check_status(d_status, st, "block reordering"));
    // within-block order: the UC pivot order of each original block
    for (int b = 0; b < r; b++) {
      k_permute_block<<<1, 512, 0, st>>>(diagS + (size_t)b * m * m, ptmp, d_idx + (size_t)b * m, d_a + (size_t)b * m,
                                         d_b + (size_t)b * m, d_order + (size_t)b * m, sizes[b], m, d_urows, 0, cap);
      TLR_CUDA(cudaGetLastError());
    }
    std::vector<double> p(r);
    TLR_CUDA(cudaMemcpyAsync(p.data(), d_logp, r * 8, cudaMemcpyDeviceToHost, st));
    TLR_CUDA(cudaStreamSynchronize(st));
    for (int j = 0; j < r; j++) {
      int best = j;
      for (int l = j + 1; l < r; l++)
        if (p[pos2blk[l]] < p[pos2blk[best]]) best = l;
      std::swap(pos2blk[j], pos2blk[best]);
    }
  }

  std::vector<int> slot((size_t)r * r, -1), rank((size_t)r * r, 0);
  int next_slot = 0;
  auto Uslot = [&](int s) { return pool + (size_t)s * 2 * m * cap; };
  auto Vslot = [&](int s) { return pool + (size_t)s * 2 * m * cap + (size_t)m * cap; };
  std::vector<GemmEntry> ent;
  std::vector<GemmSeg> seg;

  // ---- tile-low-rank arithmetic (TLRMVN_SCHUR_TLR): Algorithm 5 as printed -------------------
  // Every unordered cluster pair {p, q} owns pool slot sid(p, q): Sigma_pq ~ U V^T, U on the
  // variables of cluster rowc[s] (Sigma_qp = V U^T).  The slots first hold the ACA-compressed
  // covariance; position by position they are overwritten by the factor tiles L_ij (rowc = the
  // cluster at position i) and, further right, by the truncated Schur tiles.
  auto tlr_schur_loop = [&]() -> int {
    auto sid = [&](int p, int q) -> size_t {
      if (p > q) std::swap(p, q);
      return (size_t)p * r - (size_t)p * (p + 1) / 2 + (size_t)(q - p - 1);
    };
    std::vector<int> rowc(std::max<size_t>(npairs, 1), 0), rk(std::max<size_t>(npairs, 1), 0);
    auto side = [&](size_t s, int c) { return rowc[s] == c ? Uslot((int)s) : Vslot((int)s); };
    struct Trunc {
      size_t s;
      int rc, mi, mj;
    };
    // ACA of the dense tiles Sij[t] (t < jobs.size()) into their slots
    auto truncate = [&](const std::vector<Trunc>& jobs) -> int {
      if (jobs.empty()) return TLRMVN_OK;
      std::vector<AcaJob> aj(jobs.size());
      for (size_t t = 0; t < jobs.size(); t++)
        aj[t] = AcaJob{Sij + t * m * m, Uslot((int)jobs[t].s), Vslot((int)jobs[t].s), jobs[t].mi, jobs[t].mj};
      TLR_CHECK(upload(d_aj, aj, st));
      k_aca<<<(unsigned)aj.size(), 512, 2 * m * sizeof(double), st>>>(d_aj, m, cap, o.tol, d_ranks, d_capped);
      TLR_CUDA(cudaGetLastError());
      std::vector<int> got(jobs.size());
      TLR_CUDA(cudaMemcpyAsync(got.data(), d_ranks, got.size() * sizeof(int), cudaMemcpyDeviceToHost, st));
      TLR_CUDA(cudaStreamSynchronize(st));
      for (size_t t = 0; t < jobs.size(); t++) {
        rk[jobs[t].s] = got[t];
        rowc[jobs[t].s] = jobs[t].rc;
      }
      return TLRMVN_OK;
    };
    // -- the TLR covariance: every off-diagonal block compressed by ACA at tol
    {
      std::vector<TileJob> tj;
      std::vector<Trunc> jobs;
      auto flush = [&]() -> int {
        if (tj.empty()) return TLRMVN_OK;
        TLR_CHECK(upload(d_tj, tj, st));
        k_cov_tiles<<<dim3(std::max(1, (m * m + 255) / 256 / 4), (unsigned)tj.size()), 256, 0, st>>>(d_tj, src, m);
        TLR_CUDA(cudaGetLastError());
        TLR_CHECK(truncate(jobs));
        tj.clear();
        jobs.clear();
        return TLRMVN_OK;
      };
      for (int p = 0; p < r; p++)
        for (int q = p + 1; q < r; q++) {
          tj.push_back(TileJob{Sij + tj.size() * m * m, d_idx + (size_t)p * m, d_idx + (size_t)q * m, sizes[p], sizes[q]});
          jobs.push_back(Trunc{sid(p, q), p, sizes[p], sizes[q]});
          if (tj.size() == tbatch) TLR_CHECK(flush());
        }
      TLR_CHECK(flush());
    }
    for (int j = 0; j < r; j++) {
      int chosen = 0;
      if (o.reorder == TLRMVN_REORDER_ITERATIVE) {
        // -- lines 4-8: UC of every remaining block; the smallest estimate takes position j
        std::vector<int> bl(pos2blk.begin() + j, pos2blk.end());
        TLR_CHECK(upload(d_blist, bl, st));
        k_uc<<<(unsigned)bl.size(), uc_threads, uc_smem, st>>>(d_blist, diagS, d_bsize, m, d_a, d_b, work, d_logp, 1,
                                                               d_order, d_y, d_status);
        TLR_CUDA(cudaGetLastError());
        TLR_CHECK(check_status(d_status, st, "iterative block reordering"));
        std::vector<double> p(bl.size());
        TLR_CUDA(cudaMemcpyAsync(p.data(), d_logp, p.size() * 8, cudaMemcpyDeviceToHost, st));
        TLR_CUDA(cudaStreamSynchronize(st));
        int best = 0;
        for (size_t l = 1; l < p.size(); l++)
          if (p[l] < p[best]) best = (int)l;
        chosen = best;
        std::swap(pos2blk[j], pos2blk[j + best]);
        // its within-block order: the diagonal block, indices and limits, and the
        // cluster's variables in every tile that involves it
        const int c = pos2blk[j];
        const int* ord = d_order + (size_t)chosen * m;
        k_permute_block<<<1, 512, 0, st>>>(diagS + (size_t)c * m * m, ptmp, d_idx + (size_t)c * m, d_a + (size_t)c * m,
                                           d_b + (size_t)c * m, ord, sizes[c], m, d_urows, 0, cap);
        TLR_CUDA(cudaGetLastError());
        std::vector<PermJob> pj;
        for (int q = 0; q < r; q++) {
          if (q == c) continue;
          const size_t s = sid(c, q);
          if (rk[s]) pj.push_back(PermJob{side(s, c), rk[s]});
        }
        if (!pj.empty()) {
          TLR_CHECK(upload(d_pmj, pj, st));
          k_permute_rows<<<(unsigned)pj.size(), 256, 0, st>>>(d_pmj, ord, sizes[c], cap);
          TLR_CUDA(cudaGetLastError());
        }
        TLR_CUDA(cudaStreamSynchronize(st));
      }
      const int cj = pos2blk[j], mj = sizes[cj];
      double* Sjj = diagS + (size_t)cj * m * m;
      // -- line 10: L_jj and its inverse
      TLR_CHECK(chol_inverse(Sjj, mj, m, Linv, Pch, Pinv, d_ent, d_seg, ent_cap, seg_cap, d_status, st,
                             "diagonal Cholesky"));
      if (j == r - 1) break;
      // -- line 12: L_ij = Sigma_ij (.) Sigma_jj^-T = U (L_jj^-1 V)^T, truncated; in batches
      {
        std::vector<int> qs;
        for (int i = j + 1; i < r; i++)
          if (rk[sid(pos2blk[i], cj)]) qs.push_back(i);
        for (size_t q0 = 0; q0 < qs.size(); q0 += tbatch) {
          const size_t nb = std::min(tbatch, qs.size() - q0);
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < nb; t++) {  // W_t = L_jj^-1 V (mj x k) into Ys
            const size_t s = sid(pos2blk[qs[q0 + t]], cj);
            seg.push_back(GemmSeg{Linv, side(s, cj), m, cap, mj});
            ent.push_back(GemmEntry{Ys + t * m * cap, cap, mj, rk[s], (int)t, (int)t + 1, 1.0, 0.0});
          }
          TLR_CHECK((run_batched<false, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          std::vector<Trunc> jobs;
          for (size_t t = 0; t < nb; t++) {  // D_t = U W_t^T (mi x mj)
            const int ci = pos2blk[qs[q0 + t]];
            const size_t s = sid(ci, cj);
            seg.push_back(GemmSeg{side(s, ci), Ys + t * m * cap, cap, cap, rk[s]});
            ent.push_back(GemmEntry{Sij + t * m * m, m, sizes[ci], mj, (int)t, (int)t + 1, 1.0, 0.0});
            jobs.push_back(Trunc{s, ci, sizes[ci], mj});
          }
          TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          TLR_CHECK(truncate(jobs));
        }
      }
      // -- line 13 (Algorithm 5): a_i, b_i -= L_ij y_j
      if (o.reorder == TLRMVN_REORDER_ITERATIVE) {
        std::vector<CondJob> cj_jobs;
        for (int i = j + 1; i < r; i++) {
          const int ci = pos2blk[i];
          const size_t s = sid(ci, cj);
          if (!rk[s]) continue;
          cj_jobs.push_back(CondJob{Uslot((int)s), Vslot((int)s), d_a + (size_t)ci * m, d_b + (size_t)ci * m, sizes[ci],
                                    mj, rk[s]});
        }
        if (!cj_jobs.empty()) {
          TLR_CHECK(upload(d_cj, cj_jobs, st));
          k_condition<<<(unsigned)cj_jobs.size(), 256, 0, st>>>(d_cj, d_y + (size_t)chosen * m, cap);
          TLR_CUDA(cudaGetLastError());
          TLR_CUDA(cudaStreamSynchronize(st));
        }
      }
      // -- lines 15-19, diagonal blocks (dense, exact): S_ii -= U_ij (V_ij^T V_ij) U_ij^T
      {
        std::vector<int> is;
        for (int i = j + 1; i < r; i++)
          if (rk[sid(pos2blk[i], cj)]) is.push_back(i);
        if (!is.empty()) {
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < is.size(); t++) {
            const size_t s = sid(pos2blk[is[t]], cj);
            seg.push_back(GemmSeg{Vslot((int)s), Vslot((int)s), cap, cap, mj});
            ent.push_back(GemmEntry{Xs + t * cap * cap, rk[s], rk[s], rk[s], (int)t, (int)t + 1, 1.0, 0.0});
          }
          TLR_CHECK((run_batched<true, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < is.size(); t++) {
            const int ci = pos2blk[is[t]];
            const size_t s = sid(ci, cj);
            seg.push_back(GemmSeg{Xs + t * cap * cap, Uslot((int)s), rk[s], cap, rk[s]});
            ent.push_back(GemmEntry{Ys + t * m * cap, m, rk[s], sizes[ci], (int)t, (int)t + 1, 1.0, 0.0});
          }
          TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < is.size(); t++) {
            const int ci = pos2blk[is[t]];
            const size_t s = sid(ci, cj);
            seg.push_back(GemmSeg{Uslot((int)s), Ys + t * m * cap, cap, m, rk[s]});
            ent.push_back(GemmEntry{diagS + (size_t)ci * m * m, m, sizes[ci], sizes[ci], (int)t, (int)t + 1, -1.0, 1.0});
          }
          TLR_CHECK((run_batched<false, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
        }
      }
      // -- lines 15-19, off-diagonal: Sigma_i1j1 (-) L_i1j L_j1j^T, truncated; in batches
      {
        std::vector<std::pair<int, int>> pr;  // (i1, j1), j < j1 < i1, both factor tiles nonzero
        for (int j1 = j + 1; j1 < r; j1++) {
          if (!rk[sid(pos2blk[j1], cj)]) continue;
          for (int i1 = j1 + 1; i1 < r; i1++)
            if (rk[sid(pos2blk[i1], cj)]) pr.push_back({i1, j1});
        }
        for (size_t p0 = 0; p0 < pr.size(); p0 += tbatch) {
          const size_t nb = std::min(tbatch, pr.size() - p0);
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < nb; t++) {  // X_t = V_i1j^T V_j1j (k1 x k2)
            const size_t s1 = sid(pos2blk[pr[p0 + t].first], cj), s2 = sid(pos2blk[pr[p0 + t].second], cj);
            seg.push_back(GemmSeg{side(s1, cj), side(s2, cj), cap, cap, mj});
            ent.push_back(GemmEntry{Xs + t * cap * cap, rk[s2], rk[s1], rk[s2], (int)t, (int)t + 1, 1.0, 0.0});
          }
          TLR_CHECK((run_batched<true, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < nb; t++) {  // Z_t = -U_i1j X_t (mi1 x k2)
            const int ci1 = pos2blk[pr[p0 + t].first];
            const size_t s1 = sid(ci1, cj), s2 = sid(pos2blk[pr[p0 + t].second], cj);
            seg.push_back(GemmSeg{side(s1, ci1), Xs + t * cap * cap, cap, rk[s2], rk[s1]});
            ent.push_back(GemmEntry{Ys + t * m * cap, cap, sizes[ci1], rk[s2], (int)t, (int)t + 1, -1.0, 0.0});
          }
          TLR_CHECK((run_batched<false, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          std::vector<Trunc> jobs;
          for (size_t t = 0; t < nb; t++) {  // D_t = U V^T + Z_t U_j1j^T (mi1 x mj1)
            const int ci1 = pos2blk[pr[p0 + t].first], cj1 = pos2blk[pr[p0 + t].second];
            const size_t s = sid(ci1, cj1), s2 = sid(cj1, cj);
            const int g0 = (int)seg.size();
            seg.push_back(GemmSeg{side(s, ci1), side(s, cj1), cap, cap, rk[s]});
            seg.push_back(GemmSeg{Ys + t * m * cap, side(s2, cj1), cap, cap, rk[s2]});
            ent.push_back(GemmEntry{Sij + t * m * m, m, sizes[ci1], sizes[cj1], g0, g0 + 2, 1.0, 0.0});
            jobs.push_back(Trunc{s, ci1, sizes[ci1], sizes[cj1]});
          }
          TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          TLR_CHECK(truncate(jobs));
        }
      }
    }
    // the finished factor: L_ij in slot sid(cluster of i, cluster of j), U on i's variables
    for (int i = 0; i < r; i++)
      for (int j = 0; j < i; j++) {
        const size_t s = sid(pos2blk[i], pos2blk[j]);
        if (rk[s] && rowc[s] != pos2blk[i]) return fail(TLRMVN_E_CUDA, "internal: factor tile orientation");
        slot[(size_t)i * r + j] = (int)s;
        rank[(size_t)i * r + j] = rk[s];
      }
    return TLRMVN_OK;
  };

  if (tlr) {
    TLR_CHECK(tlr_schur_loop());
  } else {
    for (int j = 0; j < r; j++) {
      // -- choose the block of position j and its within-block order
      bool permute = false;
      int chosen = 0;
      if (o.reorder == TLRMVN_REORDER_ITERATIVE) {
        std::vector<int> bl(pos2blk.begin() + j, pos2blk.end());
        TLR_CHECK(upload(d_blist, bl, st));
        k_uc<<<(unsigned)bl.size(), uc_threads, uc_smem, st>>>(d_blist, diagS, d_bsize, m, d_a, d_b, work, d_logp, 1,
                                                               d_order, d_y, d_status);
        TLR_CUDA(cudaGetLastError());
        TLR_CHECK(check_status(d_status, st, "iterative block reordering"));
        std::vector<double> p(bl.size());
        TLR_CUDA(cudaMemcpyAsync(p.data(), d_logp, p.size() * 8, cudaMemcpyDeviceToHost, st));
        TLR_CUDA(cudaStreamSynchronize(st));
        int best = 0;
        for (size_t l = 1; l < p.size(); l++)
          if (p[l] < p[best]) best = (int)l;
        const int jt = j + best;
        chosen = best;
        if (jt != j) {
          std::swap(pos2blk[j], pos2blk[jt]);
          for (int k = 0; k < j; k++) {
            std::swap(slot[(size_t)j * r + k], slot[(size_t)jt * r + k]);
            std::swap(rank[(size_t)j * r + k], rank[(size_t)jt * r + k]);
          }
        }
        permute = true;
      }
      const int bj = pos2blk[j];
      const int mj = sizes[bj];
      double* Sjj = diagS + (size_t)bj * m * m;
      const double* yj = d_y + (size_t)chosen * m;
      if (permute) {
        std::vector<double*> ur;
        for (int k = 0; k < j; k++)
          if (rank[(size_t)j * r + k] > 0) ur.push_back(Uslot(slot[(size_t)j * r + k]));
        TLR_CHECK(upload(d_urows, ur, st));
        k_permute_block<<<1, 512, 0, st>>>(Sjj, ptmp, d_idx + (size_t)bj * m, d_a + (size_t)bj * m, d_b + (size_t)bj * m,
                                           d_order + (size_t)chosen * m, mj, m, d_urows, (int)ur.size(), cap);
        TLR_CUDA(cudaGetLastError());
        TLR_CUDA(cudaStreamSynchronize(st));
      }
      // -- L_jj and its inverse
      TLR_CHECK(chol_inverse(Sjj, mj, m, Linv, Pch, Pinv, d_ent, d_seg, ent_cap, seg_cap, d_status, st,
                             "diagonal Cholesky"));
      const int nrem = r - 1 - j;
      if (nrem == 0) break;
      // -- Sigma_ij for the remaining blocks
      {
        std::vector<TileJob> tj(nrem);
        for (int q = 0; q < nrem; q++) {
          int bi = pos2blk[j + 1 + q];
          tj[q] = TileJob{Sij + (size_t)q * m * m, d_idx + (size_t)bi * m, d_idx + (size_t)bj * m, sizes[bi], mj};
        }
        TLR_CHECK(upload(d_tj, tj, st));
        k_cov_tiles<<<dim3(std::max(1, (m * m + 255) / 256 / 4), nrem), 256, 0, st>>>(d_tj, src, m);
        TLR_CUDA(cudaGetLastError());
        TLR_CUDA(cudaStreamSynchronize(st));
      }
      // -- left-looking update S_ij -= sum_k U_ik (V_ik^T V_jk) U_jk^T
      {
        struct P {
          int q, k;
          size_t xo, yo;
        };
        std::vector<P> pairs;
        size_t xo = 0, yo = 0;
        for (int q = 0; q < nrem; q++) {
          int i = j + 1 + q;
          for (int k = 0; k < j; k++) {
            int kik = rank[(size_t)i * r + k], kjk = rank[(size_t)j * r + k];
            if (!kik || !kjk) continue;
            pairs.push_back(P{q, k, xo, yo});
            xo += (size_t)kik * kjk;
            yo += (size_t)kik * m;
          }
        }
        if (!pairs.empty()) {
          if (xo > max_pairs_step * cap * cap || yo > max_pairs_step * cap * m)
            return fail(TLRMVN_E_CUDA, "internal: left-looking scratch overflow");
          ent.clear();
          seg.clear();
          for (auto& pr : pairs) {  // X_ik = V_ik^T V_jk
            int i = j + 1 + pr.q;
            int kik = rank[(size_t)i * r + pr.k], kjk = rank[(size_t)j * r + pr.k];
            int mk = sizes[pos2blk[pr.k]];
            seg.push_back(GemmSeg{Vslot(slot[(size_t)i * r + pr.k]), Vslot(slot[(size_t)j * r + pr.k]), cap, cap, mk});
            ent.push_back(GemmEntry{Xs + pr.xo, kjk, kik, kjk, (int)seg.size() - 1, (int)seg.size(), 1.0, 0.0});
          }
          TLR_CHECK((run_batched<true, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          for (auto& pr : pairs) {  // Y_ik = X_ik U_jk^T
            int i = j + 1 + pr.q;
            int kik = rank[(size_t)i * r + pr.k], kjk = rank[(size_t)j * r + pr.k];
            seg.push_back(GemmSeg{Xs + pr.xo, Uslot(slot[(size_t)j * r + pr.k]), kjk, cap, kjk});
            ent.push_back(GemmEntry{Ys + pr.yo, m, kik, mj, (int)seg.size() - 1, (int)seg.size(), 1.0, 0.0});
          }
          TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          size_t p0 = 0;
          for (int q = 0; q < nrem; q++) {  // S_ij -= sum_k U_ik Y_ik
            int i = j + 1 + q;
            int s0 = (int)seg.size();
            while (p0 < pairs.size() && pairs[p0].q == q) {
              auto& pr = pairs[p0++];
              int kik = rank[(size_t)i * r + pr.k];
              seg.push_back(GemmSeg{Uslot(slot[(size_t)i * r + pr.k]), Ys + pr.yo, cap, m, kik});
            }
            if ((int)seg.size() > s0)
              ent.push_back(GemmEntry{Sij + (size_t)q * m * m, m, sizes[pos2blk[i]], mj, s0, (int)seg.size(), -1.0, 1.0});
          }
          TLR_CHECK((run_batched<false, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
        }
      }
      // -- L_ij = S_ij L_jj^-T
      ent.clear();
      seg.clear();
      for (int q = 0; q < nrem; q++) {
        int mi = sizes[pos2blk[j + 1 + q]];
        seg.push_back(GemmSeg{Sij + (size_t)q * m * m, Linv, m, m, mj});
        ent.push_back(GemmEntry{Lij + (size_t)q * m * m, m, mi, mj, q, q + 1, 1.0, 0.0});
      }
      TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
      // -- ACA of every L_ij into fresh slots
      {
        std::vector<AcaJob> aj(nrem);
        for (int q = 0; q < nrem; q++) {
          int i = j + 1 + q;
          int s = next_slot++;
          slot[(size_t)i * r + j] = s;
          aj[q] = AcaJob{Lij + (size_t)q * m * m, Uslot(s), Vslot(s), sizes[pos2blk[i]], mj};
        }
        TLR_CHECK(upload(d_aj, aj, st));
        k_aca<<<nrem, 512, 2 * m * sizeof(double), st>>>(d_aj, m, cap, o.tol, d_ranks, d_capped);
        TLR_CUDA(cudaGetLastError());
        std::vector<int> rk(nrem);
        TLR_CUDA(cudaMemcpyAsync(rk.data(), d_ranks, nrem * sizeof(int), cudaMemcpyDeviceToHost, st));
        TLR_CUDA(cudaStreamSynchronize(st));
        for (int q = 0; q < nrem; q++) rank[(size_t)(j + 1 + q) * r + j] = rk[q];
      }
      // -- Algorithm 5: condition the limits of the remaining blocks
      if (o.reorder == TLRMVN_REORDER_ITERATIVE) {
        std::vector<CondJob> cj;
        for (int q = 0; q < nrem; q++) {
          int i = j + 1 + q, bi = pos2blk[i], k = rank[(size_t)i * r + j];
          if (!k) continue;
          int s = slot[(size_t)i * r + j];
          cj.push_back(CondJob{Uslot(s), Vslot(s), d_a + (size_t)bi * m, d_b + (size_t)bi * m, sizes[bi], mj, k});
        }
        if (!cj.empty()) {
          TLR_CHECK(upload(d_cj, cj, st));
          k_condition<<<(unsigned)cj.size(), 256, 0, st>>>(d_cj, yj, cap);
          TLR_CUDA(cudaGetLastError());
          TLR_CUDA(cudaStreamSynchronize(st));
        }
      }
      // -- diagonal Schur blocks: S_ii -= U_ij (V_ij^T V_ij) U_ij^T
      {
        std::vector<int> qs;
        size_t xo = 0, yo = 0;
        std::vector<size_t> xof, yof;
        for (int q = 0; q < nrem; q++) {
          int k = rank[(size_t)(j + 1 + q) * r + j];
          if (!k) continue;
          qs.push_back(q);
          xof.push_back(xo);
          yof.push_back(yo);
          xo += (size_t)k * k;
          yo += (size_t)k * m;
        }
        if (!qs.empty()) {
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < qs.size(); t++) {
            int i = j + 1 + qs[t], k = rank[(size_t)i * r + j], s = slot[(size_t)i * r + j];
            seg.push_back(GemmSeg{Vslot(s), Vslot(s), cap, cap, mj});
            ent.push_back(GemmEntry{Xs + xof[t], k, k, k, (int)t, (int)t + 1, 1.0, 0.0});
          }
          TLR_CHECK((run_batched<true, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < qs.size(); t++) {
            int i = j + 1 + qs[t], k = rank[(size_t)i * r + j], s = slot[(size_t)i * r + j];
            int mi = sizes[pos2blk[i]];
            seg.push_back(GemmSeg{Xs + xof[t], Uslot(s), k, cap, k});
            ent.push_back(GemmEntry{Ys + yof[t], m, k, mi, (int)t, (int)t + 1, 1.0, 0.0});
          }
          TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
          ent.clear();
          seg.clear();
          for (size_t t = 0; t < qs.size(); t++) {
            int i = j + 1 + qs[t], k = rank[(size_t)i * r + j], s = slot[(size_t)i * r + j];
            int bi = pos2blk[i], mi = sizes[bi];
            seg.push_back(GemmSeg{Uslot(s), Ys + yof[t], cap, m, k});
            ent.push_back(GemmEntry{diagS + (size_t)bi * m * m, m, mi, mi, (int)t, (int)t + 1, -1.0, 1.0});
          }
          TLR_CHECK((run_batched<false, false>(ent, seg, d_ent, d_seg, ent_cap, seg_cap, st)));
        }
      }
    }
  }
  // -- assemble the handle
  F.n = n;
  F.r = r;
  F.m = m;
  F.tile_off.assign(r + 1, 0);
  for (int j = 0; j < r; j++) F.tile_off[j + 1] = F.tile_off[j] + sizes[pos2blk[j]];
  F.rank = std::vector<int32_t>(rank.begin(), rank.end());
  TLR_CUDA(cudaMemcpyAsync(&F.capped, d_capped, sizeof(int), cudaMemcpyDeviceToHost, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  if (o.strict_rank && F.capped > 0)
    return fail(TLRMVN_E_RANK, std::to_string(F.capped) + " off-diagonal tiles reached the rank cap " +
                                   std::to_string(cap) + " before the tolerance");
  TLR_CHECK(factor_alloc_compact(F, st));
  for (int j = 0; j < r; j++)
    TLR_CUDA(cudaMemcpyAsync(F.B + (size_t)j * m * m, diagS + (size_t)pos2blk[j] * m * m, (size_t)m * m * 8,
                             cudaMemcpyDeviceToDevice, st));
  {
    std::vector<PackJob> pj;
    for (int i = 0; i < r; i++) {
      int64_t col = 0;
      for (int j = 0; j < i; j++) {
        int k = rank[(size_t)i * r + j];
        if (!k) continue;
        int64_t vr = 0;
        for (int t = j + 1; t < i; t++) vr += rank[(size_t)t * r + j];
        int s = slot[(size_t)i * r + j];
        pj.push_back(PackJob{Uslot(s), Vslot(s), F.Ucat + (size_t)m * F.krow_off[i], F.krow(i), col,
                             F.Vcat + (size_t)m * (F.kcol_off[j] + vr), F.vmap + F.kcol_off[j] + vr,
                             F.krow_off[i] + col, sizes[pos2blk[i]], sizes[pos2blk[j]], k});
        col += k;
      }
    }
    if (!pj.empty()) {
      TLR_CHECK(upload(d_pj, pj, st));
      k_pack<<<(unsigned)pj.size(), 256, 0, st>>>(d_pj, m, cap);
      TLR_CUDA(cudaGetLastError());
    }
  }
  std::vector<int64_t> idx_fin((size_t)r * m);
  TLR_CUDA(cudaMemcpyAsync(idx_fin.data(), d_idx, idx_fin.size() * 8, cudaMemcpyDeviceToHost, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  F.perm.resize(n);
  for (int j = 0; j < r; j++)
    for (int t = 0; t < sizes[pos2blk[j]]; t++) F.perm[F.tile_off[j] + t] = idx_fin[(size_t)pos2blk[j] * m + t];
  return factor_finish(F, st);
}

// ---- post-hoc within-tile reordering of a finished factor for new limits ----------------------
// (No counterpart in the paper; derived from its factor structure.)  The block
// reorderings of Section 3.3 also order the variables within each diagonal
// block by the limits, which a resident factor meets anew in every request.
// For each tile j: P_j is the pivot order of univariate conditioning on the
// tile's conditional covariance B_j B_j^T with the new limits; the new diagonal
// block is Lt_j = chol(P_j B_j B_j^T P_j^T), and Q_j = B_j^-1 P_j^T Lt_j is
// orthogonal, so L' = diag(P) L diag(Q) has diagonal blocks Lt_j, satisfies
// L' L'^T = P L L^T P^T, and keeps every off-diagonal rank: the tile's rows in
// the row blocks are permuted (U_jk -> P_j U_jk) and its column blocks rotated
// (V_ij -> Q_j^T V_ij, i.e. the stored V^T rows times Q_j).

// Xp_j[v][w] = S_j[p_j(v)][p_j(w)] for v, w < mb_j (one tile per block row)
__global__ void k_gather_sym(const double* S, const int* order, const int* bsize, int m, double* Xp) {
  const int j = blockIdx.y, mb = bsize[j];
  const double* Sj = S + (size_t)j * m * m;
  const int* p = order + (size_t)j * m;
  double* X = Xp + (size_t)j * m * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m * m; t += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)(t / m), w = (int)(t % m);
    X[t] = (v < mb && w < mb) ? Sj[(size_t)p[v] * m + p[w]] : 0.0;
  }
}
// X_j[p_j(v)][c] = L_j[v][c] (rows scattered back: X = P^T L)
__global__ void k_scatter_rows(const double* L, const int* order, const int* bsize, int m, double* X) {
  const int j = blockIdx.y, mb = bsize[j];
  const int* p = order + (size_t)j * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m * m; t += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)(t / m), c = (int)(t % m);
    if (v < mb) X[(size_t)j * m * m + (size_t)p[v] * m + c] = L[(size_t)j * m * m + t];
    else X[(size_t)j * m * m + t] = 0.0;
  }
}
// rows of row block j of Ucat permuted: Unew_j[v][k] = Uold_j[p_j(v)][k]
__global__ void k_permute_urows(const double* Uold, double* Unew, const int64_t* krow_off, const int* order,
                                const int* bsize, int m) {
  const int j = blockIdx.y, mb = bsize[j];
  const int64_t K = krow_off[j + 1] - krow_off[j], base = (int64_t)m * krow_off[j];
  const int* p = order + (size_t)j * m;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)m * K; t += (int64_t)gridDim.x * blockDim.x) {
    const int v = (int)(t / K);
    const int64_t k = t % K;
    Unew[base + t] = (v < mb) ? Uold[base + (int64_t)p[v] * K + k] : Uold[base + t];
  }
}

static int reorder_tiles(Factor& F, const double* a, const double* b, cudaStream_t st, Factor& G) {
  const int r = F.r, m = F.m;
  G.n = F.n;
  G.r = r;
  G.m = m;
  G.capped = F.capped;
  G.device = F.device;
  G.tile_off = F.tile_off;
  G.rank = F.rank;
  TLR_CHECK(factor_alloc_compact(G, st));
  Build bd;
  int *d_bsize, *d_blist, *d_order, *d_status;
  double *d_a, *d_b, *S, *X, *Binv, *Qm, *work, *d_logp, *d_y;
  int64_t* d_kro;
  GemmEntry* d_ent;
  GemmSeg* d_seg;
  const size_t mm = (size_t)m * m;
  TLR_CHECK(bd.get(&d_bsize, r));
  TLR_CHECK(bd.get(&d_blist, r));
  TLR_CHECK(bd.get(&d_order, (size_t)r * m));
  TLR_CHECK(bd.get(&d_status, 1));
  TLR_CHECK(bd.get(&d_a, (size_t)r * m));
  TLR_CHECK(bd.get(&d_b, (size_t)r * m));
  TLR_CHECK(bd.get(&S, r * mm));
  TLR_CHECK(bd.get(&X, r * mm));
  TLR_CHECK(bd.get(&Binv, r * mm));
  TLR_CHECK(bd.get(&Qm, r * mm));
  TLR_CHECK(bd.get(&work, r * mm));
  TLR_CHECK(bd.get(&d_logp, r));
  TLR_CHECK(bd.get(&d_y, (size_t)r * m));
  TLR_CHECK(bd.get(&d_kro, (size_t)r + 1));
  TLR_CHECK(bd.get(&d_ent, (size_t)r));
  TLR_CHECK(bd.get(&d_seg, (size_t)r));
  std::vector<int> sizes(r), bl(r);
  std::vector<double> ha((size_t)r * m, 0.0), hb((size_t)r * m, 0.0);
  for (int j = 0; j < r; j++) {
    sizes[j] = (int)F.tsize(j);
    bl[j] = j;
    for (int v = 0; v < sizes[j]; v++) {
      const int64_t orig = F.perm[F.tile_off[j] + v];
      ha[(size_t)j * m + v] = a[orig];
      hb[(size_t)j * m + v] = b[orig];
    }
  }
  TLR_CHECK(upload(d_bsize, sizes, st));
  TLR_CHECK(upload(d_blist, bl, st));
  TLR_CHECK(upload(d_a, ha, st));
  TLR_CHECK(upload(d_b, hb, st));
  TLR_CHECK(upload(d_kro, F.krow_off, st));
  TLR_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
  std::vector<GemmEntry> ent;
  std::vector<GemmSeg> seg;
  // S_j = B_j B_j^T, the tile's conditional covariance given all earlier tiles
  for (int j = 0; j < r; j++) {
    seg.push_back(GemmSeg{F.B + j * mm, F.B + j * mm, m, m, sizes[j]});
    ent.push_back(GemmEntry{S + j * mm, m, sizes[j], sizes[j], j, j + 1, 1.0, 0.0});
  }
  TLR_CUDA(cudaMemsetAsync(S, 0, r * mm * 8, st));
  TLR_CHECK((run_batched<false, true>(ent, seg, d_ent, d_seg, (size_t)r, (size_t)r, st)));
  // P_j: the univariate-conditioning pivot order with the new limits
  const size_t uc_smem = (size_t)m * (5 * sizeof(double) + sizeof(int));
  TLR_CHECK(raise_smem_limit((const void*)k_uc, uc_smem));
  TLR_CHECK(raise_smem_limit((const void*)k_potrf, m * sizeof(double)));
  k_uc<<<r, m >= 256 ? 512 : 256, uc_smem, st>>>(d_blist, S, d_bsize, m, d_a, d_b, work, d_logp, 1, d_order, d_y,
                                                  d_status);
  TLR_CUDA(cudaGetLastError());
  TLR_CHECK(check_status(d_status, st, "within-tile reordering"));
  // Lt_j = chol(P S_j P^T) (in work); X_j = P^T Lt_j; Binv_j = B_j^-1; Q_j = Binv_j X_j
  const unsigned gx = (unsigned)std::max<size_t>(1, std::min<size_t>(64, (mm + 255) / 256));
  k_gather_sym<<<dim3(gx, r), 256, 0, st>>>(S, d_order, d_bsize, m, work);
  // (all tiles at once: one CTA per tile for the Cholesky factors, a warp per column of the inverses)
  TLR_CHECK(raise_smem_limit((const void*)k_trinv_cols, 8 * (size_t)m * sizeof(double)));
  k_potrf<<<r, 512, m * sizeof(double), st>>>(work, 0, m, d_status, d_bsize);
  k_trinv_cols<<<dim3((m + 7) / 8, r), 256, 8 * (size_t)m * sizeof(double), st>>>(F.B, m, mm, Binv, m, mm, 0, d_bsize,
                                                                                   m);
  TLR_CUDA(cudaGetLastError());
  TLR_CHECK(check_status(d_status, st, "within-tile reordering (Cholesky)"));
  k_scatter_rows<<<dim3(gx, r), 256, 0, st>>>(work, d_order, d_bsize, m, X);
  ent.clear();
  seg.clear();
  for (int j = 0; j < r; j++) {
    seg.push_back(GemmSeg{Binv + j * mm, X + j * mm, m, m, sizes[j]});
    ent.push_back(GemmEntry{Qm + j * mm, m, sizes[j], sizes[j], j, j + 1, 1.0, 0.0});
  }
  TLR_CUDA(cudaMemsetAsync(Qm, 0, r * mm * 8, st));
  TLR_CHECK((run_batched<false, false>(ent, seg, d_ent, d_seg, (size_t)r, (size_t)r, st)));
  // the new factor: B_j = Lt_j; V^T rows of column block j times Q_j; rows of U permuted
  TLR_CUDA(cudaMemcpyAsync(G.B, work, r * mm * 8, cudaMemcpyDeviceToDevice, st));
  if (F.ktot > 0) {
    TLR_CUDA(cudaMemsetAsync(G.Vcat, 0, (size_t)m * F.ktot * 8, st));
    ent.clear();
    seg.clear();
    for (int j = 0; j < r; j++) {
      const int64_t kc = F.kcol(j);
      if (!kc) continue;
      seg.push_back(GemmSeg{F.Vcat + (size_t)m * F.kcol_off[j], Qm + j * mm, m, m, sizes[j]});
      ent.push_back(GemmEntry{G.Vcat + (size_t)m * F.kcol_off[j], m, (int)kc, sizes[j], (int)seg.size() - 1,
                              (int)seg.size(), 1.0, 0.0});
    }
    TLR_CHECK((run_batched<false, false>(ent, seg, d_ent, d_seg, (size_t)r, (size_t)r, st)));
    int64_t kmax = 0;
    for (int j = 0; j < r; j++) kmax = std::max(kmax, F.krow(j));
    const unsigned gu = (unsigned)std::max<int64_t>(1, std::min<int64_t>(256, ((int64_t)m * kmax + 255) / 256));
    k_permute_urows<<<dim3(gu, r), 256, 0, st>>>(F.Ucat, G.Ucat, d_kro, d_order, d_bsize, m);
    TLR_CUDA(cudaMemcpyAsync(G.vmap, F.vmap, (size_t)F.ktot * 4, cudaMemcpyDeviceToDevice, st));
  }
  TLR_CUDA(cudaGetLastError());
  std::vector<int> order((size_t)r * m);
  TLR_CUDA(cudaMemcpyAsync(order.data(), d_order, order.size() * 4, cudaMemcpyDeviceToHost, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  G.perm.resize(F.n);
  for (int j = 0; j < r; j++)
    for (int v = 0; v < sizes[j]; v++)
      G.perm[F.tile_off[j] + v] = F.perm[F.tile_off[j] + order[(size_t)j * m + v]];
  return factor_finish(G, st);
}

static int check_fopts(const tlrmvn_factor_opts* o, int64_t n, const double* a, const double* b) {
  if (!o) return fail(TLRMVN_E_INVAL, "null options");
  if (n <= 0) return fail(TLRMVN_E_INVAL, "n must be positive");
  if (o->tile <= 0 || o->tile > 1024) return fail(TLRMVN_E_INVAL, "tile must be in 1..1024");
  if (!(o->tol >= 0.0)) return fail(TLRMVN_E_INVAL, "tol must be >= 0");
  if (o->max_rank < 0) return fail(TLRMVN_E_INVAL, "max_rank must be >= 0");
  if (o->reorder < 0 || o->reorder > 2) return fail(TLRMVN_E_INVAL, "bad reorder mode");
  if (o->schur != TLRMVN_SCHUR_EXACT && o->schur != TLRMVN_SCHUR_TLR) return fail(TLRMVN_E_INVAL, "bad schur mode");
  if (o->reorder != TLRMVN_REORDER_NONE) {
    if (!a || !b) return fail(TLRMVN_E_INVAL, "reordering needs limits a_ref, b_ref");
    for (int64_t i = 0; i < n; i++)
      if (std::isnan(a[i]) || std::isnan(b[i]) || a[i] > b[i] || a[i] == INFINITY || b[i] == -INFINITY)
        return fail(TLRMVN_E_INVAL, "limits must satisfy a_i <= b_i, no NaN");
  }
  return TLRMVN_OK;
}

}  // namespace tlrmvn

using namespace tlrmvn;

extern "C" int tlrmvn_factor_kernel(const double* xy, int64_t n, int kernel, const double* params, double nugget,
                                    const double* a_ref, const double* b_ref, const tlrmvn_factor_opts* opts,
                                    tlrmvn_factor_t* out) {
  if (!xy || !params || !out) return fail(TLRMVN_E_INVAL, "null argument");
  TLR_CHECK(check_fopts(opts, n, a_ref, b_ref));
  if (kernel < 0 || kernel > 2) return fail(TLRMVN_E_INVAL, "unknown kernel");
  if (!(params[0] > 0.0) || (kernel == TLRMVN_KERNEL_EXP_MATERN15 && !(params[1] > 0.0)) || !(nugget >= 0.0))
    return fail(TLRMVN_E_INVAL, "kernel parameters must be positive");
  for (int64_t i = 0; i < 2 * n; i++)
    if (!std::isfinite(xy[i])) return fail(TLRMVN_E_INVAL, "locations must be finite");
  std::vector<int64_t> geo;
  std::vector<int> sizes;
  kd_order(xy, n, opts->tile, geo, sizes);
  cudaStream_t st = pick_stream(opts->stream);
  double* dxy = nullptr;
  TLR_CHECK(dalloc(&dxy, (size_t)2 * n));
  cudaError_t e = cudaMemcpyAsync(dxy, xy, (size_t)2 * n * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    dfree(dxy);
    return cuda_fail(e, "upload locations");
  }
  CovSrc src{dxy, nullptr, 0, kernel, params[0], kernel == TLRMVN_KERNEL_EXP_MATERN15 ? params[1] : 0.0, nugget};
  Factor* F = new Factor();
  cudaGetDevice(&F->device);
  int s = factor_build(src, n, geo, sizes, a_ref, b_ref, *opts, *F);
  dfree(dxy);
  if (s != TLRMVN_OK) {
    delete F;
    return s;
  }
  *out = reinterpret_cast<tlrmvn_factor_t>(F);
  return TLRMVN_OK;
}

extern "C" int tlrmvn_factor_dense(const double* cov, int64_t n, int64_t ld, const double* a_ref, const double* b_ref,
                                   const tlrmvn_factor_opts* opts, tlrmvn_factor_t* out) {
  if (!cov || !out) return fail(TLRMVN_E_INVAL, "null argument");
  TLR_CHECK(check_fopts(opts, n, a_ref, b_ref));
  if (ld < n) return fail(TLRMVN_E_INVAL, "ld must be >= n");
  std::vector<int64_t> geo(n);
  std::iota(geo.begin(), geo.end(), 0);
  std::vector<int> sizes;
  for (int64_t off = 0; off < n; off += opts->tile) sizes.push_back((int)std::min<int64_t>(opts->tile, n - off));
  cudaStream_t st = pick_stream(opts->stream);
  double* dcov = nullptr;
  TLR_CHECK(dalloc(&dcov, (size_t)ld * n));
  cudaError_t e = cudaMemcpyAsync(dcov, cov, (size_t)ld * n * 8, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    dfree(dcov);
    return cuda_fail(e, "upload covariance");
  }
  CovSrc src{nullptr, dcov, ld, 0, 0.0, 0.0, 0.0};
  Factor* F = new Factor();
  cudaGetDevice(&F->device);
  int s = factor_build(src, n, geo, sizes, a_ref, b_ref, *opts, *F);
  dfree(dcov);
  if (s != TLRMVN_OK) {
    delete F;
    return s;
  }
  *out = reinterpret_cast<tlrmvn_factor_t>(F);
  return TLRMVN_OK;
}

extern "C" int tlrmvn_factor_reorder_tiles(tlrmvn_factor_t f, const double* a, const double* b, void* stream,
                                           tlrmvn_factor_t* out) {
  if (!f || !a || !b || !out) return fail(TLRMVN_E_INVAL, "null argument");
  Factor& F = *reinterpret_cast<Factor*>(f);
  for (int64_t i = 0; i < F.n; i++)
    if (std::isnan(a[i]) || std::isnan(b[i]) || a[i] > b[i] || a[i] == INFINITY || b[i] == -INFINITY)
      return fail(TLRMVN_E_INVAL, "limits must satisfy a_i <= b_i, a_i < +inf, b_i > -inf, no NaN");
  int cur = 0;
  cudaGetDevice(&cur);
  TLR_CUDA(cudaSetDevice(F.device));
  cudaStream_t st = pick_stream(stream);
  Factor* G = new Factor();
  const int s = reorder_tiles(F, a, b, st, *G);
  cudaSetDevice(cur);
  if (s != TLRMVN_OK) {
    delete G;
    return s;
  }
  *out = reinterpret_cast<tlrmvn_factor_t>(G);
  return TLRMVN_OK;
}
