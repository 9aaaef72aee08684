// SIMT GEMMs in float64 / float32: the low-rank shifts of the FP64 and FP32
// integrands, and the products of the FP64 factorisation.
#pragma once
#include "common.cuh"

namespace tlrmvn {

// C[rowmap[i]][:] = A (M x K, row-major) * B (K x N, row-major) (+ C when accumulate);
// rowmap may be null.  64x64 output tile per 256-thread block, 4x4 per thread, K in steps of 16.
template <typename T>
__global__ void __launch_bounds__(256) k_gemm_nn(int M, int64_t N, int64_t K, const T* __restrict__ A, int64_t lda,
                                                 const T* __restrict__ B, int64_t ldb, T* __restrict__ C, int64_t ldc,
                                                 const int32_t* __restrict__ rowmap, int accumulate) {
  __shared__ T As[16][64 + 1];
  __shared__ T Bs[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64;
  const int64_t n0 = (int64_t)blockIdx.x * 64;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = (T)0;
  for (int64_t k0 = 0; k0 < K; k0 += 16) {
    for (int l = threadIdx.x; l < 64 * 16; l += 256) {
      int mm = l >> 4, kk = l & 15;
      int gm = m0 + mm;
      int64_t gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? A[(int64_t)gm * lda + gk] : (T)0;
    }
    for (int l = threadIdx.x; l < 16 * 64; l += 256) {
      int kk = l >> 6, nn = l & 63;
      int64_t gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < K && gn < N) ? B[gk * ldb + gn] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
    int64_t row = rowmap ? (int64_t)rowmap[gm] : (int64_t)gm;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn < N) {
        T* c = C + row * ldc + gn;
        *c = accumulate ? *c + acc[i][j] : acc[i][j];
      }
    }
  }
}

template <typename T>
inline void gemm_nn(cudaStream_t st, int M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B, int64_t ldb,
                    T* C, int64_t ldc, const int32_t* rowmap, int accumulate = 0) {
  if (M <= 0 || N <= 0) return;
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64));
  k_gemm_nn<T><<<grid, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, rowmap, accumulate);
}

// ---- batched, grouped float64 GEMM for the factorisation ---------------------------
// For every batch entry e:  C_e = alpha * sum_{segments s of e} op(A_s) op(B_s) + beta * C_e
// op(X) = X or X^T (template flags).  A_s is (M x K_s) after op, B_s (K_s x N).
struct GemmSeg {
  const double* A;
  const double* B;
  int lda, ldb, K;
};
struct GemmEntry {
  double* C;
  int ldc, M, N;
  int seg0, seg1;  // segments [seg0, seg1)
  double alpha, beta;
};

template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_batched(const GemmEntry* __restrict__ ent, const GemmSeg* __restrict__ seg) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const GemmEntry e = ent[blockIdx.z];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  if (m0 >= e.M || n0 >= e.N) return;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.0;
  for (int s = e.seg0; s < e.seg1; s++) {
    const GemmSeg g = seg[s];
    for (int k0 = 0; k0 < g.K; k0 += 16) {
      for (int l = threadIdx.x; l < 64 * 16; l += 256) {
        int mm, kk;
        if (TA) { kk = l >> 6; mm = l & 63; } else { mm = l >> 4; kk = l & 15; }
        int gm = m0 + mm, gk = k0 + kk;
        double v = 0.0;
        if (gm < e.M && gk < g.K) v = TA ? g.A[(int64_t)gk * g.lda + gm] : g.A[(int64_t)gm * g.lda + gk];
        As[kk][mm] = v;
      }
      for (int l = threadIdx.x; l < 16 * 64; l += 256) {
        int kk, nn;
        if (TB) { nn = l >> 4; kk = l & 15; } else { kk = l >> 6; nn = l & 63; }
        int gk = k0 + kk, gn = n0 + nn;
        double v = 0.0;
        if (gk < g.K && gn < e.N) v = TB ? g.B[(int64_t)gn * g.ldb + gk] : g.B[(int64_t)gk * g.ldb + gn];
        Bs[kk][nn] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; kk++) {
        double a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; i++)
#pragma unroll
          for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    int gm = m0 + ty + 16 * i;
    if (gm >= e.M) continue;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      int gn = n0 + tx + 16 * j;
      if (gn >= e.N) continue;
      double* c = e.C + (int64_t)gm * e.ldc + gn;
      *c = e.alpha * acc[i][j] + (e.beta == 0.0 ? 0.0 : e.beta * *c);
    }
  }
}

}  // namespace tlrmvn
