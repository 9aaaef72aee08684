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

// float32 C = A B (+ C): 128 x 128 output tile per 256-thread block, 8 x 8 per
// thread (two 4 x 4 quadrants so that shared-memory reads are float4), K in
// steps of 8 with the next step's tile prefetched into registers while the
// current one is multiplied (shared memory double-buffered, one barrier per step).
// Requires lda, ldb, ldc multiples of 4, 16-byte aligned A, B, C and K a multiple of 8.
static __global__ void __launch_bounds__(256, 2) k_sgemm128(int M, int64_t N, int K, const float* __restrict__ A, int64_t lda,
                                                  const float* __restrict__ B, int64_t ldb, float* __restrict__ C,
                                                  int64_t ldc, const int32_t* __restrict__ rowmap, int accumulate) {
  __shared__ __align__(16) float As[2][8][128];
  __shared__ __align__(16) float Bs[2][8][128];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * 128;
  const int64_t n0 = (int64_t)blockIdx.x * 128;
  const int am = tid >> 1, ak = (tid & 1) * 4;   // A: row, first k of a float4
  const int bk = tid >> 5, bn = (tid & 31) * 4;  // B: k row, first column of a float4
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; i++)
#pragma unroll
    for (int j = 0; j < 8; j++) acc[i][j] = 0.0f;
  float4 ra, rb;
  auto load = [&](int k0) {
    const int gm = m0 + am;
    ra = (gm < M) ? *reinterpret_cast<const float4*>(A + (int64_t)gm * lda + k0 + ak) : make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t gn = n0 + bn;
    const float* brow = B + (int64_t)(k0 + bk) * ldb;
    if (gn + 3 < N) {
      rb = *reinterpret_cast<const float4*>(brow + gn);
    } else {
      rb.x = gn < N ? brow[gn] : 0.f;
      rb.y = gn + 1 < N ? brow[gn + 1] : 0.f;
      rb.z = gn + 2 < N ? brow[gn + 2] : 0.f;
      rb.w = 0.f;
    }
  };
  auto store = [&](int buf) {
    As[buf][ak][am] = ra.x;
    As[buf][ak + 1][am] = ra.y;
    As[buf][ak + 2][am] = ra.z;
    As[buf][ak + 3][am] = ra.w;
    *reinterpret_cast<float4*>(&Bs[buf][bk][bn]) = rb;
  };
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += 8) {
    const bool more = k0 + 8 < K;
    if (more) load(k0 + 8);
#pragma unroll
    for (int kk = 0; kk < 8; kk++) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; i++)
#pragma unroll
        for (int j = 0; j < 8; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; i++) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (gm >= M) continue;
    const int64_t row = rowmap ? (int64_t)rowmap[gm] : (int64_t)gm;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int64_t gn = n0 + h * 64 + tx * 4;
      float* c = C + row * ldc + gn;
      const float* v = &acc[i][4 * h];
      if (gn + 3 < N) {
        float4 o = make_float4(v[0], v[1], v[2], v[3]);
        if (accumulate) {
          const float4 p = *reinterpret_cast<const float4*>(c);
          o.x += p.x;
          o.y += p.y;
          o.z += p.z;
          o.w += p.w;
        }
        *reinterpret_cast<float4*>(c) = o;
      } else {
        for (int q = 0; q < 3; q++)
          if (gn + q < N) c[q] = accumulate ? c[q] + v[q] : v[q];
      }
    }
  }
}

// The same for M <= 64 (the in-tile coupling of 64-variable sub-tiles): a 64 x 256 output tile
// per block, 4 x 16 per thread (rows ty*4.., columns tx*4 + 64 h), so no half of the block's
// rows is padding.  Same requirements as k_sgemm128.
static __global__ void __launch_bounds__(256, 2) k_sgemm64(int M, int64_t N, int K, const float* __restrict__ A,
                                                           int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                           float* __restrict__ C, int64_t ldc,
                                                           const int32_t* __restrict__ rowmap, int accumulate) {
  __shared__ __align__(16) float As[2][8][64];
  __shared__ __align__(16) float Bs[2][8][256];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t n0 = (int64_t)blockIdx.x * 256;
  const int am = (tid & 127) >> 1, ak = (tid & 1) * 4;  // A (threads 0..127): row, first k of a float4
  const int bk = tid >> 5, bn = (tid & 31) * 4;         // B: k row, first column of the first float4 (+128)
  float acc[4][16];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 16; j++) acc[i][j] = 0.0f;
  float4 ra, rb0, rb1;
  auto ldb4 = [&](const float* brow, int64_t gn) {
    float4 r;
    if (gn + 3 < N) {
      r = *reinterpret_cast<const float4*>(brow + gn);
    } else {
      r.x = gn < N ? brow[gn] : 0.f;
      r.y = gn + 1 < N ? brow[gn + 1] : 0.f;
      r.z = gn + 2 < N ? brow[gn + 2] : 0.f;
      r.w = 0.f;
    }
    return r;
  };
  auto load = [&](int k0) {
    ra = (tid < 128 && am < M) ? *reinterpret_cast<const float4*>(A + (int64_t)am * lda + k0 + ak)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
    const float* brow = B + (int64_t)(k0 + bk) * ldb;
    rb0 = ldb4(brow, n0 + bn);
    rb1 = ldb4(brow, n0 + 128 + bn);
  };
  auto store = [&](int buf) {
    if (tid < 128) {
      As[buf][ak][am] = ra.x;
      As[buf][ak + 1][am] = ra.y;
      As[buf][ak + 2][am] = ra.z;
      As[buf][ak + 3][am] = ra.w;
    }
    *reinterpret_cast<float4*>(&Bs[buf][bk][bn]) = rb0;
    *reinterpret_cast<float4*>(&Bs[buf][bk][128 + bn]) = rb1;
  };
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += 8) {
    const bool more = k0 + 8 < K;
    if (more) load(k0 + 8);
#pragma unroll
    for (int kk = 0; kk < 8; kk++) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      float b[16];
#pragma unroll
      for (int h = 0; h < 4; h++) {
        const float4 bh = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 * h + tx * 4]);
        b[4 * h] = bh.x;
        b[4 * h + 1] = bh.y;
        b[4 * h + 2] = bh.z;
        b[4 * h + 3] = bh.w;
      }
      const float a[4] = {a0.x, a0.y, a0.z, a0.w};
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 16; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) {
      store(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int gm = ty * 4 + i;
    if (gm >= M) continue;
    const int64_t row = rowmap ? (int64_t)rowmap[gm] : (int64_t)gm;
#pragma unroll
    for (int h = 0; h < 4; h++) {
      const int64_t gn = n0 + h * 64 + tx * 4;
      float* c = C + row * ldc + gn;
      const float* v = &acc[i][4 * h];
      if (gn + 3 < N) {
        float4 o = make_float4(v[0], v[1], v[2], v[3]);
        if (accumulate) {
          const float4 q = *reinterpret_cast<const float4*>(c);
          o.x += q.x;
          o.y += q.y;
          o.z += q.z;
          o.w += q.w;
        }
        *reinterpret_cast<float4*>(c) = o;
      } else {
        for (int q = 0; q < 3; q++)
          if (gn + q < N) c[q] = accumulate ? c[q] + v[q] : v[q];
      }
    }
  }
}

template <typename T>
inline void gemm_nn(cudaStream_t st, int M, int64_t N, int64_t K, const T* A, int64_t lda, const T* B, int64_t ldb,
                    T* C, int64_t ldc, const int32_t* rowmap, int accumulate = 0) {
  if (M <= 0 || N <= 0) return;
  if constexpr (sizeof(T) == 4) {
    const bool aligned = (lda % 4 == 0) && (ldb % 4 == 0) && (ldc % 4 == 0) && (K % 8 == 0) && K > 0 &&
                         ((uintptr_t)A % 16 == 0) && ((uintptr_t)B % 16 == 0) && ((uintptr_t)C % 16 == 0);
    if (aligned && M <= 64) {
      k_sgemm64<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(M, N, (int)K, (const float*)A, lda, (const float*)B, ldb,
                                                             (float*)C, ldc, rowmap, accumulate);
      return;
    }
    if (aligned) {
      dim3 grid((unsigned)((N + 127) / 128), (unsigned)((M + 127) / 128));
      k_sgemm128<<<grid, 256, 0, st>>>(M, N, (int)K, (const float*)A, lda, (const float*)B, ldb, (float*)C, ldc,
                                       rowmap, accumulate);
      return;
    }
  }
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
      // (small ranks leave most of the last 16-deep step empty: only its kn rows are summed)
      const int kn = min(16, g.K - k0);
      if (kn == 16) {
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
      } else {
        for (int kk = 0; kk < kn; kk++) {
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
