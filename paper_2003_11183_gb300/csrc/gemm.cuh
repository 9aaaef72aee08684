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

// ---- float32 C = At^T B (+ C) with the first operand stored k-major -------------------
// At is K x M (row k holds column k of the product's first factor), so that a k-step of
// it is a plain copy: the tiles of At and B go by cp.async straight into a ring of four
// shared-memory stages (no registers held for the copies, three steps in flight while
// one is multiplied).  A BM x 128 output tile per block of 256 threads, TM x 8 outputs
// per thread (4-row by 4-column quadrants, so that shared-memory reads are float4) as
// paired float32 FMAs (two FMAs an instruction, each rounded as fmaf).  BM = 128, TM = 8:
// the shifts and projections; BM = 64, TM = 4: the in-tile coupling of 64-variable
// sub-tiles, 64 rows only, whose launches over the samples would otherwise hold about
// nine warps per SM and wait on memory.  Requires lda, ldb, ldc multiples of 4, 16-byte
// aligned At, B, C and K a multiple of 8; the ragged columns of the last row and column
// blocks are zero-filled copies.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory");
}

template <int BM, int TM>
__global__ void __launch_bounds__(256, TM == 4 ? 3 : 2)
    k_sgemm_t(int M, int64_t N, int K, const float* __restrict__ At, int64_t lda, const float* __restrict__ B,
              int64_t ldb, float* __restrict__ C, int64_t ldc, const int32_t* __restrict__ rowmap, int accumulate) {
  static_assert((BM == 128 && TM == 8) || (BM == 64 && TM == 4), "tile shapes");
  constexpr int S = 4;  // stages (256 threads: BM / TM row groups x 16 column groups)
  __shared__ __align__(16) float As[S][8][BM];
  __shared__ __align__(16) float Bs[S][8][128];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // ty < BM / TM
  const int m0 = blockIdx.y * BM;
  const int64_t n0 = (int64_t)blockIdx.x * 128;
  float2 acc[TM][4];  // acc[i][j]: columns 2j, 2j + 1 of row i
#pragma unroll
  for (int i = 0; i < TM; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = make_float2(0.0f, 0.0f);
  // the copies of k-step ks into stage buf
  auto issue = [&](int ks, int buf) {
    const int k0 = ks * 8;
    if (tid < 2 * BM) {  // the At tile: 2 BM float4
      const int kk = tid / (BM / 4), mm = (tid % (BM / 4)) * 4, gm = m0 + mm;
      const int bytes = gm + 3 < M ? 16 : (gm < M ? 4 * (M - gm) : 0);
      cp_async16(&As[buf][kk][mm], bytes ? At + (int64_t)(k0 + kk) * lda + gm : At, bytes);
    }
    {  // the B tile: 256 float4
      const int kk = tid >> 5, nn = (tid & 31) * 4;
      const int64_t gn = n0 + nn;
      const int bytes = gn + 3 < N ? 16 : (gn < N ? (int)(4 * (N - gn)) : 0);
      cp_async16(&Bs[buf][kk][nn], bytes ? B + (int64_t)(k0 + kk) * ldb + gn : B, bytes);
    }
  };
  const int nk = K / 8;
  pdl_trigger();
  pdl_wait();  // B and C may be the preceding kernels' output
#pragma unroll
  for (int s = 0; s < S - 1; s++) {
    if (s < nk) issue(s, s);
    cp_async_commit();
  }
  for (int ks = 0; ks < nk; ks++) {
    cp_async_wait<S - 2>();  // this thread's copies of step ks have landed
    __syncthreads();         // everyone's have, and everyone is done with step ks - 1's stage
    if (ks + S - 1 < nk) issue(ks + S - 1, (ks + S - 1) % S);
    cp_async_commit();
    const int buf = ks % S;
#pragma unroll
    for (int kk = 0; kk < 8; kk++) {
      float a[TM];
      {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
        a[0] = a0.x, a[1] = a0.y, a[2] = a0.z, a[3] = a0.w;
        if constexpr (TM == 8) {
          const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][BM / 2 + ty * 4]);
          a[4] = a1.x, a[5] = a1.y, a[6] = a1.z, a[7] = a1.w;
        }
      }
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + tx * 4]);
      const float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w), make_float2(b1.x, b1.y),
                           make_float2(b1.z, b1.w)};
#pragma unroll
      for (int i = 0; i < TM; i++) {
        const float2 aa = make_float2(a[i], a[i]);
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = __ffma2_rn(aa, b[j], acc[i][j]);
      }
    }
  }
  cp_async_wait<0>();  // (only empty groups remain)
#pragma unroll
  for (int i = 0; i < TM; i++) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : BM / 2 + ty * 4 + i - 4);
    if (gm >= M) continue;
    const int64_t row = rowmap ? (int64_t)rowmap[gm] : (int64_t)gm;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int64_t gn = n0 + h * 64 + tx * 4;
      float* c = C + row * ldc + gn;
      const float v[4] = {acc[i][2 * h].x, acc[i][2 * h].y, acc[i][2 * h + 1].x, acc[i][2 * h + 1].y};
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

// The same product for any shape and alignment: 64 x 64 output tile per 256-thread
// block, 4 x 4 per thread, K in steps of 16.
static __global__ void __launch_bounds__(256) k_gemm_tn_f32(int M, int64_t N, int64_t K, const float* __restrict__ At,
                                                     int64_t lda, const float* __restrict__ B, int64_t ldb,
                                                     float* __restrict__ C, int64_t ldc,
                                                     const int32_t* __restrict__ rowmap, int accumulate) {
  __shared__ float As[16][64];
  __shared__ float Bs[16][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * 64;
  const int64_t n0 = (int64_t)blockIdx.x * 64;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) acc[i][j] = 0.0f;
  pdl_trigger();
  pdl_wait();  // B and C may be the preceding kernels' output
  for (int64_t k0 = 0; k0 < K; k0 += 16) {
    for (int l = threadIdx.x; l < 16 * 64; l += 256) {
      const int kk = l >> 6, mm = l & 63;
      const int gm = m0 + mm;
      const int64_t gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? At[gk * lda + gm] : 0.0f;
    }
    for (int l = threadIdx.x; l < 16 * 64; l += 256) {
      const int kk = l >> 6, nn = l & 63;
      const int64_t gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < K && gn < N) ? B[gk * ldb + gn] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; kk++) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; i++) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
    const int64_t row = rowmap ? (int64_t)rowmap[gm] : (int64_t)gm;
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int64_t gn = n0 + tx + 16 * j;
      if (gn < N) {
        float* c = C + row * ldc + gn;
        *c = accumulate ? *c + acc[i][j] : acc[i][j];
      }
    }
  }
}

// C[rowmap[i]][:] = sum_k At[k][i] B[k][:] (+ C when accumulate): the float path's products
inline void gemm_tn_f32(cudaStream_t st, int M, int64_t N, int64_t K, const float* At, int64_t lda, const float* B,
                        int64_t ldb, float* C, int64_t ldc, const int32_t* rowmap, int accumulate = 0) {
  if (M <= 0 || N <= 0) return;
  const bool aligned = (lda % 4 == 0) && (ldb % 4 == 0) && (ldc % 4 == 0) && (K % 8 == 0) && K > 0 &&
                       ((uintptr_t)At % 16 == 0) && ((uintptr_t)B % 16 == 0) && ((uintptr_t)C % 16 == 0);
  // (programmatic dependent launches: each kernel waits for its predecessor before it reads)
  if (aligned) {
    if (M <= 64) {
      launch_pdl(k_sgemm_t<64, 4>, dim3((unsigned)((N + 127) / 128), 1), dim3(256), 0, st, M, N, (int)K, At, lda, B,
                 ldb, C, ldc, rowmap, accumulate);
    } else {
      launch_pdl(k_sgemm_t<128, 8>, dim3((unsigned)((N + 127) / 128), (unsigned)((M + 127) / 128)), dim3(256), 0, st, M,
                 N, (int)K, At, lda, B, ldb, C, ldc, rowmap, accumulate);
    }
    return;
  }
  launch_pdl(k_gemm_tn_f32, dim3((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64)), dim3(256), 0, st, M, N, K, At,
             lda, B, ldb, C, ldc, rowmap, accumulate);
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
