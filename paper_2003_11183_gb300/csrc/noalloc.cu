// tlrmvn_estimate_noalloc: the QMC estimator over per-sample log integrand values,
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a serving loop that reserved all of its
// device memory up front and must not take the implicit device-wide
// synchronisation of cudaMalloc / cudaFree between requests, or a host
// application whose device memory belongs entirely to another allocator (for
// instance a framework's caching pool).  This entry point runs the same two
// estimator kernels as tlrmvn_prob (per-shift log-sum-exp, then the
// cross-shift mean and standard error), but keeps their scratch - the per-shift
// log means - in a fixed array in this file instead of allocating it.
#include "common.cuh"

#include <mutex>

namespace tlrmvn {

// the estimator kernels (defined with the integrand)
__global__ void k_shift_reduce(const double* logP, int64_t N, double* ell);
__global__ void k_final(const double* ell, int M, double* logp, double* errp);

// Scratch of every call on a device: one log mean per shift.  Every GPU that
// loads this library holds it until the process exits.
static __device__ __align__(256) double g_noalloc_ell[TLRMVN_NOALLOC_MAX_SHIFTS];

static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {};

// Device address of the scratch array on the current device, looked up once per
// device (host code only sees a host-side stand-in under the array's name).
static int noalloc_scratch(double** out) {
  int dev = 0;
  TLR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(TLRMVN_E_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_ell);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_ell)");
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return TLRMVN_OK;
}

}  // namespace tlrmvn

using namespace tlrmvn;

extern "C" int tlrmvn_estimate_noalloc(const double* per_sample, int n_shifts, int64_t n_points, double* out,
                                       double* per_shift, void* stream) {
  if (!per_sample || !out) return fail(TLRMVN_E_INVAL, "null argument");
  if (n_shifts < 1 || n_points < 1) return fail(TLRMVN_E_INVAL, "n_shifts and n_points must be >= 1");
  if (n_shifts > TLRMVN_NOALLOC_MAX_SHIFTS)
    return fail(TLRMVN_E_INVAL, "n_shifts exceeds TLRMVN_NOALLOC_MAX_SHIFTS (" +
                                    std::to_string(TLRMVN_NOALLOC_MAX_SHIFTS) + ")");
  double* ell = nullptr;
  TLR_CHECK(noalloc_scratch(&ell));
  cudaStream_t st = stream ? (cudaStream_t)stream : pick_stream(nullptr);
  // every entry of the scratch that k_final reads is written first by k_shift_reduce
  k_shift_reduce<<<(unsigned)n_shifts, 256, 0, st>>>(per_sample, n_points, ell);
  k_final<<<1, 256, 0, st>>>(ell, n_shifts, out, out + 1);
  TLR_CUDA(cudaGetLastError());
  if (per_shift) TLR_CUDA(cudaMemcpyAsync(per_shift, ell, (size_t)n_shifts * 8, cudaMemcpyDeviceToDevice, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  return TLRMVN_OK;
}
