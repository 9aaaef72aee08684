// Host runtime of the tlrmvn library: status strings, thread-local error detail,
// the factor handle's compact layout, lattice generators, and factor
// serialisation (tlrmvn_factor_export / tlrmvn_factor_import / info / free).
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>

namespace tlrmvn {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }
int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}
int cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? TLRMVN_E_NOMEM : TLRMVN_E_CUDA;
}

static std::mutex g_stream_mu;
static cudaStream_t g_stream[64] = {};

cudaStream_t pick_stream(void* s) {
  if (s) return (cudaStream_t)s;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lk(g_stream_mu);
  if (!g_stream[dev]) cudaStreamCreateWithFlags(&g_stream[dev], cudaStreamNonBlocking);
  return g_stream[dev];
}

static std::mutex g_smem_mu;
static std::map<std::pair<int, const void*>, size_t> g_smem_limit;

int raise_smem_limit(const void* kernel, size_t bytes) {
  int dev = 0;
  TLR_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_smem_mu);
  size_t& cur = g_smem_limit[{dev, kernel}];
  if (bytes <= cur) return TLRMVN_OK;
  TLR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return TLRMVN_OK;
}

static std::mutex g_prof_mu;
static bool g_prof_on = false;
static double g_prof_ms[TLRMVN_KC_COUNT] = {};
static int64_t g_prof_n[TLRMVN_KC_COUNT] = {};

Prof::Prof(cudaStream_t s) : st(s) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  on = g_prof_on;
}
void Prof::begin(int cls) {
  if (!on) return;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaEventRecord(a, st);
  ev.push_back({cls, {a, b}});
}
void Prof::end() {
  if (!on || ev.empty()) return;
  cudaEventRecord(ev.back().second.second, st);
}
int Prof::collect() {
  if (!on) return TLRMVN_OK;
  double ms[TLRMVN_KC_COUNT] = {};
  int64_t cnt[TLRMVN_KC_COUNT] = {};
  for (auto& e : ev) {
    float t = 0.f;
    if (cudaEventElapsedTime(&t, e.second.first, e.second.second) == cudaSuccess) {
      ms[e.first] += t;
      cnt[e.first]++;
    }
  }
  cudaGetLastError();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int c = 0; c < TLRMVN_KC_COUNT; c++) {
    g_prof_ms[c] += ms[c];
    g_prof_n[c] += cnt[c];
  }
  return TLRMVN_OK;
}
Prof::~Prof() {
  for (auto& e : ev) {
    cudaEventDestroy(e.second.first);
    cudaEventDestroy(e.second.second);
  }
}

Factor::~Factor() {
  dfree(B);
  dfree(Ucat);
  dfree(Vcat);
  dfree(vmap);
  dfree(B32);
  dfree(BT32);
  dfree(inv32);
  dfree(band32);
  dfree(U32);
  dfree(V32);
  dfree(U16);
  dfree(V16);
  dfree(B16x2);
  dfree(vmap16);
  dfree(U16h);
  dfree(V16h);
  dfree(B16x2h);
  dfree(wscale16);
  dfree(Q);
  dfree(dperm);
}

int factor_alloc_compact(Factor& F, cudaStream_t st) {
  const int r = F.r;
  F.krow_off.assign(r + 1, 0);
  F.kcol_off.assign(r + 1, 0);
  for (int i = 0; i < r; i++) {
    int64_t k = 0;
    for (int j = 0; j < i; j++) k += F.rank[(size_t)i * r + j];
    F.krow_off[i + 1] = F.krow_off[i] + k;
  }
  for (int j = 0; j < r; j++) {
    int64_t k = 0;
    for (int i = j + 1; i < r; i++) k += F.rank[(size_t)i * r + j];
    F.kcol_off[j + 1] = F.kcol_off[j] + k;
  }
  F.ktot = F.krow_off[r];
  TLR_CHECK(dalloc(&F.B, (size_t)r * F.m * F.m));
  TLR_CHECK(dalloc(&F.Ucat, (size_t)F.m * F.ktot));
  TLR_CHECK(dalloc(&F.Vcat, (size_t)F.m * F.ktot));
  TLR_CHECK(dalloc(&F.vmap, (size_t)F.ktot));
  // zero padding rows / columns of short tiles; ordered on the stream that fills them
  if (F.ktot) {
    TLR_CUDA(cudaMemsetAsync(F.Ucat, 0, (size_t)F.m * F.ktot * 8, st));
    TLR_CUDA(cudaMemsetAsync(F.Vcat, 0, (size_t)F.m * F.ktot * 8, st));
  }
  TLR_CUDA(cudaMemsetAsync(F.B, 0, (size_t)r * F.m * F.m * 8, st));
  return TLRMVN_OK;
}

// Global rank index of component c of pair (i, j): row-grouped.
static inline int64_t kidx(const Factor& F, int i, int j) {
  int64_t k = F.krow_off[i];
  for (int t = 0; t < j; t++) k += F.rank[(size_t)i * F.r + t];
  return k;
}

std::vector<uint64_t> richtmyer_generators(int64_t d) {
  // first d primes by a sieve
  std::vector<uint64_t> out;
  if (d <= 0) return out;
  double dd = (double)std::max<int64_t>(d, 6);
  int64_t bound = (int64_t)(dd * (log(dd) + log(log(dd)))) + 16;
  std::vector<char> comp(bound + 1, 0);
  std::vector<uint64_t> ps;
  for (int64_t i = 2; i <= bound && (int64_t)ps.size() < d; i++) {
    if (comp[i]) continue;
    ps.push_back((uint64_t)i);
    for (int64_t j = i * i; j <= bound; j += i) comp[j] = 1;
  }
  out.resize(d);
  typedef unsigned __int128 u128;
  for (int64_t t = 0; t < d; t++) {
    uint64_t p = ps[t];
    uint64_t a = (uint64_t)floor(sqrt((double)p));
    while (a * a > p) a--;
    while ((a + 1) * (a + 1) <= p) a++;
    u128 dlt = (u128)(p - a * a);  // p - a^2
    // largest f < 2^64 with (a 2^64 + f)^2 <= p 2^128, i.e.
    // 2 a f 2^64 + f^2 <= dlt 2^128; compare after dividing by 2^64.
    uint64_t lo = 0, hi = ~(uint64_t)0;
    auto ok = [&](uint64_t f) {
      u128 f2 = (u128)f * f;
      u128 lhs = (u128)2 * a * f + (f2 >> 64);
      u128 rhs = dlt << 64;
      if (lhs < rhs) return true;
      if (lhs > rhs) return false;
      return (uint64_t)f2 == 0;
    };
    if (dlt == 0) {
      out[t] = 0;
      continue;
    }
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2 + 1;
      if (ok(mid)) lo = mid;
      else hi = mid - 1;
    }
    out[t] = lo;
  }
  return out;
}

int factor_finish(Factor& F, cudaStream_t st) {
  std::vector<uint64_t> Q = richtmyer_generators(F.n + 1);
  TLR_CHECK(dalloc(&F.Q, Q.size()));
  TLR_CHECK(dalloc(&F.dperm, (size_t)F.n));
  TLR_CUDA(cudaMemcpyAsync(F.Q, Q.data(), Q.size() * 8, cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaMemcpyAsync(F.dperm, F.perm.data(), F.n * 8, cudaMemcpyHostToDevice, st));
  TLR_CUDA(cudaStreamSynchronize(st));
  return TLRMVN_OK;
}

}  // namespace tlrmvn

using namespace tlrmvn;

static const char kMagic[8] = {'T', 'L', 'R', 'M', 'V', 'N', '0', '1'};

extern "C" const char* tlrmvn_strerror(int status) {
  switch (status) {
    case TLRMVN_OK: return "ok";
    case TLRMVN_E_INVAL: return "invalid argument";
    case TLRMVN_E_NOT_SPD: return "covariance is not positive definite";
    case TLRMVN_E_NOMEM: return "out of memory";
    case TLRMVN_E_CUDA: return "CUDA error";
    case TLRMVN_E_FORMAT: return "malformed factor buffer";
    case TLRMVN_E_NOTSUP: return "not supported";
    case TLRMVN_E_TIMEOUT: return "device-side wait timed out";
    case TLRMVN_E_RANK: return "rank cap reached before the truncation tolerance";
    case TLRMVN_E_BUSY: return "admission refused";
    default: return "unknown status";
  }
}

extern "C" const char* tlrmvn_last_error(void) { return g_last_error.c_str(); }

extern "C" int tlrmvn_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return TLRMVN_OK;
}
extern "C" int tlrmvn_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int c = 0; c < TLRMVN_KC_COUNT; c++) {
    g_prof_ms[c] = 0.0;
    g_prof_n[c] = 0;
  }
  return TLRMVN_OK;
}
extern "C" int tlrmvn_profile_get(int kernel_class, double* total_ms, int64_t* launches) {
  if (kernel_class < 0 || kernel_class >= TLRMVN_KC_COUNT) return fail(TLRMVN_E_INVAL, "bad kernel class");
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (total_ms) *total_ms = g_prof_ms[kernel_class];
  if (launches) *launches = g_prof_n[kernel_class];
  return TLRMVN_OK;
}

extern "C" int tlrmvn_factor_info(tlrmvn_factor_t f, int64_t* n, int* r, int* m, int64_t* k_total, int* capped) {
  if (!f) return fail(TLRMVN_E_INVAL, "null factor");
  Factor& F = *reinterpret_cast<Factor*>(f);
  if (n) *n = F.n;
  if (r) *r = F.r;
  if (m) *m = F.m;
  if (k_total) *k_total = F.ktot;
  if (capped) *capped = F.capped;
  return TLRMVN_OK;
}

extern "C" int tlrmvn_factor_ranks(tlrmvn_factor_t f, int32_t* ranks) {
  if (!f || !ranks) return fail(TLRMVN_E_INVAL, "null argument");
  const Factor& F = *reinterpret_cast<Factor*>(f);
  std::memcpy(ranks, F.rank.data(), F.rank.size() * sizeof(int32_t));
  return TLRMVN_OK;
}

extern "C" int tlrmvn_factor_free(tlrmvn_factor_t f) {
  if (!f) return TLRMVN_OK;
  Factor* F = reinterpret_cast<Factor*>(f);
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(F->device);
  delete F;
  cudaSetDevice(cur);
  return TLRMVN_OK;
}

static size_t export_size(const Factor& F) {
  size_t bytes = 8 + 4 * 8 + (F.r + 1) * 8 + F.n * 8 + (size_t)F.r * F.r * 4 + (size_t)F.r * F.m * F.m * 8;
  for (int i = 0; i < F.r; i++)
    for (int j = 0; j < i; j++) bytes += (size_t)(F.tsize(i) + F.tsize(j)) * F.rank[(size_t)i * F.r + j] * 8;
  return bytes;
}

extern "C" int tlrmvn_factor_export(tlrmvn_factor_t f, void* buf, size_t* bytes) {
  if (!f || !bytes) return fail(TLRMVN_E_INVAL, "null argument");
  Factor& F = *reinterpret_cast<Factor*>(f);
  size_t need = export_size(F);
  if (!buf) {
    *bytes = need;
    return TLRMVN_OK;
  }
  if (*bytes < need) return fail(TLRMVN_E_INVAL, "export buffer too small");
  int cur = 0;
  cudaGetDevice(&cur);
  TLR_CUDA(cudaSetDevice(F.device));
  const int r = F.r, m = F.m;
  std::vector<double> Uh((size_t)m * F.ktot), Vh((size_t)m * F.ktot);
  TLR_CUDA(cudaMemcpy(Uh.data(), F.Ucat, Uh.size() * 8, cudaMemcpyDeviceToHost));
  TLR_CUDA(cudaMemcpy(Vh.data(), F.Vcat, Vh.size() * 8, cudaMemcpyDeviceToHost));
  char* p = (char*)buf;
  memcpy(p, kMagic, 8);
  p += 8;
  int64_t hdr[4] = {F.n, F.r, F.m, F.ktot};
  memcpy(p, hdr, 32);
  p += 32;
  memcpy(p, F.tile_off.data(), (r + 1) * 8);
  p += (r + 1) * 8;
  memcpy(p, F.perm.data(), F.n * 8);
  p += F.n * 8;
  memcpy(p, F.rank.data(), (size_t)r * r * 4);
  p += (size_t)r * r * 4;
  TLR_CUDA(cudaMemcpy(p, F.B, (size_t)r * m * m * 8, cudaMemcpyDeviceToHost));
  p += (size_t)r * m * m * 8;
  for (int i = 0; i < r; i++) {
    for (int j = 0; j < i; j++) {
      int k = F.rank[(size_t)i * r + j];
      if (!k) continue;
      int64_t mi = F.tsize(i), mj = F.tsize(j);
      // U_ij: columns [kl, kl+k) of row block i
      int64_t kl = kidx(F, i, j) - F.krow_off[i];
      int64_t Kr = F.krow(i);
      std::vector<double> U((size_t)mi * k), V((size_t)mj * k);
      for (int64_t v = 0; v < mi; v++)
        for (int c = 0; c < k; c++) U[v * k + c] = Uh[(size_t)m * F.krow_off[i] + v * Kr + kl + c];
      memcpy(p, U.data(), U.size() * 8);
      p += mi * k * 8;
      // V_ij: rows of column block j, stored transposed
      int64_t vr = 0;
      for (int t = j + 1; t < i; t++) vr += F.rank[(size_t)t * r + j];
      for (int64_t u = 0; u < mj; u++)
        for (int c = 0; c < k; c++) V[u * k + c] = Vh[(size_t)m * (F.kcol_off[j] + vr + c) + u];
      memcpy(p, V.data(), V.size() * 8);
      p += mj * k * 8;
    }
  }
  *bytes = need;
  cudaSetDevice(cur);
  return TLRMVN_OK;
}

namespace tlrmvn {
// Fills Ucat/Vcat/vmap from host pair arrays (Uh[(i,j)] m_i x k, Vh[(i,j)] m_j x k) and uploads B.
int factor_upload_pairs(Factor& F, const double* Bh, const std::vector<const double*>& Up,
                        const std::vector<const double*>& Vp, cudaStream_t st) {
  const int r = F.r, m = F.m;
  TLR_CHECK(factor_alloc_compact(F, st));
  std::vector<double> Uc((size_t)m * F.ktot, 0.0), Vc((size_t)m * F.ktot, 0.0);
  std::vector<int32_t> vm(F.ktot);
  for (int i = 0; i < r; i++) {
    for (int j = 0; j < i; j++) {
      int k = F.rank[(size_t)i * r + j];
      if (!k) continue;
      const double* U = Up[(size_t)i * r + j];
      const double* V = Vp[(size_t)i * r + j];
      int64_t mi = F.tsize(i), mj = F.tsize(j);
      int64_t g = kidx(F, i, j);
      int64_t kl = g - F.krow_off[i], Kr = F.krow(i);
      for (int64_t v = 0; v < mi; v++)
        for (int c = 0; c < k; c++) Uc[(size_t)m * F.krow_off[i] + v * Kr + kl + c] = U[v * k + c];
      int64_t vr = 0;
      for (int t = j + 1; t < i; t++) vr += F.rank[(size_t)t * r + j];
      for (int c = 0; c < k; c++) {
        int64_t row = F.kcol_off[j] + vr + c;
        vm[row] = (int32_t)(g + c);
        for (int64_t u = 0; u < mj; u++) Vc[(size_t)m * row + u] = V[u * k + c];
      }
    }
  }
  TLR_CUDA(cudaMemcpyAsync(F.B, Bh, (size_t)r * m * m * 8, cudaMemcpyHostToDevice, st));
  if (F.ktot) {
    TLR_CUDA(cudaMemcpyAsync(F.Ucat, Uc.data(), Uc.size() * 8, cudaMemcpyHostToDevice, st));
    TLR_CUDA(cudaMemcpyAsync(F.Vcat, Vc.data(), Vc.size() * 8, cudaMemcpyHostToDevice, st));
    TLR_CUDA(cudaMemcpyAsync(F.vmap, vm.data(), vm.size() * 4, cudaMemcpyHostToDevice, st));
  }
  TLR_CUDA(cudaStreamSynchronize(st));
  return factor_finish(F, st);
}
}  // namespace tlrmvn

extern "C" int tlrmvn_factor_import(const void* buf, size_t bytes, tlrmvn_factor_t* out) {
  if (!buf || !out) return fail(TLRMVN_E_INVAL, "null argument");
  const char* p = (const char*)buf;
  const char* end = p + bytes;
  if (bytes < 40 || memcmp(p, kMagic, 8) != 0) return fail(TLRMVN_E_FORMAT, "bad magic");
  int64_t hdr[4];
  memcpy(hdr, p + 8, 32);
  p += 40;
  int64_t n = hdr[0], r = hdr[1], m = hdr[2];
  if (n <= 0 || r <= 0 || m <= 0 || r > n || m > 4096 || r * m < n) return fail(TLRMVN_E_FORMAT, "bad header");
  size_t fixed = (r + 1) * 8 + n * 8 + (size_t)r * r * 4 + (size_t)r * m * m * 8;
  if ((size_t)(end - p) < fixed) return fail(TLRMVN_E_FORMAT, "truncated buffer");
  Factor* F = new Factor();
  cudaGetDevice(&F->device);
  F->n = n;
  F->r = (int)r;
  F->m = (int)m;
  F->tile_off.resize(r + 1);
  memcpy(F->tile_off.data(), p, (r + 1) * 8);
  p += (r + 1) * 8;
  F->perm.resize(n);
  memcpy(F->perm.data(), p, n * 8);
  p += n * 8;
  F->rank.resize((size_t)r * r);
  memcpy(F->rank.data(), p, (size_t)r * r * 4);
  p += (size_t)r * r * 4;
  // copy into aligned storage: the rank table may leave the doubles 4-byte aligned
  std::vector<double> Bh((size_t)r * m * m);
  memcpy(Bh.data(), p, Bh.size() * 8);
  p += (size_t)r * m * m * 8;
  std::vector<double> pairs((size_t)((end - p) / 8) + 1);
  const char* pair_base = p;
  // validate the tiling and permutation
  bool okt = F->tile_off[0] == 0 && F->tile_off[r] == n;
  for (int64_t t = 0; t < r && okt; t++) okt = F->tile_off[t + 1] > F->tile_off[t] && F->tile_off[t + 1] - F->tile_off[t] <= m;
  std::vector<char> seen(n, 0);
  for (int64_t i = 0; i < n && okt; i++) {
    int64_t q = F->perm[i];
    okt = q >= 0 && q < n && !seen[q];
    if (okt) seen[q] = 1;
  }
  if (!okt) {
    delete F;
    return fail(TLRMVN_E_FORMAT, "bad tiling or permutation");
  }
  std::vector<const double*> Up((size_t)r * r, nullptr), Vp((size_t)r * r, nullptr);
  for (int i = 0; i < r; i++)
    for (int j = 0; j < i; j++) {
      int k = F->rank[(size_t)i * r + j];
      if (k < 0 || k > m) {
        delete F;
        return fail(TLRMVN_E_FORMAT, "bad rank");
      }
      if (!k) continue;
      size_t need = (size_t)(F->tsize(i) + F->tsize(j)) * k * 8;
      if ((size_t)(end - p) < need) {
        delete F;
        return fail(TLRMVN_E_FORMAT, "truncated low-rank data");
      }
      size_t off = (size_t)(p - pair_base) / 8;
      memcpy(pairs.data() + off, p, need);
      Up[(size_t)i * r + j] = pairs.data() + off;
      p += F->tsize(i) * k * 8;
      Vp[(size_t)i * r + j] = pairs.data() + off + F->tsize(i) * k;
      p += F->tsize(j) * k * 8;
    }
  cudaStream_t st = pick_stream(nullptr);
  int s = factor_upload_pairs(*F, Bh.data(), Up, Vp, st);
  if (s != TLRMVN_OK) {
    delete F;
    return s;
  }
  *out = reinterpret_cast<tlrmvn_factor_t>(F);
  return TLRMVN_OK;
}

// Section 2.1 estimate pooled over shift batches gathered on the host: the same
// formula as the device reduction (k_final), in float64 on the host.
extern "C" int tlrmvn_estimate_pooled(const double* per_shift, int64_t count, double* logp, double* err) {
  if (!per_shift || !logp || !err) return fail(TLRMVN_E_INVAL, "null argument");
  if (count < 1) return fail(TLRMVN_E_INVAL, "count must be >= 1");
  double mx = -INFINITY;
  for (int64_t s = 0; s < count; s++) {
    if (std::isnan(per_shift[s]) || per_shift[s] == INFINITY)
      return fail(TLRMVN_E_INVAL, "per-shift logs must be finite or -INFINITY");
    mx = std::max(mx, per_shift[s]);
  }
  if (mx == -INFINITY) {
    *logp = -INFINITY;
    *err = NAN;
    return TLRMVN_OK;
  }
  double sum = 0.0;
  for (int64_t s = 0; s < count; s++) sum += std::exp(per_shift[s] - mx);
  const double mean = sum / (double)count;
  double sq = 0.0;
  for (int64_t s = 0; s < count; s++) {
    const double d = std::exp(per_shift[s] - mx) - mean;
    sq += d * d;
  }
  *logp = mx + std::log(sum) - std::log((double)count);
  *err = count > 1 ? std::sqrt(sq / (double)(count - 1) / (double)count) / mean : NAN;
  return TLRMVN_OK;
}
