// Autotuner of the integrand's launch choices (tlrmvn_autotune).
//
// For one factor, precision and solve size it times a small set of candidate
// launch choices (Tuning: sweep sub-tile, sweep block size, samples per pass,
// whole-tile sweeps per SM) with CUDA events on real solves of the caller's own
// problem, keeps the fastest on the factor (every later tlrmvn_prob on that
// factor and precision uses it) and records it in a cache file, so that the next
// process with the same device, shape and rank mass reads it back instead of
// timing again.  The candidates only change how the work is launched, never what
// is computed: every candidate gives the same samples, sums and estimate up to
// the rounding order of the sweep's dense products.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

namespace tlrmvn {

int prob_impl(Factor& F, const double* a_dev, const double* b_dev, double nu, const tlrmvn_opts& o,
              double* logp_dev, double* err_dev, double* ell_dev_out, double* per_sample_dev, cudaStream_t st);

// Cache key: device name, precision, n, tile, total rank rounded to 2 significant
// bits of its binary logarithm, samples per solve (binary logarithm), and whether
// the problem is a Student-t one (its extra per-sample scale).
static std::string tune_key(const Factor& F, int precision, int64_t S, bool mvt) {
  cudaDeviceProp prop;
  std::string dev = "unknown";
  if (cudaGetDeviceProperties(&prop, F.device) == cudaSuccess) dev = prop.name;
  for (char& c : dev)
    if (c == ' ' || c == '\t') c = '_';
  const int kbin = F.ktot > 0 ? (int)std::lround(4.0 * std::log2((double)F.ktot)) : -1;
  const int sbin = (int)std::lround(std::log2((double)std::max<int64_t>(S, 1)));
  std::ostringstream k;
  k << dev << " p" << precision << " n" << F.n << " m" << F.m << " k" << kbin << " s" << sbin << " t" << (mvt ? 1 : 0);
  return k.str();
}

static std::vector<Tuning> candidates(const Factor& F, int precision, int64_t S) {
  std::vector<Tuning> c;
  if (precision == TLRMVN_BF16_SHIFT || precision == TLRMVN_FP16_SHIFT) {
    for (int spt : {1, 2})
      for (int ctas : {6, 4}) {
        if (spt == 2 && ctas > 4) continue;  // (two samples per thread: at most four CTAs per SM)
        for (int64_t chunk : {(int64_t)0, (S / 2 + 255) / 256 * 256}) {
          Tuning t;
          t.tc_ctas = ctas;
          t.chunk = chunk;
          t.spt = spt;
          c.push_back(t);
        }
      }
  } else if (precision == TLRMVN_FP32) {
    for (int sub : {64, 128})
      for (int threads : {0, 64, 128, 256}) {
        Tuning t;
        t.sub = sub;
        t.threads = threads;
        c.push_back(t);
      }
  } else {
    for (int sub : {32, 64}) {
      Tuning t;
      t.sub = sub;
      c.push_back(t);
    }
  }
  // candidates that change nothing for this factor (tiles no larger than the sub-tile) are dropped
  std::vector<Tuning> out;
  for (const Tuning& t : c) {
    bool dup = false;
    for (const Tuning& u : out)
      dup = dup || (std::min(t.sub, F.m) == std::min(u.sub, F.m) && t.threads == u.threads && t.chunk == u.chunk &&
                    t.tc_ctas == u.tc_ctas && t.spt == u.spt);
    if (!dup) out.push_back(t);
  }
  return out;
}

static bool cache_lookup(const char* path, const std::string& key, Tuning& t) {
  if (!path || !*path) return false;
  std::ifstream in(path);
  std::string line;
  bool found = false;
  while (std::getline(in, line)) {  // the last entry of a key wins
    const size_t bar = line.find(" | ");
    if (bar == std::string::npos || line.compare(0, bar, key) != 0 || bar != key.size()) continue;
    std::istringstream v(line.substr(bar + 3));
    Tuning u;
    long long chunk = 0;
    if (v >> u.sub >> u.threads >> chunk >> u.tc_ctas) {
      u.chunk = chunk;
      int spt = 1;
      if (v >> spt && (spt == 1 || spt == 2)) u.spt = spt;  // (entries without it: one sample per thread)
      t = u;
      found = true;
    }
  }
  return found;
}

static void cache_store(const char* path, const std::string& key, const Tuning& t, double ms) {
  if (!path || !*path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s | %d %d %lld %d %d # %.4f ms\n", key.c_str(), t.sub, t.threads, (long long)t.chunk, t.tc_ctas, t.spt,
          ms);
  fclose(f);
}

// Device milliseconds of one solve with tuning t (after one untimed solve).
static int time_solve(Factor& F, int precision, const Tuning& t, const double* a, const double* b, double nu,
                      const tlrmvn_opts& o, double* out2, cudaStream_t st, int reps, double& ms) {
  {
    std::lock_guard<std::mutex> lk(F.tune_mu);
    F.tune[precision] = t;
  }
  TLR_CHECK(prob_impl(F, a, b, nu, o, out2, out2 + 1, nullptr, nullptr, st));
  cudaEvent_t e0, e1;
  TLR_CUDA(cudaEventCreate(&e0));
  TLR_CUDA(cudaEventCreate(&e1));
  int s = TLRMVN_OK;
  cudaError_t e = cudaEventRecord(e0, st);
  for (int r = 0; r < reps && s == TLRMVN_OK && e == cudaSuccess; r++)
    s = prob_impl(F, a, b, nu, o, out2, out2 + 1, nullptr, nullptr, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t_ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t_ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TLR_CHECK(s);
  if (e != cudaSuccess) return cuda_fail(e, "autotune timing");
  ms = (double)t_ms / reps;
  return TLRMVN_OK;
}

}  // namespace tlrmvn

using namespace tlrmvn;

extern "C" int tlrmvn_autotune(tlrmvn_factor_t f, const double* a, const double* b, double nu,
                               const tlrmvn_opts* opts, const char* cache_path, int force, tlrmvn_tuning* out) {
  if (!f || !a || !b || !opts) return fail(TLRMVN_E_INVAL, "null argument");
  if (opts->n_shifts < 1 || opts->n_points < 1) return fail(TLRMVN_E_INVAL, "n_shifts and n_points must be >= 1");
  if (opts->precision < TLRMVN_FP64 || opts->precision > TLRMVN_FP16_SHIFT) return fail(TLRMVN_E_INVAL, "bad precision");
  if (!(nu > 0.0)) return fail(TLRMVN_E_INVAL, "nu must be > 0 (INFINITY for the normal case)");
  Factor& F = *reinterpret_cast<Factor*>(f);
  const int prec = opts->precision;
  const int64_t S = (int64_t)opts->n_shifts * opts->n_points;
  const std::string key = tune_key(F, prec, S, std::isfinite(nu));
  Tuning best;
  double best_ms = -1.0;
  int tried = 0;
  if (!force && cache_lookup(cache_path, key, best)) {
    std::lock_guard<std::mutex> lk(F.tune_mu);
    F.tune[prec] = best;
  } else {
    int cur = 0;
    cudaGetDevice(&cur);
    TLR_CUDA(cudaSetDevice(F.device));
    cudaStream_t st = pick_stream(opts->stream);
    tlrmvn_opts o = *opts;
    o.sample_chunk = 0;  // (the candidates choose it)
    double* dev = nullptr;
    int s = dalloc(&dev, (size_t)2 * F.n + 2);
    if (s == TLRMVN_OK) {
      cudaError_t e = cudaMemcpyAsync(dev, a, F.n * 8, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(dev + F.n, b, F.n * 8, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) s = cuda_fail(e, "autotune: copy limits");
    }
    const Tuning before = F.tuning(prec);
    for (const Tuning& t : candidates(F, prec, S)) {
      if (s != TLRMVN_OK) break;
      double ms = 0.0;
      s = time_solve(F, prec, t, dev, dev + F.n, nu, o, dev + 2 * F.n, st, 2, ms);
      tried++;
      if (s == TLRMVN_OK && (best_ms < 0.0 || ms < best_ms)) {
        best_ms = ms;
        best = t;
      }
    }
    dfree(dev);
    {
      std::lock_guard<std::mutex> lk(F.tune_mu);
      F.tune[prec] = (s == TLRMVN_OK) ? best : before;
    }
    cudaSetDevice(cur);
    TLR_CHECK(s);
    cache_store(cache_path, key, best, best_ms);
  }
  if (out) {
    out->sub = best.sub;
    out->threads = best.threads;
    out->chunk = best.chunk;
    out->tc_ctas = best.tc_ctas;
    out->spt = best.spt;
    out->ms = best_ms;
    out->candidates = tried;
  }
  return TLRMVN_OK;
}

extern "C" int tlrmvn_get_tuning(tlrmvn_factor_t f, int precision, tlrmvn_tuning* out) {
  if (!f || !out) return fail(TLRMVN_E_INVAL, "null argument");
  if (precision < TLRMVN_FP64 || precision > TLRMVN_FP16_SHIFT) return fail(TLRMVN_E_INVAL, "bad precision");
  const Tuning t = reinterpret_cast<Factor*>(f)->tuning(precision);
  out->sub = t.sub;
  out->threads = t.threads;
  out->chunk = t.chunk;
  out->tc_ctas = t.tc_ctas;
  out->spt = t.spt;
  out->ms = -1.0;
  out->candidates = 0;
  return TLRMVN_OK;
}

extern "C" int tlrmvn_set_tuning(tlrmvn_factor_t f, int precision, const tlrmvn_tuning* t) {
  if (!f || !t) return fail(TLRMVN_E_INVAL, "null argument");
  if (precision < TLRMVN_FP64 || precision > TLRMVN_FP16_SHIFT) return fail(TLRMVN_E_INVAL, "bad precision");
  if ((t->sub != 32 && t->sub != 64 && t->sub != 128) || (precision != TLRMVN_FP64 && t->sub == 32) ||
      (precision == TLRMVN_FP64 && t->sub == 128))
    return fail(TLRMVN_E_INVAL, "sub must be 64 or 128 (float32) / 32 or 64 (float64)");
  if (t->threads != 0 && (t->threads < 32 || t->threads > 256 || t->threads % 32))
    return fail(TLRMVN_E_INVAL, "threads must be 0 or a multiple of 32 in 32..256");
  if (t->chunk < 0 || t->tc_ctas < 1 || t->tc_ctas > 6) return fail(TLRMVN_E_INVAL, "bad chunk or tc_ctas");
  if (t->spt != 1 && t->spt != 2) return fail(TLRMVN_E_INVAL, "spt must be 1 or 2");
  Factor& F = *reinterpret_cast<Factor*>(f);
  Tuning u;
  u.sub = t->sub;
  u.threads = t->threads;
  u.chunk = t->chunk;
  u.tc_ctas = t->tc_ctas;
  u.spt = t->spt;
  std::lock_guard<std::mutex> lk(F.tune_mu);
  F.tune[precision] = u;
  return TLRMVN_OK;
}
