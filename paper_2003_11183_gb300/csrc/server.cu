// Serving loop: continuous admission of probability requests on resident factors.
//
// Requests (factor index, limits, nu, options) are queued in arrival order.
// A fixed set of lanes - worker threads, each with its own CUDA stream - takes
// them from the head of the queue: the head is admitted as soon as a lane is
// free and its scratch (prob_scratch_bytes) fits in what is left of the memory
// budget.  Requests that arrive while others are on the GPU therefore start as
// lanes and memory free up, and their kernels overlap on the device with the
// ones already running.  Scratch is stream-ordered (cudaMallocAsync), so lanes
// never synchronise the device.  Each request's result depends only on its own
// inputs, so it is the same alone and in the mix.
#include "common.cuh"

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace tlrmvn {

int prob_impl(Factor& F, const double* a_dev, const double* b_dev, double nu, const tlrmvn_opts& o,
              double* logp_dev, double* err_dev, double* ell_dev_out, double* per_sample_dev, cudaStream_t st);
int64_t prob_scratch_bytes(const Factor& F, const tlrmvn_opts& o);

using Clock = std::chrono::steady_clock;

struct Request {
  int64_t id;
  int factor;
  std::vector<double> a, b;
  std::vector<uint64_t> shifts;
  double nu;
  tlrmvn_opts opts;
  int64_t bytes;
  Clock::time_point t_submit, t_start, t_done;
  int status = -1;  // -1 pending
  double logp = 0.0, err = 0.0;
  std::string msg;  // failure detail from the lane's thread
};

struct Server {
  std::vector<Factor*> factors;
  int device = 0;
  int64_t budget = 0, in_use = 0, peak_in_use = 0;
  int lanes = 0, busy = 0, peak_busy = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::unordered_map<int64_t, Request*> all;
  std::vector<double> latencies_ms;
  std::vector<std::thread> workers;
  int64_t next_id = 1, completed = 0, overlapped = 0;
  bool stop = false;

  void worker() {
    cudaSetDevice(device);
    cudaStream_t st;
    cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (;;) {
      Request* r = nullptr;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stop || (!queue.empty() && in_use + queue.front()->bytes <= budget); });
        if (stop && queue.empty()) break;
        if (queue.empty() || in_use + queue.front()->bytes > budget) continue;
        r = queue.front();
        queue.pop_front();
        in_use += r->bytes;
        peak_in_use = std::max(peak_in_use, in_use);
        if (busy > 0) overlapped++;
        busy++;
        peak_busy = std::max(peak_busy, busy);
      }
      r->t_start = Clock::now();
      r->opts.stream = st;
      if (!r->shifts.empty()) r->opts.shifts = r->shifts.data();
      const int64_t n = (int64_t)r->a.size();
      double* dev = nullptr;  // a, b, (logp, err)
      int s = TLRMVN_OK;
      cudaError_t e = cudaMallocAsync((void**)&dev, (size_t)(2 * n + 2) * 8, st);
      if (e != cudaSuccess) {
        cudaGetLastError();
        s = TLRMVN_E_NOMEM;
      }
      if (s == TLRMVN_OK) {
        e = cudaMemcpyAsync(dev, r->a.data(), n * 8, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dev + n, r->b.data(), n * 8, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) s = cuda_fail(e, "server: copy limits");
      }
      if (s == TLRMVN_OK) s = prob_impl(*factors[r->factor], dev, dev + n, r->nu, r->opts, dev + 2 * n,
                                        dev + 2 * n + 1, nullptr, nullptr, st);
      double out[2] = {NAN, NAN};
      if (s == TLRMVN_OK) {
        e = cudaMemcpyAsync(out, dev + 2 * n, 16, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "server: copy result");
      }
      if (dev) cudaFreeAsync(dev, st);
      cudaStreamSynchronize(st);
      {
        std::lock_guard<std::mutex> lk(mu);
        r->t_done = Clock::now();
        r->status = s;
        if (s != TLRMVN_OK) r->msg = tlrmvn_last_error();
        r->logp = out[0];
        r->err = out[1];
        in_use -= r->bytes;
        busy--;
        completed++;
        latencies_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
      }
      cv_done.notify_all();
      cv_work.notify_all();
    }
    cudaStreamDestroy(st);
  }

  ~Server() {
    {
      std::lock_guard<std::mutex> lk(mu);
      stop = true;
    }
    cv_work.notify_all();
    for (auto& t : workers) t.join();
    for (auto& kv : all) delete kv.second;
    for (Request* r : queue)
      if (!all.count(r->id)) delete r;
  }
};

static double percentile(std::vector<double> v, double q) {
  if (v.empty()) return NAN;
  std::sort(v.begin(), v.end());
  double pos = q * (v.size() - 1);
  size_t lo = (size_t)pos, hi = std::min(v.size() - 1, lo + 1);
  return v[lo] + (pos - lo) * (v[hi] - v[lo]);
}

}  // namespace tlrmvn

using namespace tlrmvn;

extern "C" int tlrmvn_server_create(const tlrmvn_factor_t* factors, int n_factors, int lanes, int64_t memory_budget,
                                    tlrmvn_server_t* out) {
  if (!factors || n_factors < 1 || lanes < 1 || lanes > 64 || memory_budget <= 0 || !out)
    return fail(TLRMVN_E_INVAL, "bad server arguments");
  Server* S = new Server();
  for (int i = 0; i < n_factors; i++) {
    if (!factors[i]) {
      delete S;
      return fail(TLRMVN_E_INVAL, "null factor");
    }
    S->factors.push_back(reinterpret_cast<Factor*>(factors[i]));
  }
  S->device = S->factors[0]->device;
  S->budget = memory_budget;
  S->lanes = lanes;
  for (int i = 0; i < lanes; i++) S->workers.emplace_back([S] { S->worker(); });
  *out = reinterpret_cast<tlrmvn_server_t>(S);
  return TLRMVN_OK;
}

extern "C" int tlrmvn_server_submit(tlrmvn_server_t srv, int factor, const double* a, const double* b, double nu,
                                    const tlrmvn_opts* opts, int64_t* request_id) {
  if (!srv || !a || !b || !opts || !request_id) return fail(TLRMVN_E_INVAL, "null argument");
  Server& S = *reinterpret_cast<Server*>(srv);
  if (factor < 0 || factor >= (int)S.factors.size()) return fail(TLRMVN_E_INVAL, "factor index out of range");
  if (opts->n_shifts < 1 || opts->n_points < 1 || opts->precision < 0 || opts->precision > 3 || !(nu > 0.0))
    return fail(TLRMVN_E_INVAL, "bad options");
  const Factor& F = *S.factors[factor];
  Request* r = new Request();
  r->factor = factor;
  r->a.assign(a, a + F.n);
  r->b.assign(b, b + F.n);
  r->nu = nu;
  r->opts = *opts;
  if (opts->shifts) r->shifts.assign(opts->shifts, opts->shifts + (size_t)opts->n_shifts * (F.n + 1));
  r->opts.shifts = nullptr;
  r->bytes = prob_scratch_bytes(F, r->opts) + (2 * F.n + 2) * 8;
  if (r->bytes > S.budget) {
    const int64_t r_bytes = r->bytes;
    delete r;
    return fail(TLRMVN_E_BUSY, "admission refused: the request needs more scratch (" + std::to_string(r_bytes) +
                                   " bytes) than the server's memory budget");
  }
  r->t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(S.mu);
    r->id = S.next_id++;
    S.all[r->id] = r;
    S.queue.push_back(r);
  }
  S.cv_work.notify_all();
  *request_id = r->id;
  return TLRMVN_OK;
}

extern "C" int tlrmvn_server_wait(tlrmvn_server_t srv, int64_t request_id, double* logp, double* err,
                                  double* latency_ms) {
  if (!srv) return fail(TLRMVN_E_INVAL, "null server");
  Server& S = *reinterpret_cast<Server*>(srv);
  std::unique_lock<std::mutex> lk(S.mu);
  auto it = S.all.find(request_id);
  if (it == S.all.end()) return fail(TLRMVN_E_INVAL, "unknown request id");
  Request* r = it->second;
  S.cv_done.wait(lk, [&] { return r->status != -1; });
  int s = r->status;
  const std::string msg = r->msg;
  if (logp) *logp = r->logp;
  if (err) *err = r->err;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  S.all.erase(it);
  delete r;
  if (s != TLRMVN_OK) return fail(s, "request failed: " + msg);
  return TLRMVN_OK;
}

extern "C" int tlrmvn_server_stats(tlrmvn_server_t srv, tlrmvn_server_stats_t* out) {
  if (!srv || !out) return fail(TLRMVN_E_INVAL, "null argument");
  Server& S = *reinterpret_cast<Server*>(srv);
  std::lock_guard<std::mutex> lk(S.mu);
  out->completed = S.completed;
  out->queued = (int64_t)S.queue.size();
  out->in_flight = S.busy;
  out->peak_in_flight = S.peak_busy;
  out->overlapped = S.overlapped;
  out->peak_bytes = S.peak_in_use;
  out->p50_ms = percentile(S.latencies_ms, 0.50);
  out->p99_ms = percentile(S.latencies_ms, 0.99);
  return TLRMVN_OK;
}

extern "C" int tlrmvn_prob_scratch_bytes(tlrmvn_factor_t f, const tlrmvn_opts* opts, int64_t* bytes) {
  if (!f || !opts || !bytes) return fail(TLRMVN_E_INVAL, "null argument");
  const Factor& F = *reinterpret_cast<Factor*>(f);
  *bytes = prob_scratch_bytes(F, *opts) + (2 * F.n + 2) * 8;
  return TLRMVN_OK;
}

extern "C" int tlrmvn_server_free(tlrmvn_server_t srv) {
  delete reinterpret_cast<Server*>(srv);
  return TLRMVN_OK;
}
