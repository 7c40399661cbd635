// Request server: continuous batching of simulation requests on one GPU.
//
// A request is (plan, bitstrings, path selection), the problem statement of
// Sections 2-3. Requests are admitted in arrival order while the sum of the
// admitted requests' device footprints (level buffers of the path tree plus
// bitstrings and accumulators, the M_proc model of Section 8) fits the
// budget; a request that does not fit lets later, smaller ones pass until it
// has waited one second, after which it blocks admission until memory frees.
// Each admitted request runs on a worker thread with its own CUDA stream,
// workspace and resident-node cache, so the kernels of concurrent requests
// overlap on the device. Results equal sf_amplitudes on the same input.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>

#include "sf_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

enum { Q_QUEUED, Q_RUNNING, Q_DONE, Q_FAILED, Q_CANCELLED };

struct Request {
  uint64_t ticket = 0;
  sf::Plan* plan = nullptr;
  std::vector<uint64_t> bits;
  std::vector<uint64_t> list;
  sf_path_sel sel;
  size_t ws_bytes = 0;
  int64_t footprint = 0;
  double terms[4] = {0, 0, 0, 0};  // runtime-model features (Eq. t_tot)
  std::vector<double> out;
  int state = Q_QUEUED;
  int err_code = 0;
  std::string err;
  volatile int cancel = 0;
  Clock::time_point t_submit, t_start, t_done;
};

}  // namespace

struct sf_server {
  int64_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  int64_t in_use = 0;
  int running = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<std::thread> workers;
  // runtime model: when set, admission prefers the shortest predicted request
  bool model = false;
  double coeffs[4] = {0, 0, 0, 0};
  double max_wait_s = 1.0;
};

namespace {

void cuda_ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) sf::fail(e == cudaErrorMemoryAllocation ? SF_ENOMEM : SF_ECUDA,
                                 std::string(what) + ": " + cudaGetErrorString(e));
}

// Pick the next request to admit (caller holds the lock): the oldest one that
// fits, unless the oldest has waited > 1 s and does not fit. With a runtime
// model set, requests that have waited less than max_wait_s go in order of
// predicted time (shortest first) after any that have waited longer.
std::shared_ptr<Request> pick(sf_server& s) {
  if (s.queue.empty()) return nullptr;
  auto now = Clock::now();
  if (s.model) {
    const auto aged = std::chrono::duration<double>(s.max_wait_s);
    int best = -1;
    double best_t = 0;
    for (size_t i = 0; i < s.queue.size(); i++) {
      auto& r = s.queue[i];
      const bool old = now - r->t_submit > aged;
      const bool fits = s.in_use + r->footprint <= s.budget || s.running == 0;
      if (old) {
        if (best >= 0 && now - s.queue[best]->t_submit > aged) continue;  // an older aged one wins
        if (!fits) return nullptr;  // the oldest aged request blocks until memory frees
        best = (int)i;
        best_t = -1;
        continue;
      }
      if (!fits || (best >= 0 && best_t < 0)) continue;
      const double t = sf_cost_predict(r->terms, s.coeffs);
      if (best < 0 || t < best_t) {
        best = (int)i;
        best_t = t;
      }
    }
    if (best < 0) return nullptr;
    auto out = s.queue[best];
    s.queue.erase(s.queue.begin() + best);
    return out;
  }
  for (size_t i = 0; i < s.queue.size(); i++) {
    auto& r = s.queue[i];
    if (s.in_use + r->footprint <= s.budget || s.running == 0) {
      auto out = r;
      s.queue.erase(s.queue.begin() + i);
      return out;
    }
    if (i == 0 && now - r->t_submit > std::chrono::seconds(1)) return nullptr;
  }
  return nullptr;
}

void run_request(sf_server& s, Request& r, cudaStream_t st, void** cache) {
  uint64_t* d_bits = nullptr;
  double* d_out = nullptr;
  void* d_ws = nullptr;
  const int64_t n = (int64_t)r.bits.size();
  try {
    cuda_ok(cudaSetDevice(s.device), "cudaSetDevice");
    if (n > 0) {
      cuda_ok(cudaMallocAsync((void**)&d_bits, (size_t)n * 8, st), "cudaMallocAsync");
      cuda_ok(cudaMallocAsync((void**)&d_out, (size_t)n * 16, st), "cudaMallocAsync");
      cuda_ok(cudaMallocAsync(&d_ws, r.ws_bytes, st), "cudaMallocAsync");
      cuda_ok(cudaMemcpyAsync(d_bits, r.bits.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st),
              "cudaMemcpyAsync");
      sf::ExecCtx ctx;
      ctx.cache_slot = cache;
      ctx.profile = false;
      ctx.cancel = &r.cancel;
      sf::exec_run(*r.plan, d_bits, n, r.sel, d_out, 0, d_ws, r.ws_bytes, st, false, &ctx);
      r.out.resize((size_t)2 * n);
      cuda_ok(cudaMemcpyAsync(r.out.data(), d_out, (size_t)n * 16, cudaMemcpyDeviceToHost, st),
              "cudaMemcpyAsync");
    }
    cuda_ok(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    r.err_code = 0;
  } catch (const sf::Error& e) {
    cudaStreamSynchronize(st);
    r.err_code = e.code;
    r.err = e.msg;
  } catch (const std::exception& e) {
    cudaStreamSynchronize(st);
    r.err_code = SF_EINVAL;
    r.err = e.what();
  }
  if (d_bits) cudaFreeAsync(d_bits, st);
  if (d_out) cudaFreeAsync(d_out, st);
  if (d_ws) cudaFreeAsync(d_ws, st);
  cudaStreamSynchronize(st);
}

void worker(sf_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  void* cache = nullptr;
  while (true) {
    std::shared_ptr<Request> r;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
      r = pick(*s);
      if (!r) continue;
      s->in_use += r->footprint;
      s->running++;
      r->state = Q_RUNNING;
      r->t_start = Clock::now();
    }
    run_request(*s, *r, st, &cache);
    sf::exec_free_cache(cache);
    cache = nullptr;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->in_use -= r->footprint;
      s->running--;
      r->t_done = Clock::now();
      if (r->err_code == 0) r->state = Q_DONE;
      else if (r->err_code == SF_ECANCELLED) r->state = Q_CANCELLED;
      else r->state = Q_FAILED;
      r->bits.clear();
      r->bits.shrink_to_fit();
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  if (st) cudaStreamDestroy(st);
}

}  // namespace

#define SF_SGUARD_BEGIN try {
#define SF_SGUARD_END                       \
  }                                         \
  catch (const sf::Error& e) {              \
    sf::set_error(e.msg);                   \
    return e.code;                          \
  }                                         \
  catch (const std::exception& e) {         \
    sf::set_error(e.what());                \
    return SF_EINVAL;                       \
  }

extern "C" {

int sf_server_create(int64_t budget, int max_concurrent, sf_server** out) {
  SF_SGUARD_BEGIN
  if (!out) sf::fail(SF_EINVAL, "null output pointer");
  *out = nullptr;
  if (budget < 0 || max_concurrent < 0 || max_concurrent > 64) sf::fail(SF_EINVAL, "bad budget or concurrency");
  auto* s = new sf_server();
  cuda_ok(cudaGetDevice(&s->device), "cudaGetDevice");
  if (budget == 0) {
    size_t fr = 0, tot = 0;
    cuda_ok(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
    budget = (int64_t)(fr / 4 * 3);
  }
  s->budget = budget;
  int nw = max_concurrent > 0 ? max_concurrent : 4;
  for (int i = 0; i < nw; i++) s->workers.emplace_back(worker, s);
  *out = s;
  return SF_OK;
  SF_SGUARD_END
}

int sf_server_submit(sf_server* s, sf_plan* p, const uint64_t* bits, int64_t n, const sf_path_sel* sel,
                     uint64_t* ticket) {
  SF_SGUARD_BEGIN
  if (!s || !p || !sel || !ticket || n < 0 || (n > 0 && !bits)) sf::fail(SF_EINVAL, "bad argument");
  auto r = std::make_shared<Request>();
  r->plan = p->p;
  r->bits.assign(bits, bits + n);
  r->sel = *sel;
  if (sel->mode == SF_SEL_LIST && sel->n_list > 0) {
    r->list.assign(sel->list, sel->list + sel->n_list);
    r->sel.list = r->list.data();
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    sf::ensure_device(*r->plan);  // tables and budget, once per plan
  }
  r->ws_bytes = sf::exec_workspace_bytes(*r->plan, n, r->sel);
  r->footprint = (int64_t)r->ws_bytes + 24 * n;
  sf::cost_terms(*r->plan, r->sel, n, r->terms);
  if (r->footprint > s->budget)
    sf::fail(SF_ENOMEM, "request footprint " + std::to_string(r->footprint) + " exceeds the server budget");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->ticket = s->next_ticket++;
    r->t_submit = Clock::now();
    s->all[r->ticket] = r;
    s->queue.push_back(r);
    *ticket = r->ticket;
  }
  s->cv_work.notify_all();
  return SF_OK;
  SF_SGUARD_END
}

int sf_server_wait(sf_server* s, uint64_t ticket, int timeout_ms, double* out) {
  SF_SGUARD_BEGIN
  if (!s) sf::fail(SF_EINVAL, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) sf::fail(SF_EINVAL, "unknown ticket");
  auto r = it->second;
  auto done = [&] { return r->state == Q_DONE || r->state == Q_FAILED || r->state == Q_CANCELLED; };
  if (timeout_ms < 0) s->cv_done.wait(lk, done);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
    sf::fail(SF_ETIMEOUT, "request not finished");
  s->all.erase(ticket);
  if (r->state == Q_CANCELLED) sf::fail(SF_ECANCELLED, "request cancelled");
  if (r->state == Q_FAILED) sf::fail(r->err_code, r->err);
  if (out && !r->out.empty()) std::memcpy(out, r->out.data(), r->out.size() * sizeof(double));
  return SF_OK;
  SF_SGUARD_END
}

int sf_server_cancel(sf_server* s, uint64_t ticket) {
  SF_SGUARD_BEGIN
  if (!s) sf::fail(SF_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) sf::fail(SF_EINVAL, "unknown ticket");
    auto r = it->second;
    r->cancel = 1;
    if (r->state == Q_QUEUED) {
      for (size_t i = 0; i < s->queue.size(); i++)
        if (s->queue[i] == r) {
          s->queue.erase(s->queue.begin() + i);
          break;
        }
      r->state = Q_CANCELLED;
      r->t_start = r->t_done = Clock::now();
    }
  }
  s->cv_done.notify_all();
  return SF_OK;
  SF_SGUARD_END
}

int sf_server_set_cost_model(sf_server* s, const double* coeffs, double max_wait_s) {
  SF_SGUARD_BEGIN
  if (!s || !(max_wait_s >= 0)) sf::fail(SF_EINVAL, "bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  s->model = coeffs != nullptr;
  if (coeffs)
    for (int j = 0; j < 4; j++) {
      if (!(coeffs[j] >= 0)) sf::fail(SF_EINVAL, "model coefficients must be >= 0");
      s->coeffs[j] = coeffs[j];
    }
  s->max_wait_s = max_wait_s;
  return SF_OK;
  SF_SGUARD_END
}

int sf_server_times(sf_server* s, uint64_t ticket, double* queued_s, double* total_s) {
  SF_SGUARD_BEGIN
  if (!s) sf::fail(SF_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) sf::fail(SF_EINVAL, "unknown ticket");
  auto& r = *it->second;
  if (r.state != Q_DONE && r.state != Q_FAILED && r.state != Q_CANCELLED)
    sf::fail(SF_ETIMEOUT, "request not finished");
  using D = std::chrono::duration<double>;
  if (queued_s) *queued_s = D(r.t_start - r.t_submit).count();
  if (total_s) *total_s = D(r.t_done - r.t_submit).count();
  return SF_OK;
  SF_SGUARD_END
}

void sf_server_destroy(sf_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    for (auto& kv : s->all) {
      kv.second->cancel = 1;
      if (kv.second->state == Q_QUEUED) kv.second->state = Q_CANCELLED;
    }
    s->queue.clear();
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  delete s;
}

}  // extern "C"
