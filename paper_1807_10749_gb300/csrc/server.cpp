// Request server: continuous batching of simulation requests on one GPU.
//
// A request is (plan, bitstrings, path selection), the problem statement of
// Sections 2-3. Worker threads, each with its own CUDA stream, take requests
// from one queue:
//  * admission: a request runs only while the device memory it needs (the
//    path-tree workspace plus bitstrings and amplitudes, the M_proc model of
//    Section 8) fits the budget next to everything the other workers hold; a
//    request that does not fit lets later, smaller ones pass until it has
//    waited one second, after which it blocks admission until memory frees
//    (or, with a runtime model set, shortest predicted time first);
//  * batching across requests: a worker that takes a request also takes the
//    queued requests on the same plan, and runs them as one batch - their
//    paths share one path tree and every pass launch carries all of them
//    (Section 2: the paths of a circuit are independent, so requests that
//    share a circuit share its work); each request is gathered into its own
//    output, bit for bit what it gets alone;
//  * resident state: a worker keeps its device buffers between batches, and
//    the path-tree nodes too while consecutive batches use the same plan, so
//    a request that repeats a selected prefix does not evolve it again;
//  * failure: every pass wait is bounded; each worker checks its own
//    wait-timeout flag after a batch and fails that batch's requests with
//    SF_ECUDA.
// Kernels of different workers' batches overlap on the device.
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

constexpr int kMaxBatch = 16;  // requests per batch

struct Request {
  uint64_t ticket = 0;
  sf::Plan* plan = nullptr;
  std::vector<uint64_t> bits;
  std::vector<uint64_t> list;
  sf_path_sel sel;
  std::vector<sf::Range> rs;
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

// Device memory a worker keeps between batches.
struct Pool {
  void* ws = nullptr;
  size_t ws_bytes = 0;
  uint64_t* bits = nullptr;
  double* out = nullptr;
  int64_t cap_n = 0;
  int64_t bytes() const { return (int64_t)ws_bytes + 24 * cap_n; }
};

}  // namespace

struct sf_server {
  int64_t budget = 0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> queue;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  int64_t in_use = 0;  // pools of all workers (running batches grow their pool first)
  int running = 0;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::vector<std::thread> workers;
  // runtime model: when set, admission prefers the shortest predicted request
  bool model = false;
  double coeffs[4] = {0, 0, 0, 0};
  double max_wait_s = 1.0;
  int64_t n_batches = 0, n_batched = 0, max_batch = 0;
};

namespace {

void cuda_ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) sf::fail(e == cudaErrorMemoryAllocation ? SF_ENOMEM : SF_ECUDA,
                                 std::string(what) + ": " + cudaGetErrorString(e));
}

// Does a batch of footprint f fit for a worker that holds `pool` bytes?
bool fits(const sf_server& s, int64_t pool, int64_t f) {
  return s.in_use - pool + std::max(pool, f) <= s.budget || s.running == 0;
}

// Pick the next request to admit (caller holds the lock): the oldest one that
// fits, unless the oldest has waited > 1 s and does not fit. With a runtime
// model set, requests that have waited less than max_wait_s go in order of
// predicted time (shortest first) after any that have waited longer.
std::shared_ptr<Request> pick(sf_server& s, int64_t pool) {
  if (s.queue.empty()) return nullptr;
  auto now = Clock::now();
  if (s.model) {
    const auto aged = std::chrono::duration<double>(s.max_wait_s);
    int best = -1;
    double best_t = 0;
    for (size_t i = 0; i < s.queue.size(); i++) {
      auto& r = s.queue[i];
      const bool old = now - r->t_submit > aged;
      const bool ok = fits(s, pool, r->footprint);
      if (old) {
        if (best >= 0 && now - s.queue[best]->t_submit > aged) continue;  // an older aged one wins
        if (!ok) return nullptr;  // the oldest aged request blocks until memory frees
        best = (int)i;
        best_t = -1;
        continue;
      }
      if (!ok || (best >= 0 && best_t < 0)) continue;
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
    if (fits(s, pool, r->footprint)) {
      auto out = r;
      s.queue.erase(s.queue.begin() + i);
      return out;
    }
    if (i == 0 && now - r->t_submit > std::chrono::seconds(1)) return nullptr;
  }
  return nullptr;
}

// Device bytes of a batch: its workspace (the union of its paths) plus the
// bitstrings and amplitudes of every request.
int64_t batch_footprint(const std::vector<std::shared_ptr<Request>>& b, size_t* ws) {
  std::vector<sf::ExecReq> v(b.size());
  int64_t nb = 0;
  for (size_t i = 0; i < b.size(); i++) {
    v[i].rs = b[i]->rs;
    v[i].n = (int64_t)b[i]->bits.size();
    nb += v[i].n;
  }
  *ws = sf::exec_workspace_bytes(*b[0]->plan, v);
  return (int64_t)*ws + 24 * nb;
}

// Add the queued requests on the batch's plan while the batch still fits
// (caller holds the lock).
void extend_batch(sf_server& s, std::vector<std::shared_ptr<Request>>& b, int64_t pool, size_t* ws,
                  int64_t* foot) {
  for (size_t i = 0; i < s.queue.size() && b.size() < (size_t)kMaxBatch;) {
    auto& r = s.queue[i];
    if (r->plan != b[0]->plan) {
      i++;
      continue;
    }
    b.push_back(r);
    size_t w2 = 0;
    int64_t f2 = 0;
    try {
      f2 = batch_footprint(b, &w2);
    } catch (const sf::Error&) {
      f2 = s.budget + 1;
    }
    if (f2 > s.budget || !fits(s, pool, f2)) {
      b.pop_back();
      i++;
      continue;
    }
    *ws = w2;
    *foot = f2;
    s.queue.erase(s.queue.begin() + i);
  }
}

void release_pool(Pool& p) {
  if (p.ws) {
    sf::exec_forget_workspace(p.ws);
    cudaFree(p.ws);
  }
  if (p.bits) cudaFree(p.bits);
  if (p.out) cudaFree(p.out);
  p = Pool();
}

// Run one batch on the worker's stream with its pooled buffers; fills each
// request's output or error.
void run_batch(sf_server& s, std::vector<std::shared_ptr<Request>>& b, size_t ws_need, cudaStream_t st,
               Pool& pool, void** cache, sf::Plan** cache_plan, int* d_err) {
  int64_t ntot = 0;
  for (auto& r : b) ntot += (int64_t)r->bits.size();
  int code = 0;
  std::string msg;
  std::vector<sf::ExecReq> v(b.size());
  int64_t layout_budget = 0;  // the plan's own, unless the device is short of memory
  try {
    cuda_ok(cudaSetDevice(s.device), "cudaSetDevice");
    for (size_t i = 0; i < b.size(); i++) {
      v[i].rs = b[i]->rs;
      v[i].n = (int64_t)b[i]->bits.size();
    }
    if (pool.ws_bytes < ws_need) {
      if (pool.ws) {
        sf::exec_forget_workspace(pool.ws);
        cudaFree(pool.ws);
      }
      pool.ws = nullptr;
      pool.ws_bytes = 0;
      sf::exec_free_cache(*cache);  // its buffers were in the old workspace
      *cache = nullptr;
      size_t got = 0;
      layout_budget = sf::exec_alloc_workspace(*b[0]->plan, v, 0, &pool.ws, &got);
      pool.ws_bytes = got;
    }
    if (pool.cap_n < ntot) {
      if (pool.bits) cudaFree(pool.bits);
      if (pool.out) cudaFree(pool.out);
      pool.bits = nullptr;
      pool.out = nullptr;
      pool.cap_n = 0;
      cuda_ok(cudaMalloc((void**)&pool.bits, (size_t)ntot * 8), "cudaMalloc bitstrings");
      cuda_ok(cudaMalloc((void**)&pool.out, (size_t)ntot * 16), "cudaMalloc amplitudes");
      pool.cap_n = ntot;
    }
    if (*cache_plan != b[0]->plan) {  // resident nodes belong to one plan
      sf::exec_free_cache(*cache);
      *cache = nullptr;
      *cache_plan = b[0]->plan;
    }
    int64_t at = 0;
    for (size_t i = 0; i < b.size(); i++) {
      const int64_t n = (int64_t)b[i]->bits.size();
      if (n > 0)
        cuda_ok(cudaMemcpyAsync(pool.bits + at, b[i]->bits.data(), (size_t)n * 8, cudaMemcpyHostToDevice, st),
                "cudaMemcpyAsync");
      v[i].rs = b[i]->rs;
      v[i].d_bits = pool.bits + at;
      v[i].n = n;
      v[i].d_out = pool.out + 2 * at;
      v[i].accumulate = 0;
      v[i].cancel = &b[i]->cancel;
      at += n;
    }
    sf::ExecCtx ctx;
    ctx.cache_slot = cache;
    ctx.profile = false;
    ctx.err = d_err;
    ctx.budget = layout_budget;
    sf::exec_run(*b[0]->plan, v, pool.ws, pool.ws_bytes, st, true, &ctx);
    at = 0;
    for (size_t i = 0; i < b.size(); i++) {
      const int64_t n = (int64_t)b[i]->bits.size();
      b[i]->out.resize((size_t)2 * n);
      if (n > 0 && !v[i].cancelled)
        cuda_ok(cudaMemcpyAsync(b[i]->out.data(), pool.out + 2 * at, (size_t)n * 16, cudaMemcpyDeviceToHost, st),
                "cudaMemcpyAsync");
      at += n;
    }
    sf::check_wait_flag(d_err, st);
  } catch (const sf::Error& e) {
    cudaStreamSynchronize(st);
    code = e.code;
    msg = e.msg;
  } catch (const std::exception& e) {
    cudaStreamSynchronize(st);
    code = SF_EINVAL;
    msg = e.what();
  }
  if (code != 0) {  // node buffers may be half written
    sf::exec_free_cache(*cache);
    *cache = nullptr;
  }
  for (size_t i = 0; i < b.size(); i++) {
    Request& r = *b[i];
    if (code == SF_ECANCELLED || (code == 0 && (v[i].cancelled || r.cancel))) {
      r.err_code = SF_ECANCELLED;
      r.err = "request cancelled";
    } else {
      r.err_code = code;
      r.err = msg;
    }
  }
}

void worker(sf_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  int* d_err = nullptr;
  if (cudaMalloc(&d_err, sizeof(int)) == cudaSuccess) cudaMemset(d_err, 0, sizeof(int));
  Pool pool;
  void* cache = nullptr;
  sf::Plan* cache_plan = nullptr;
  while (true) {
    std::vector<std::shared_ptr<Request>> batch;
    size_t ws_need = 0;
    int64_t foot = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->stop || !s->queue.empty(); });
      if (s->stop) break;
      auto r = pick(*s, pool.bytes());
      if (!r) {
        // something is queued that does not fit: give back this worker's
        // idle buffers
        if (!s->queue.empty() && pool.bytes() > 0) {
          s->in_use -= pool.bytes();
          sf::exec_free_cache(cache);
          cache = nullptr;
          cache_plan = nullptr;
          release_pool(pool);
        }
        continue;
      }
      batch.push_back(r);
      ws_need = r->ws_bytes;
      foot = r->footprint;
      extend_batch(*s, batch, pool.bytes(), &ws_need, &foot);
      // the pool grows to the batch's footprint (it is counted while held)
      const int64_t grow = std::max<int64_t>(0, foot - pool.bytes());
      s->in_use += grow;
      s->running++;
      s->n_batches++;
      s->n_batched += (int64_t)batch.size();
      s->max_batch = std::max<int64_t>(s->max_batch, (int64_t)batch.size());
      for (auto& q : batch) {
        q->state = Q_RUNNING;
        q->t_start = Clock::now();
      }
    }
    const int64_t before = pool.bytes();
    if (!d_err) {
      for (auto& q : batch) {
        q->err_code = SF_ECUDA;
        q->err = "worker has no device error flag";
      }
    } else {
      run_batch(*s, batch, ws_need, st, pool, &cache, &cache_plan, d_err);
    }
    {
      std::lock_guard<std::mutex> lk(s->mu);
      // account the pool as actually held now
      s->in_use += pool.bytes() - std::max(before, foot);
      s->running--;
      for (auto& q : batch) {
        q->t_done = Clock::now();
        if (q->err_code == 0) q->state = Q_DONE;
        else if (q->err_code == SF_ECANCELLED) q->state = Q_CANCELLED;
        else q->state = Q_FAILED;
        q->bits.clear();
        q->bits.shrink_to_fit();
      }
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
  sf::exec_free_cache(cache);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->in_use -= pool.bytes();
  }
  release_pool(pool);
  if (d_err) cudaFree(d_err);
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
  double fa = 0;
  r->rs = sf::select_ranges(*r->plan, r->sel, &fa);
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

int sf_server_stats(sf_server* s, int64_t* batches, int64_t* requests, int64_t* max_batch) {
  SF_SGUARD_BEGIN
  if (!s) sf::fail(SF_EINVAL, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (batches) *batches = s->n_batches;
  if (requests) *requests = s->n_batched;
  if (max_batch) *max_batch = s->max_batch;
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
