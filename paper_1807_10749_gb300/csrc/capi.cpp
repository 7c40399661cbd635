// C ABI of the sfsim library (include/sfsim.h). Every entry point converts
// internal failures into a status code and a thread-local message.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>

#include "sf_internal.h"

using HostBuffers = SfHostBuffers;

namespace sf {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

void fail(int code, const std::string& msg) { throw Error{code, msg}; }

}  // namespace sf

using sf::Error;

#define SF_GUARD_BEGIN try {
#define SF_GUARD_END                                  \
  }                                                   \
  catch (const Error& e) {                            \
    sf::set_error(e.msg);                             \
    return e.code;                                    \
  }                                                   \
  catch (const std::bad_alloc&) {                     \
    sf::set_error("host allocation failed");          \
    return SF_ENOMEM;                                 \
  }                                                   \
  catch (const std::exception& e) {                   \
    sf::set_error(e.what());                          \
    return SF_EINVAL;                                 \
  }                                                   \
  catch (...) {                                       \
    sf::set_error("unknown internal error");          \
    return SF_EINVAL;                                 \
  }

static void cuda_check(cudaError_t e, const char* what) {
  if (e != cudaSuccess) sf::fail(e == cudaErrorMemoryAllocation ? SF_ENOMEM : SF_ECUDA,
                                 std::string(what) + ": " + cudaGetErrorString(e));
}

// Device-side state of a plan: the gather byte tables, the wait-timeout
// flag, the profile's count ring and the memory budget; every kernel the plan
// runs is loaded into the device's context here as well. Set up when the plan
// is created if a device is present, else on first use.
namespace sf {

static std::atomic<int> g_inject_timeouts{0};

void check_wait_flag(int* d_flag, void* stream) {
  cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "cudaStreamSynchronize");
  int flag = 0;
  if (d_flag) cuda_check(cudaMemcpy(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost), "cudaMemcpy");
  if (flag) {
    cuda_check(cudaMemset(d_flag, 0, sizeof(int)), "cudaMemset");
    fail(SF_ECUDA, "a kernel wait timed out (error flag set); the results of that call are invalid");
  }
  int v = g_inject_timeouts.load();
  while (v > 0 && !g_inject_timeouts.compare_exchange_weak(v, v - 1)) {
  }
  if (v > 0) fail(SF_ECUDA, "a kernel wait timed out (injected); the results of that call are invalid");
}

void ensure_device(sf::Plan& p) {
  if (p.d_tabA) return;
  cuda_check(cudaGetDevice(&p.device), "cudaGetDevice");
  if (p.opts.hbm_budget_bytes == 0) {
    size_t fr = 0, tot = 0;
    cuda_check(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
    p.opts.hbm_budget_bytes = (int64_t)(fr / 4 * 3);
  }
  uint32_t *a = nullptr, *b = nullptr, *cnt = nullptr;
  int* e = nullptr;
  try {
    cuda_check(cudaMalloc(&e, sizeof(int)), "cudaMalloc");
    cuda_check(cudaMemset(e, 0, sizeof(int)), "cudaMemset");
    cuda_check(cudaMalloc(&cnt, 2 * sf::kCountRing * sizeof(uint32_t)), "cudaMalloc");
    cuda_check(cudaMalloc(&a, 8 * 256 * sizeof(uint32_t)), "cudaMalloc");
    cuda_check(cudaMalloc(&b, 8 * 256 * sizeof(uint32_t)), "cudaMalloc");
    cuda_check(cudaMemcpy(a, p.A.tab.data(), 8 * 256 * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
    cuda_check(cudaMemcpy(b, p.B.tab.data(), 8 * 256 * 4, cudaMemcpyHostToDevice), "cudaMemcpy");
  } catch (...) {
    if (a) cudaFree(a);
    if (b) cudaFree(b);
    if (e) cudaFree(e);
    if (cnt) cudaFree(cnt);
    throw;
  }
  p.d_err = e;
  p.d_cnt = cnt;
  p.d_tabA = a;
  p.d_tabB = b;
  preload_kernels();
  if (p.opts.jit) jit_load(p);
  noalloc_prepare(p.device);
}

static bool have_device() {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}
}  // namespace sf
using sf::ensure_device;

extern "C" {

const char* sf_last_error(void) { return sf::g_last_error.c_str(); }

int sf_circuit_create(int rows, int cols, const sf_gate* gates, int64_t n_gates, sf_circuit** out) {
  SF_GUARD_BEGIN
  if (!out) sf::fail(SF_EINVAL, "null output pointer");
  *out = nullptr;
  sf::Circuit* c = sf::circuit_from_gates(rows, cols, gates, n_gates);
  sf_circuit* h = new sf_circuit();
  h->c = *c;
  delete c;
  *out = h;
  return SF_OK;
  SF_GUARD_END
}

int sf_circuit_parse(const char* text, sf_circuit** out) {
  SF_GUARD_BEGIN
  if (!out) sf::fail(SF_EINVAL, "null output pointer");
  *out = nullptr;
  sf::Circuit* c = sf::circuit_parse(text);
  sf_circuit* h = new sf_circuit();
  h->c = *c;
  delete c;
  *out = h;
  return SF_OK;
  SF_GUARD_END
}

int sf_circuit_info(const sf_circuit* c, int* rows, int* cols, int64_t* n_gates) {
  SF_GUARD_BEGIN
  if (!c) sf::fail(SF_EINVAL, "null circuit");
  if (rows) *rows = c->c.rows;
  if (cols) *cols = c->c.cols;
  if (n_gates) *n_gates = (int64_t)c->c.gates.size();
  return SF_OK;
  SF_GUARD_END
}

void sf_circuit_destroy(sf_circuit* c) { delete c; }

void sf_plan_opts_default(sf_plan_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->decomposition = SF_DEC_SCHMIDT;
  o->select_prefix_bits = -1;
  o->exec_mode = SF_EXEC_BATCHED;
  o->defer_last_level = 1;
  o->jit = 1;
  o->fp32x2 = 1;
  o->precision = SF_PREC_F64;
}

int sf_plan_create(const sf_circuit* c, const sf_plan_opts* opts, sf_plan** out) {
  SF_GUARD_BEGIN
  if (!c || !out) sf::fail(SF_EINVAL, "null argument");
  *out = nullptr;
  sf_plan_opts o;
  if (opts) o = *opts;
  else sf_plan_opts_default(&o);
  if (o.decomposition != SF_DEC_SCHMIDT && o.decomposition != SF_DEC_BLOCK4)
    sf::fail(SF_EINVAL, "unknown decomposition");
  if (o.exec_mode != SF_EXEC_BATCHED && o.exec_mode != SF_EXEC_PLAIN) sf::fail(SF_EINVAL, "unknown exec mode");
  if (o.tile_bits < 0 || o.tile_bits > sf::MAX_K) sf::fail(SF_EINVAL, "tile_bits out of range (0..14)");
  if (o.fuse_bits < 0 || o.fuse_bits > sf::MAX_R) sf::fail(SF_EINVAL, "fuse_bits out of range (0..5)");
  if (o.run_bits < 0 || o.run_bits > 8) sf::fail(SF_EINVAL, "run_bits out of range (0..8)");
  if (o.hbm_budget_bytes < 0 || o.batch_paths < 0) sf::fail(SF_EINVAL, "negative budget or batch");
  if (o.exec_mode == SF_EXEC_PLAIN) {
    o.defer_last_level = 0;
    o.batch_paths = 1;
  }
  if (o.jit != 0 && o.jit != 1) sf::fail(SF_EINVAL, "jit must be 0 or 1");
  if (o.dense_finals != 0 && o.dense_finals != 1) sf::fail(SF_EINVAL, "dense_finals must be 0 or 1");
  if (o.precision != SF_PREC_F64 && o.precision != SF_PREC_COMPENSATED) sf::fail(SF_EINVAL, "unknown precision");
  if (o.projector_side != SF_PROJ_A && o.projector_side != SF_PROJ_ALTERNATE)
    sf::fail(SF_EINVAL, "unknown projector side");
  if (o.tile_buffers != 0 && o.tile_buffers != 2 && o.tile_buffers != 3)
    sf::fail(SF_EINVAL, "tile_buffers must be 0, 2 or 3");
  if (o.cycle_segments != 0 && o.cycle_segments != 1) sf::fail(SF_EINVAL, "cycle_segments must be 0 or 1");
  sf::Plan* p = sf::plan_create(c->c, o);
  sf_plan* h = new sf_plan();
  h->p = p;
  try {
    if (o.jit) sf::jit_prepare(*p);
    if (sf::have_device()) ensure_device(*p);
  } catch (...) {
    sf_plan_destroy(h);
    throw;
  }
  *out = h;
  return SF_OK;
  SF_GUARD_END
}

int sf_plan_info(const sf_plan* h, int* n_cross, int* path_bits, int* m_a, int* m_b, int* n_levels) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  const sf::Plan& p = *h->p;
  if (n_cross) *n_cross = (int)p.cross.size();
  if (path_bits) *path_bits = p.path_bits;
  if (m_a) *m_a = p.A.m;
  if (m_b) *m_b = p.B.m;
  if (n_levels) *n_levels = (int)p.levels.size();
  return SF_OK;
  SF_GUARD_END
}

int sf_plan_stats(const sf_plan* h, int* passes_a, int* passes_b, int* stages_a, int* stages_b,
                  int* deferred) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  const sf::Plan& p = *h->p;
  int pa = 0, pb = 0, sa = 0, sb = 0;
  for (auto& s : p.A.seg) {
    pa += (int)s.passes.size();
    sa += s.n_stages;
  }
  for (auto& s : p.B.seg) {
    pb += (int)s.passes.size();
    sb += s.n_stages;
  }
  if (passes_a) *passes_a = pa;
  if (passes_b) *passes_b = pb;
  if (stages_a) *stages_a = sa;
  if (stages_b) *stages_b = sb;
  if (deferred) *deferred = p.deferred ? p.levels.back().n_cross : 0;
  return SF_OK;
  SF_GUARD_END
}



int sf_plan_segment_stats(const sf_plan* h, int half, int segment, int* passes, int* stages,
                          double* bytes_per_node) {
  SF_GUARD_BEGIN
  if (!h || half < 0 || half > 1) sf::fail(SF_EINVAL, "bad plan or half");
  const sf::Plan& p = *h->p;
  const sf::HalfPlan& H = half ? p.B : p.A;
  const int nL = (int)p.levels.size();
  const sf::SegmentPlan* seg = nullptr;
  if (segment >= 0 && segment <= nL) seg = &H.seg[segment];
  else if (segment == nL + 1 && p.deferred) seg = p.merged_last ? &H.last_merged : &H.last_deferred;
  else sf::fail(SF_EINVAL, "segment out of range");
  if (passes) *passes = (int)seg->passes.size();
  if (stages) *stages = seg->n_stages;
  if (bytes_per_node) *bytes_per_node = sf::segment_bytes(*seg);
  return SF_OK;
  SF_GUARD_END
}

int sf_plan_describe(const sf_plan* h, char* buf, size_t cap, size_t* len) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  std::string t = sf::plan_describe(*h->p);
  if (len) *len = t.size();
  if (buf && cap) {
    size_t n = std::min(cap - 1, t.size());
    std::memcpy(buf, t.data(), n);
    buf[n] = 0;
  }
  return SF_OK;
  SF_GUARD_END
}

static void free_host_buffers(HostBuffers& hb) {
  if (hb.ws) {
    sf::exec_forget_workspace(hb.ws);
    cudaFree(hb.ws);
  }
  if (hb.bits) cudaFree(hb.bits);
  if (hb.out) cudaFree(hb.out);
  if (hb.stream) cudaStreamDestroy((cudaStream_t)hb.stream);
  hb = HostBuffers();
}

void sf_plan_destroy(sf_plan* h) {
  if (!h) return;
  free_host_buffers(h->hb);
  if (h->p) {
    sf::prof_release(*h->p);
    if (h->p->d_err) cudaFree(h->p->d_err);
    if (h->p->d_cnt) cudaFree(h->p->d_cnt);
    if (h->p->d_tabA) cudaFree(h->p->d_tabA);
    if (h->p->d_tabB) cudaFree(h->p->d_tabB);
    sf::plan_destroy(h->p);
  }
  delete h;
}

int sf_plan_profile(sf_plan* h, int enable_timing) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  sf::Plan& p = *h->p;
  sf::prof_collect(p);
  for (int k = 0; k < 3; k++) {
    p.prof.launches[k] = 0;
    p.prof.bytes[k] = 0;
    p.prof.seconds[k] = 0;
  }
  p.prof.timing = enable_timing != 0;
  return SF_OK;
  SF_GUARD_END
}

int sf_plan_profile_read(sf_plan* h, int kernel, int64_t* launches, double* seconds, double* bytes) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  if (kernel < 0 || kernel > 2) sf::fail(SF_EINVAL, "kernel must be 0, 1 or 2");
  sf::Plan& p = *h->p;
  sf::prof_collect(p);
  if (launches) *launches = p.prof.launches[kernel];
  if (seconds) *seconds = p.prof.seconds[kernel];
  if (bytes) *bytes = p.prof.bytes[kernel];
  return SF_OK;
  SF_GUARD_END
}

int sf_selection_size(const sf_plan* h, const sf_path_sel* sel, uint64_t* n_paths, double* f_actual) {
  SF_GUARD_BEGIN
  if (!h || !sel) sf::fail(SF_EINVAL, "null argument");
  double fa = 0;
  auto rs = sf::select_ranges(*h->p, *sel, &fa);
  uint64_t n = 0;
  for (auto& r : rs) n += r.hi - r.lo;
  if (n_paths) *n_paths = n;
  if (f_actual) *f_actual = fa;
  return SF_OK;
  SF_GUARD_END
}

int sf_selection_ids(const sf_plan* h, const sf_path_sel* sel, uint64_t* ids, uint64_t cap,
                     uint64_t* n_written) {
  SF_GUARD_BEGIN
  if (!h || !sel || (cap && !ids)) sf::fail(SF_EINVAL, "null argument");
  double fa = 0;
  auto rs = sf::select_ranges(*h->p, *sel, &fa);
  uint64_t w = 0;
  for (auto& r : rs)
    for (uint64_t v = r.lo; v < r.hi && w < cap; v++) ids[w++] = v;
  if (n_written) *n_written = w;
  return SF_OK;
  SF_GUARD_END
}

int sf_workspace_size(const sf_plan* h, int64_t n, const sf_path_sel* sel, size_t* bytes) {
  SF_GUARD_BEGIN
  if (!h || !sel || !bytes) sf::fail(SF_EINVAL, "null argument");
  if (n < 0) sf::fail(SF_EINVAL, "negative bitstring count");
  // the size depends on the device only through the default memory budget
  if (h->p->opts.hbm_budget_bytes == 0) ensure_device(*const_cast<sf::Plan*>(h->p));
  *bytes = sf::exec_workspace_bytes(*h->p, n, *sel);
  return SF_OK;
  SF_GUARD_END
}

int sf_amplitudes_device(sf_plan* h, const uint64_t* d_bits, int64_t n, const sf_path_sel* sel,
                         double* d_out, int accumulate, void* d_ws, size_t ws_bytes, void* stream) {
  SF_GUARD_BEGIN
  if (!h || !sel) sf::fail(SF_EINVAL, "null argument");
  if (n < 0) sf::fail(SF_EINVAL, "negative bitstring count");
  if (n > 0 && (!d_bits || !d_out)) sf::fail(SF_EINVAL, "null device buffer");
  ensure_device(*h->p);
  sf::exec_run(*h->p, d_bits, n, *sel, d_out, accumulate, d_ws, ws_bytes, stream, true);
  return SF_OK;
  SF_GUARD_END
}

static std::vector<sf::ExecReq> batch_reqs(const sf::Plan& p, const sf_request* reqs, int n_req) {
  if (n_req < 0 || (n_req > 0 && !reqs)) sf::fail(SF_EINVAL, "bad request array");
  std::vector<sf::ExecReq> v(n_req);
  for (int i = 0; i < n_req; i++) {
    const sf_request& r = reqs[i];
    if (!r.sel) sf::fail(SF_EINVAL, "request without a selection");
    if (r.n < 0) sf::fail(SF_EINVAL, "negative bitstring count");
    if (r.n > 0 && (!r.d_bitstrings || !r.d_out_amps)) sf::fail(SF_EINVAL, "null device buffer");
    double fa = 0;
    v[i].rs = sf::select_ranges(p, *r.sel, &fa);
    v[i].d_bits = r.d_bitstrings;
    v[i].n = r.n;
    v[i].d_out = r.d_out_amps;
    v[i].accumulate = r.accumulate;
  }
  return v;
}

int sf_workspace_size_batch(const sf_plan* h, const sf_request* reqs, int n_req, size_t* bytes) {
  SF_GUARD_BEGIN
  if (!h || !bytes) sf::fail(SF_EINVAL, "null argument");
  if (h->p->opts.hbm_budget_bytes == 0) ensure_device(*const_cast<sf::Plan*>(h->p));
  auto v = batch_reqs(*h->p, reqs, n_req);
  *bytes = sf::exec_workspace_bytes(*h->p, v);
  return SF_OK;
  SF_GUARD_END
}

int sf_amplitudes_device_batch(sf_plan* h, const sf_request* reqs, int n_req, void* d_ws, size_t ws_bytes,
                               void* stream) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  ensure_device(*h->p);
  auto v = batch_reqs(*h->p, reqs, n_req);
  sf::exec_run(*h->p, v, d_ws, ws_bytes, stream, true);
  return SF_OK;
  SF_GUARD_END
}

int sf_plan_drop_resident(sf_plan* h) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  sf::exec_release_cache(*h->p);
  free_host_buffers(h->hb);
  return SF_OK;
  SF_GUARD_END
}

int sf_plan_status(sf_plan* h, void* stream) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  sf::check_wait_flag(h->p->d_err, stream);
  return SF_OK;
  SF_GUARD_END
}

int sf_debug_inject_wait_timeouts(int count) {
  SF_GUARD_BEGIN
  if (count < 0) sf::fail(SF_EINVAL, "negative count");
  sf::g_inject_timeouts.store(count);
  return SF_OK;
  SF_GUARD_END
}

int sf_debug_set_wait_flag(sf_plan* h, int value) {
  SF_GUARD_BEGIN
  if (!h) sf::fail(SF_EINVAL, "null plan");
  ensure_device(*h->p);
  cuda_check(cudaMemcpy(h->p->d_err, &value, sizeof(int), cudaMemcpyHostToDevice), "cudaMemcpy");
  return SF_OK;
  SF_GUARD_END
}

int sf_probabilities_device(const double* d_amps, int64_t n, double scale, double* d_probs, void* stream) {
  SF_GUARD_BEGIN
  if (n < 0 || (n > 0 && (!d_amps || !d_probs))) sf::fail(SF_EINVAL, "bad argument");
  if (!(scale >= 0)) sf::fail(SF_EINVAL, "the scale must be >= 0");
  sf::launch_prob(d_amps, n, scale, d_probs, stream);
  return SF_OK;
  SF_GUARD_END
}

int sf_frugal_accept_device(const double* d_amps, const double* d_u, int64_t n, double N, double mprime,
                            double prob_scale, uint8_t* d_accept, int64_t* d_count, void* stream) {
  SF_GUARD_BEGIN
  if (n < 0) sf::fail(SF_EINVAL, "negative count");
  if (!d_count || (n > 0 && (!d_amps || !d_u || !d_accept))) sf::fail(SF_EINVAL, "null device buffer");
  if (!(N > 0) || !(mprime > 0) || !(prob_scale > 0)) sf::fail(SF_EINVAL, "N, M' and the scale must be positive");
  sf::launch_frugal(d_amps, d_u, n, N, mprime, prob_scale, d_accept, d_count, stream);
  return SF_OK;
  SF_GUARD_END
}

int sf_overlap_device(const double* a, const double* b, int64_t n, double* out, void* stream) {
  SF_GUARD_BEGIN
  if (n < 0 || !out || (n > 0 && (!a || !b))) sf::fail(SF_EINVAL, "bad argument");
  sf::launch_overlap(a, b, n, out, stream);
  return SF_OK;
  SF_GUARD_END
}

// The host-buffer forms: bitstrings in, amplitudes (prob = 0) or
// probabilities (prob = 1, divided by f_actual when divide_by_f) out.
static int host_form(sf_plan* h, const uint64_t* bits, int64_t n, const sf_path_sel* sel, double* out,
                     double* f_actual, int prob, int divide_by_f) {
  if (!h || !sel) sf::fail(SF_EINVAL, "null argument");
  if (n < 0) sf::fail(SF_EINVAL, "negative bitstring count");
  if (n > 0 && (!bits || !out)) sf::fail(SF_EINVAL, "null host buffer");
  double fa = 0;
  auto rs = sf::select_ranges(*h->p, *sel, &fa);
  if (f_actual) *f_actual = fa;
  if (n == 0) return SF_OK;
  HostBuffers& hb = h->hb;
  ensure_device(*h->p);
  size_t need = sf::exec_workspace_bytes(*h->p, n, *sel);
  if (!hb.stream) {
    cudaStream_t st = nullptr;
    cuda_check(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "cudaStreamCreate");
    hb.stream = st;
  }
  cudaStream_t hst = (cudaStream_t)hb.stream;
  sf::ExecCtx ctx;  // the plan's defaults; a smaller layout when memory is short
  if (hb.ws_bytes < need) {
    if (hb.ws) {
      sf::exec_forget_workspace(hb.ws);
      cudaFree(hb.ws);
    }
    hb.ws = nullptr;
    hb.ws_bytes = 0;
    std::vector<sf::ExecReq> one(1);
    one[0].rs = rs;
    one[0].n = n;
    size_t got = 0;
    ctx.budget = sf::exec_alloc_workspace(*h->p, one, 0, &hb.ws, &got);
    hb.ws_bytes = got;
  }
  if (hb.cap_n < n) {
    if (hb.bits) cudaFree(hb.bits);
    if (hb.out) cudaFree(hb.out);
    hb.bits = nullptr;
    hb.out = nullptr;
    hb.cap_n = 0;
    cuda_check(cudaMalloc(&hb.bits, (size_t)n * 8), "cudaMalloc bitstrings");
    cuda_check(cudaMalloc(&hb.out, (size_t)n * 24), "cudaMalloc output");
    hb.cap_n = n;
  }
  cuda_check(cudaMemcpyAsync(hb.bits, bits, (size_t)n * 8, cudaMemcpyHostToDevice, hst), "cudaMemcpyAsync");
  sf::exec_run(*h->p, hb.bits, n, *sel, hb.out, 0, hb.ws, hb.ws_bytes, hst, true, &ctx);
  if (prob) {
    sf::launch_prob(hb.out, n, divide_by_f ? (fa > 0 ? 1.0 / fa : 0.0) : 1.0, hb.probs(n), hst);
    cuda_check(cudaMemcpyAsync(out, hb.probs(n), (size_t)n * 8, cudaMemcpyDeviceToHost, hst), "cudaMemcpyAsync");
  } else {
    cuda_check(cudaMemcpyAsync(out, hb.out, (size_t)n * 16, cudaMemcpyDeviceToHost, hst), "cudaMemcpyAsync");
  }
  sf::check_wait_flag(h->p->d_err, hst);
  return SF_OK;
}

int sf_amplitudes(sf_plan* h, const uint64_t* bits, int64_t n, const sf_path_sel* sel, double* out,
                  double* f_actual) {
  SF_GUARD_BEGIN
  return host_form(h, bits, n, sel, out, f_actual, 0, 0);
  SF_GUARD_END
}

int sf_probabilities(sf_plan* h, const uint64_t* bits, int64_t n, const sf_path_sel* sel, int divide_by_f,
                     double* out, double* f_actual) {
  SF_GUARD_BEGIN
  return host_form(h, bits, n, sel, out, f_actual, 1, divide_by_f);
  SF_GUARD_END
}

}  // extern "C"
