// Autotuner: picks the tile size, fusion width (register bits per thread),
// copy-run width and paths per launch (finals per block) of a plan by
// timing candidates on the device, on a sample of the request.
#include <cuda_runtime.h>

#include <algorithm>
#include <memory>
#include <vector>

#include "sf_internal.h"

namespace {

void ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) sf::fail(SF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

// Time one candidate: plan it, compile its kernels (jit), run the sample
// once to warm up and once timed. Returns seconds, or a negative value when
// the candidate cannot run (invalid shape, or no memory for its workspace).
double time_candidate(const sf_circuit* c, const sf_plan_opts& o, const sf_path_sel& s, const uint64_t* d_bits,
                      int64_t n, double* d_out, cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1) {
  std::unique_ptr<sf::Plan> P;
  try {
    P.reset(sf::plan_create(c->c, o));
    if (o.jit) sf::jit_prepare(*P);  // time the kernels the plan will run
    sf::ensure_device(*P);
  } catch (const sf::Error&) {
    return -1;
  }
  struct Free {
    sf::Plan* p;
    ~Free() {
      if (p->d_tabA) cudaFree(p->d_tabA);
      if (p->d_tabB) cudaFree(p->d_tabB);
      if (p->d_err) cudaFree(p->d_err);
      if (p->d_cnt) cudaFree(p->d_cnt);
      p->d_tabA = p->d_tabB = nullptr;
      p->d_err = nullptr;
      p->d_cnt = nullptr;
    }
  } fr{P.get()};
  DevBuf ws;
  size_t need = 0;
  try {
    need = sf::exec_workspace_bytes(*P, n, s);
  } catch (const sf::Error&) {
    return -1;
  }
  if (cudaMalloc(&ws.p, need) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  sf::ExecCtx ctx;
  void* cache = nullptr;
  ctx.cache_slot = &cache;
  ctx.profile = false;
  float ms = 0;
  try {
    sf::exec_run(*P, d_bits, n, s, d_out, 0, ws.p, need, st, false, &ctx);  // warm up
    ok(cudaEventRecord(e0, st), "cudaEventRecord");
    sf::exec_run(*P, d_bits, n, s, d_out, 0, ws.p, need, st, false, &ctx);
    ok(cudaEventRecord(e1, st), "cudaEventRecord");
    ok(cudaEventSynchronize(e1), "cudaEventSynchronize");
    ok(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
    sf::check_wait_flag(P->d_err, st);
  } catch (...) {
    sf::exec_free_cache(cache);
    throw;
  }
  sf::exec_free_cache(cache);
  return ms * 1e-3;
}

}  // namespace

extern "C" int sf_plan_autotune(const sf_circuit* c, const sf_plan_opts* base, const sf_path_sel* sel,
                                int64_t sample_paths, const uint64_t* d_bits, int64_t n, sf_plan_opts* best,
                                double* best_seconds, double* base_seconds) {
  try {
    if (!c || !base || !sel || !best || sample_paths <= 0 || n <= 0 || !d_bits)
      sf::fail(SF_EINVAL, "bad argument");
    sf_plan_opts b = *base;
    if (b.exec_mode != SF_EXEC_BATCHED && b.exec_mode != SF_EXEC_PLAIN) sf::fail(SF_EINVAL, "bad exec mode");
    // the sample: the first sample_paths ids of the selection, as a list
    std::vector<uint64_t> ids;
    {
      std::unique_ptr<sf::Plan> probe(sf::plan_create(c->c, b));
      double fa = 0;
      auto rs = sf::select_ranges(*probe, *sel, &fa);
      for (auto& r : rs)
        for (uint64_t v = r.lo; v < r.hi && (int64_t)ids.size() < sample_paths; v++) ids.push_back(v);
      if (ids.empty()) sf::fail(SF_EINVAL, "empty selection");
    }
    sf_path_sel s{};
    s.mode = SF_SEL_LIST;
    s.list = ids.data();
    s.n_list = (int64_t)ids.size();
    cudaStream_t st = nullptr;
    ok(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "cudaStreamCreate");
    DevBuf out;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double best_t = 1e300, base_t = -1;
    sf_plan_opts best_o = b;
    try {
      ok(cudaMalloc(&out.p, (size_t)n * 16), "cudaMalloc");
      ok(cudaEventCreate(&e0), "cudaEventCreate");
      ok(cudaEventCreate(&e1), "cudaEventCreate");
      auto consider = [&](const sf_plan_opts& o) {
        const double t = time_candidate(c, o, s, d_bits, n, (double*)out.p, st, e0, e1);
        if (t >= 0 && t < best_t) {
          best_t = t;
          best_o = o;
        }
        return t;
      };
      base_t = consider(b);
      // stage 1: the pass shape - tile size (0: the planner's per-segment
      // choice), fusion width k = fuse_bits register qubits per thread block
      // (2..5), copy-run width (0: per segment)
      for (int tb : {0, 12, 13})
        for (int fb : {2, 3, 4, 5})
          for (int rb : {0, 3, 4}) {
            if ((tb == 0) != (rb == 0)) continue;  // automatic tile and run choice go together
            sf_plan_opts o = b;
            o.tile_bits = tb;
            o.fuse_bits = fb;
            o.run_bits = rb;
            if (o.tile_bits == b.tile_bits && o.fuse_bits == b.fuse_bits && o.run_bits == b.run_bits) continue;
            consider(o);
          }
      // stage 2: paths per launch (finals per block) at the best shape
      const sf_plan_opts shape = best_o;
      for (int bp : {1, 4, 16, 64, 256, 1024}) {
        if (bp > (int)ids.size()) break;
        sf_plan_opts o = shape;
        o.batch_paths = bp;
        if (o.batch_paths == shape.batch_paths) continue;
        consider(o);
      }
    } catch (...) {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      cudaStreamDestroy(st);
      throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (best_t >= 1e300) sf::fail(SF_ENOMEM, "no candidate configuration could run");
    *best = best_o;
    if (best_seconds) *best_seconds = best_t;
    if (base_seconds) *base_seconds = base_t;
    return SF_OK;
  } catch (const sf::Error& e) {
    sf::set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    sf::set_error(e.what());
    return SF_EINVAL;
  }
}
