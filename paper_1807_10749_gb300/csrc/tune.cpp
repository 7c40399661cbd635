// Autotuner: picks the tile size, fusion width (register bits per thread) and
// copy-run width of the fused passes by timing them on the device.
#include <cuda_runtime.h>

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

}  // namespace

extern "C" int sf_plan_autotune(const sf_circuit* c, const sf_plan_opts* base, const sf_path_sel* sel,
                                int64_t sample_paths, const uint64_t* d_bits, int64_t n, sf_plan_opts* best,
                                double* best_seconds) {
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
    ok(cudaMalloc(&out.p, (size_t)n * 16), "cudaMalloc");
    cudaEvent_t e0, e1;
    ok(cudaEventCreate(&e0), "cudaEventCreate");
    ok(cudaEventCreate(&e1), "cudaEventCreate");
    double best_t = 1e300;
    sf_plan_opts best_o = b;
    for (int tb : {11, 12, 13})
      for (int fb : {4, 5})
        for (int rb : {3, 4, 5}) {
          sf_plan_opts o = b;
          o.tile_bits = tb;
          o.fuse_bits = fb;
          o.run_bits = rb;
          std::unique_ptr<sf::Plan> P;
          try {
            P.reset(sf::plan_create(c->c, o));
          } catch (const sf::Error&) {
            continue;  // not a valid shape for this circuit
          }
          if (o.jit) sf::jit_prepare(*P);  // time the kernels the plan will run
          sf::ensure_device(*P);
          DevBuf ws;
          const size_t need = sf::exec_workspace_bytes(*P, n, s);
          if (cudaMalloc(&ws.p, need) != cudaSuccess) {
            cudaGetLastError();
            continue;
          }
          sf::ExecCtx ctx;
          void* cache = nullptr;
          ctx.cache_slot = &cache;
          ctx.profile = false;
          sf::exec_run(*P, d_bits, n, s, (double*)out.p, 0, ws.p, need, st, true, &ctx);  // warm up
          ok(cudaEventRecord(e0, st), "cudaEventRecord");
          sf::exec_run(*P, d_bits, n, s, (double*)out.p, 0, ws.p, need, st, false, &ctx);
          ok(cudaEventRecord(e1, st), "cudaEventRecord");
          ok(cudaEventSynchronize(e1), "cudaEventSynchronize");
          float ms = 0;
          ok(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
          sf::exec_free_cache(cache);
          if (P->d_tabA) cudaFree(P->d_tabA);
          if (P->d_tabB) cudaFree(P->d_tabB);
          if (P->d_err) cudaFree(P->d_err);
          if (P->d_cnt) cudaFree(P->d_cnt);
          P->d_tabA = P->d_tabB = nullptr;
          P->d_err = nullptr;
          P->d_cnt = nullptr;
          if (ms * 1e-3 < best_t) {
            best_t = ms * 1e-3;
            best_o = o;
          }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (best_t >= 1e300) sf::fail(SF_ENOMEM, "no candidate configuration could run");
    *best = best_o;
    if (best_seconds) *best_seconds = best_t;
    return SF_OK;
  } catch (const sf::Error& e) {
    sf::set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    sf::set_error(e.what());
    return SF_EINVAL;
  }
}
