// sf_amplitudes_device_noalloc: the device-buffer amplitude call with its
// scratch memory taken from one fixed array compiled into this library, so
// that the call itself never allocates device memory.
//
// Who needs it: callers that must not call cudaMalloc once they are running.
// cudaMalloc can synchronise the whole device and can fail when another
// allocator in the process (for example a framework's caching allocator) has
// already reserved the free memory; a service with a fixed memory plan, or
// one that cannot afford an implicit device-wide synchronisation in its
// request path, wants every byte decided before its requests start.
//
// The scratch array holds what sf_amplitudes_device takes from its caller's
// workspace: the path-tree node buffers, the compact-final maps and buffers,
// and (SF_PREC_COMPENSATED) the compensation terms. Its size is fixed at
// SF_NOALLOC_SCRATCH_BYTES (64 MiB); every GPU that loads this module keeps
// that much device memory until the process exits. The plan's gather tables
// and wait-timeout flag are allocated when the plan is created, and its
// kernels are loaded then, so a call only enqueues kernels.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "sf_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)SF_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device with that device
// current. In host code `g_scratch` names a host-side stand-in, never the
// device memory, so kernels only ever receive this looked-up address.
std::mutex g_mu;
void* g_base[128] = {nullptr};

}  // namespace

namespace sf {

// Called from the plan's device set-up (the device current), and by the call
// itself on a device where no plan was set up yet.
void* noalloc_prepare(int device) {
  if (device < 0 || device >= 128) fail(SF_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      fail(e == cudaErrorMemoryAllocation ? SF_ENOMEM : SF_ECUDA,
           std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_base[device] = p;
  }
  return g_base[device];
}

}  // namespace sf

extern "C" int sf_amplitudes_device_noalloc(sf_plan* h, const uint64_t* d_bits, int64_t n,
                                            const sf_path_sel* sel, double* d_out, int accumulate,
                                            void* stream) {
  try {
    if (!h || !sel) sf::fail(SF_EINVAL, "null argument");
    if (n < 0) sf::fail(SF_EINVAL, "negative bitstring count");
    if (n > 0 && (!d_bits || !d_out)) sf::fail(SF_EINVAL, "null device buffer");
    sf::Plan& p = *h->p;
    int device = 0;
    cudaError_t ce = cudaGetDevice(&device);
    if (ce != cudaSuccess) sf::fail(SF_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce));
    if (!p.d_tabA || p.device != device)
      sf::fail(SF_EINVAL,
               "sf_amplitudes_device_noalloc: the plan has no device state on the current device (create the "
               "plan with this device current)");
    // the executor reserves 256 bytes to align the workspace base
    const int64_t room = (int64_t)kScratchBytes - 256;
    size_t need = 0;
    try {
      need = sf::exec_workspace_bytes(p, n, *sel, room);
    } catch (const sf::Error& e) {
      if (e.code != SF_ENOMEM) throw;
      need = kScratchBytes + 1;
    }
    if (need > kScratchBytes)
      sf::fail(SF_ENOMEM, "sf_amplitudes_device_noalloc: this plan and request need " + std::to_string(need) +
                              " bytes, more than the " + std::to_string(kScratchBytes >> 20) +
                              " MiB fixed scratch (use sf_amplitudes_device with a caller workspace)");
    void* base = sf::noalloc_prepare(device);
    sf::ExecCtx ctx;
    void* cache = nullptr;
    ctx.cache_slot = &cache;
    ctx.profile = false;
    ctx.budget = room;
    try {
      sf::exec_run(p, d_bits, n, *sel, d_out, accumulate, base, kScratchBytes, stream, false, &ctx);
    } catch (...) {
      sf::exec_free_cache(cache);
      throw;
    }
    sf::exec_free_cache(cache);
    return SF_OK;
  } catch (const sf::Error& e) {
    sf::set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    sf::set_error(e.what());
    return SF_EINVAL;
  }
}
