// sf_amplitudes_device_noalloc: the device-buffer amplitude call with every
// piece of scratch memory taken from one fixed array compiled into this
// library, so that the call itself never allocates device memory.
//
// Who needs it: callers that must not call cudaMalloc once they are running.
// cudaMalloc can synchronise the whole device and can fail when another
// allocator in the process (for example a framework's caching allocator) has
// already reserved the free memory; a service with a fixed memory plan, or
// one that cannot afford an implicit device-wide synchronisation in its
// request path, wants every byte decided when the library is loaded.
//
// The scratch array holds the two 8 x 256-entry gather tables, the wait
// error flag and the path-tree node buffers (the workspace that
// sf_amplitudes_device takes from its caller). Its size is fixed at
// SF_NOALLOC_SCRATCH_BYTES (64 MiB); every GPU that loads the library keeps
// that much device memory until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "sf_internal.h"

namespace {

constexpr size_t kScratchBytes = (size_t)SF_NOALLOC_SCRATCH_BYTES;
constexpr size_t kTabBytes = 8 * 256 * sizeof(uint32_t);
constexpr size_t kHeader = 2 * kTabBytes + 256;  // tables A, B, error flag

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Device address of g_scratch, looked up once per device with that device
// current. In host code `g_scratch` names a host-side stand-in, never the
// device memory, so kernels only ever receive this looked-up address.
std::mutex g_mu;
void* g_base[128] = {nullptr};

void* scratch_base(int device) {
  if (device < 0 || device >= 128) sf::fail(SF_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_base[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      sf::fail(SF_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
    g_base[device] = p;
  }
  return g_base[device];
}

void ok(cudaError_t e, const char* what) {
  if (e != cudaSuccess) sf::fail(SF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" int sf_amplitudes_device_noalloc(sf_plan* h, const uint64_t* d_bits, int64_t n,
                                            const sf_path_sel* sel, double* d_out, int accumulate,
                                            void* stream) {
  try {
    if (!h || !sel) sf::fail(SF_EINVAL, "null argument");
    if (n < 0) sf::fail(SF_EINVAL, "negative bitstring count");
    if (n > 0 && (!d_bits || !d_out)) sf::fail(SF_EINVAL, "null device buffer");
    sf::Plan& p = *h->p;
    int device = 0;
    ok(cudaGetDevice(&device), "cudaGetDevice");
    const int64_t room = (int64_t)(kScratchBytes - kHeader);
    size_t need = 0;
    try {
      need = sf::exec_workspace_bytes(p, n, *sel, room);
    } catch (const sf::Error& e) {
      if (e.code != SF_ENOMEM) throw;
      need = (size_t)room + 1;
    }
    if (need > (size_t)room)
      sf::fail(SF_ENOMEM, "sf_amplitudes_device_noalloc: one path of this plan needs more than the " +
                              std::to_string(kScratchBytes >> 20) +
                              " MiB fixed scratch (use sf_amplitudes_device with a caller workspace)");
    unsigned char* base = static_cast<unsigned char*>(scratch_base(device));
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t* tabA = reinterpret_cast<uint32_t*>(base);
    uint32_t* tabB = reinterpret_cast<uint32_t*>(base + kTabBytes);
    int* err = reinterpret_cast<int*>(base + 2 * kTabBytes);
    // the array keeps the previous call's contents: refresh the tables and
    // clear the error flag; node buffers are always written before read
    ok(cudaMemcpyAsync(tabA, p.A.tab.data(), kTabBytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    ok(cudaMemcpyAsync(tabB, p.B.tab.data(), kTabBytes, cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    ok(cudaMemsetAsync(err, 0, sizeof(int), st), "cudaMemsetAsync");
    sf::ExecCtx ctx;
    void* cache = nullptr;
    ctx.cache_slot = &cache;
    ctx.profile = false;
    ctx.tabA = tabA;
    ctx.tabB = tabB;
    ctx.err = err;
    ctx.budget = room;
    try {
      sf::exec_run(p, d_bits, n, *sel, d_out, accumulate, base + kHeader, (size_t)room, st, false, &ctx);
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
