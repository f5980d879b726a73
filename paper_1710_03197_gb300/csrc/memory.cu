// memory.cu - the library's device allocations, with a host-side fault
// injection hook for tests and a count of the bytes held.
//
// Every device buffer the library owns (plan arrays, work spaces, solver and
// batch buffers, temporaries) is allocated by dev_malloc_bytes and released
// by dev_free.  nufft_debug_fail_allocation arms a one-shot failure: the n-th
// allocation from then on returns cudaErrorMemoryAllocation without calling
// CUDA, so the NUFFT_ENOMEM paths run on a healthy device and leave no CUDA
// error behind.  nufft_debug_device_bytes reports the bytes held, so a test
// can check that a failed call released what it had taken.
#include <mutex>
#include <unordered_map>

#include "internal.cuh"

namespace nufft {
namespace {
std::mutex g_mem_mu;
std::unordered_map<void*, size_t> g_live;   // device pointer -> bytes
int64_t g_live_bytes = 0;
int64_t g_fail_countdown = -1;              // < 0: disarmed
}  // namespace

cudaError_t dev_malloc_bytes(void** ptr, size_t bytes) {
  *ptr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    if (g_fail_countdown == 0) {
      g_fail_countdown = -1;
      return cudaErrorMemoryAllocation;
    }
    if (g_fail_countdown > 0) --g_fail_countdown;
  }
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return e;
  }
  std::lock_guard<std::mutex> lock(g_mem_mu);
  g_live[*ptr] = bytes;
  g_live_bytes += (int64_t)bytes;
  return cudaSuccess;
}

cudaError_t dev_free(void* ptr) {
  if (!ptr) return cudaSuccess;
  {
    std::lock_guard<std::mutex> lock(g_mem_mu);
    auto it = g_live.find(ptr);
    if (it != g_live.end()) {
      g_live_bytes -= (int64_t)it->second;
      g_live.erase(it);
    }
  }
  return cudaFree(ptr);
}

}  // namespace nufft

extern "C" int nufft_debug_fail_allocation(int64_t n) {
  std::lock_guard<std::mutex> lock(nufft::g_mem_mu);
  nufft::g_fail_countdown = n < 0 ? -1 : n;
  return NUFFT_OK;
}

extern "C" int64_t nufft_debug_device_bytes(void) {
  std::lock_guard<std::mutex> lock(nufft::g_mem_mu);
  return nufft::g_live_bytes;
}
