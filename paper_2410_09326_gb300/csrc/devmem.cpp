// Device allocations of the library with an optional process-wide budget
// (qs_set_memory_limit): a request that would take the library's live
// device bytes above the budget is refused before cudaMalloc runs, so a
// caller sharing the GPU can bound what the simulator takes and tests can
// exercise the allocation-failure paths without exhausting a GPU.
#include <mutex>
#include <unordered_map>

#include "qs_internal.h"

namespace qs {

namespace {

std::mutex g_mu;
std::unordered_map<void *, size_t> g_sizes;
size_t g_in_use = 0;
size_t g_limit = 0;
thread_local bool t_refused = false;

}  // namespace

bool dev_refused_by_budget() { return t_refused; }

cudaError_t dev_malloc(void **p, size_t bytes) {
  *p = nullptr;
  t_refused = false;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_limit && (bytes > g_limit || g_in_use > g_limit - bytes)) {
      t_refused = true;
      return cudaErrorMemoryAllocation;
    }
    g_in_use += bytes;  // reserved until the allocation is known
  }
  cudaError_t e = cudaMalloc(p, bytes);
  std::lock_guard<std::mutex> lk(g_mu);
  if (e != cudaSuccess) {
    g_in_use -= bytes;
    *p = nullptr;
    cudaGetLastError();
    return e;
  }
  g_sizes[*p] = bytes;
  return cudaSuccess;
}

void dev_free(void *p) {
  if (!p) return;
  cudaFree(p);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_sizes.find(p);
  if (it != g_sizes.end()) {
    g_in_use -= it->second;
    g_sizes.erase(it);
  }
}

}  // namespace qs

extern "C" {

void qs_set_memory_limit(uint64_t bytes) {
  std::lock_guard<std::mutex> lk(qs::g_mu);
  qs::g_limit = (size_t)bytes;
}

uint64_t qs_memory_in_use(void) {
  std::lock_guard<std::mutex> lk(qs::g_mu);
  return (uint64_t)qs::g_in_use;
}

}  // extern "C"
