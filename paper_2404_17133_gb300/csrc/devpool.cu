// Per-stream cache of work buffers and the shared-memory attribute cache
// (declared in common.cuh).
#include <map>
#include <mutex>
#include <unordered_map>
#include <utility>
#include <vector>

#include "common.cuh"

namespace tddft {

namespace {

constexpr size_t kCacheMax = 64ull << 20;           // larger blocks are not cached
constexpr size_t kCachedPerStream = 4ull << 30;     // cap on idle cached bytes per stream

// size class: 256 B minimum, powers of two up to 1 MiB, then 1 MiB multiples
size_t size_class(size_t n) {
  if (n <= 256) return 256;
  if (n <= (1u << 20)) {
    size_t c = 512;
    while (c < n) c <<= 1;
    return c;
  }
  return (n + (1u << 20) - 1) & ~(size_t)((1u << 20) - 1);
}

struct StreamCache {
  std::unordered_map<size_t, std::vector<void*>> free;
  size_t idle = 0;
};

std::mutex g_pool_mu;
std::unordered_map<cudaStream_t, StreamCache>& caches() {
  static auto* m = new std::unordered_map<cudaStream_t, StreamCache>();   // outlives exit-time frees
  return *m;
}

}  // namespace

void* pool_get(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (bytes > kCacheMax) {
    TD_CUDA(cudaMallocAsync(&p, bytes, s));
    return p;
  }
  const size_t c = size_class(bytes);
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = caches().find(s);
    if (it != caches().end()) {
      auto f = it->second.free.find(c);
      if (f != it->second.free.end() && !f->second.empty()) {
        p = f->second.back();
        f->second.pop_back();
        it->second.idle -= c;
        return p;
      }
    }
  }
  TD_CUDA(cudaMallocAsync(&p, c, s));
  return p;
}

void pool_put(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (bytes <= kCacheMax) {
    const size_t c = size_class(bytes);
    std::lock_guard<std::mutex> lk(g_pool_mu);
    StreamCache& sc = caches()[s];
    if (sc.idle + c <= kCachedPerStream) {
      sc.free[c].push_back(p);
      sc.idle += c;
      return;
    }
  }
  cudaFreeAsync(p, s);
}

void pool_trim(cudaStream_t s) {
  std::vector<void*> all;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = caches().find(s);
    if (it == caches().end()) return;
    for (auto& kv : it->second.free)
      for (void* p : kv.second) all.push_back(p);
    caches().erase(it);
  }
  for (void* p : all) cudaFreeAsync(p, s);
}

void ensure_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  TD_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{kernel, dev}];
  if (bytes > have) {
    TD_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    have = bytes;
  }
}

}  // namespace tddft
